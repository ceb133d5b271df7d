// Host-side setup of the scaled-ILU smoother: CSR validation, incomplete
// factorisation (ILU(0), ILU(k), ILUT), row scaling and level sets.
// Pure C++; no CUDA.  Compiled with -ffp-contract=off: every pivot division
// and update rounds separately, so drop decisions are reproducible.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace silu {

struct Csr {
  int64_t n = 0;
  std::vector<int64_t> rp;  // n+1
  std::vector<int32_t> ci;
  std::vector<double> va;
  int64_t nnz() const { return rp.empty() ? 0 : rp.back(); }
};

// Host setup calls made on the calling thread use up to `budget` host
// threads for large systems (0: the default, up to 16 and the hardware's
// count).  Callers that already run several setups side by side (the solve
// server's workers, a batch's per-system threads) lower it, so that their
// threads do not multiply.
void set_setup_thread_budget(int budget);
int setup_thread_budget();

enum class Kind { ILU0 = 0, ILUK = 1, ILUT = 2, GS = 3, SGS = 4 };

// Result codes mirror silu_status.
enum HostStatus { H_OK = 0, H_BADARG = 1, H_ZERO_PIVOT = 2, H_OOM = 4 };

// Validate and canonicalise user CSR (sort columns, sum duplicates, check
// finiteness).  Returns H_OK or H_BADARG with a message.
int csr_canonical(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* va, Csr& out,
                  std::string& msg);

// Factor storage: L strict lower, U upper with the diagonal first per row.
struct Factors {
  Csr L, U;
  // symbolic data kept for a numeric refactorisation (ILU0 / ILUK):
  // pattern of L+U merged per row is implied by L and U themselves.
};

int factor_ilu0(const Csr& A, Factors& F, std::string& msg);
int factor_iluk(const Csr& A, int k, Factors& F, std::string& msg);
int factor_ilut(const Csr& A, double tau, int p, Factors& F, std::string& msg);
// Gauss-Seidel splitting written as factors (no elimination): with
// A = D + L_A + U_A, forward Gauss-Seidel M = D + L_A = (I + L_A D^{-1}) D,
// so L_s = L_A D^{-1} and U = D; symmetric Gauss-Seidel
// M = (D + L_A) D^{-1} (D + U_A) = (I + L_A D^{-1}) D (I + D^{-1} U_A), so
// U = D + U_A.  A zero, missing or non-finite diagonal gives H_ZERO_PIVOT.
int factor_gs(const Csr& A, bool symmetric, Factors& F, std::string& msg);
// Dispatch on the kind (0..4); `fill` is k for ILU(k) and p for ILUT.
int factor_kind(const Csr& A, int kind, double tau, int fill, Factors& F, std::string& msg);
// numeric phase only, on the pattern already in F (values overwritten)
int refactor_numeric(const Csr& A, Factors& F, std::string& msg);

// Row scaling: Us = strict part of D^{-1} U, dinv = 1 / diag(U).
int row_scale(const Csr& U, Csr& Us, std::vector<double>& dinv, std::string& msg);

// Row/column scaling (Eq. rowcolScale): Ruiz equilibration of U gives the
// column scaling dc (each step divides every row and every column of
// diag(r) U diag(dc) by the square root of its largest magnitude, both taken
// on the same matrix; at most `maxit` steps, stopping once every row and
// column maximum is within `tol` of one), then dr_i = 1 / (u_ii dc_i) so that
// Uhat = D_r U D_c has a unit diagonal.  Us = strict part of Uhat.  `steps`
// receives the number of equilibration steps taken.
int rowcol_scale(const Csr& U, int maxit, double tol, Csr& Us, std::vector<double>& dr, std::vector<double>& dc,
                 int& steps, std::string& msg);

// Level sets.  lev[i] of each row; rows grouped by level in ascending row
// order: level_ptr[nlev+1], level_rows[n].  Lower: from the top; upper
// (strict or with diagonal first): from the bottom.
int32_t levels_lower(const Csr& L, std::vector<int32_t>& lev);
int32_t levels_upper(const Csr& U, bool diag_first, std::vector<int32_t>& lev);
void group_levels(const std::vector<int32_t>& lev, int32_t nlev, std::vector<int32_t>& level_ptr,
                  std::vector<int32_t>& level_rows);

}  // namespace silu
