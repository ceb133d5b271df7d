// Host-side algebraic multigrid setup (Sec. 3): the hierarchy of Galerkin
// coarse operators built by Ruge-Stueben coarsening.  Pure C++; no CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "host_factor.h"

namespace silu {

// Largest coarsest level whose dense inverse is formed (8 * 4096^2 = 128 MiB).
constexpr int64_t kAmgMaxCoarse = 4096;

struct AmgLevel {
  Csr A;                      // A_l
  Csr P, R;                   // P_l (n_l x n_{l+1}) and R_l = P_l^T; empty on the coarsest level
  std::vector<int32_t> cf;    // 1 = coarse point (not on the coarsest level)
  std::vector<double> l1inv;  // 1 / sum_j |a_ij| (l1-Jacobi)
  Csr Lgs;                    // L D^{-1}: strict lower part of A, column j divided by a_jj (polynomial GS)
  std::vector<double> dinv;   // 1 / a_ii (polynomial GS)
};

struct AmgHost {
  std::vector<AmgLevel> lev;
  std::vector<double> coarse_inv;  // dense row-major inverse of the coarsest A
};

// Build the hierarchy from A (copied as level 0).  Strength: j strongly
// influences i when |a_ij| >= theta max_{k != i} |a_ik|.  C/F split: the
// Ruge-Stueben first pass (largest measure first, smallest index on ties;
// points left with measure 0 become F).  Interpolation: direct (Stueben).
// Coarse operators: A_{l+1} = P^T A_l P.  Coarsening stops at max_levels
// levels, at coarse_size rows or fewer, or when a split gives no or only C
// points.  Returns H_OK, H_BADARG (bad parameters, or a coarsest level above
// kAmgMaxCoarse rows) or H_ZERO_PIVOT (empty row, singular coarsest level).
int amg_build(const Csr& A, double theta, int max_levels, int64_t coarse_size, AmgHost& H, std::string& msg);
// Polynomial Gauss-Seidel data of every level below the finest (Lgs, dinv).
// H_ZERO_PIVOT for a zero or missing diagonal entry.
int amg_gs_factors(AmgHost& H, std::string& msg);

}  // namespace silu
