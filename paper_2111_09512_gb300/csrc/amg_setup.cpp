// Host-side setup of the algebraic multigrid hierarchy (Sec. 3 of the paper:
// strength of connection with threshold theta, Ruge-Stueben coarsening,
// interpolation P, Galerkin coarse operators A_{l+1} = P^T A_l P), and the
// inverse of the coarsest operator for its direct solve.
//
// Compiled with -ffp-contract=off: every product and sum rounds as written,
// in the fixed orders stated below, so the hierarchy (C/F splits, patterns
// and values) is reproducible bit for bit.
#include "amg_setup.h"

#include <algorithm>
#include <cmath>
#include <set>
#include <utility>

namespace silu {

namespace {

// s[p] = 1 when entry p of row i (column j != i) is a strong connection:
// |a_ij| >= theta * max_{k != i} |a_ik| (rows without off-diagonals have none).
void strength(const Csr& A, double theta, std::vector<char>& s) {
  s.assign(A.ci.size(), 0);
  for (int64_t i = 0; i < A.n; ++i) {
    double mx = 0.0;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (A.ci[p] != i) mx = std::max(mx, std::fabs(A.va[p]));
    if (mx == 0.0) continue;
    const double cut = theta * mx;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (A.ci[p] != i && std::fabs(A.va[p]) >= cut) s[p] = 1;
  }
}

// Ruge-Stueben first pass with an ordered set keyed by (-measure, index):
// the front is always the undecided point of largest measure, smallest
// index among equals.
void split(const Csr& A, const std::vector<char>& s, std::vector<int32_t>& cf) {
  const int64_t n = A.n;
  // transpose of the strength graph: for point k, the rows j with k in S_j
  std::vector<int64_t> tp(n + 1, 0);
  for (int64_t p = 0; p < (int64_t)s.size(); ++p)
    if (s[p]) tp[A.ci[p] + 1]++;
  for (int64_t k = 0; k < n; ++k) tp[k + 1] += tp[k];
  std::vector<int32_t> tj(tp[n]);
  {
    std::vector<int64_t> f(tp.begin(), tp.end() - 1);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = A.rp[j]; p < A.rp[j + 1]; ++p)
        if (s[p]) tj[f[A.ci[p]]++] = (int32_t)j;
  }
  std::vector<int64_t> lam(n);
  std::vector<char> und(n, 1);
  std::set<std::pair<int64_t, int64_t>> order;
  for (int64_t k = 0; k < n; ++k) {
    lam[k] = tp[k + 1] - tp[k];
    order.insert({-lam[k], k});
  }
  cf.assign(n, 0);
  while (!order.empty()) {
    const auto top = *order.begin();
    const int64_t best = top.second;
    if (lam[best] == 0) break;  // the remaining undecided points become F
    order.erase(order.begin());
    und[best] = 0;
    cf[best] = 1;
    for (int64_t t = tp[best]; t < tp[best + 1]; ++t) {
      const int32_t j = tj[t];
      if (!und[j]) continue;
      und[j] = 0;  // F
      order.erase({-lam[j], j});
      for (int64_t p = A.rp[j]; p < A.rp[j + 1]; ++p) {
        const int32_t k = A.ci[p];
        if (!s[p] || !und[k]) continue;
        order.erase({-lam[k], k});
        lam[k]++;
        order.insert({-lam[k], k});
      }
    }
  }
}

// Direct interpolation.  C point: its coarse value.  F point i with strong
// coarse neighbours C_i: sneg / spos = sums of the negative / positive
// off-diagonal entries of row i, cneg / cpos the same over C_i (each summed
// in column order); d = a_ii (+ spos when cpos = 0, + sneg when cneg = 0);
// w_ij = -(f a_ij) / d with f = sneg / cneg (a_ij < 0) or spos / cpos.
void interpolation(const Csr& A, const std::vector<char>& s, const std::vector<int32_t>& cf, Csr& P, int64_t& nc) {
  const int64_t n = A.n;
  std::vector<int64_t> cidx(n, -1);
  nc = 0;
  for (int64_t i = 0; i < n; ++i)
    if (cf[i]) cidx[i] = nc++;
  P.n = n;
  P.rp.assign(n + 1, 0);
  P.ci.clear();
  P.va.clear();
  for (int64_t i = 0; i < n; ++i) {
    if (cf[i]) {
      P.ci.push_back((int32_t)cidx[i]);
      P.va.push_back(1.0);
    } else {
      double aii = 0.0, sneg = 0.0, spos = 0.0, cneg = 0.0, cpos = 0.0;
      for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        const double a = A.va[p];
        if (A.ci[p] == i) {
          aii += a;
          continue;
        }
        if (a < 0.0) sneg += a;
        if (a > 0.0) spos += a;
        if (s[p] && cf[A.ci[p]]) {
          if (a < 0.0) cneg += a;
          if (a > 0.0) cpos += a;
        }
      }
      double d = aii;
      if (cpos == 0.0) d += spos;
      if (cneg == 0.0) d += sneg;
      const double fneg = cneg != 0.0 ? sneg / cneg : 0.0;
      const double fpos = cpos != 0.0 ? spos / cpos : 0.0;
      for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        const int32_t j = A.ci[p];
        if (j == i || !s[p] || !cf[j]) continue;
        const double f = A.va[p] < 0.0 ? fneg : fpos;
        P.ci.push_back((int32_t)cidx[j]);
        P.va.push_back(-(f * A.va[p]) / d);
      }
    }
    P.rp[i + 1] = (int64_t)P.ci.size();
  }
}

// R = P^T as CSR (coarse rows, fine columns ascending).
void transpose_p(const Csr& P, int64_t nc, Csr& R) {
  R.n = nc;
  R.rp.assign(nc + 1, 0);
  for (int32_t c : P.ci) R.rp[c + 1]++;
  for (int64_t I = 0; I < nc; ++I) R.rp[I + 1] += R.rp[I];
  R.ci.resize(P.ci.size());
  R.va.resize(P.va.size());
  std::vector<int64_t> f(R.rp.begin(), R.rp.end() - 1);
  for (int64_t i = 0; i < P.n; ++i)
    for (int64_t q = P.rp[i]; q < P.rp[i + 1]; ++q) {
      const int64_t t = f[P.ci[q]]++;
      R.ci[t] = (int32_t)i;
      R.va[t] = P.va[q];
    }
}

// A_c = R A P, row I accumulated as sum over i in row I of R (ascending),
// j in row i of A (ascending), J in row j of P of (r_Ii a_ij) p_jJ, in that
// order, into a dense accumulator with a list of touched columns (sorted
// before the row is stored).
void galerkin(const Csr& A, const Csr& P, const Csr& R, Csr& Ac) {
  const int64_t nc = R.n;
  Ac.n = nc;
  Ac.rp.assign(nc + 1, 0);
  Ac.ci.clear();
  Ac.va.clear();
  std::vector<double> acc(nc, 0.0);
  std::vector<char> hit(nc, 0);
  std::vector<int32_t> cols;
  for (int64_t I = 0; I < nc; ++I) {
    cols.clear();
    for (int64_t t = R.rp[I]; t < R.rp[I + 1]; ++t) {
      const int64_t i = R.ci[t];
      const double rIi = R.va[t];
      for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        const int64_t j = A.ci[p];
        const double w = rIi * A.va[p];
        for (int64_t q = P.rp[j]; q < P.rp[j + 1]; ++q) {
          const int32_t J = P.ci[q];
          acc[J] += w * P.va[q];
          if (!hit[J]) {
            hit[J] = 1;
            cols.push_back(J);
          }
        }
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t J : cols) {
      Ac.ci.push_back(J);
      Ac.va.push_back(acc[J]);
      acc[J] = 0.0;
      hit[J] = 0;
    }
    Ac.rp[I + 1] = (int64_t)Ac.ci.size();
  }
}

// Dense inverse of a small matrix by LU with partial pivoting (row-major).
bool dense_inverse(const Csr& A, std::vector<double>& inv) {
  const int64_t m = A.n;
  std::vector<double> M(m * m, 0.0);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) M[i * m + A.ci[p]] += A.va[p];
  std::vector<int64_t> piv(m);
  for (int64_t k = 0; k < m; ++k) {
    int64_t r = k;
    for (int64_t i = k + 1; i < m; ++i)
      if (std::fabs(M[i * m + k]) > std::fabs(M[r * m + k])) r = i;
    if (M[r * m + k] == 0.0 || !std::isfinite(M[r * m + k])) return false;
    piv[k] = r;
    if (r != k)
      for (int64_t j = 0; j < m; ++j) std::swap(M[k * m + j], M[r * m + j]);
    for (int64_t i = k + 1; i < m; ++i) {
      const double f = M[i * m + k] / M[k * m + k];
      M[i * m + k] = f;
      for (int64_t j = k + 1; j < m; ++j) M[i * m + j] -= f * M[k * m + j];
    }
  }
  inv.assign(m * m, 0.0);
  std::vector<double> col(m);
  for (int64_t c = 0; c < m; ++c) {
    std::fill(col.begin(), col.end(), 0.0);
    col[c] = 1.0;
    for (int64_t k = 0; k < m; ++k) std::swap(col[k], col[piv[k]]);
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < i; ++j) col[i] -= M[i * m + j] * col[j];
    for (int64_t i = m - 1; i >= 0; --i) {
      for (int64_t j = i + 1; j < m; ++j) col[i] -= M[i * m + j] * col[j];
      col[i] /= M[i * m + i];
    }
    for (int64_t i = 0; i < m; ++i) inv[i * m + c] = col[i];
  }
  return true;
}

}  // namespace

int amg_build(const Csr& A, double theta, int max_levels, int64_t coarse_size, AmgHost& H, std::string& msg) {
  if (!(theta > 0.0 && theta <= 1.0) || max_levels < 1 || coarse_size < 1) {
    msg = "AMG needs 0 < theta <= 1, max_levels >= 1, coarse_size >= 1";
    return H_BADARG;
  }
  H.lev.clear();
  H.lev.emplace_back();
  H.lev[0].A = A;
  while ((int)H.lev.size() < max_levels && H.lev.back().A.n > coarse_size) {
    AmgLevel& L = H.lev.back();
    std::vector<char> s;
    strength(L.A, theta, s);
    std::vector<int32_t> cf;
    split(L.A, s, cf);
    int64_t nc = 0;
    for (int32_t c : cf) nc += c;
    if (nc == 0 || nc == L.A.n) break;
    interpolation(L.A, s, cf, L.P, nc);
    L.cf = std::move(cf);
    transpose_p(L.P, nc, L.R);
    AmgLevel C;
    galerkin(L.A, L.P, L.R, C.A);
    H.lev.push_back(std::move(C));
  }
  for (AmgLevel& L : H.lev) {  // l1-Jacobi diagonal: 1 / sum_j |a_ij|
    L.l1inv.assign(L.A.n, 0.0);
    for (int64_t i = 0; i < L.A.n; ++i) {
      double d = 0.0;
      for (int64_t p = L.A.rp[i]; p < L.A.rp[i + 1]; ++p) d += std::fabs(L.A.va[p]);
      if (d == 0.0) {
        msg = "AMG level with an empty row";
        return H_ZERO_PIVOT;
      }
      L.l1inv[i] = 1.0 / d;
    }
  }
  const Csr& Am = H.lev.back().A;
  if (Am.n > kAmgMaxCoarse) {
    msg = "coarsening stalled with " + std::to_string(Am.n) + " rows on the coarsest level (limit " +
          std::to_string(kAmgMaxCoarse) + ")";
    return H_BADARG;
  }
  if (!dense_inverse(Am, H.coarse_inv)) {
    msg = "singular coarsest operator";
    return H_ZERO_PIVOT;
  }
  return H_OK;
}

}  // namespace silu
