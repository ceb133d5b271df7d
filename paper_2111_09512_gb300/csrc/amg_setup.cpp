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
#include <memory>
#include <thread>
#include <utility>

namespace silu {

namespace {

// Host threads for row-parallel setup work (contiguous row ranges; results
// never depend on the count).
int setup_threads(int64_t work) {
  if (work < (1 << 16)) return 1;
  return setup_thread_budget();
}

// fn(r0, r1, t) on nt contiguous ranges of [0, n), in parallel.
template <class Fn>
void for_row_ranges(int64_t n, int nt, Fn fn) {
  if (nt <= 1) {
    fn(0, n, 0);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back([&, t]() { fn(n * t / nt, n * (t + 1) / nt, t); });
  for (std::thread& th : pool) th.join();
}

// s[p] = 1 when entry p of row i (column j != i) is a strong connection:
// |a_ij| >= theta * max_{k != i} |a_ik| (rows without off-diagonals have none).
void strength(const Csr& A, double theta, std::vector<char>& s) {
  s.assign(A.ci.size(), 0);
  for_row_ranges(A.n, setup_threads(A.nnz()), [&](int64_t r0, int64_t r1, int) {
    for (int64_t i = r0; i < r1; ++i) {
      double mx = 0.0;
      for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
        if (A.ci[p] != i) mx = std::max(mx, std::fabs(A.va[p]));
      if (mx == 0.0) continue;
      const double cut = theta * mx;
      for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
        if (A.ci[p] != i && std::fabs(A.va[p]) >= cut) s[p] = 1;
    }
  });
}

// A set of indices in [0, n) with the smallest member found in a few word
// scans: one bit per index, and above it summary levels with one bit per
// non-zero word of the level below.
class IndexSet {
 public:
  explicit IndexSet(int64_t n) {
    int64_t len = n;
    do {
      len = (len + 63) / 64;
      lv_.emplace_back((size_t)len, 0ull);
    } while (len > 1);
  }
  void insert(int64_t i) {
    for (auto& w : lv_) {
      const bool was = w[(size_t)(i >> 6)] != 0;
      w[(size_t)(i >> 6)] |= 1ull << (i & 63);
      if (was) return;
      i >>= 6;
    }
  }
  void erase(int64_t i) {
    for (auto& w : lv_) {
      w[(size_t)(i >> 6)] &= ~(1ull << (i & 63));
      if (w[(size_t)(i >> 6)] != 0) return;
      i >>= 6;
    }
  }
  bool empty() const { return lv_.back()[0] == 0; }
  int64_t first() const {  // smallest member (the set must not be empty)
    int64_t i = 0;
    for (size_t l = lv_.size(); l-- > 0;) i = (i << 6) | __builtin_ctzll(lv_[l][(size_t)i]);
    return i;
  }

 private:
  std::vector<std::vector<uint64_t>> lv_;
};

// Ruge-Stueben first pass.  Undecided points sit in buckets by measure; the
// pick is the smallest index of the highest non-empty bucket (largest
// measure, smallest index among equals).  Measures only grow.
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
  std::vector<std::unique_ptr<IndexSet>> bucket;
  auto at = [&](int64_t m) -> IndexSet& {
    while ((int64_t)bucket.size() <= m) bucket.emplace_back(nullptr);
    if (!bucket[m]) bucket[m].reset(new IndexSet(n));
    return *bucket[m];
  };
  int64_t top = -1;
  for (int64_t k = 0; k < n; ++k) {
    lam[k] = tp[k + 1] - tp[k];
    at(lam[k]).insert(k);
    top = std::max(top, lam[k]);
  }
  cf.assign(n, 0);
  for (;;) {
    while (top > 0 && (!bucket[top] || bucket[top]->empty())) --top;
    if (top <= 0) break;  // the remaining undecided points (measure 0) become F
    const int64_t best = bucket[top]->first();
    bucket[top]->erase(best);
    und[best] = 0;
    cf[best] = 1;
    for (int64_t t = tp[best]; t < tp[best + 1]; ++t) {
      const int32_t j = tj[t];
      if (!und[j]) continue;
      und[j] = 0;  // F
      bucket[lam[j]]->erase(j);
      for (int64_t p = A.rp[j]; p < A.rp[j + 1]; ++p) {
        const int32_t k = A.ci[p];
        if (!s[p] || !und[k]) continue;
        bucket[lam[k]]->erase(k);
        lam[k]++;
        at(lam[k]).insert(k);
        top = std::max(top, lam[k]);
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
  struct Part {
    std::vector<int64_t> len;
    std::vector<int32_t> ci;
    std::vector<double> va;
  };
  const int nt = setup_threads(A.nnz());
  std::vector<Part> parts(nt);
  for_row_ranges(n, nt, [&](int64_t r0, int64_t r1, int t) {
    Part& out = parts[t];
    out.len.assign((size_t)(r1 - r0), 0);
    for (int64_t i = r0; i < r1; ++i) {
      const size_t before = out.ci.size();
      if (cf[i]) {
        out.ci.push_back((int32_t)cidx[i]);
        out.va.push_back(1.0);
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
          out.ci.push_back((int32_t)cidx[j]);
          out.va.push_back(-(f * A.va[p]) / d);
        }
      }
      out.len[(size_t)(i - r0)] = (int64_t)(out.ci.size() - before);
    }
  });
  P.n = n;
  P.rp.assign(n + 1, 0);
  P.ci.clear();
  P.va.clear();
  int64_t i = 0;
  for (Part& pt : parts) {
    for (int64_t l : pt.len) {
      P.rp[i + 1] = P.rp[i] + l;
      ++i;
    }
    P.ci.insert(P.ci.end(), pt.ci.begin(), pt.ci.end());
    P.va.insert(P.va.end(), pt.va.begin(), pt.va.end());
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
// before the row is stored).  Rows are independent: contiguous ranges of
// them go to host threads, each with its own accumulator, and the ranges
// are concatenated in order, so the result does not depend on the thread
// count.
void galerkin(const Csr& A, const Csr& P, const Csr& R, Csr& Ac) {
  const int64_t nc = R.n;
  struct Part {
    std::vector<int64_t> len;
    std::vector<int32_t> ci;
    std::vector<double> va;
  };
  const int64_t work = R.nnz() + nc;
  const int nt = setup_threads(work);
  std::vector<Part> parts(nt);
  auto run = [&](int t) {
    const int64_t I0 = nc * t / nt, I1 = nc * (t + 1) / nt;
    Part& out = parts[t];
    out.len.assign((size_t)(I1 - I0), 0);
    std::vector<double> acc((size_t)nc, 0.0);
    std::vector<char> hit((size_t)nc, 0);
    std::vector<int32_t> cols;
    for (int64_t I = I0; I < I1; ++I) {
      cols.clear();
      for (int64_t t2 = R.rp[I]; t2 < R.rp[I + 1]; ++t2) {
        const int64_t i = R.ci[t2];
        const double rIi = R.va[t2];
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
        out.ci.push_back(J);
        out.va.push_back(acc[J]);
        acc[J] = 0.0;
        hit[J] = 0;
      }
      out.len[(size_t)(I - I0)] = (int64_t)cols.size();
    }
  };
  if (nt == 1) {
    run(0);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(run, t);
    for (std::thread& th : pool) th.join();
  }
  Ac.n = nc;
  Ac.rp.assign(nc + 1, 0);
  Ac.ci.clear();
  Ac.va.clear();
  int64_t I = 0;
  for (Part& pt : parts) {
    for (int64_t l : pt.len) {
      Ac.rp[I + 1] = Ac.rp[I] + l;
      ++I;
    }
    Ac.ci.insert(Ac.ci.end(), pt.ci.begin(), pt.ci.end());
    Ac.va.insert(Ac.va.end(), pt.va.begin(), pt.va.end());
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
    std::vector<char> empty(setup_threads(L.A.nnz()), 0);
    for_row_ranges(L.A.n, (int)empty.size(), [&](int64_t r0, int64_t r1, int t) {
      for (int64_t i = r0; i < r1; ++i) {
        double d = 0.0;
        for (int64_t p = L.A.rp[i]; p < L.A.rp[i + 1]; ++p) d += std::fabs(L.A.va[p]);
        if (d == 0.0) empty[t] = 1;
        L.l1inv[i] = d != 0.0 ? 1.0 / d : 0.0;
      }
    });
    for (char e : empty)
      if (e) {
        msg = "AMG level with an empty row";
        return H_ZERO_PIVOT;
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

int amg_gs_factors(AmgHost& H, std::string& msg) {
  for (size_t l = 1; l < H.lev.size(); ++l) {
    AmgLevel& L = H.lev[l];
    Factors F;
    const int st = factor_gs(L.A, false, F, msg);  // L_s = L_A D^{-1}, U = D
    if (st != H_OK) return st;
    L.Lgs = std::move(F.L);
    L.dinv.resize(L.A.n);
    for (int64_t i = 0; i < L.A.n; ++i) L.dinv[i] = 1.0 / F.U.va[F.U.rp[i]];
  }
  return H_OK;
}

}  // namespace silu
