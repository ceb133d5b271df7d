// Host-side setup of the scaled-ILU smoother (see host_factor.h).
//
// The factorisations follow the paper's setup step (Sec. 4.2, Sec. 5.1): an
// incomplete LU with pivoting off, L unit lower, U upper, then the row
// scaling D = diag(U), Utilde = D^{-1} U (Eq. extractD, Eq. newD).  ILU(k)
// uses Saad's level-of-fill and ILUT Saad's dual threshold, the readings of
// the paper's "fill level" and "droptol / lfill".
#include "host_factor.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>

namespace silu {

namespace {

thread_local int g_thread_budget = 0;

// Host threads for row-parallel setup work on `work` stored entries: none
// below a million (thread start-up would dominate), else the calling
// thread's budget.
int host_threads(int64_t work) {
  if (work < ((int64_t)1 << 20)) return 1;
  return setup_thread_budget();
}

// fn(r0, r1, t) on nt contiguous ranges of rows [0, n), in parallel.
template <class Fn>
void row_ranges(int64_t n, int nt, Fn fn) {
  if (nt <= 1) {
    fn((int64_t)0, n, 0);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back([&, t]() { fn(n * t / nt, n * (t + 1) / nt, t); });
  for (std::thread& th : pool) th.join();
}

}  // namespace

void set_setup_thread_budget(int budget) { g_thread_budget = budget < 0 ? 0 : budget; }
int setup_thread_budget() {
  const int hw = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
  return g_thread_budget > 0 ? std::min(g_thread_budget, hw) : hw;
}

int csr_canonical(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci, const double* va, Csr& out,
                  std::string& msg) {
  if (n < 0 || nnz < 0 || n >= INT32_MAX || nnz >= INT32_MAX) {
    msg = "n and nnz must be in [0, 2^31 - 1)";
    return H_BADARG;
  }
  if (!rp || (nnz > 0 && (!ci || !va))) {
    msg = "null CSR array";
    return H_BADARG;
  }
  if (rp[0] != 0 || rp[n] != nnz) {
    msg = "row_ptr must start at 0 and end at nnz";
    return H_BADARG;
  }
  // row pointers first: every row's entries must lie inside [0, nnz) before
  // any is read
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i] || rp[i + 1] > nnz) {
      msg = "row_ptr is not monotone at row " + std::to_string(i);
      return H_BADARG;
    }
  // Rows are checked, sorted (stably) and their duplicates summed
  // independently, in two passes over contiguous row ranges on host threads:
  // the first checks and counts each row's distinct columns, the second writes
  // the rows in place at their final offsets.  The first bad row of the lowest
  // range that has one is the first bad row of the matrix.
  const int nt = host_threads(nnz);
  std::vector<int64_t> bad(nt, -1);
  std::vector<std::string> why(nt);
  out.n = n;
  out.rp.assign(n + 1, 0);
  auto sorted_row = [&](int64_t i, std::vector<std::pair<int32_t, double>>& row) {
    row.clear();
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) row.emplace_back(ci[p], va[p]);
    std::stable_sort(row.begin(), row.end(),
                     [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
                       return x.first < y.first;
                     });
  };
  row_ranges(n, nt, [&](int64_t r0, int64_t r1, int t) {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = r0; i < r1; ++i) {
      bool sorted = true;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        if (ci[p] < 0 || ci[p] >= n) {
          bad[t] = i;
          why[t] = "column index out of range in row ";
          return;
        }
        if (!std::isfinite(va[p])) {
          bad[t] = i;
          why[t] = "non-finite value in row ";
          return;
        }
        if (p > rp[i] && ci[p] <= ci[p - 1]) sorted = false;
      }
      int64_t distinct = rp[i + 1] - rp[i];
      if (!sorted) {
        sorted_row(i, row);
        distinct = 0;
        for (size_t q = 0; q < row.size(); ++q)
          if (q == 0 || row[q].first != row[q - 1].first) ++distinct;
      }
      out.rp[i + 1] = distinct;
    }
  });
  for (int t = 0; t < nt; ++t)
    if (bad[t] >= 0) {
      msg = why[t] + std::to_string(bad[t]);
      return H_BADARG;
    }
  for (int64_t i = 0; i < n; ++i) out.rp[i + 1] += out.rp[i];
  out.ci.resize((size_t)out.rp[n]);
  out.va.resize((size_t)out.rp[n]);
  row_ranges(n, nt, [&](int64_t r0, int64_t r1, int) {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = r0; i < r1; ++i) {
      int64_t o = out.rp[i];
      if (out.rp[i + 1] - o == rp[i + 1] - rp[i]) {  // sorted, no duplicates: copied as is
        std::copy(ci + rp[i], ci + rp[i + 1], out.ci.begin() + o);
        std::copy(va + rp[i], va + rp[i + 1], out.va.begin() + o);
        bool in_order = true;
        for (int64_t p = rp[i] + 1; p < rp[i + 1]; ++p) in_order = in_order && ci[p] > ci[p - 1];
        if (in_order) continue;
      }
      // duplicates or unsorted: stable sort, then sum equal columns in order
      sorted_row(i, row);
      o = out.rp[i] - 1;
      for (size_t q = 0; q < row.size(); ++q) {
        if (q > 0 && row[q].first == row[q - 1].first) {
          out.va[(size_t)o] += row[q].second;
        } else {
          ++o;
          out.ci[(size_t)o] = row[q].first;
          out.va[(size_t)o] = row[q].second;
        }
      }
    }
  });
  return H_OK;
}

namespace {

// Position of column c inside the sorted row [b, e) of ci, or -1.
int64_t find_col(const std::vector<int32_t>& ci, int64_t b, int64_t e, int32_t c) {
  auto it = std::lower_bound(ci.begin() + b, ci.begin() + e, c);
  if (it == ci.begin() + e || *it != c) return -1;
  return it - ci.begin();
}

// One row of the numeric incomplete LU on pattern P, IKJ order: for each
// k < i of P(i) in ascending order, l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj
// for the j > k of row k that are in P(i).  slot[] is -1 everywhere on entry
// and on return.  Returns H_OK, or H_ZERO_PIVOT for a structurally zero,
// zero or non-finite pivot.
int numeric_row(const Csr& A, const std::vector<int64_t>& prp, const std::vector<int32_t>& pci, int64_t i,
                std::vector<double>& lu, std::vector<int64_t>& dpos, int32_t* slot) {
  const int64_t b = prp[i], e = prp[i + 1];
  for (int64_t p = b; p < e; ++p) slot[pci[p]] = (int32_t)p;
  for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) lu[slot[A.ci[p]]] = A.va[p];
  const int64_t di = slot[i];
  if (di < 0) {
    for (int64_t p = b; p < e; ++p) slot[pci[p]] = -1;
    return H_ZERO_PIVOT;
  }
  dpos[i] = di;
  for (int64_t p = b; p < di; ++p) {
    const int32_t k = pci[p];
    lu[p] = lu[p] / lu[dpos[k]];
    const double lik = lu[p];
    for (int64_t q = dpos[k] + 1; q < prp[k + 1]; ++q) {
      const int64_t t = slot[pci[q]];
      if (t >= 0) lu[t] = lu[t] - lik * lu[q];
    }
  }
  for (int64_t p = b; p < e; ++p) slot[pci[p]] = -1;
  const double piv = lu[di];
  return (piv == 0.0 || !std::isfinite(piv)) ? H_ZERO_PIVOT : H_OK;
}

// Numeric incomplete LU on a fixed pattern P (which contains the pattern of
// A), row by row as numeric_row; lu receives the values on P.
//
// Row i reads only rows k < i of P(i), so the rows of one level of P's lower
// part (level(i) = 1 + the largest level of those k) are independent: large
// systems run level after level, the rows of a large level split over host
// threads (each with its own slot array).  Every row does the same
// arithmetic in the same order as in a row-by-row pass, so the factors are
// the same bits.  A failure reruns the row-by-row pass, which reports the
// first failing row.
int numeric_on_pattern(const Csr& A, const std::vector<int64_t>& prp, const std::vector<int32_t>& pci,
                       std::vector<double>& lu, std::vector<int64_t>& dpos, std::string& msg) {
  const int64_t n = A.n;
  lu.assign(pci.size(), 0.0);
  dpos.assign(n, -1);
  const int64_t nnz = prp[n];
  int nt = host_threads(nnz);
  // per-thread slot arrays of n int32: at most about 1 GB in all
  nt = (int)std::min<int64_t>(nt, std::max<int64_t>(1, ((int64_t)1 << 30) / (4 * std::max<int64_t>(n, 1))));
  if (n > 0 && nnz >= ((int64_t)1 << 20) && nt > 1) {
    std::vector<int32_t> lev(n, 0);
    int32_t nlev = 0;
    for (int64_t i = 0; i < n; ++i) {
      int32_t l = 0;
      for (int64_t p = prp[i]; p < prp[i + 1] && pci[p] < i; ++p) l = std::max(l, lev[pci[p]] + 1);
      lev[i] = l;
      nlev = std::max(nlev, l + 1);
    }
    std::vector<int64_t> lptr(nlev + 1, 0);
    for (int64_t i = 0; i < n; ++i) lptr[lev[i] + 1]++;
    for (int32_t l = 0; l < nlev; ++l) lptr[l + 1] += lptr[l];
    std::vector<int64_t> rows(n), fill(lptr.begin(), lptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) rows[fill[lev[i]]++] = i;  // ascending within a level
    std::vector<std::vector<int32_t>> slots(nt, std::vector<int32_t>(n, -1));
    std::vector<char> bad(nt, 0);
    bool failed = false;
    for (int32_t l = 0; l < nlev && !failed; ++l) {
      const int64_t r0 = lptr[l], r1 = lptr[l + 1];
      int64_t work = 0;  // entries of the level's rows: a proxy for its updates
      for (int64_t r = r0; r < r1; ++r) work += prp[rows[r] + 1] - prp[rows[r]];
      const int use = work >= (1 << 14) ? nt : 1;
      auto run = [&](int t) {
        const int64_t q0 = r0 + (r1 - r0) * t / use, q1 = r0 + (r1 - r0) * (t + 1) / use;
        for (int64_t r = q0; r < q1; ++r)
          if (numeric_row(A, prp, pci, rows[r], lu, dpos, slots[t].data()) != H_OK) {
            bad[t] = 1;
            return;
          }
      };
      if (use == 1) {
        run(0);
      } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < use; ++t) pool.emplace_back(run, t);
        for (std::thread& th : pool) th.join();
      }
      for (char c : bad) failed = failed || c;
    }
    if (!failed) return H_OK;
    lu.assign(pci.size(), 0.0);
    dpos.assign(n, -1);
  }
  std::vector<int32_t> slot(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    if (numeric_row(A, prp, pci, i, lu, dpos, slot.data()) != H_OK) {
      msg = (dpos[i] < 0 ? "structurally zero pivot in row " : "zero or non-finite pivot in row ") + std::to_string(i);
      return H_ZERO_PIVOT;
    }
  }
  return H_OK;
}

// Split values on pattern P at the diagonal into L (strict) and U (diagonal first).
void split_lu(int64_t n, const std::vector<int64_t>& prp, const std::vector<int32_t>& pci,
              const std::vector<double>& lu, const std::vector<int64_t>& dpos, Factors& F) {
  F.L.n = F.U.n = n;
  F.L.rp.assign(n + 1, 0);
  F.U.rp.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    F.L.rp[i + 1] = F.L.rp[i] + (dpos[i] - prp[i]);
    F.U.rp[i + 1] = F.U.rp[i] + (prp[i + 1] - dpos[i]);
  }
  F.L.ci.resize((size_t)F.L.rp[n]);
  F.L.va.resize((size_t)F.L.rp[n]);
  F.U.ci.resize((size_t)F.U.rp[n]);
  F.U.va.resize((size_t)F.U.rp[n]);
  row_ranges(n, host_threads(prp[n]), [&](int64_t r0, int64_t r1, int) {
    for (int64_t i = r0; i < r1; ++i) {
      std::copy(pci.begin() + prp[i], pci.begin() + dpos[i], F.L.ci.begin() + F.L.rp[i]);
      std::copy(lu.begin() + prp[i], lu.begin() + dpos[i], F.L.va.begin() + F.L.rp[i]);
      std::copy(pci.begin() + dpos[i], pci.begin() + prp[i + 1], F.U.ci.begin() + F.U.rp[i]);
      std::copy(lu.begin() + dpos[i], lu.begin() + prp[i + 1], F.U.va.begin() + F.U.rp[i]);
    }
  });
}

}  // namespace

int factor_ilu0(const Csr& A, Factors& F, std::string& msg) {
  std::vector<double> lu;
  std::vector<int64_t> dpos;
  int st = numeric_on_pattern(A, A.rp, A.ci, lu, dpos, msg);
  if (st != H_OK) return st;
  split_lu(A.n, A.rp, A.ci, lu, dpos, F);
  return H_OK;
}

// Level-of-fill symbolic phase.  Row i keeps a sorted singly linked list of
// its columns (next[] indexed by column, -1 terminated, head = n as a
// sentinel); walking it visits the L part in ascending order while fill is
// spliced in behind the walker.
int factor_iluk(const Csr& A, int kfill, Factors& F, std::string& msg) {
  if (kfill < 0) {
    msg = "ILU(k) needs k >= 0";
    return H_BADARG;
  }
  const int64_t n = A.n;
  std::vector<int64_t> prp(n + 1, 0);
  std::vector<int32_t> pci;
  std::vector<int32_t> plev;   // level of every pattern entry
  std::vector<int64_t> pdiag(n, -1);
  std::vector<int32_t> next(n + 1, -1);
  std::vector<int32_t> lev(n, 0);
  const int32_t head = (int32_t)n;
  pci.reserve(A.ci.size() * 2);
  plev.reserve(A.ci.size() * 2);
  for (int64_t i = 0; i < n; ++i) {
    // initial list: the sorted columns of A's row, level 0
    int32_t tail = head;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      next[tail] = A.ci[p];
      tail = A.ci[p];
      lev[A.ci[p]] = 0;
    }
    next[tail] = -1;
    for (int32_t k = next[head]; k != -1 && k < i; k = next[k]) {
      const int32_t lik = lev[k];
      int32_t prev = k;
      for (int64_t q = pdiag[k] + 1; q < prp[k + 1]; ++q) {
        const int32_t j = pci[q];
        const int32_t nl = lik + plev[q] + 1;
        while (next[prev] != -1 && next[prev] < j) prev = next[prev];
        if (next[prev] == j) {
          if (nl < lev[j]) lev[j] = nl;
        } else if (nl <= kfill) {
          next[j] = next[prev];
          next[prev] = j;
          lev[j] = nl;
        }
        if (next[prev] == j) prev = j;
      }
    }
    for (int32_t c = next[head]; c != -1; c = next[c]) {
      if (c == i) pdiag[i] = (int64_t)pci.size();
      pci.push_back(c);
      plev.push_back(lev[c]);
    }
    prp[i + 1] = (int64_t)pci.size();
    if (pdiag[i] < 0) {
      msg = "structurally zero pivot in row " + std::to_string(i);
      return H_ZERO_PIVOT;
    }
  }
  std::vector<double> lu;
  std::vector<int64_t> dpos;
  int st = numeric_on_pattern(A, prp, pci, lu, dpos, msg);
  if (st != H_OK) return st;
  split_lu(n, prp, pci, lu, dpos, F);
  return H_OK;
}

int factor_gs(const Csr& A, bool symmetric, Factors& F, std::string& msg) {
  const int64_t n = A.n;
  std::vector<double> d(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = find_col(A.ci, A.rp[i], A.rp[i + 1], (int32_t)i);
    if (q < 0 || A.va[q] == 0.0 || !std::isfinite(A.va[q])) {
      msg = "zero diagonal entry in row " + std::to_string(i);
      return H_ZERO_PIVOT;
    }
    d[i] = A.va[q];
  }
  F.L.n = F.U.n = n;
  F.L.rp.assign(n + 1, 0);
  F.U.rp.assign(n + 1, 0);
  F.L.ci.clear();
  F.L.va.clear();
  F.U.ci.clear();
  F.U.va.clear();
  for (int64_t i = 0; i < n; ++i) {
    F.U.ci.push_back((int32_t)i);
    F.U.va.push_back(d[i]);
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int32_t j = A.ci[p];
      if (j < i) {
        F.L.ci.push_back(j);
        F.L.va.push_back(A.va[p] / d[j]);
      } else if (j > i && symmetric) {
        F.U.ci.push_back(j);
        F.U.va.push_back(A.va[p]);
      }
    }
    F.L.rp[i + 1] = (int64_t)F.L.ci.size();
    F.U.rp[i + 1] = (int64_t)F.U.ci.size();
  }
  return H_OK;
}

int factor_kind(const Csr& A, int kind, double tau, int fill, Factors& F, std::string& msg) {
  switch (kind) {
    case (int)Kind::ILU0: return factor_ilu0(A, F, msg);
    case (int)Kind::ILUK: return factor_iluk(A, fill, F, msg);
    case (int)Kind::ILUT: return factor_ilut(A, tau, fill, F, msg);
    case (int)Kind::GS: return factor_gs(A, false, F, msg);
    case (int)Kind::SGS: return factor_gs(A, true, F, msg);
    default: msg = "bad factorisation kind"; return H_BADARG;
  }
}

int refactor_numeric(const Csr& A, Factors& F, std::string& msg) {
  const int64_t n = A.n;
  std::vector<int64_t> prp(n + 1, 0);
  std::vector<int32_t> pci;
  pci.reserve(F.L.ci.size() + F.U.ci.size());
  for (int64_t i = 0; i < n; ++i) {
    pci.insert(pci.end(), F.L.ci.begin() + F.L.rp[i], F.L.ci.begin() + F.L.rp[i + 1]);
    pci.insert(pci.end(), F.U.ci.begin() + F.U.rp[i], F.U.ci.begin() + F.U.rp[i + 1]);
    prp[i + 1] = (int64_t)pci.size();
    // the pattern must contain A's row
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (find_col(pci, prp[i], prp[i + 1], A.ci[p]) < 0) {
        msg = "new values do not fit the factor pattern";
        return H_BADARG;
      }
  }
  std::vector<double> lu;
  std::vector<int64_t> dpos;
  int st = numeric_on_pattern(A, prp, pci, lu, dpos, msg);
  if (st != H_OK) return st;
  split_lu(n, prp, pci, lu, dpos, F);
  return H_OK;
}

// ILUT(tau, p) with pivoting off.  The working row is a dense array w with a
// membership flag; the L part's columns sit in a sorted linked list that the
// elimination walks in ascending order (fill spliced in behind the walker),
// the U part's columns in a plain list.
int factor_ilut(const Csr& A, double tau, int pfill, Factors& F, std::string& msg) {
  if (!(tau >= 0.0) || pfill < 0) {
    msg = "ILUT needs tau >= 0 and fill >= 0";
    return H_BADARG;
  }
  const int64_t n = A.n;
  F.L.n = F.U.n = n;
  F.L.rp.assign(n + 1, 0);
  F.U.rp.assign(n + 1, 0);
  F.L.ci.clear();
  F.L.va.clear();
  F.U.ci.clear();
  F.U.va.clear();
  std::vector<double> w(n, 0.0);
  std::vector<char> member(n, 0);
  std::vector<int32_t> next(n + 1, -1);
  std::vector<int32_t> upper;
  std::vector<int32_t> kept;
  std::vector<std::pair<double, int32_t>> cand;
  const int32_t head = (int32_t)n;
  auto by_magnitude = [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
    return a.first > b.first || (a.first == b.first && a.second < b.second);
  };
  for (int64_t i = 0; i < n; ++i) {
    double ss = 0.0;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) ss = ss + A.va[p] * A.va[p];
    const double tau_i = tau * std::sqrt(ss);
    upper.clear();
    kept.clear();
    int32_t tail = head;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int32_t j = A.ci[p];
      w[j] = A.va[p];
      member[j] = 1;
      if (j < i) {
        next[tail] = j;
        tail = j;
      } else {
        upper.push_back(j);
      }
    }
    next[tail] = -1;
    for (int32_t k = next[head]; k != -1; k = next[k]) {
      w[k] = w[k] / F.U.va[F.U.rp[k]];
      if (std::fabs(w[k]) < tau_i) {
        w[k] = 0.0;
        continue;
      }
      kept.push_back(k);
      const double wk = w[k];
      int32_t prev = k;
      for (int64_t q = F.U.rp[k] + 1; q < F.U.rp[k + 1]; ++q) {
        const int32_t j = F.U.ci[q];
        if (!member[j]) {
          member[j] = 1;
          w[j] = 0.0;
          if (j < i) {
            while (next[prev] != -1 && next[prev] < j) prev = next[prev];
            next[j] = next[prev];
            next[prev] = j;
          } else {
            upper.push_back(j);
          }
        }
        w[j] = w[j] - wk * F.U.va[q];
      }
    }
    const double piv = member[i] ? w[i] : 0.0;
    if (piv == 0.0 || !std::isfinite(piv)) {
      for (int32_t k = next[head]; k != -1; k = next[k]) member[k] = 0, w[k] = 0.0;
      for (int32_t j : upper) member[j] = 0, w[j] = 0.0;
      msg = "zero or non-finite pivot in row " + std::to_string(i);
      return H_ZERO_PIVOT;
    }
    // L part: the kept multipliers, at most p of the largest
    cand.clear();
    for (int32_t k : kept) cand.emplace_back(std::fabs(w[k]), k);
    if ((int64_t)cand.size() > pfill) {
      std::nth_element(cand.begin(), cand.begin() + pfill, cand.end(), by_magnitude);
      cand.resize(pfill);
    }
    std::sort(cand.begin(), cand.end(),
              [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
                return a.second < b.second;
              });
    for (auto& c : cand) {
      F.L.ci.push_back(c.second);
      F.L.va.push_back(w[c.second]);
    }
    // U part: off-diagonals above the threshold, at most p of the largest
    cand.clear();
    for (int32_t j : upper)
      if (j > i && std::fabs(w[j]) >= tau_i) cand.emplace_back(std::fabs(w[j]), j);
    if ((int64_t)cand.size() > pfill) {
      std::nth_element(cand.begin(), cand.begin() + pfill, cand.end(), by_magnitude);
      cand.resize(pfill);
    }
    std::sort(cand.begin(), cand.end(),
              [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
                return a.second < b.second;
              });
    F.U.ci.push_back((int32_t)i);
    F.U.va.push_back(piv);
    for (auto& c : cand) {
      F.U.ci.push_back(c.second);
      F.U.va.push_back(w[c.second]);
    }
    F.L.rp[i + 1] = (int64_t)F.L.ci.size();
    F.U.rp[i + 1] = (int64_t)F.U.ci.size();
    for (int32_t k = next[head]; k != -1; k = next[k]) member[k] = 0, w[k] = 0.0;
    for (int32_t j : upper) member[j] = 0, w[j] = 0.0;
  }
  return H_OK;
}

int row_scale(const Csr& U, Csr& Us, std::vector<double>& dinv, std::string& msg) {
  const int64_t n = U.n;
  Us.n = n;
  Us.rp.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t b = U.rp[i], e = U.rp[i + 1];
    if (e <= b || U.ci[b] != i) {
      msg = "upper factor row without leading diagonal";
      return H_BADARG;
    }
    const double d = U.va[b];
    if (d == 0.0 || !std::isfinite(d)) {
      msg = "zero pivot in row scaling";
      return H_ZERO_PIVOT;
    }
    Us.rp[i + 1] = Us.rp[i] + (e - b - 1);
  }
  Us.ci.resize((size_t)Us.rp[n]);
  Us.va.resize((size_t)Us.rp[n]);
  dinv.assign(n, 0.0);
  // rows are independent: u_ij / u_ii and 1 / u_ii on host threads
  row_ranges(n, host_threads(U.rp[n]), [&](int64_t r0, int64_t r1, int) {
    for (int64_t i = r0; i < r1; ++i) {
      const int64_t b = U.rp[i], e = U.rp[i + 1];
      const double d = U.va[b];
      dinv[i] = 1.0 / d;
      int64_t o = Us.rp[i];
      for (int64_t p = b + 1; p < e; ++p, ++o) {
        Us.ci[o] = U.ci[p];
        Us.va[o] = U.va[p] / d;
      }
    }
  });
  return H_OK;
}

int rowcol_scale(const Csr& U, int maxit, double tol, Csr& Us, std::vector<double>& dr, std::vector<double>& dc,
                 int& steps, std::string& msg) {
  const int64_t n = U.n;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t b = U.rp[i];
    if (U.rp[i + 1] <= b || U.ci[b] != i) {
      msg = "upper factor row without leading diagonal";
      return H_BADARG;
    }
    if (U.va[b] == 0.0 || !std::isfinite(U.va[b])) {
      msg = "zero pivot in row/column scaling";
      return H_ZERO_PIVOT;
    }
  }
  std::vector<double> r(n, 1.0), rmax(n), cmax(n);
  dc.assign(n, 1.0);
  steps = 0;
  for (;;) {
    std::fill(rmax.begin(), rmax.end(), 0.0);
    std::fill(cmax.begin(), cmax.end(), 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = U.rp[i]; p < U.rp[i + 1]; ++p) {
        const double a = std::fabs(r[i] * U.va[p] * dc[U.ci[p]]);
        rmax[i] = std::max(rmax[i], a);
        cmax[U.ci[p]] = std::max(cmax[U.ci[p]], a);
      }
    double dev = 0.0;
    for (int64_t i = 0; i < n; ++i) dev = std::max(dev, std::max(std::fabs(1.0 - rmax[i]), std::fabs(1.0 - cmax[i])));
    if (dev <= tol || steps >= maxit) break;
    for (int64_t i = 0; i < n; ++i) {
      r[i] /= std::sqrt(rmax[i]);
      dc[i] /= std::sqrt(cmax[i]);
    }
    ++steps;
  }
  dr.resize(n);
  Us.n = n;
  Us.rp.assign(n + 1, 0);
  Us.ci.clear();
  Us.va.clear();
  for (int64_t i = 0; i < n; ++i) {
    dr[i] = 1.0 / (U.va[U.rp[i]] * dc[i]);
    for (int64_t p = U.rp[i] + 1; p < U.rp[i + 1]; ++p) {
      Us.ci.push_back(U.ci[p]);
      Us.va.push_back(dr[i] * U.va[p] * dc[U.ci[p]]);
    }
    Us.rp[i + 1] = (int64_t)Us.ci.size();
  }
  return H_OK;
}

int32_t levels_lower(const Csr& L, std::vector<int32_t>& lev) {
  const int64_t n = L.n;
  lev.assign(n, 0);
  int32_t top = -1;
  for (int64_t i = 0; i < n; ++i) {
    int32_t l = 0;
    for (int64_t p = L.rp[i]; p < L.rp[i + 1]; ++p) l = std::max(l, lev[L.ci[p]] + 1);
    lev[i] = l;
    top = std::max(top, l);
  }
  return top + 1;
}

int32_t levels_upper(const Csr& U, bool diag_first, std::vector<int32_t>& lev) {
  const int64_t n = U.n;
  lev.assign(n, 0);
  int32_t top = -1;
  for (int64_t i = n - 1; i >= 0; --i) {
    int32_t l = 0;
    for (int64_t p = U.rp[i] + (diag_first ? 1 : 0); p < U.rp[i + 1]; ++p) l = std::max(l, lev[U.ci[p]] + 1);
    lev[i] = l;
    top = std::max(top, l);
  }
  return top + 1;
}

void group_levels(const std::vector<int32_t>& lev, int32_t nlev, std::vector<int32_t>& level_ptr,
                  std::vector<int32_t>& level_rows) {
  const int64_t n = (int64_t)lev.size();
  level_ptr.assign((size_t)nlev + 1, 0);
  for (int64_t i = 0; i < n; ++i) level_ptr[lev[i] + 1]++;
  for (int32_t l = 0; l < nlev; ++l) level_ptr[l + 1] += level_ptr[l];
  level_rows.assign(n, 0);
  std::vector<int32_t> fillp(level_ptr.begin(), level_ptr.end() - 1);
  for (int64_t i = 0; i < n; ++i) level_rows[fillp[lev[i]]++] = (int32_t)i;
}

}  // namespace silu
