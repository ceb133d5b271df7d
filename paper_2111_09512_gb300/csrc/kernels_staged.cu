// Staged Richardson sweep (sm_103a): out = epilogue(c - T in), one RHS.
//
// The sweep is a CSR SpMV that the paper's performance model treats as
// bandwidth-bound (one full read of the factor per sweep, Sec. 6.3).  On
// GB300 FP64 arithmetic is also scarce (about two FP64 lanes per clock per
// SM), so at 12 bytes per FP64 entry the FP64 pipe saturates at nearly the
// same rate as HBM: the kernel spends one FP64 fused multiply-add per entry
// of the longest row in each warp and nothing else, and keeps the FP64 unit
// fed while other warps wait on memory.
//
// Work is cut into warp tiles of consecutive rows: 32 rows (one per lane),
// or 16 / 8 with two / four lanes sharing a long row, or 64 / 128 with one
// lane taking two / four short rows in turn.  When row lengths vary, a second
// copy of the factor stores the rows of every 512-row window sorted by length
// (with their row numbers), so a warp's rows are about equally long and few
// FMA slots are spent on padding.
// Every warp walks its own fixed sequence of tiles with its own two-stage
// shared-memory ring: lane 0 issues three bulk asynchronous copies per tile
// (values, column indices, row pointers; a fourth with the row numbers of a
// sorted copy) that complete on the stage's
// mbarrier, marked evict-first in L2; the warp computes one tile while the
// next one lands.  Warps never wait for each other, so their gather and FMA
// phases interleave on the SM.  A lane's accumulator starts at c_i and takes
// acc <- acc - t_ij * in_j for each entry in column order, so c - T in costs
// one FMA per entry; the iterate vectors are read and written evict-last so
// they stay resident in L2 from one sweep to the next.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "device.cuh"

namespace silu {

int staged_lanes(const int64_t* rp, int64_t n) {
  const double avg = n ? (double)rp[n] / (double)n : 0.0;
  return avg <= 16.0 ? 1 : (avg <= 32.0 ? 2 : 4);
}

int staged_passes(const int64_t* rp, int64_t n, int lanes) {
  if (lanes != 1) return 1;
  const double avg = n ? (double)rp[n] / (double)n : 0.0;
  const double room = (double)(kTileNnz - 8) / (double)kTileRows;  // entries per row at one pass
  return avg * 4.0 <= room ? 4 : (avg * 2.0 <= room ? 2 : 1);
}

bool make_tiles(const int64_t* rp, int64_t n, int lanes, int passes, std::vector<int>& desc, int max_nnz) {
  desc.clear();
  const int rows = kTileRows * passes / lanes;
  int64_t r0 = 0;
  while (r0 < n) {
    int64_t r1 = r0;
    while (r1 < n && r1 - r0 < rows && rp[r1 + 1] - rp[r0] <= max_nnz - 8) ++r1;
    if (r1 == r0) return false;  // a single row does not fit
    desc.push_back((int)r0);
    desc.push_back((int)r1);
    desc.push_back((int)rp[r0]);
    desc.push_back((int)rp[r1]);
    r0 = r1;
  }
  return true;
}

bool narrow_fits(const int64_t* rp, int64_t n) {
  if (n <= 0) return false;
  int64_t longest = 0;
  for (int64_t r = 0; r < n; ++r) longest = std::max<int64_t>(longest, rp[r + 1] - rp[r]);
  const double mean = (double)rp[n] / (double)n;
  return longest <= kNarrowChunkRows && mean <= kNarrowMeanRow;
}

double tile_pad(const int64_t* rp, int64_t n) {
  std::vector<int> d;
  if (n <= 0 || rp[n] == 0 || !make_tiles(rp, n, 1, 1, d)) return 0.0;
  double slots = 0.0;
  for (size_t t = 0; t < d.size(); t += 4) {
    int64_t wmax = 0;
    for (int64_t r = d[t]; r < d[t + 1]; ++r) wmax = std::max<int64_t>(wmax, rp[r + 1] - rp[r]);
    slots += 32.0 * (double)wmax;
  }
  return slots / (double)rp[n];
}

void window_sort(const int64_t* rp, int64_t n, std::vector<int32_t>& perm, std::vector<int64_t>& srp) {
  perm.resize((size_t)n);
  for (int64_t w0 = 0; w0 < n; w0 += kSortWindow) {
    const int64_t w1 = std::min<int64_t>(n, w0 + kSortWindow);
    for (int64_t r = w0; r < w1; ++r) perm[(size_t)r] = (int32_t)r;
    std::stable_sort(perm.begin() + w0, perm.begin() + w1,
                     [rp](int32_t a, int32_t b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
  }
  srp.assign((size_t)n + 1, 0);
  for (int64_t s = 0; s < n; ++s) {
    const int32_t r = perm[(size_t)s];
    srp[(size_t)s + 1] = srp[(size_t)s] + (rp[r + 1] - rp[r]);
  }
}

bool sorting_pays(double natural, double sorted) {
  return natural >= kSortPadMin && sorted > 0.0 && natural - sorted >= kSortGain;
}

bool make_sorted(const int64_t* rp, const int32_t* ci, const double* va, int64_t n, std::vector<int64_t>& srp,
                 std::vector<int32_t>& sci, std::vector<double>& sva, std::vector<int32_t>& perm) {
  if (n <= 0 || rp[n] == 0) return false;
  const double pad0 = tile_pad(rp, n);
  if (pad0 < kSortPadMin) return false;
  window_sort(rp, n, perm, srp);
  if (!sorting_pays(pad0, tile_pad(srp.data(), n))) return false;
  sci.resize((size_t)rp[n]);
  sva.resize((size_t)rp[n]);
  for (int64_t s = 0; s < n; ++s) {
    const int32_t r = perm[(size_t)s];
    std::copy(ci + rp[r], ci + rp[r + 1], sci.begin() + srp[(size_t)s]);
    std::copy(va + rp[r], va + rp[r + 1], sva.begin() + srp[(size_t)s]);
  }
  return true;
}

namespace {

constexpr int kWarpStages = 2;
// Warps per CTA (one CTA per SM; shared memory holds one two-stage ring per
// warp).  FP32 stages are smaller, so more warps fit beside them.
constexpr int kWarpsF64 = 20;
constexpr int kWarpsF32 = 24;
template <class MT>
__host__ __device__ constexpr int warps_of() {
  return sizeof(MT) == 4 ? kWarpsF32 : kWarpsF64;
}
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of bar, giving up after kWaitNs.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Vector accesses that keep the iterates resident in L2 across sweeps.
__device__ __forceinline__ double ld_keep(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_keep(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_keep(double* p, double v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(float* p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

// One stage: a 16-byte header (the tile descriptor, written by the issuing
// lane), then values, column indices and row pointers as copied, and, for a
// length-sorted layout, the tile's row numbers in the vectors.
template <class MT, int RL, bool PERM, int NNZ = kTileNnz>
struct StageLayout {
  static constexpr int kValAlign = 16 / (int)sizeof(MT);  // elements per 16 bytes
  static constexpr size_t kHdr = 16;
  static constexpr size_t kVal = sizeof(MT) * (NNZ + 8);
  static constexpr size_t kCol = sizeof(int) * (NNZ + 8);
  static constexpr size_t kRp = sizeof(int) * (RL * kTileRows + 8);
  static constexpr size_t kPerm = PERM ? sizeof(int) * (kTileRows + 8) : 0;
  static constexpr size_t kBytes = kHdr + kVal + kCol + kRp + kPerm;  // all multiples of 16
};

// Issuing lane: record the descriptor d of a tile in the stage header and
// issue its copies into stage buffer `st` (three, or four with the row
// numbers of a sorted layout).  The header store precedes the arrive on the
// stage's mbarrier, so waiters see it.
template <class MT, int RL, bool PERM, bool RP = true, int NNZ = kTileNnz>
__device__ __forceinline__ void issue_tile(int4 d, unsigned char* st, uint64_t* bar, const int* __restrict__ rp,
                                           const int* __restrict__ ci, const MT* __restrict__ va,
                                           const int* __restrict__ perm, uint64_t pol) {
  using L = StageLayout<MT, RL, PERM, NNZ>;
  const int r0 = d.x, r1 = d.y, p0 = d.z, p1 = d.w;
  const int a0 = p0 & ~(L::kValAlign - 1), a1 = (p1 + L::kValAlign - 1) & ~(L::kValAlign - 1);
  const int c0 = p0 & ~3, c1 = (p1 + 3) & ~3;
  const int q0 = r0 & ~3, q1 = (r1 + 1 + 3) & ~3;
  const int m1 = (r1 + 3) & ~3;
  const uint32_t bv = (uint32_t)(a1 - a0) * (uint32_t)sizeof(MT);
  const uint32_t bc = (uint32_t)(c1 - c0) * 4u;
  const uint32_t br = RP ? (uint32_t)(q1 - q0) * 4u : 0u;
  const uint32_t bp = PERM ? (uint32_t)(m1 - q0) * 4u : 0u;
  *(int4*)st = d;
  fence_proxy_async();
  mbar_expect_tx(bar, bv + bc + br + bp);
  if (bv) bulk_g2s(st + L::kHdr, va + a0, bv, bar, pol);
  if (bc) bulk_g2s(st + L::kHdr + L::kVal, ci + c0, bc, bar, pol);
  if (RP) bulk_g2s(st + L::kHdr + L::kVal + L::kCol, rp + q0, br, bar, pol);
  if (PERM && bp) bulk_g2s(st + L::kHdr + L::kVal + L::kCol + L::kRp, perm + q0, bp, bar, pol);
}

// Epilogue operands (dinv_row, x_row) are read after the accumulation; a
// prefetch into L1 issued before it takes their memory latency off the end
// of the tile without holding registers through the gathers.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_epilogue(int epi, int row, const double* dinv, const double* x) {
  switch (epi) {
    case EPI_SCALE:
      prefetch_l1(dinv + row);
      break;
    case EPI_SCALE_ADDX:
    case EPI_JAC_ADDX:
      prefetch_l1(dinv + row);
      prefetch_l1(x + row);
      break;
    case EPI_SCALE_SETX:
    case EPI_JAC:
    case EPI_JAC_SETX:
      prefetch_l1(dinv + row);
      break;
    case EPI_ADDX:
    case EPI_RICH_ADDX:
      prefetch_l1(x + row);
      break;
    default:
      break;
  }
}

// t = c_row - (T in)_row, already formed by the accumulation
template <class MT, class VI, class VO>
__device__ __forceinline__ void epilogue(int epi, int row, MT t, const VI* in, VO* out, const double* dinv,
                                         double* x, uint64_t keep) {
  switch (epi) {
    case EPI_STORE: st_keep(out + row, (VO)t, keep); break;
    case EPI_SCALE: st_keep(out + row, (VO)(dinv[row] * (double)t), keep); break;
    case EPI_ADDX: x[row] += (double)t; break;
    case EPI_SETX: x[row] = (double)t; break;
    case EPI_SCALE_ADDX: x[row] += dinv[row] * (double)t; break;
    case EPI_SCALE_SETX: x[row] = dinv[row] * (double)t; break;
    case EPI_JAC: st_keep(out + row, (VO)((MT)in[row] + (MT)dinv[row] * t), keep); break;
    case EPI_JAC_ADDX: x[row] += (double)((MT)in[row] + (MT)dinv[row] * t); break;
    case EPI_JAC_SETX: x[row] = (double)((MT)in[row] + (MT)dinv[row] * t); break;
    case EPI_RICH: st_keep(out + row, (VO)(t + (MT)in[row]), keep); break;
    case EPI_RICH_ADDX: x[row] += (double)(t + (MT)in[row]); break;
    case EPI_RICH_SETX: x[row] = (double)(t + (MT)in[row]); break;
    default: break;
  }
}

// The same epilogues for column k of R interleaved right-hand sides: vector
// entries at o = row * ldx + k, dinv at row.
template <class MT, class VI, class VO>
__device__ __forceinline__ void epilogue_col(int epi, int row, size_t o, MT t, const VI* in, VO* out,
                                             const double* dinv, double* x, uint64_t keep) {
  switch (epi) {
    case EPI_STORE: st_keep(out + o, (VO)t, keep); break;
    case EPI_SCALE: st_keep(out + o, (VO)(dinv[row] * (double)t), keep); break;
    case EPI_ADDX: x[o] += (double)t; break;
    case EPI_SETX: x[o] = (double)t; break;
    case EPI_SCALE_ADDX: x[o] += dinv[row] * (double)t; break;
    case EPI_SCALE_SETX: x[o] = dinv[row] * (double)t; break;
    case EPI_JAC: st_keep(out + o, (VO)((MT)in[o] + (MT)dinv[row] * t), keep); break;
    case EPI_JAC_ADDX: x[o] += (double)((MT)in[o] + (MT)dinv[row] * t); break;
    case EPI_JAC_SETX: x[o] = (double)((MT)in[o] + (MT)dinv[row] * t); break;
    case EPI_RICH: st_keep(out + o, (VO)(t + (MT)in[o]), keep); break;
    case EPI_RICH_ADDX: x[o] += (double)(t + (MT)in[o]); break;
    case EPI_RICH_SETX: x[o] = (double)(t + (MT)in[o]); break;
    case EPI_SPMV: st_keep(out + o, (VO)t, keep); break;
    default: break;
  }
}

// R interleaved right-hand sides, one lane per row: acc[k] -/+= sum v[p]
// in[col[p] ldx + k] over the row's entries in column order.  All gathers
// of a chunk of CH entries (R values each, adjacent in memory) are issued
// before the first FMA; the FMA loop runs to the warp's longest row.  One
// factor entry read from shared memory feeds R FMAs.
template <class MT, class VI, bool NEG, int R, int CH>
__device__ __forceinline__ void row_accumulate_cols(const MT* sv, const int* sc, int len, const VI* __restrict__ in,
                                                    int ldx, MT (&acc)[R], uint64_t keep) {
  const int wmax = __reduce_max_sync(0xffffffffu, len);
  for (int k0 = 0; k0 < wmax; k0 += CH) {
    MT v[CH], xv[CH][R];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      if (k0 + q < len) {
        v[q] = sv[k0 + q];
        const VI* pin = in + (size_t)sc[k0 + q] * (size_t)ldx;
#pragma unroll
        for (int k = 0; k < R; ++k) xv[q][k] = (MT)ld_keep(pin + k, keep);
      } else {
        v[q] = MT(0);
#pragma unroll
        for (int k = 0; k < R; ++k) xv[q][k] = MT(0);
      }
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      if (k0 + q >= wmax) break;
#pragma unroll
      for (int k = 0; k < R; ++k) acc[k] = fma(NEG ? -v[q] : v[q], xv[q][k], acc[k]);
    }
  }
}

// acc -/+= sum v[p] * in[col[p]] over the entries p = sub, sub + G, ... of one
// row held in shared memory (G lanes share a row; sub is this lane's place).
// All gathers of a chunk of kChunk entries are issued before the first FMA
// (one latency round per chunk); the FMA loop runs to the warp's largest
// per-lane count (a warp-uniform bound) and padded slots multiply zeros,
// which leaves acc exactly unchanged.  The G partial sums are then combined
// with log2(G) shuffles.  Cost: one FP64 FMA per entry of the warp's longest
// lane, plus log2(G) adds per row.
template <class MT, class VI, bool NEG, int G, int kChunk>
__device__ __forceinline__ MT row_accumulate(const MT* sv, const int* sc, int len, int sub,
                                             const VI* __restrict__ in, MT acc, uint64_t keep) {
  const int cnt = len > sub ? (len - sub + G - 1) / G : 0;  // this lane's entries
  const int wmax = __reduce_max_sync(0xffffffffu, cnt);
  for (int k0 = 0; k0 < wmax; k0 += kChunk) {
    MT v[kChunk], xv[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      if (k0 + k < cnt) {
        const int p = (k0 + k) * G + sub;
        v[k] = sv[p];
        xv[k] = (MT)ld_keep(in + sc[p], keep);
      } else {
        v[k] = MT(0);
        xv[k] = MT(0);
      }
    }
    // warp-uniform exit: a predicated FMA would still occupy the FP64 pipe
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      if (k0 + k >= wmax) break;
      acc = fma(NEG ? -v[k] : v[k], xv[k], acc);
    }
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  return acc;
}

// One lane per row and RL rows per lane (rows r0 + p * 32 + lane of the
// tile, p < RL): the short-row case.  Taking the rows one after another costs
// RL dependent gather rounds per tile; here a round gathers up to CH / RL
// entries of every row at once (about the registers of CH entries of one row), then
// runs the FMAs of all RL independent accumulators, then stores the RL
// results.  Each row still accumulates c - sum t_ij in_j in column order, so
// results are bitwise those of the one-row-at-a-time loop.  The round count
// is the warp's longest row over all RL passes (warp-uniform).
template <class MT, class VI, class VO, int CH, int RL, bool PERM>
__device__ __forceinline__ void rows_accumulate(const MT* sv, const int* sc, const int* sr, const int* sp, int r0,
                                                int r1, int q0, int a0, int c0, int p0, int lane,
                                                const VI* __restrict__ c, const VI* __restrict__ in,
                                                VO* __restrict__ out, const double* __restrict__ dinv,
                                                double* __restrict__ x, int epi, uint64_t keep) {
  // entries of each row per round: CH / RL, at most 3 in FP64 (the 96
  // registers a thread has here hold 4 x 3 values and gathers without spills)
  constexpr int KP0 = CH / RL > 0 ? CH / RL : 1;
  constexpr int KP = (sizeof(MT) == 8 && KP0 > 3) ? 3 : KP0;
  int b[RL], len[RL], o[RL];
  MT acc[RL];
  int wmax = 0;
#pragma unroll
  for (int p = 0; p < RL; ++p) {
    const int r = r0 + p * 32 + lane;
    const bool act = r < r1;
    b[p] = act ? sr[r - q0] : p0;
    len[p] = act ? sr[r + 1 - q0] - b[p] : 0;
    o[p] = act ? (PERM ? sp[r - q0] : r) : -1;
    acc[p] = (act && c) ? (MT)ld_keep(c + o[p], keep) : MT(0);
    wmax = len[p] > wmax ? len[p] : wmax;
  }
  wmax = __reduce_max_sync(0xffffffffu, wmax);
  const bool neg = epi != EPI_SPMV;
  for (int k0 = 0; k0 < wmax; k0 += KP) {
    MT v[RL][KP], xv[RL][KP];
#pragma unroll
    for (int p = 0; p < RL; ++p)
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        if (k0 + k < len[p]) {
          v[p][k] = sv[b[p] - a0 + k0 + k];
          xv[p][k] = (MT)ld_keep(in + sc[b[p] - c0 + k0 + k], keep);
        } else {
          v[p][k] = MT(0);
          xv[p][k] = MT(0);
        }
      }
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      if (k0 + k >= wmax) break;  // warp-uniform; padded slots multiply zeros
#pragma unroll
      for (int p = 0; p < RL; ++p) acc[p] = fma(neg ? -v[p][k] : v[p][k], xv[p][k], acc[p]);
    }
  }
#pragma unroll
  for (int p = 0; p < RL; ++p) {
    if (o[p] < 0) continue;
    if (epi == EPI_SPMV)
      st_keep(out + o[p], (VO)acc[p], keep);
    else
      epilogue<MT, VI, VO>(epi, o[p], acc[p], in, out, dinv, x, keep);
  }
}

template <class MT, class VI, class VO, int G, int CH, int RL, bool PERM>
__global__ void __launch_bounds__(warps_of<MT>() * 32, 1)
    k_sweep_staged(int ntiles, const int4* __restrict__ tiles, const int* __restrict__ rp, const int* __restrict__ ci,
                   const MT* __restrict__ va, const int* __restrict__ perm, const VI* __restrict__ c,
                   const VI* __restrict__ in, VO* __restrict__ out, const double* __restrict__ dinv,
                   double* __restrict__ x, int epi, int flags, int* __restrict__ err) {
  using L = StageLayout<MT, RL, PERM>;
  constexpr int kWarps = warps_of<MT>();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kWarps][kWarpStages];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int w = 0; w < kWarps; ++w)
      for (int s = 0; s < kWarpStages; ++s) mbar_init(&full[w][s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int gw = blockIdx.x * kWarps + warp;  // this warp's first tile
  const int nw = gridDim.x * kWarps;          // tile stride
  unsigned char* ring = smem + (size_t)warp * kWarpStages * L::kBytes;
  // flags: kFlagReverse walks the tiles last to first (a warp's k-th tile is
  // ntiles - 1 - (gw + k nw)); kFlagFactorNormal / kFlagVectorNormal give the
  // factor copies / the vector accesses the normal L2 priority instead of
  // evict-first / evict-last
  const bool rev = (flags & kFlagReverse) != 0;
  const uint64_t stream = (flags & kFlagFactorNormal) ? policy_evict_normal() : policy_evict_first();
  const uint64_t keep = (flags & kFlagVectorNormal) ? policy_evict_normal() : policy_evict_last();
  grid_launch_dependents();
  // the factor and its tiles are never written by a sweep: the first copies
  // may start before the kernel that produced c and in has finished
  if (lane == 0)
    for (int s = 0; s < kWarpStages; ++s) {
      const int t = gw + s * nw;
      if (t < ntiles)
        issue_tile<MT, RL, PERM>(__ldg(tiles + (rev ? ntiles - 1 - t : t)), ring + s * L::kBytes, &full[warp][s], rp,
                                 ci, va, perm, stream);
    }
  grid_wait_prior();  // c, in, out and x below belong to the previous kernel until it completes
  int k = 0;
  for (int t = gw; t < ntiles; t += nw, ++k) {
    // the issuing lane fetches the descriptor of the tile it will issue next
    const int tn = t + kWarpStages * nw;
    int4 dn = make_int4(0, 0, 0, 0);
    if (lane == 0 && tn < ntiles) dn = __ldg(tiles + (rev ? ntiles - 1 - tn : tn));
    const int s = k % kWarpStages;
    const bool ok = mbar_wait_bounded(&full[warp][s], (uint32_t)(k / kWarpStages) & 1u);
    if (!__all_sync(0xffffffffu, ok)) {
      // a copy did not land in time: report, let the other stage's copy land, leave
      if (lane == 0) {
        atomicOr(err, 1);
        for (int d = 1; d < kWarpStages; ++d) {
          const int kd = k + d;
          if (t + d * nw < ntiles) mbar_wait_bounded(&full[warp][kd % kWarpStages], (uint32_t)(kd / kWarpStages) & 1u);
        }
      }
      return;
    }
    const unsigned char* st = ring + s * L::kBytes;
    const int4 d = *(const int4*)st;
    const MT* sv = (const MT*)(st + L::kHdr);
    const int* sc = (const int*)(st + L::kHdr + L::kVal);
    const int* sr = (const int*)(st + L::kHdr + L::kVal + L::kCol);
    const int* sp = (const int*)(st + L::kHdr + L::kVal + L::kCol + L::kRp);  // sorted layout only
    const int r0 = d.x, r1 = d.y, p0 = d.z;
    const int q0 = r0 & ~3;
    const int a0 = p0 & ~(L::kValAlign - 1);
    const int c0 = p0 & ~3;
    const int sub = lane % G;
    if constexpr (RL > 1 && G == 1) {
      // several short rows per lane: gather for all of them before any FMA
      rows_accumulate<MT, VI, VO, CH, RL, PERM>(sv, sc, sr, sp, r0, r1, q0, a0, c0, p0, lane, c, in, out, dinv, x,
                                                epi, keep);
    } else {
#pragma unroll 1
    for (int pass = 0; pass < RL; ++pass) {
      const int r = r0 + pass * (32 / G) + lane / G;  // stored row
      const bool act = r < r1;
      const int b = act ? sr[r - q0] : p0;
      const int len = act ? sr[r + 1 - q0] - b : 0;
      const int o = (PERM && act) ? sp[r - q0] : r;  // the row's place in the vectors
      // c enters once per row, through the lane that writes the result
      MT acc = (act && c && sub == 0) ? (MT)ld_keep(c + o, keep) : MT(0);
      if (epi == EPI_SPMV)
        acc = row_accumulate<MT, VI, false, G, CH>(sv + (b - a0), sc + (b - c0), len, sub, in, acc, keep);
      else
        acc = row_accumulate<MT, VI, true, G, CH>(sv + (b - a0), sc + (b - c0), len, sub, in, acc, keep);
      if (act && sub == 0) {
        if (epi == EPI_SPMV)
          st_keep(out + o, (VO)acc, keep);
        else
          epilogue<MT, VI, VO>(epi, o, acc, in, out, dinv, x, keep);
      }
    }
    }
    __syncwarp();
    if (lane == 0 && tn < ntiles)
      issue_tile<MT, RL, PERM>(dn, ring + s * L::kBytes, &full[warp][s], rp, ci, va, perm, stream);
  }
}

// R = 2 or 4 interleaved right-hand sides (row-major vectors, leading
// dimension ldx >= R), one lane per row, natural row order, RL rows per
// lane taken one after another: the factor tile is staged once and each of
// its entries feeds R FMAs, so the factor is read once for all R columns.
// The pipeline (per-warp two-stage ring of bulk copies, bounded waits,
// programmatic launch, alternating direction) is k_sweep_staged's.
template <class MT, class VI, class VO, int CH, int RL, int R>
__global__ void __launch_bounds__(warps_of<MT>() * 32, 1)
    k_sweep_multi(int ntiles, const int4* __restrict__ tiles, const int* __restrict__ rp, const int* __restrict__ ci,
                  const MT* __restrict__ va, const VI* __restrict__ c, const VI* __restrict__ in, VO* __restrict__ out,
                  int ldx, const double* __restrict__ dinv, double* __restrict__ x, int epi, int flags,
                  int* __restrict__ err) {
  using L = StageLayout<MT, RL, false>;
  constexpr int kWarps = warps_of<MT>();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kWarps][kWarpStages];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int w = 0; w < kWarps; ++w)
      for (int s = 0; s < kWarpStages; ++s) mbar_init(&full[w][s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int gw = blockIdx.x * kWarps + warp;
  const int nw = gridDim.x * kWarps;
  unsigned char* ring = smem + (size_t)warp * kWarpStages * L::kBytes;
  const bool rev = (flags & kFlagReverse) != 0;
  const uint64_t stream = (flags & kFlagFactorNormal) ? policy_evict_normal() : policy_evict_first();
  const uint64_t keep = (flags & kFlagVectorNormal) ? policy_evict_normal() : policy_evict_last();
  grid_launch_dependents();
  if (lane == 0)
    for (int s = 0; s < kWarpStages; ++s) {
      const int t = gw + s * nw;
      if (t < ntiles)
        issue_tile<MT, RL, false>(__ldg(tiles + (rev ? ntiles - 1 - t : t)), ring + s * L::kBytes, &full[warp][s], rp,
                                  ci, va, nullptr, stream);
    }
  grid_wait_prior();
  int k = 0;
  for (int t = gw; t < ntiles; t += nw, ++k) {
    const int tn = t + kWarpStages * nw;
    int4 dn = make_int4(0, 0, 0, 0);
    if (lane == 0 && tn < ntiles) dn = __ldg(tiles + (rev ? ntiles - 1 - tn : tn));
    const int s = k % kWarpStages;
    const bool ok = mbar_wait_bounded(&full[warp][s], (uint32_t)(k / kWarpStages) & 1u);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) {
        atomicOr(err, 1);
        for (int d = 1; d < kWarpStages; ++d) {
          const int kd = k + d;
          if (t + d * nw < ntiles) mbar_wait_bounded(&full[warp][kd % kWarpStages], (uint32_t)(kd / kWarpStages) & 1u);
        }
      }
      return;
    }
    const unsigned char* st = ring + s * L::kBytes;
    const int4 d = *(const int4*)st;
    const MT* sv = (const MT*)(st + L::kHdr);
    const int* sc = (const int*)(st + L::kHdr + L::kVal);
    const int* sr = (const int*)(st + L::kHdr + L::kVal + L::kCol);
    const int r0 = d.x, r1 = d.y, p0 = d.z;
    const int q0 = r0 & ~3;
    const int a0 = p0 & ~(L::kValAlign - 1);
    const int c0 = p0 & ~3;
#pragma unroll 1
    for (int pass = 0; pass < RL; ++pass) {
      const int r = r0 + pass * 32 + lane;
      const bool act = r < r1;
      const int b = act ? sr[r - q0] : p0;
      const int len = act ? sr[r + 1 - q0] - b : 0;
      const size_t o = (size_t)r * (size_t)ldx;
      MT acc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] = (act && c) ? (MT)ld_keep(c + o + j, keep) : MT(0);
      if (epi == EPI_SPMV)
        row_accumulate_cols<MT, VI, false, R, CH>(sv + (b - a0), sc + (b - c0), len, in, ldx, acc, keep);
      else
        row_accumulate_cols<MT, VI, true, R, CH>(sv + (b - a0), sc + (b - c0), len, in, ldx, acc, keep);
      if (act)
#pragma unroll
        for (int j = 0; j < R; ++j) epilogue_col<MT, VI, VO>(epi, r, o + j, acc[j], in, out, dinv, x, keep);
    }
    __syncwarp();
    if (lane == 0 && tn < ntiles)
      issue_tile<MT, RL, false>(dn, ring + s * L::kBytes, &full[warp][s], rp, ci, va, nullptr, stream);
  }
}

template <class MT, class VI, class VO, int CH, int RL, int R>
cudaError_t multi_attr() {
  using L = StageLayout<MT, RL, false>;
  const size_t smem = (size_t)warps_of<MT>() * kWarpStages * L::kBytes;
  return cudaFuncSetAttribute(k_sweep_multi<MT, VI, VO, CH, RL, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// Entries gathered before the FMAs with R columns (about the registers of
// sixteen entries of one column).
template <int R>
constexpr int multi_chunk() {
  return R == 2 ? 8 : 4;
}

template <class MT, class VI, class VO, int RL, int R>
cudaError_t multi_g(const DevCsr& T, const LaunchEnv& env, int ldx, const void* c, const void* in, void* out,
                    const double* dinv, double* x, int epi, cudaStream_t s) {
  using L = StageLayout<MT, RL, false>;
  constexpr int kWarps = warps_of<MT>();
  constexpr int CH = multi_chunk<R>();
  const int nt = T.ntiles;
  if (nt == 0) return cudaSuccess;
  const int want = (nt + kWarps - 1) / kWarps;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(want < env.sms ? want : env.sms));
  cfg.blockDim = dim3(kWarps * 32);
  cfg.dynamicSmemBytes = (size_t)kWarps * kWarpStages * L::kBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = env.overlap ? 1 : 0;
  int flags = env.l2 & (kFlagFactorNormal | kFlagVectorNormal);
  if ((env.l2 & kFlagReverse) && (env.flips++ & 1u)) flags |= kFlagReverse;
  return cudaLaunchKernelEx(&cfg, k_sweep_multi<MT, VI, VO, CH, RL, R>, nt, (const int4*)T.tiles, (const int*)T.rp,
                            (const int*)T.ci, (const MT*)T.va, (const VI*)c, (const VI*)in, (VO*)out, ldx, dinv, x,
                            epi, flags, env.err);
}

template <class MT, class VI, class VO, int R>
cudaError_t multi_rl(const DevCsr& T, const LaunchEnv& env, int ldx, const void* c, const void* in, void* out,
                     const double* dinv, double* x, int epi, cudaStream_t s) {
  if (T.tile_passes == 4) return multi_g<MT, VI, VO, 4, R>(T, env, ldx, c, in, out, dinv, x, epi, s);
  if (T.tile_passes == 2) return multi_g<MT, VI, VO, 2, R>(T, env, ldx, c, in, out, dinv, x, epi, s);
  return multi_g<MT, VI, VO, 1, R>(T, env, ldx, c, in, out, dinv, x, epi, s);
}

template <class MT, class VI, class VO>
cudaError_t multi(const DevCsr& T, const LaunchEnv& env, int R, int ldx, const void* c, const void* in, void* out,
                  const double* dinv, double* x, int epi, cudaStream_t s) {
  if (R == 2) return multi_rl<MT, VI, VO, 2>(T, env, ldx, c, in, out, dinv, x, epi, s);
  if (R == 4) return multi_rl<MT, VI, VO, 4>(T, env, ldx, c, in, out, dinv, x, epi, s);
  return cudaErrorInvalidValue;
}

template <class MT, class VI, class VO>
cudaError_t prepare_multi() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = multi_attr<MT, VI, VO, multi_chunk<2>(), 1, 2>();
  if (e == cudaSuccess) e = multi_attr<MT, VI, VO, multi_chunk<2>(), 2, 2>();
  if (e == cudaSuccess) e = multi_attr<MT, VI, VO, multi_chunk<2>(), 4, 2>();
  if (e == cudaSuccess) e = multi_attr<MT, VI, VO, multi_chunk<4>(), 1, 4>();
  if (e == cudaSuccess) e = multi_attr<MT, VI, VO, multi_chunk<4>(), 2, 4>();
  if (e == cudaSuccess) e = multi_attr<MT, VI, VO, multi_chunk<4>(), 4, 4>();
  return e;
}

__device__ __forceinline__ int4 shfl_int4(int4 v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  v.z = __shfl_sync(0xffffffffu, v.z, src);
  v.w = __shfl_sync(0xffffffffu, v.w, src);
  return v;
}

// The one-row-per-lane shape in natural row order (most factors): the same
// sweep as k_sweep_staged, with the tile descriptors held by every lane in
// registers and each lane's row bounds loaded from global memory one tile
// ahead, so that a tile's critical path is the column-index read from
// shared memory, the gather and the FMA chain, not a chain of dependent
// shared-memory reads (descriptor, row pointers, columns).  The stage holds
// only the values and column indices of the tile.  Each row still
// accumulates c - sum t_ij in_j in column order, so the results are the
// bits of k_sweep_staged.
template <class MT, class VI, class VO, int CH, int W = warps_of<MT>(), int NNZ = kTileNnz>
__global__ void __launch_bounds__(W * 32, 1)
    k_sweep_rows(int ntiles, const int4* __restrict__ tiles, const int* __restrict__ rp, const int* __restrict__ ci,
                 const MT* __restrict__ va, const VI* __restrict__ c, const VI* __restrict__ in, VO* __restrict__ out,
                 const double* __restrict__ dinv, double* __restrict__ x, int epi, int flags, int* __restrict__ err) {
  using L = StageLayout<MT, 1, false, NNZ>;
  constexpr int kWarps = W;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kWarps][kWarpStages];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int w = 0; w < kWarps; ++w)
      for (int s = 0; s < kWarpStages; ++s) mbar_init(&full[w][s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int gw = blockIdx.x * kWarps + warp;
  const int nw = gridDim.x * kWarps;
  unsigned char* ring = smem + (size_t)warp * kWarpStages * L::kBytes;
  const bool rev = (flags & kFlagReverse) != 0;
  const uint64_t stream = (flags & kFlagFactorNormal) ? policy_evict_normal() : policy_evict_first();
  const uint64_t keep = (flags & kFlagVectorNormal) ? policy_evict_normal() : policy_evict_last();
  grid_launch_dependents();
  // descriptors of this warp's first two tiles, in every lane
  int4 dcur = make_int4(0, 0, 0, 0), dnext = make_int4(0, 0, 0, 0);
  if (lane == 0) {
    if (gw < ntiles) dcur = __ldg(tiles + (rev ? ntiles - 1 - gw : gw));
    if (gw + nw < ntiles) dnext = __ldg(tiles + (rev ? ntiles - 1 - (gw + nw) : gw + nw));
    // the factor and its tiles are never written by a sweep: the first copies
    // may start before the kernel that produced c and in has finished
    if (gw < ntiles) issue_tile<MT, 1, false, false, NNZ>(dcur, ring, &full[warp][0], rp, ci, va, nullptr, stream);
    if (gw + nw < ntiles)
      issue_tile<MT, 1, false, false, NNZ>(dnext, ring + L::kBytes, &full[warp][1], rp, ci, va, nullptr, stream);
  }
  dcur = shfl_int4(dcur, 0);
  dnext = shfl_int4(dnext, 0);
  int rb = 0, re = 0;  // bounds of this lane's row of the current tile
  if (dcur.x + lane < dcur.y) {
    rb = __ldg(rp + dcur.x + lane);
    re = __ldg(rp + dcur.x + lane + 1);
  }
  grid_wait_prior();  // c, in, out and x below belong to the previous kernel until it completes
  int k = 0;
  for (int t = gw; t < ntiles; t += nw, ++k) {
    const int tn = t + kWarpStages * nw;
    int4 dn = make_int4(0, 0, 0, 0);
    if (lane == 0 && tn < ntiles) dn = __ldg(tiles + (rev ? ntiles - 1 - tn : tn));
    // bounds of this lane's row of the next tile, a whole tile ahead
    int nb = 0, ne = 0;
    if (t + nw < ntiles && dnext.x + lane < dnext.y) {
      nb = __ldg(rp + dnext.x + lane);
      ne = __ldg(rp + dnext.x + lane + 1);
    }
    // the row's constant term and the epilogue's operands: their addresses
    // are known before the stage lands, so their loads are issued before the
    // wait (left to the compiler, where they went depended on unrelated code
    // in the same file, and the lower sweep of the 128^3 cut-cell ILUT factor
    // took 45 or 49 us depending on it)
    const int r = dcur.x + lane;
    const bool act = r < dcur.y;
    MT acc = (act && c) ? (MT)ld_keep(c + r, keep) : MT(0);
    if (act) prefetch_epilogue(epi, r, dinv, x);
    const int s = k % kWarpStages;
    const bool ok = mbar_wait_bounded(&full[warp][s], (uint32_t)(k / kWarpStages) & 1u);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) {
        atomicOr(err, 1);
        for (int d = 1; d < kWarpStages; ++d) {
          const int kd = k + d;
          if (t + d * nw < ntiles) mbar_wait_bounded(&full[warp][kd % kWarpStages], (uint32_t)(kd / kWarpStages) & 1u);
        }
      }
      return;
    }
    const unsigned char* st = ring + s * L::kBytes;
    const MT* sv = (const MT*)(st + L::kHdr);
    const int* sc = (const int*)(st + L::kHdr + L::kVal);
    const int a0 = dcur.z & ~(L::kValAlign - 1);
    const int c0 = dcur.z & ~3;
    const int len = act ? re - rb : 0;
    const int off = act ? rb : dcur.z;  // inactive lanes read nothing
    if (epi == EPI_SPMV)
      acc = row_accumulate<MT, VI, false, 1, CH>(sv + (off - a0), sc + (off - c0), len, 0, in, acc, keep);
    else
      acc = row_accumulate<MT, VI, true, 1, CH>(sv + (off - a0), sc + (off - c0), len, 0, in, acc, keep);
    if (act) {
      if (epi == EPI_SPMV)
        st_keep(out + r, (VO)acc, keep);
      else
        epilogue<MT, VI, VO>(epi, r, acc, in, out, dinv, x, keep);
    }
    __syncwarp();
    if (lane == 0 && tn < ntiles)
      issue_tile<MT, 1, false, false, NNZ>(dn, ring + s * L::kBytes, &full[warp][s], rp, ci, va, nullptr, stream);
    dcur = dnext;
    dnext = shfl_int4(dn, 0);
    rb = nb;
    re = ne;
  }
}

template <class MT, class VI, class VO, int CH, int W = warps_of<MT>(), int NNZ = kTileNnz>
cudaError_t rows_attr() {
  using L = StageLayout<MT, 1, false, NNZ>;
  const size_t smem = (size_t)W * kWarpStages * L::kBytes;
  return cudaFuncSetAttribute(k_sweep_rows<MT, VI, VO, CH, W, NNZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// The narrow configuration of the one-row-per-lane sweep for FP64 factors
// whose rows fit one gather round of kNarrowChunk entries: tiles of at most
// kTileNnzNarrow - 8 entries, so that the stages are smaller and
// kNarrowWarps warps (more rows in processing per SM) fit beside them, with
// kNarrowChunk gathers in flight per lane (the registers of 24 warps).
constexpr int kNarrowWarps = 24;
constexpr int kNarrowChunk = kNarrowChunkRows;

template <class MT, class VI, class VO>
cudaError_t narrow_launch(const DevCsr& T, const LaunchEnv& env, const void* c, const void* in, void* out,
                          const double* dinv, double* x, int epi, cudaStream_t s) {
  using L = StageLayout<MT, 1, false, kTileNnzNarrow>;
  const int nt = T.ntiles;
  if (nt == 0) return cudaSuccess;
  const int want = (nt + kNarrowWarps - 1) / kNarrowWarps;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(want < env.sms ? want : env.sms));
  cfg.blockDim = dim3(kNarrowWarps * 32);
  cfg.dynamicSmemBytes = (size_t)kNarrowWarps * kWarpStages * L::kBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = env.overlap ? 1 : 0;
  int flags = env.l2 & (kFlagFactorNormal | kFlagVectorNormal);
  if ((env.l2 & kFlagReverse) && (env.flips++ & 1u)) flags |= kFlagReverse;
  return cudaLaunchKernelEx(&cfg, k_sweep_rows<MT, VI, VO, kNarrowChunk, kNarrowWarps, kTileNnzNarrow>, nt,
                            (const int4*)T.tiles, (const int*)T.rp, (const int*)T.ci, (const MT*)T.va, (const VI*)c,
                            (const VI*)in, (VO*)out, dinv, x, epi, flags, env.err);
}

template <class MT, class VI, class VO, int G, int CH, int RL, bool PERM>
cudaError_t staged_attr() {
  using L = StageLayout<MT, RL, PERM>;
  const size_t smem = (size_t)warps_of<MT>() * kWarpStages * L::kBytes;
  return cudaFuncSetAttribute(k_sweep_staged<MT, VI, VO, G, CH, RL, PERM>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class MT, class VI, class VO, int G, int CH, int RL, bool PERM>
cudaError_t staged_g(const DevCsr& T, const LaunchEnv& env, const void* c, const void* in, void* out,
                     const double* dinv, double* x, int epi, cudaStream_t s) {
  using L = StageLayout<MT, RL, PERM>;
  constexpr int kWarps = warps_of<MT>();
  const size_t smem = (size_t)kWarps * kWarpStages * L::kBytes;
  const int nt = PERM ? T.nstiles : T.ntiles;
  if (nt == 0) return cudaSuccess;
  const int want = (nt + kWarps - 1) / kWarps;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(want < env.sms ? want : env.sms));
  cfg.blockDim = dim3(kWarps * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = env.overlap ? 1 : 0;
  // consecutive launches alternate their direction, so each starts on the
  // rows (vector entries, and factor tiles when the matrix is the same) that
  // the previous one touched last, while they are still in L2
  int flags = env.l2 & (kFlagFactorNormal | kFlagVectorNormal);
  if ((env.l2 & kFlagReverse) && (env.flips++ & 1u)) flags |= kFlagReverse;
  if constexpr (G == 1 && RL == 1 && !PERM) {
    return cudaLaunchKernelEx(&cfg, k_sweep_rows<MT, VI, VO, CH>, nt, (const int4*)T.tiles, (const int*)T.rp,
                              (const int*)T.ci, (const MT*)T.va, (const VI*)c, (const VI*)in, (VO*)out, dinv, x, epi,
                              flags, env.err);
  }
  if (PERM)
    return cudaLaunchKernelEx(&cfg, k_sweep_staged<MT, VI, VO, G, CH, RL, PERM>, nt, (const int4*)T.stiles,
                              (const int*)T.srp, (const int*)T.sci, (const MT*)T.sva, (const int*)T.perm,
                              (const VI*)c, (const VI*)in, (VO*)out, dinv, x, epi, flags, env.err);
  return cudaLaunchKernelEx(&cfg, k_sweep_staged<MT, VI, VO, G, CH, RL, PERM>, nt, (const int4*)T.tiles,
                            (const int*)T.rp, (const int*)T.ci, (const MT*)T.va, (const int*)nullptr, (const VI*)c,
                            (const VI*)in, (VO*)out, dinv, x, epi, flags, env.err);
}

template <class MT, class VI, class VO, int G, int RL, bool PERM>
cudaError_t staged_c(const DevCsr& T, const LaunchEnv& env, const void* c, const void* in, void* out,
                     const double* dinv, double* x, int epi, cudaStream_t s) {
  if (T.chunk == 8) return staged_g<MT, VI, VO, G, 8, RL, PERM>(T, env, c, in, out, dinv, x, epi, s);
  return staged_g<MT, VI, VO, G, 16, RL, PERM>(T, env, c, in, out, dinv, x, epi, s);
}

template <class MT, class VI, class VO>
cudaError_t staged(const DevCsr& T, const LaunchEnv& env, const void* c, const void* in, void* out,
                   const double* dinv, double* x, int epi, cudaStream_t s) {
  if (T.use_sorted && T.nstiles > 0) return staged_c<MT, VI, VO, 1, 1, true>(T, env, c, in, out, dinv, x, epi, s);
  if (T.tile_nnz == kTileNnzNarrow) {
    // tiles cut for the narrow configuration (one lane per row, FP64 values)
    if constexpr (sizeof(MT) == 8) {
      if (T.tile_lanes == 1 && T.tile_passes == 1) return narrow_launch<MT, VI, VO>(T, env, c, in, out, dinv, x, epi, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (T.tile_lanes) {
    case 1:
      if (T.tile_passes == 4) return staged_c<MT, VI, VO, 1, 4, false>(T, env, c, in, out, dinv, x, epi, s);
      if (T.tile_passes == 2) return staged_c<MT, VI, VO, 1, 2, false>(T, env, c, in, out, dinv, x, epi, s);
      return staged_c<MT, VI, VO, 1, 1, false>(T, env, c, in, out, dinv, x, epi, s);
    case 2: return staged_c<MT, VI, VO, 2, 1, false>(T, env, c, in, out, dinv, x, epi, s);
    case 4: return staged_c<MT, VI, VO, 4, 1, false>(T, env, c, in, out, dinv, x, epi, s);
  }
  return cudaErrorInvalidValue;
}

template <class MT, class VI, class VO, int G, int RL, bool PERM>
cudaError_t prepare_shape() {
  cudaError_t e = staged_attr<MT, VI, VO, G, 8, RL, PERM>();
  if (e == cudaSuccess) e = staged_attr<MT, VI, VO, G, 16, RL, PERM>();
  if (G == 1 && RL == 1 && !PERM) {
    if (e == cudaSuccess) e = rows_attr<MT, VI, VO, 8>();
    if (e == cudaSuccess) e = rows_attr<MT, VI, VO, 16>();
  }
  return e;
}

template <class MT, class VI, class VO>
cudaError_t prepare_mode() {
  cudaError_t e = prepare_shape<MT, VI, VO, 1, 1, false>();
  if (e == cudaSuccess) e = prepare_shape<MT, VI, VO, 1, 2, false>();
  if (e == cudaSuccess) e = prepare_shape<MT, VI, VO, 1, 4, false>();
  if (e == cudaSuccess) e = prepare_shape<MT, VI, VO, 2, 1, false>();
  if (e == cudaSuccess) e = prepare_shape<MT, VI, VO, 4, 1, false>();
  if (e == cudaSuccess) e = prepare_shape<MT, VI, VO, 1, 1, true>();
  if constexpr (sizeof(MT) == 8) {
    if (e == cudaSuccess) e = rows_attr<MT, VI, VO, kNarrowChunk, kNarrowWarps, kTileNnzNarrow>();
  }
  return e;
}

// Waits up to timeout_ns for *flag to become non-zero; nothing sets it, so
// the wait runs out and the error word records it (bit 1).
__global__ void k_wait_flag(const int* flag, unsigned long long timeout_ns, int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long t0 = global_ns();
  while (atomicAdd((int*)flag, 0) == 0)
    if (global_ns() - t0 > timeout_ns) {
      atomicOr(err, 2);
      return;
    }
}

}  // namespace

cudaError_t launch_wait_flag(const int* flag, unsigned long long timeout_ns, int* err, cudaStream_t s) {
  k_wait_flag<<<1, 32, 0, s>>>(flag, timeout_ns, err);
  return cudaGetLastError();
}

cudaError_t staged_prepare() {
  cudaError_t e = prepare_mode<double, double, double>();
  if (e == cudaSuccess) e = prepare_mode<float, float, float>();
  if (e == cudaSuccess) e = prepare_mode<double, double, float>();
  if (e == cudaSuccess) e = prepare_multi<double, double, double>();
  if (e == cudaSuccess) e = prepare_multi<float, float, float>();
  if (e == cudaSuccess) e = prepare_multi<double, double, float>();
  return e;
}

bool staged_multi_ok(const DevCsr& T, int R) {
  return (R == 2 || R == 4) && T.ntiles > 0 && T.tile_lanes == 1;
}

cudaError_t launch_sweep_staged_multi(const DevCsr& T, Mode mode, const LaunchEnv& env, int R, int ldx, const void* c,
                                      const void* in, void* out, const double* dinv, double* x, int epi,
                                      cudaStream_t s) {
  if (!staged_multi_ok(T, R) || ldx < R) return cudaErrorInvalidValue;
  switch (mode) {
    case MODE_D: return multi<double, double, double>(T, env, R, ldx, c, in, out, dinv, x, epi, s);
    case MODE_F: return multi<float, float, float>(T, env, R, ldx, c, in, out, dinv, x, epi, s);
    case MODE_DF: return multi<double, double, float>(T, env, R, ldx, c, in, out, dinv, x, epi, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_staged(const DevCsr& T, Mode mode, const LaunchEnv& env, const void* c, const void* in,
                                void* out, const double* dinv, double* x, int epi, cudaStream_t s) {
  switch (mode) {
    case MODE_D: return staged<double, double, double>(T, env, c, in, out, dinv, x, epi, s);
    case MODE_F: return staged<float, float, float>(T, env, c, in, out, dinv, x, epi, s);
    case MODE_DF: return staged<double, double, float>(T, env, c, in, out, dinv, x, epi, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace silu
