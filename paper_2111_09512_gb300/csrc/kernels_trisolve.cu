// Exact triangular solves of the comparison path in one persistent launch
// (sm_103a): y = L^{-1} r, c = D^{-1} y, v = Utilde^{-1} c, x (+)= (D_c) v.
//
// The level-set schedule of Sec. 4 orders the rows: a row of level l reads
// only rows of levels below l.  Launching one kernel per level makes every
// level pay a launch and a device-wide ordering point, a few microseconds
// each; the 27-point 256^3 factors have 1786 levels per triangle.  Here one
// grid processes every level.  Rows are stored in level order (host copies
// of L_s and Utilde_s, rows permuted, columns unchanged) and cut into items
// of at most 32 rows of one level; the L items come first, then the U items.
// A warp takes the next item from a device ticket counter, so items are
// claimed in level order by warps that are running, and a row waits only for
// the rows it reads (no level waits for the whole previous level).  Because
// every row an item waits for belongs to an earlier ticket, already held by
// a running warp, the waits always end; each is also bounded in time, after
// which the kernel records a device error and finishes with what it has.
//
// Readiness travels with the value: every published entry of y and v has its
// lowest significand bit set to the solve's tag (0 or 1, alternating from
// solve to solve), so one 8-byte store makes the value visible and ready at
// once, and a reader polls the entry itself.  Readers (and the update of x)
// use the entry with that bit cleared, so the results are the same bits
// whatever the tag.  The cost is one bit of the 53-bit FP64 significand of
// the intermediates (a relative change of at most 2^-52 per entry).  Every solve writes every entry of its tagged
// arrays, so at the start of a solve all of them carry the previous tag.
// The last warp to finish resets the ticket and flips the tag for the next
// solve, so the launch needs no preparation and can be captured in a graph.
// With several right-hand sides a lane publishes its row from inside its
// polling loop, as soon as its own entries are in (with one column that
// measured slower on short rows, so one column waits, sums and publishes
// after the loop).
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace silu {
namespace {

constexpr int kTriThreads = 256;
constexpr unsigned long long kTriWaitNs = 2000000000ull;  // 2 s bound on any wait

__device__ __forceinline__ unsigned long long tri_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ long long ld_poll(const double* p) {
  long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_poll_i(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_publish(double* p, long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Published form of v (lowest significand bit replaced by the tag) and the
// value every reader uses (that bit cleared), so results do not depend on
// the tag, i.e. on how many solves came before.
__device__ __forceinline__ long long tag_of(double v, long long tag) {
  return (__double_as_longlong(v) & ~1ll) | tag;
}
__device__ __forceinline__ double untag(long long b) { return __longlong_as_double(b & ~1ll); }

// Resident blocks per SM at most.
constexpr int kTriMaxBlocksPerSm = 8;
// Pauses (ns) between reads of entries not yet published: none for the
// entries a row reads (they are re-read at once), longer for an item's gate
// (below).
constexpr unsigned kTriPause = 0;
constexpr unsigned kTriGatePause = 128;

// Wait until *p carries the tag: reads after fixed pauses, bounded by
// kTriWaitNs, and cut short when another wait has already given up (error
// word non-zero).
__device__ __forceinline__ void wait_gate(const double* p, long long tag, int* err) {
  long long b = ld_poll(p);
  if ((b & 1ll) == tag) return;
  const unsigned long long t0 = tri_ns();
  for (unsigned spins = 1;; ++spins) {
    __nanosleep(kTriGatePause);
    b = ld_poll(p);
    if ((b & 1ll) == tag) return;
    if ((spins & 15u) == 0) {
      if (ld_poll_i(err) != 0) return;
      if (tri_ns() - t0 > kTriWaitNs) {
        atomicOr(err, 4);
        return;
      }
    }
  }
}

// Entries a run of at most CH consecutive entries of a row reads, R columns
// each: b[q][k] holds vec[j[q] R + k] once its tag bit equals `tag`.  All
// loads are issued before any is waited for; the ones not yet published are
// all read again after each pause until they are (bounded as in wait_gate).
template <int R, int CH>
__device__ __forceinline__ void gather_ready(const double* vec, const int (&j)[CH], int cnt, long long tag,
                                             long long (&b)[CH][R], int* err) {
#pragma unroll
  for (int q = 0; q < CH; ++q)
    if (q < cnt)
#pragma unroll
      for (int k = 0; k < R; ++k) b[q][k] = ld_poll(vec + (size_t)j[q] * R + k);
  bool ready = true;
#pragma unroll
  for (int q = 0; q < CH; ++q)
    if (q < cnt)
#pragma unroll
      for (int k = 0; k < R; ++k) ready = ready && ((b[q][k] & 1ll) == tag);
  if (ready) return;
  const unsigned long long t0 = tri_ns();
  for (unsigned spins = 1;; ++spins) {
    __nanosleep(kTriPause);
    ready = true;
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (q < cnt)
#pragma unroll
        for (int k = 0; k < R; ++k)
          if ((b[q][k] & 1ll) != tag) {
            b[q][k] = ld_poll(vec + (size_t)j[q] * R + k);
            ready = ready && ((b[q][k] & 1ll) == tag);
          }
    if (ready) return;
    if ((spins & 63u) == 0) {
      if (ld_poll_i(err) != 0) return;
      if (tri_ns() - t0 > kTriWaitNs) {
        atomicOr(err, 4);
        return;
      }
    }
  }
}

// Entries whose loads are issued together: more in flight for one column.
template <int R>
__host__ __device__ constexpr int tri_chunk() {
  return R == 1 ? 8 : 4;
}

// The row's entries [p0, p1) read from vec (R columns each), CH at a time:
// acc[k] -= T_oj vec_jk in column order, waiting for each entry's tag; the
// FMAs of a run and, after the last run, publish(acc) happen inside the
// polling loop, so a lane publishes its row as soon as its own entries are
// in, whatever the other lanes of its warp still wait for.
template <int R, int CH, class Publish>
__device__ __forceinline__ void solve_row(const double* vec, const int* __restrict__ ci, const double* __restrict__ va,
                                          int p0, int p1, long long tag, double (&acc)[R], int* err,
                                          Publish publish) {
  if (p0 >= p1) {
    publish(acc);
    return;
  }
  int p = p0;
  int cnt = p1 - p < CH ? p1 - p : CH;
  int j[CH];
  double w[CH];
  long long b[CH][R];
#pragma unroll
  for (int q = 0; q < CH; ++q)
    if (q < cnt) {
      j[q] = __ldg(ci + p + q);
      w[q] = __ldg(va + p + q);
    }
#pragma unroll
  for (int q = 0; q < CH; ++q)
    if (q < cnt)
#pragma unroll
      for (int k = 0; k < R; ++k) b[q][k] = ld_poll(vec + (size_t)j[q] * R + k);
  unsigned long long t0 = 0;
  bool gave_up = false;
  for (unsigned spins = 0;; ++spins) {
    bool ready = true;
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (q < cnt)
#pragma unroll
        for (int k = 0; k < R; ++k) ready = ready && ((b[q][k] & 1ll) == tag);
    if (ready || gave_up) {
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (q < cnt)
#pragma unroll
          for (int k = 0; k < R; ++k) acc[k] = fma(-w[q], untag(b[q][k]), acc[k]);
      p += CH;
      if (p >= p1) {
        publish(acc);
        return;
      }
      cnt = p1 - p < CH ? p1 - p : CH;
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (q < cnt) {
          j[q] = __ldg(ci + p + q);
          w[q] = __ldg(va + p + q);
        }
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (q < cnt)
#pragma unroll
          for (int k = 0; k < R; ++k) b[q][k] = ld_poll(vec + (size_t)j[q] * R + k);
      continue;
    }
    if (t0 == 0) t0 = tri_ns();
    __nanosleep(kTriPause);
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (q < cnt)
#pragma unroll
        for (int k = 0; k < R; ++k)
          if ((b[q][k] & 1ll) != tag) b[q][k] = ld_poll(vec + (size_t)j[q] * R + k);
    if ((spins & 63u) == 63u) {
      if (ld_poll_i(err) != 0) gave_up = true;
      else if (tri_ns() - t0 > kTriWaitNs) {
        atomicOr(err, 4);
        gave_up = true;
      }
    }
  }
}

struct TriArgs {
  int nitemsL, nitems;
  const int4* items;  // {first, last + 1, gate row or -1, gate in v (1) or y (0)}
  const int* rowsL;   // row of each level-ordered L row
  const int* lrp;
  const int* lci;
  const double* lva;
  const int* rowsU;
  const int* urp;
  const int* uci;
  const double* uva;
  const double* r;  // right-hand side of the lower solve, row-major, leading dimension ldr
  int ldr;
  const double* dinv;  // D^{-1} (D_r under row/column scaling)
  const double* dcol;  // D_c or null
  double* y;           // tagged L^{-1} r, n x R
  double* v;           // tagged Utilde^{-1} c, n x R
  double* x;
  int ldx;
  int x_zero;
  unsigned* state;  // [0] ticket, [1] finished warps, [2] solves done (its parity gives the tag)
  unsigned total_warps;
  int* err;
};

// y_o = r_o - sum_j L_oj y_j over the row's entries in column order.
template <int R>
__device__ __forceinline__ void lower_row(const TriArgs& a, int idx, long long tag) {
  constexpr int CH = tri_chunk<R>();
  const int o = __ldg(a.rowsL + idx);
  double acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = a.r[(size_t)o * a.ldr + k];
  const int p0 = __ldg(a.lrp + idx), p1 = __ldg(a.lrp + idx + 1);
  if constexpr (R > 1) {
    // several columns: publish from inside the polling loop (see solve_row)
    solve_row<R, CH>(a.y, a.lci, a.lva, p0, p1, tag, acc, a.err, [&](double (&v)[R]) {
#pragma unroll
      for (int k = 0; k < R; ++k) st_publish(a.y + (size_t)o * R + k, tag_of(v[k], tag));
    });
    return;
  }
  for (int p = p0; p < p1; p += CH) {
    const int cnt = p1 - p < CH ? p1 - p : CH;
    int j[CH];
    double w[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (q < cnt) {
        j[q] = __ldg(a.lci + p + q);
        w[q] = __ldg(a.lva + p + q);
      }
    long long yb[CH][R];
    gather_ready<R, CH>(a.y, j, cnt, tag, yb, a.err);
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (q < cnt)
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = fma(-w[q], untag(yb[q][k]), acc[k]);
  }
#pragma unroll
  for (int k = 0; k < R; ++k) st_publish(a.y + (size_t)o * R + k, tag_of(acc[k], tag));
}

// v_o = dinv_o y_o - sum_j Utilde_oj v_j; x_o (+)= (D_c)_o v_o.
template <int R>
__device__ __forceinline__ void upper_row(const TriArgs& a, int idx, long long tag) {
  constexpr int CH = tri_chunk<R>();
  const int o = __ldg(a.rowsU + idx);
  const double d = __ldg(a.dinv + o);
  double acc[R];
  {
    const int jo[1] = {o};
    long long yo[1][R];
    gather_ready<R, 1>(a.y, jo, 1, tag, yo, a.err);
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = d * untag(yo[0][k]);
  }
  const int p0 = __ldg(a.urp + idx), p1 = __ldg(a.urp + idx + 1);
  const double dc = a.dcol ? __ldg(a.dcol + o) : 1.0;
  auto publish = [&](double (&v)[R]) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const long long pub = tag_of(v[k], tag);
      st_publish(a.v + (size_t)o * R + k, pub);
      const double vo = untag(pub);
      double* xo = a.x + (size_t)o * a.ldx + k;
      const double add = a.dcol ? dc * vo : vo;
      *xo = a.x_zero ? add : *xo + add;
    }
  };
  if constexpr (R > 1) {
    solve_row<R, CH>(a.v, a.uci, a.uva, p0, p1, tag, acc, a.err, publish);
    return;
  }
  for (int p = p0; p < p1; p += CH) {
    const int cnt = p1 - p < CH ? p1 - p : CH;
    int j[CH];
    double w[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (q < cnt) {
        j[q] = __ldg(a.uci + p + q);
        w[q] = __ldg(a.uva + p + q);
      }
    long long vb[CH][R];
    gather_ready<R, CH>(a.v, j, cnt, tag, vb, a.err);
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (q < cnt)
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = fma(-w[q], untag(vb[q][k]), acc[k]);
  }
  publish(acc);
}

// Resident blocks per SM the register budget is set for: many warps keep
// many items in flight while earlier levels finish.
template <int R>
__host__ __device__ constexpr int tri_min_blocks() {
  return R == 1 ? 2 : (R == 2 ? 3 : 2);
}

template <int R>
__global__ void __launch_bounds__(kTriThreads, tri_min_blocks<R>()) k_trisolve(TriArgs a) {
  const int lane = threadIdx.x & 31;
  // solves finished so far: this solve publishes with the opposite parity
  const long long tag = (long long)((ld_poll_i((const int*)a.state + 2) & 1) ^ 1);
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(a.state, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.nitems) break;
    const int4 it = __ldg(a.items + t);
    if (it.z >= 0) {
      // the gate: a row a few levels back (the plan's choice; three by
      // default) whose publication means the rows this item reads are
      // about to be published; only then do the lanes
      // start reading them, so items far ahead of the finished levels wait
      // on one entry each instead of flooding L2 with reads
      if (lane == 0) wait_gate((it.w ? a.v : a.y) + (size_t)it.z * R, tag, a.err);
      __syncwarp();
    }
    const int idx = it.x + lane;
    if (idx < it.y) {
      if (t < a.nitemsL)
        lower_row<R>(a, idx, tag);
      else
        upper_row<R>(a, idx, tag);
    }
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    const unsigned fin = atomicAdd(a.state + 1, 1u);
    if (fin == a.total_warps - 1) {
      // every warp has taken its last ticket and read the tag: reset for the next solve
      a.state[0] = 0u;
      a.state[1] = 0u;
      a.state[2] = a.state[2] + 1u;
      __threadfence();
    }
  }
}

template <int R>
cudaError_t trisolve_r(TriArgs a, int window, int sms, cudaStream_t s) {
  static int occ = 0;  // resident blocks per SM (same on every GB300)
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trisolve<R>, kTriThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (occ > kTriMaxBlocksPerSm) occ = kTriMaxBlocksPerSm;
  }
  const int items = window < a.nitems ? window : a.nitems;
  const int want = (items + kTriThreads / 32 - 1) / (kTriThreads / 32);
  int blocks = sms * occ;
  if (blocks > want) blocks = want;
  if (blocks < 1) return cudaSuccess;
  a.total_warps = (unsigned)blocks * (kTriThreads / 32);
  k_trisolve<R><<<blocks, kTriThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trisolve(const TriPlan& P, int R, const double* r, int ldr, const double* dinv, const double* dcol,
                            double* y, double* v, unsigned* state, double* x, int ldx, bool x_zero, int sms, int* err,
                            cudaStream_t s) {
  if (P.nitems == 0) return cudaSuccess;
  TriArgs a;
  a.nitemsL = P.nitemsL;
  a.nitems = P.nitems;
  a.items = (const int4*)P.items;
  a.rowsL = P.rowsL;
  a.lrp = P.lrp;
  a.lci = P.lci;
  a.lva = P.lva;
  a.rowsU = P.rowsU;
  a.urp = P.urp;
  a.uci = P.uci;
  a.uva = P.uva;
  a.r = r;
  a.ldr = ldr;
  a.dinv = dinv;
  a.dcol = dcol;
  a.y = y;
  a.v = v;
  a.x = x;
  a.ldx = ldx;
  a.x_zero = x_zero ? 1 : 0;
  a.state = state;
  a.total_warps = 0;
  a.err = err;
  switch (R) {
    case 1: return trisolve_r<1>(a, P.window > 0 ? P.window : P.nitems, sms, s);
    case 2: return trisolve_r<2>(a, P.window > 0 ? P.window : P.nitems, sms, s);
    case 4: return trisolve_r<4>(a, P.window > 0 ? P.window : P.nitems, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace silu
