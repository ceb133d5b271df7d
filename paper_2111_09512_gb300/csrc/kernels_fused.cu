// One whole smoother application in one cooperative launch, for small
// systems (sm_103a).
//
// On a system of a few ten thousand rows every sweep of Alg. ILUJac is a
// few microseconds of work, and a launch per sweep (residual, m_L - 1 lower
// sweeps, m_U - 1 upper sweeps, each with its start-up and drain) costs more
// than the arithmetic.  Here one grid, every block resident at once
// (cooperative launch), runs the same sequence of steps -- residual,
// r - L_s y, D^{-1} y, c - Utilde_s v, the update of x -- and separates them
// by grid-wide barriers.  Each thread takes rows in a grid-stride loop and
// all R right-hand sides of its row; each row accumulates c - sum_j T_ij in_j
// in column order with one FMA per entry, as the sweep kernels do.  The
// vectors of a small system stay in L2, so the rows are read straight from
// the CSR arrays without staging.
//
// The barrier: block leaders count arrivals on a device word; the last one
// to arrive resets the count and advances a generation word that the others
// wait on.  Every wait is bounded (2 s of %globaltimer); one that gives up
// sets bit 3 (value 8) of the context's error word and the kernel finishes
// without waiting again, so a broken barrier costs a wrong result reported
// by silu_ctx_check, never a hang.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace silu {
namespace {

constexpr int kFusedThreads = 256;
constexpr unsigned long long kFusedWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long fused_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier over gridDim.x resident blocks.  bar[0] counts the
// blocks that arrived at the current barrier, bar[1] is the generation.
// Returns false (and every later call returns false at once) after a wait
// gave up.
__device__ bool grid_barrier(unsigned* bar, int* err, bool& alive) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = alive ? 1 : 0;
    if (alive) {
      const unsigned gen = ld_acquire_u32(bar + 1);
      __threadfence();
      if (atomicAdd(bar, 1u) == gridDim.x - 1) {
        bar[0] = 0u;
        __threadfence();
        st_release_u32(bar + 1, gen + 1u);
      } else {
        const unsigned long long t0 = fused_ns();
        unsigned spins = 0;
        while (ld_acquire_u32(bar + 1) == gen) {
          if ((++spins & 255u) == 0 && fused_ns() - t0 > kFusedWaitNs) {
            atomicOr(err, 8);
            ok = 0;
            break;
          }
        }
      }
    }
  }
  __syncthreads();
  alive = ok != 0;
  return alive;
}

// A CSR operator of the fused application, or none (a step with no sum).
template <class MT>
struct Op {
  const int* rp;
  const int* ci;
  const MT* va;
};

// One step over all rows: for each row i and column k,
//   t = c[i] - sum_j T_ij in[j]       (t = c[i] without an operator)
// then the epilogue writes out[i] or updates x[i] (as the sweep kernels'
// epilogues: EPI_STORE, EPI_SCALE, EPI_ADDX, EPI_SETX, EPI_SCALE_ADDX,
// EPI_SCALE_SETX).  Vectors are row-major with leading dimension ldx.
template <int R, class MT, class CT, class IT, class OT>
__device__ __forceinline__ void fused_step(int n, int ldx, Op<MT> T, const CT* c, const IT* in, OT* out,
                                           const double* dinv, double* x, int epi) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const size_t o = (size_t)i * (size_t)ldx;
    MT acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = (MT)c[o + k];
    if (T.rp) {
      const int p0 = __ldg(T.rp + i), p1 = __ldg(T.rp + i + 1);
      for (int p = p0; p < p1; ++p) {
        const MT a = __ldg(T.va + p);
        const size_t j = (size_t)__ldg(T.ci + p) * (size_t)ldx;
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = fma(-a, (MT)in[j + k], acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const double t = (double)acc[k];
      if (!T.rp) {
        // a step without an operator rounds the scaling and the update
        // separately, as the launch-per-sweep path's elementwise kernels do
        const double v = (epi == EPI_SCALE || epi == EPI_SCALE_ADDX || epi == EPI_SCALE_SETX) ? __dmul_rn(dinv[i], t) : t;
        if (epi == EPI_STORE || epi == EPI_SCALE)
          out[o + k] = (OT)v;
        else if (epi == EPI_ADDX || epi == EPI_SCALE_ADDX)
          x[o + k] = __dadd_rn(x[o + k], v);
        else
          x[o + k] = v;
        continue;
      }
      switch (epi) {
        case EPI_STORE: out[o + k] = (OT)acc[k]; break;
        case EPI_SCALE: out[o + k] = (OT)(dinv[i] * t); break;
        case EPI_ADDX: x[o + k] += t; break;
        case EPI_SETX: x[o + k] = t; break;
        case EPI_SCALE_ADDX: x[o + k] += dinv[i] * t; break;
        case EPI_SCALE_SETX: x[o + k] = dinv[i] * t; break;
        default: break;
      }
    }
  }
}

struct FusedArgs {
  int n, ldx, mL, mU, x_zero, rowcol;
  Op<double> A;
  const int* lrp;
  const int* lci;
  const void* lva;
  const int* urp;
  const int* uci;
  const void* uva;
  const double* dinv;  // D^{-1} (D_r under row/column scaling)
  const double* dcol;  // D_c under row/column scaling, else null
  const double* b;
  double* x;
  void* r;
  void* c;
  void* p0;
  void* p1;
  unsigned* bar;
  int* err;
};

// The step sequence of one application with row-scaled (or row/column
// scaled) factors, as the launch-per-sweep path orders it:
//   r = b - A x (r = b from a zero guess);
//   y^1 = r, y^k = r - L_s y^{k-1}, k = 2..m_L;
//   then, by m_U: x (+)= y (m_U = 0); x (+)= D^{-1} y (m_U = 1, row
//   scaling); else c = D^{-1} y (D_r y), v^1 = c, v^k = c - Utilde_s v^{k-1},
//   k = 2..m_U, the last one fused with x (+)= v (x (+)= D_c v).
// VI is the type of the workspace vectors (FP32 with FP32 factors), MT the
// factors' type.
template <int R, class MT, class VI>
__global__ void __launch_bounds__(kFusedThreads) k_smooth_fused(FusedArgs a) {
  bool alive = true;
  const int n = a.n, ldx = a.ldx;
  VI* r = (VI*)a.r;
  VI* cbuf = (VI*)a.c;
  VI* pp[2] = {(VI*)a.p0, (VI*)a.p1};
  const Op<MT> L = {a.lrp, a.lci, (const MT*)a.lva};
  const Op<MT> U = {a.urp, a.uci, (const MT*)a.uva};
  const Op<MT> none = {nullptr, nullptr, nullptr};
  const Op<double> noneD = {nullptr, nullptr, nullptr};
  const bool xz = a.x_zero != 0;
  enum { FINAL_Y, FINAL_DY, NEED_C };
  const int after = a.mU == 0 ? FINAL_Y : ((a.mU == 1 && !a.rowcol) ? FINAL_DY : NEED_C);
  // residual
  if (xz)
    fused_step<R, double, double, double, VI>(n, ldx, noneD, a.b, a.b, r, nullptr, nullptr, EPI_STORE);
  else
    fused_step<R, double, double, double, VI>(n, ldx, a.A, a.b, a.x, r, nullptr, nullptr, EPI_STORE);
  grid_barrier(a.bar, a.err, alive);
  // lower sweeps
  const VI* y = r;
  bool done = false;
  for (int k = 2; k <= a.mL; ++k) {
    if (!alive) return;
    const bool last = k == a.mL;
    VI* out = pp[k & 1];
    int epi = EPI_STORE;
    if (last) {
      if (after == FINAL_Y) epi = xz ? EPI_SETX : EPI_ADDX;
      else if (after == FINAL_DY) epi = xz ? EPI_SCALE_SETX : EPI_SCALE_ADDX;
      else {
        epi = EPI_SCALE;
        out = cbuf;
      }
    }
    fused_step<R, MT, VI, VI, VI>(n, ldx, L, r, y, out, a.dinv, a.x, epi);
    grid_barrier(a.bar, a.err, alive);
    y = out;
    if (last && after != NEED_C) done = true;
  }
  if (done || !alive) return;
  if (after == FINAL_Y || after == FINAL_DY) {
    // m_L <= 1: y = r
    fused_step<R, MT, VI, VI, VI>(n, ldx, none, y, y, (VI*)nullptr, a.dinv, a.x,
                                  after == FINAL_Y ? (xz ? EPI_SETX : EPI_ADDX)
                                                   : (xz ? EPI_SCALE_SETX : EPI_SCALE_ADDX));
    return;
  }
  if (a.mL <= 1) {
    // c = D^{-1} r
    fused_step<R, MT, VI, VI, VI>(n, ldx, none, y, y, cbuf, a.dinv, nullptr, EPI_SCALE);
    grid_barrier(a.bar, a.err, alive);
    if (!alive) return;
  }
  const double* xs = a.rowcol ? a.dcol : nullptr;  // x (+)= D_c v under row/column scaling
  if (a.mU == 1) {
    // row/column scaling with one upper term: x (+)= D_c c
    fused_step<R, MT, VI, VI, VI>(n, ldx, none, cbuf, cbuf, (VI*)nullptr, xs, a.x,
                                  xz ? EPI_SCALE_SETX : EPI_SCALE_ADDX);
    return;
  }
  const VI* v = cbuf;
  for (int k = 2; k <= a.mU; ++k) {
    if (!alive) return;
    const bool last = k == a.mU;
    VI* out = pp[k & 1];
    int epi = EPI_STORE;
    if (last) epi = a.rowcol ? (xz ? EPI_SCALE_SETX : EPI_SCALE_ADDX) : (xz ? EPI_SETX : EPI_ADDX);
    fused_step<R, MT, VI, VI, VI>(n, ldx, U, cbuf, v, last ? (VI*)nullptr : out, xs, a.x, epi);
    if (!last) grid_barrier(a.bar, a.err, alive);
    v = out;
  }
}

template <int R, class MT, class VI>
cudaError_t fused_r(const FusedArgs& a, int sms, cudaStream_t s) {
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_smooth_fused<R, MT, VI>, kFusedThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
  }
  int blocks = (a.n + kFusedThreads - 1) / kFusedThreads;
  if (blocks > sms * occ) blocks = sms * occ;
  if (blocks < 1) blocks = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_smooth_fused<R, MT, VI>, a);
}

template <class MT, class VI>
cudaError_t fused_mode(const FusedArgs& a, int R, int sms, cudaStream_t s) {
  switch (R) {
    case 1: return fused_r<1, MT, VI>(a, sms, s);
    case 2: return fused_r<2, MT, VI>(a, sms, s);
    case 4: return fused_r<4, MT, VI>(a, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_smooth_fused(const DevCsr& A, const DevCsr& Ls, const DevCsr& Us, bool f32, int R, int ldx,
                                int mL, int mU, bool x_zero, bool rowcol, const double* dinv, const double* dcol,
                                const double* b, double* x, void* r, void* c, void* p0, void* p1, unsigned* bar,
                                int sms, int* err, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  FusedArgs a;
  a.n = A.n;
  a.ldx = ldx;
  a.mL = mL;
  a.mU = mU;
  a.x_zero = x_zero ? 1 : 0;
  a.rowcol = rowcol ? 1 : 0;
  a.A = {A.rp, A.ci, (const double*)A.va};
  a.lrp = Ls.rp;
  a.lci = Ls.ci;
  a.lva = Ls.va;
  a.urp = Us.rp;
  a.uci = Us.ci;
  a.uva = Us.va;
  a.dinv = dinv;
  a.dcol = dcol;
  a.b = b;
  a.x = x;
  a.r = r;
  a.c = c;
  a.p0 = p0;
  a.p1 = p1;
  a.bar = bar;
  a.err = err;
  return f32 ? fused_mode<float, float>(a, R, sms, s) : fused_mode<double, double>(a, R, sms, s);
}

}  // namespace silu
