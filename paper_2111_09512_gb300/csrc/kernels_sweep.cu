// Sweep kernels of the scaled-ILU smoother (sm_103a).
//
// Every step of the smoother is one CSR SpMV with a fused epilogue:
//   residual      r = b - A x                         (Eq. ILUsplit)
//   L sweep       y^{k+1} = r - L_s y^k               (Alg. ILUJac)
//   U sweep       v^{k+1} = D^{-1} y - Utilde_s v^k   (Eq. richard)
// This is bandwidth-bound sparse work (about 0.17 flop per byte), so the
// tensor cores have no role; the kernel streams the factor's column indices
// and values once per sweep, with `lanes` threads cooperating on a row and a
// shuffle reduction, and gathers the iterate through L1/L2.
#include "device.cuh"

namespace silu {
namespace {

constexpr int kThreads = 256;

template <class MT, class VI, class VO, int R, int G>
__global__ void __launch_bounds__(kThreads) k_sweep(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                    const MT* __restrict__ va, const VI* __restrict__ c,
                                                    const VI* __restrict__ in, VO* __restrict__ out, int ldx,
                                                    const double* __restrict__ dinv, double* __restrict__ x, int epi) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = (int)(gt / G);
  const int lane = (int)(threadIdx.x & (G - 1));
  MT acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = MT(0);
  int p0 = 0, p1 = 0;
  if (row < n) {
    p0 = __ldg(rp + row);
    p1 = __ldg(rp + row + 1);
  }
  for (int p = p0 + lane; p < p1; p += G) {
    const MT a = __ldg(va + p);
    const size_t j = (size_t)__ldg(ci + p) * (size_t)ldx;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += a * (MT)__ldg(in + j + r);
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
  if (row >= n) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (lane != (r % G)) continue;
    const size_t o = (size_t)row * (size_t)ldx + r;
    const MT cv = c ? (MT)c[o] : MT(0);
    const MT t = cv - acc[r];
    switch (epi) {
      case EPI_STORE:
        out[o] = (VO)t;
        break;
      case EPI_SCALE:
        out[o] = (VO)(dinv[row] * (double)t);
        break;
      case EPI_ADDX:
        x[o] += (double)t;
        break;
      case EPI_SETX:
        x[o] = (double)t;
        break;
      case EPI_SCALE_ADDX:
        x[o] += dinv[row] * (double)t;
        break;
      case EPI_SCALE_SETX:
        x[o] = dinv[row] * (double)t;
        break;
      case EPI_JAC:
        out[o] = (VO)((MT)in[o] + (MT)dinv[row] * t);
        break;
      case EPI_JAC_ADDX:
        x[o] += (double)((MT)in[o] + (MT)dinv[row] * t);
        break;
      case EPI_JAC_SETX:
        x[o] = (double)((MT)in[o] + (MT)dinv[row] * t);
        break;
      case EPI_RICH:
        out[o] = (VO)(t + (MT)in[o]);
        break;
      case EPI_RICH_ADDX:
        x[o] += (double)(t + (MT)in[o]);
        break;
      case EPI_RICH_SETX:
        x[o] = (double)(t + (MT)in[o]);
        break;
      case EPI_SPMV:
        out[o] = (VO)acc[r];
        break;
      default:
        break;
    }
  }
}

template <class MT, class VI, class VO, int R>
cudaError_t sweep_g(const DevCsr& T, int lanes, int ldx, const void* c, const void* in, void* out, const double* dinv,
                    double* x, int epi, cudaStream_t s) {
  const long long threads = (long long)T.n * lanes;
  const unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
  if (blocks == 0) return cudaSuccess;
  const MT* va = (const MT*)T.va;
  const VI* cc = (const VI*)c;
  const VI* ii = (const VI*)in;
  VO* oo = (VO*)out;
  switch (lanes) {
    case 1: k_sweep<MT, VI, VO, R, 1><<<blocks, kThreads, 0, s>>>(T.n, T.rp, T.ci, va, cc, ii, oo, ldx, dinv, x, epi); break;
    case 2: k_sweep<MT, VI, VO, R, 2><<<blocks, kThreads, 0, s>>>(T.n, T.rp, T.ci, va, cc, ii, oo, ldx, dinv, x, epi); break;
    case 4: k_sweep<MT, VI, VO, R, 4><<<blocks, kThreads, 0, s>>>(T.n, T.rp, T.ci, va, cc, ii, oo, ldx, dinv, x, epi); break;
    case 8: k_sweep<MT, VI, VO, R, 8><<<blocks, kThreads, 0, s>>>(T.n, T.rp, T.ci, va, cc, ii, oo, ldx, dinv, x, epi); break;
    case 16: k_sweep<MT, VI, VO, R, 16><<<blocks, kThreads, 0, s>>>(T.n, T.rp, T.ci, va, cc, ii, oo, ldx, dinv, x, epi); break;
    case 32: k_sweep<MT, VI, VO, R, 32><<<blocks, kThreads, 0, s>>>(T.n, T.rp, T.ci, va, cc, ii, oo, ldx, dinv, x, epi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class MT, class VI, class VO>
cudaError_t sweep_r(const DevCsr& T, int R, int lanes, int ldx, const void* c, const void* in, void* out,
                    const double* dinv, double* x, int epi, cudaStream_t s) {
  switch (R) {
    case 1: return sweep_g<MT, VI, VO, 1>(T, lanes, ldx, c, in, out, dinv, x, epi, s);
    case 2: return sweep_g<MT, VI, VO, 2>(T, lanes, ldx, c, in, out, dinv, x, epi, s);
    case 4: return sweep_g<MT, VI, VO, 4>(T, lanes, ldx, c, in, out, dinv, x, epi, s);
    default: return cudaErrorInvalidValue;
  }
}

// Level-scheduled substitution: the rows of one level only read entries of
// earlier levels, which earlier launches finished (Sec. 4).
template <int R, int G>
__global__ void __launch_bounds__(kThreads) k_level(int nrows, const int* __restrict__ rows,
                                                    const int* __restrict__ rp, const int* __restrict__ ci,
                                                    const double* __restrict__ va, double* y, int ldx,
                                                    const double* __restrict__ dinv, double* c_out, double* x) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int idx = (int)(gt / G);
  const int lane = (int)(threadIdx.x & (G - 1));
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  int row = -1, p0 = 0, p1 = 0;
  if (idx < nrows) {
    row = __ldg(rows + idx);
    p0 = __ldg(rp + row);
    p1 = __ldg(rp + row + 1);
  }
  // the level's rows and pointers are fixed; y is not until the previous level is done
  grid_wait_prior();
  grid_launch_dependents();
  for (int p = p0 + lane; p < p1; p += G) {
    const double a = __ldg(va + p);
    const size_t j = (size_t)__ldg(ci + p) * (size_t)ldx;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += a * y[j + r];
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off);
  if (row < 0) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (lane != (r % G)) continue;
    const size_t o = (size_t)row * (size_t)ldx + r;
    const double v = y[o] - acc[r];
    y[o] = v;
    if (c_out) c_out[o] = dinv[row] * v;
    if (x) x[o] += v;
  }
}

template <int R>
cudaError_t level_g(const DevCsr& T, const int* rows, int nrows, int lanes, int ldx, double* y, const double* dinv,
                    double* c_out, double* x, bool overlap, cudaStream_t s) {
  const long long threads = (long long)nrows * lanes;
  const unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
  if (blocks == 0) return cudaSuccess;
  const double* va = (const double*)T.va;
  // each level is a programmatic dependent of the one before: its CTAs load
  // their rows' pointers while the previous level finishes
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap ? 1 : 0;
  const int* rp = T.rp;
  const int* ci = T.ci;
  switch (lanes) {
    case 1: return cudaLaunchKernelEx(&cfg, k_level<R, 1>, nrows, rows, rp, ci, va, y, ldx, dinv, c_out, x);
    case 2: return cudaLaunchKernelEx(&cfg, k_level<R, 2>, nrows, rows, rp, ci, va, y, ldx, dinv, c_out, x);
    case 4: return cudaLaunchKernelEx(&cfg, k_level<R, 4>, nrows, rows, rp, ci, va, y, ldx, dinv, c_out, x);
    case 8: return cudaLaunchKernelEx(&cfg, k_level<R, 8>, nrows, rows, rp, ci, va, y, ldx, dinv, c_out, x);
    case 16: return cudaLaunchKernelEx(&cfg, k_level<R, 16>, nrows, rows, rp, ci, va, y, ldx, dinv, c_out, x);
    case 32: return cudaLaunchKernelEx(&cfg, k_level<R, 32>, nrows, rows, rp, ci, va, y, ldx, dinv, c_out, x);
  }
  return cudaErrorInvalidValue;
}

template <class VI, class VO>
__global__ void k_scale(int n, int R, int ldx, const VI* __restrict__ in, const double* __restrict__ dinv,
                        VO* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * R) return;
  // one right-hand side (the common case) needs no 64-bit division
  const int row = R == 1 ? (int)t : (int)(t / R), r = R == 1 ? 0 : (int)(t % R);
  const size_t o = (size_t)row * (size_t)ldx + r;
  const double v = (double)in[o];
  out[o] = (VO)(dinv ? dinv[row] * v : v);
}

template <class VI>
__global__ void k_addx(int n, int R, int ldx, const VI* __restrict__ in, const double* __restrict__ dinv,
                       double* __restrict__ x, int accumulate) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * R) return;
  const int row = R == 1 ? (int)t : (int)(t / R), r = R == 1 ? 0 : (int)(t % R);
  const size_t o = (size_t)row * (size_t)ldx + r;
  double v = (double)in[o];
  if (dinv) v = dinv[row] * v;
  x[o] = accumulate ? x[o] + v : v;
}

}  // namespace

cudaError_t launch_sweep(const DevCsr& T, Mode mode, int R, int lanes, int ldx, const void* c, const void* in,
                         void* out, const double* dinv, double* x, int epi, cudaStream_t s) {
  switch (mode) {
    case MODE_D: return sweep_r<double, double, double>(T, R, lanes, ldx, c, in, out, dinv, x, epi, s);
    case MODE_F: return sweep_r<float, float, float>(T, R, lanes, ldx, c, in, out, dinv, x, epi, s);
    case MODE_DF: return sweep_r<double, double, float>(T, R, lanes, ldx, c, in, out, dinv, x, epi, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_level(const DevCsr& T, const int* rows, int nrows, int R, int lanes, int ldx, double* y,
                         const double* dinv, double* c_out, double* x, bool overlap, cudaStream_t s) {
  switch (R) {
    case 1: return level_g<1>(T, rows, nrows, lanes, ldx, y, dinv, c_out, x, overlap, s);
    case 2: return level_g<2>(T, rows, nrows, lanes, ldx, y, dinv, c_out, x, overlap, s);
    case 4: return level_g<4>(T, rows, nrows, lanes, ldx, y, dinv, c_out, x, overlap, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_scale(int n, int R, int ldx, const void* in, bool in_f32, const double* dinv, void* out,
                         bool out_f32, cudaStream_t s) {
  const long long tot = (long long)n * R;
  if (tot == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((tot + kThreads - 1) / kThreads);
  if (in_f32 && out_f32)
    k_scale<float, float><<<blocks, kThreads, 0, s>>>(n, R, ldx, (const float*)in, dinv, (float*)out);
  else if (in_f32)
    k_scale<float, double><<<blocks, kThreads, 0, s>>>(n, R, ldx, (const float*)in, dinv, (double*)out);
  else if (out_f32)
    k_scale<double, float><<<blocks, kThreads, 0, s>>>(n, R, ldx, (const double*)in, dinv, (float*)out);
  else
    k_scale<double, double><<<blocks, kThreads, 0, s>>>(n, R, ldx, (const double*)in, dinv, (double*)out);
  return cudaGetLastError();
}

cudaError_t launch_addx(int n, int R, int ldx, const void* in, bool in_f32, const double* dinv, double* x,
                        bool accumulate, cudaStream_t s) {
  const long long tot = (long long)n * R;
  if (tot == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((tot + kThreads - 1) / kThreads);
  if (in_f32)
    k_addx<float><<<blocks, kThreads, 0, s>>>(n, R, ldx, (const float*)in, dinv, x, accumulate ? 1 : 0);
  else
    k_addx<double><<<blocks, kThreads, 0, s>>>(n, R, ldx, (const double*)in, dinv, x, accumulate ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace silu
