// FP64 Krylov kernels of the flexible GMRES solve (Sec. 6: FGMRES with
// modified Gram-Schmidt, Givens rotations, Eq. relres stopping test).
//
// Reductions are two-stage and deterministic: a fixed grid writes one
// partial sum per block, and every consumer reduces the partials in the same
// fixed order.  The same inputs therefore give bitwise the same results
// whatever else runs on the device.
#include <cmath>

#include "device.cuh"
#include "krylov.cuh"

namespace silu {
namespace {

constexpr int KB = 256;
constexpr int kMaxParts = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block-wide sum in a fixed order; the result is returned to every thread.
__device__ double block_sum(double v) {
  __shared__ double red[KB / 32];
  __shared__ double total;
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < KB / 32; ++i) s += red[i];
    total = s;
  }
  __syncthreads();
  const double out = total;
  __syncthreads();
  return out;
}

__device__ double sum_parts(const double* __restrict__ part, int nparts) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += KB) v += part[i];
  return block_sum(v);
}

// The streaming loops below visit a thread's elements i0, i0 + S, i0 + 2S, ...
// (S = the grid's thread count) in that order, as a plain grid-stride loop
// would, but load two of them before using either: twice the bytes in
// flight per thread, the same accumulation order, the same bits.  Indices are
// unsigned 32-bit (n < 2^31, so i + 2S cannot wrap), which keeps each kernel
// within 32 registers: all 1024 blocks of the largest grid are resident at
// once (eight per SM) and none waits for a second wave.
__global__ void __launch_bounds__(KB, 8) k_dot_part(int n, const double* __restrict__ a, const double* __restrict__ b,
                                                    double* __restrict__ part) {
  const unsigned N = (unsigned)n, S = gridDim.x * KB;
  unsigned i = blockIdx.x * KB + threadIdx.x;
  double acc = 0.0;
  for (; i + S < N; i += 2 * S) {
    const double a0 = a[i], a1 = a[i + S];
    const double b0 = b[i], b1 = b[i + S];
    acc += a0 * b0;
    acc += a1 * b1;
  }
  for (; i < N; i += S) acc += a[i] * b[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(KB, 8) k_mgs_step(int n, const double* __restrict__ part_in, int nparts,
                                                    double* __restrict__ hout, double* __restrict__ w,
                                                    const double* __restrict__ vi, const double* __restrict__ vnext,
                                                    double* __restrict__ part_out) {
  const double h = sum_parts(part_in, nparts);
  if (blockIdx.x == 0 && threadIdx.x == 0 && hout) *hout = h;
  const unsigned N = (unsigned)n, S = gridDim.x * KB;
  unsigned i = blockIdx.x * KB + threadIdx.x;
  double acc = 0.0;
  if (vnext) {
    for (; i + S < N; i += 2 * S) {
      const double w0 = w[i], w1 = w[i + S];
      const double v0 = vi[i], v1 = vi[i + S];
      const double u0 = vnext[i], u1 = vnext[i + S];
      const double n0 = w0 - h * v0, n1 = w1 - h * v1;
      w[i] = n0;
      w[i + S] = n1;
      acc += n0 * u0;
      acc += n1 * u1;
    }
    for (; i < N; i += S) {
      const double wn = w[i] - h * vi[i];
      w[i] = wn;
      acc += wn * vnext[i];
    }
  } else {  // last step: the partial sums of ||w||^2 for the normalisation
    for (; i + S < N; i += 2 * S) {
      const double w0 = w[i], w1 = w[i + S];
      const double v0 = vi[i], v1 = vi[i + S];
      const double n0 = w0 - h * v0, n1 = w1 - h * v1;
      w[i] = n0;
      w[i + S] = n1;
      acc += n0 * n0;
      acc += n1 * n1;
    }
    for (; i < N; i += S) {
      const double wn = w[i] - h * vi[i];
      w[i] = wn;
      acc += wn * wn;
    }
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part_out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(KB, 8) k_normalize(int n, const double* __restrict__ part_in, int nparts,
                                                     double* __restrict__ hout, const double* w, double* vout) {
  const double h = sqrt(sum_parts(part_in, nparts));
  if (blockIdx.x == 0 && threadIdx.x == 0 && hout) *hout = h;
  if (h == 0.0) return;
  const unsigned N = (unsigned)n, S = gridDim.x * KB;
  unsigned i = blockIdx.x * KB + threadIdx.x;
  for (; i + S < N; i += 2 * S) {  // w may be vout: each element is read, then written, by one thread
    const double w0 = w[i], w1 = w[i + S];
    vout[i] = w0 / h;
    vout[i + S] = w1 / h;
  }
  for (; i < N; i += S) vout[i] = w[i] / h;
}

// Minimal-residual step: alpha = sum(part_num) / sum(part_den) (0 when the
// denominator is 0), y = alpha s.
__global__ void __launch_bounds__(KB) k_mr_step(int n, const double* __restrict__ part_num,
                                                const double* __restrict__ part_den, int nparts,
                                                const double* __restrict__ s, double* __restrict__ y) {
  const double num = sum_parts(part_num, nparts);
  const double den = sum_parts(part_den, nparts);
  const double alpha = den != 0.0 ? num / den : 0.0;
  for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB)
    y[i] = alpha * s[i];
}

__global__ void k_norm_final(const double* __restrict__ part_in, int nparts, double* __restrict__ out) {
  const double h = sqrt(sum_parts(part_in, nparts));
  if (threadIdx.x == 0) *out = h;
}

// One thread: apply the earlier rotations to column j, make the new one,
// rotate g (right-hand side of the least-squares problem).
__global__ void k_givens(int j, int m, double* H, double* cs, double* sn, double* g, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], b = H[(i + 1) * m + j];
    H[i * m + j] = cs[i] * a + sn[i] * b;
    H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
  }
  const double a = H[j * m + j], b = H[(j + 1) * m + j];
  const double den = hypot(a, b);
  const double c = den != 0.0 ? a / den : 1.0;
  const double s = den != 0.0 ? b / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  res[0] = fabs(g[j + 1]);
  res[1] = b;  // h_{j+1,j}: zero means the Krylov space is exhausted
}

// Every block solves the small triangle (redundantly, same order) and then
// updates its slice of x with the combination of the preconditioned vectors.
__global__ void __launch_bounds__(KB) k_update_x(int n, int jend, int m, const double* __restrict__ H,
                                                 const double* __restrict__ g, double* __restrict__ yout,
                                                 const double* __restrict__ Z, double* __restrict__ x) {
  extern __shared__ double ys[];
  if (threadIdx.x == 0) {
    for (int i = jend - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < jend; ++t) s -= H[i * m + t] * ys[t];
      ys[i] = s / H[i * m + i];
    }
    if (blockIdx.x == 0)
      for (int i = 0; i < jend; ++i) yout[i] = ys[i];
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * KB + threadIdx.x; i < n; i += (long long)gridDim.x * KB) {
    double acc = x[i];
    for (int k = 0; k < jend; ++k) acc += ys[k] * Z[(size_t)k * (size_t)n + i];
    x[i] = acc;
  }
}

}  // namespace

int krylov_parts(int n) {
  long long p = ((long long)n + 8 * KB - 1) / (8 * KB);
  if (p < 1) p = 1;
  if (p > kMaxParts) p = kMaxParts;
  return (int)p;
}

cudaError_t launch_dot_part(int n, const double* a, const double* b, double* part, cudaStream_t s) {
  k_dot_part<<<krylov_parts(n), KB, 0, s>>>(n, a, b, part);
  return cudaGetLastError();
}

cudaError_t launch_mgs_step(int n, const double* part_in, double* hout, double* w, const double* vi,
                            const double* vnext, double* part_out, cudaStream_t s) {
  const int np = krylov_parts(n);
  k_mgs_step<<<np, KB, 0, s>>>(n, part_in, np, hout, w, vi, vnext, part_out);
  return cudaGetLastError();
}

cudaError_t launch_normalize(int n, const double* part_in, double* hout, const double* w, double* vout,
                             cudaStream_t s) {
  const int np = krylov_parts(n);
  k_normalize<<<np, KB, 0, s>>>(n, part_in, np, hout, w, vout);
  return cudaGetLastError();
}

cudaError_t launch_mr_step(int n, const double* part_num, const double* part_den, const double* sv, double* y,
                           cudaStream_t s) {
  const int np = krylov_parts(n);
  k_mr_step<<<np, KB, 0, s>>>(n, part_num, part_den, np, sv, y);
  return cudaGetLastError();
}

cudaError_t launch_norm_final(int n, const double* part_in, double* out, cudaStream_t s) {
  k_norm_final<<<1, KB, 0, s>>>(part_in, krylov_parts(n), out);
  return cudaGetLastError();
}

cudaError_t launch_givens(int j, int m, double* H, double* cs, double* sn, double* g, double* res, cudaStream_t s) {
  k_givens<<<1, 32, 0, s>>>(j, m, H, cs, sn, g, res);
  return cudaGetLastError();
}

cudaError_t launch_update_x(int n, int jend, int m, const double* H, const double* g, double* y, const double* Z,
                            double* x, cudaStream_t s) {
  if (jend <= 0) return cudaSuccess;
  k_update_x<<<krylov_parts(n), KB, sizeof(double) * (size_t)jend, s>>>(n, jend, m, H, g, y, Z, x);
  return cudaGetLastError();
}

}  // namespace silu
