// silu_smooth_noalloc: one smoother application that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they apply
// the smoother: an application whose device memory is owned up front by its
// own pool or by another framework's allocator, or a latency-critical
// time-stepping loop that must not pay the implicit device synchronisation
// of cudaMalloc / cudaFree.  They keep the factors in arrays they own and
// call this entry point, which takes its working vectors from a fixed
// device array compiled into the library instead of allocating them.
//
// The scratch array holds four vectors of kNoAllocMaxRows doubles (16 MiB);
// every device that loads the library keeps it until the process exits.
// Its device address is looked up once per device, with that device
// current, on the first call that uses the device.  With CUDA's lazy module
// loading (the default), that lookup is also what loads this file's device
// code on the device and so reserves the 16 MiB: the first call on a device
// can fail with SILU_ERR_OOM when the caller's pool already holds all device
// memory, so callers make one call before their pool claims the memory (and
// before any stream capture); from then on no call needs device memory.  The
// address is cached for the life of the process, so calls after
// cudaDeviceReset (or a reset of the primary context) are not supported.
// Every call shares the array and it keeps whatever the previous call left
// in it; this entry point writes each scratch vector before reading it, so
// nothing has to start at zero.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "device.cuh"
#include "silu.h"

namespace {

constexpr int64_t kNoAllocMaxRows = 524288;  // 2^19 rows
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[4 * kNoAllocMaxRows];

std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).
cudaError_t scratch_on(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

silu::DevCsr csr_view(int64_t n, const int32_t* rp, const int32_t* ci, const double* va) {
  silu::DevCsr d;
  d.n = (int)n;
  d.rp = const_cast<int*>(rp);
  d.ci = const_cast<int*>(ci);
  d.va = const_cast<double*>(va);
  return d;
}

cudaError_t run(int64_t n64, cudaStream_t s, double* scratch, const silu::DevCsr& A, const silu::DevCsr& L,
                const silu::DevCsr& U, const double* dinv, double* x, const double* b, int mL, int mU) {
  const int n = (int)n64;
  double* R = scratch;
  double* C = scratch + kNoAllocMaxRows;
  double* P[2] = {scratch + 2 * kNoAllocMaxRows, scratch + 3 * kNoAllocMaxRows};
  const int gA = 8, gT = 4;  // lanes per row: any power of two is correct
  cudaError_t e = silu::launch_sweep(A, silu::MODE_D, 1, gA, 1, b, x, R, nullptr, nullptr, silu::EPI_STORE, s);
  if (e != cudaSuccess) return e;
  // y^1 = r, y^k = r - L_s y^{k-1}
  const double* y = R;
  for (int k = 2; k <= mL; ++k) {
    e = silu::launch_sweep(L, silu::MODE_D, 1, gT, 1, R, y, P[k & 1], nullptr, nullptr, silu::EPI_STORE, s);
    if (e != cudaSuccess) return e;
    y = P[k & 1];
  }
  if (mU == 0) return silu::launch_addx(n, 1, 1, y, false, nullptr, x, true, s);
  // c = D^{-1} y; v^1 = c, v^k = c - Utilde_s v^{k-1}; x += v
  e = silu::launch_scale(n, 1, 1, y, false, dinv, C, false, s);
  if (e != cudaSuccess) return e;
  if (mU == 1) return silu::launch_addx(n, 1, 1, C, false, nullptr, x, true, s);
  const double* v = C;
  for (int k = 2; k <= mU; ++k) {
    const bool last = (k == mU);
    e = silu::launch_sweep(U, silu::MODE_D, 1, gT, 1, C, v, last ? nullptr : P[k & 1], nullptr, x,
                           last ? silu::EPI_ADDX : silu::EPI_STORE, s);
    if (e != cudaSuccess) return e;
    v = P[k & 1];
  }
  return cudaSuccess;
}

}  // namespace

extern "C" silu_status silu_smooth_noalloc(int device, void* cuda_stream, int64_t n, const int32_t* A_rp,
                                           const int32_t* A_ci, const double* A_val, const int32_t* L_rp,
                                           const int32_t* L_ci, const double* L_val, const int32_t* U_rp,
                                           const int32_t* U_ci, const double* U_val, const double* dinv,
                                           double* x, const double* b, int sweeps_L, int sweeps_U) {
  if (n < 0 || sweeps_L < 0 || sweeps_U < 0 || device < 0 || device >= kMaxDevices) return SILU_ERR_INVALID_ARG;
  if (n > kNoAllocMaxRows) return SILU_ERR_TOO_LARGE;
  if (n == 0) return SILU_OK;
  if (!A_rp || !A_ci || !A_val || !L_rp || !L_ci || !L_val || !U_rp || !U_ci || !U_val || !dinv || !x || !b)
    return SILU_ERR_INVALID_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return SILU_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return SILU_ERR_NO_DEVICE;
  double* scratch = nullptr;
  cudaError_t e = scratch_on(device, &scratch);
  if (e == cudaErrorMemoryAllocation) {
    // loading the array onto the device needs 16 MiB that are not free
    if (prev != device) cudaSetDevice(prev);
    return SILU_ERR_OOM;
  }
  if (e == cudaSuccess)
    e = run(n, (cudaStream_t)cuda_stream, scratch, csr_view(n, A_rp, A_ci, A_val), csr_view(n, L_rp, L_ci, L_val),
            csr_view(n, U_rp, U_ci, U_val), dinv, x, b, sweeps_L, sweeps_U);
  if (prev != device) cudaSetDevice(prev);
  return e == cudaSuccess ? SILU_OK : SILU_ERR_CUDA;
}
