// Batches of independent systems (many small pressure solves of uneven size).
//
// The systems are factored independently and in parallel on the host, then
// concatenated into one block-diagonal system: the incomplete factors of a
// block-diagonal matrix are the block-diagonal of the systems' factors, so a
// sweep over the concatenation is exactly every system's sweep, done by one
// launch that load-balances entries across the whole GPU.  The flexible GMRES
// of each system stays its own: dot products are segmented by system (fixed
// row chunks that never straddle two systems, reduced in a fixed order), and
// each system keeps its own Hessenberg matrix, Givens rotations, iteration
// count and convergence state; a system that converges stops updating while
// the others go on.  Each inner iteration is one CUDA graph (captured once per
// Arnoldi index on the batch's fixed buffers) followed by one read of the
// number of systems still active.
#include <thread>

#include "internal.h"

using namespace silu;

namespace {

constexpr int kChunkRows = 4096;
constexpr int KB = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block-wide sum in a fixed order, returned to every thread.
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

// Sum of system s's chunk partials, in chunk order (thread 0), broadcast.
__device__ double system_sum(const double* __restrict__ part, const int* __restrict__ sys_chunk0, int s) {
  __shared__ double v;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int c = sys_chunk0[s]; c < sys_chunk0[s + 1]; ++c) a += part[c];
    v = a;
  }
  __syncthreads();
  const double out = v;
  __syncthreads();
  return out;
}

// The chunk loops below visit a thread's rows d.y + t, d.y + t + KB, ... in
// that order, two loaded before either is used (the same accumulation order
// as one at a time, the same bits); eight blocks fit on an SM.

// part[c] = sum over chunk c of a_i * b_i
__global__ void __launch_bounds__(KB, 8) k_bdot(int nch, const int4* __restrict__ ch, const double* __restrict__ a,
                                                const double* __restrict__ b, double* __restrict__ part) {
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int4 d = ch[c];
    double acc = 0.0;
    int i = d.y + threadIdx.x;
    for (; i + KB < d.z; i += 2 * KB) {
      const double a0 = a[i], a1 = a[i + KB], b0 = b[i], b1 = b[i + KB];
      acc += a0 * b0;
      acc += a1 * b1;
    }
    for (; i < d.z; i += KB) acc += a[i] * b[i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[c] = s;
  }
}

// MGS step i of Arnoldi column j for every active system:
//   h = <w, v_i>_s (from part_in);  H_s[i][j] = h;  w -= h v_i;
//   part_out = chunk partials of <w, v_next> (or |w|^2 when v_next is null).
__global__ void __launch_bounds__(KB, 8) k_bmgs(int nch, const int4* __restrict__ ch, const int* __restrict__ sys_chunk0,
                                             const double* __restrict__ part_in, double* __restrict__ H, int m,
                                             int i, int j, double* __restrict__ w, const double* __restrict__ vi,
                                             const double* __restrict__ vnext, double* __restrict__ part_out,
                                             const int* __restrict__ act) {
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int4 d = ch[c];
    const int s = d.x;
    if (!act[s]) {
      if (threadIdx.x == 0) part_out[c] = 0.0;
      continue;
    }
    const double h = system_sum(part_in, sys_chunk0, s);
    if (threadIdx.x == 0 && c == sys_chunk0[s]) H[((size_t)s * (m + 1) + i) * m + j] = h;
    double acc = 0.0;
    int r = d.y + threadIdx.x;
    if (vnext) {
      for (; r + KB < d.z; r += 2 * KB) {
        const double w0 = w[r], w1 = w[r + KB], v0 = vi[r], v1 = vi[r + KB], u0 = vnext[r], u1 = vnext[r + KB];
        const double n0 = w0 - h * v0, n1 = w1 - h * v1;
        w[r] = n0;
        w[r + KB] = n1;
        acc += n0 * u0;
        acc += n1 * u1;
      }
    } else {
      for (; r + KB < d.z; r += 2 * KB) {
        const double w0 = w[r], w1 = w[r + KB], v0 = vi[r], v1 = vi[r + KB];
        const double n0 = w0 - h * v0, n1 = w1 - h * v1;
        w[r] = n0;
        w[r + KB] = n1;
        acc += n0 * n0;
        acc += n1 * n1;
      }
    }
    for (; r < d.z; r += KB) {
      const double wn = w[r] - h * vi[r];
      w[r] = wn;
      acc += wn * (vnext ? vnext[r] : wn);
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part_out[c] = t;
  }
}

// h = sqrt(<w, w>_s); H_s[j+1][j] = h; v_{j+1} = w / h (active systems, h != 0)
__global__ void __launch_bounds__(KB, 8) k_bnormalize(int nch, const int4* __restrict__ ch,
                                                   const int* __restrict__ sys_chunk0,
                                                   const double* __restrict__ part_in, double* __restrict__ H, int m,
                                                   int j, const double* __restrict__ w, double* __restrict__ vout,
                                                   const int* __restrict__ act) {
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int4 d = ch[c];
    const int s = d.x;
    if (!act[s]) continue;
    const double h = sqrt(system_sum(part_in, sys_chunk0, s));
    if (threadIdx.x == 0 && c == sys_chunk0[s]) H[((size_t)s * (m + 1) + j + 1) * m + j] = h;
    if (h == 0.0) continue;
    int r = d.y + threadIdx.x;
    for (; r + KB < d.z; r += 2 * KB) {
      const double w0 = w[r], w1 = w[r + KB];
      vout[r] = w0 / h;
      vout[r + KB] = w1 / h;
    }
    for (; r < d.z; r += KB) vout[r] = w[r] / h;
  }
}

// out[s] = sqrt(sum of system s's partials)
__global__ void k_bsysnorm(int ns, const int* __restrict__ sys_chunk0, const double* __restrict__ part,
                           double* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int c = sys_chunk0[s]; c < sys_chunk0[s + 1]; ++c) a += part[c];
    out[s] = sqrt(a);
  }
}

// Start of a restart cycle, one block: relres_s = beta_s / |b_s|; a system is
// done once relres <= tol (or |b_s| = 0); the others with iterations left
// become active with g = (beta, 0, ...).  count = active systems.
__global__ void k_bstart(int ns, int m, const double* __restrict__ beta, const double* __restrict__ bnorm, double tol,
                         int maxit, const int* __restrict__ its, int* __restrict__ done, int* __restrict__ act,
                         int* __restrict__ jend, double* __restrict__ g, double* __restrict__ relres,
                         int* __restrict__ count) {
  __shared__ int cnt[KB];
  int mine = 0;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    const double bn = bnorm[s];
    const double rr = bn > 0.0 ? beta[s] / bn : 0.0;
    relres[s] = rr;
    const int d = (bn == 0.0 || rr <= tol) ? 1 : 0;
    done[s] = d;
    const int a = (!d && its[s] < maxit && beta[s] > 0.0) ? 1 : 0;
    act[s] = a;
    jend[s] = 0;
    for (int t = 0; t <= m; ++t) g[(size_t)s * (m + 1) + t] = 0.0;
    if (a) g[(size_t)s * (m + 1)] = beta[s];
    mine += a;
  }
  cnt[threadIdx.x] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < blockDim.x; ++k) t += cnt[k];
    *count = t;
  }
}

// Givens step j, one block, one thread per system.
__global__ void k_bgivens(int ns, int j, int m, double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                          double* __restrict__ g, const double* __restrict__ bnorm, double tol, int maxit,
                          int* __restrict__ act, int* __restrict__ its, int* __restrict__ jend,
                          int* __restrict__ count) {
  __shared__ int cnt[KB];
  int mine = 0;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    if (!act[s]) continue;
    double* Hs = H + (size_t)s * (m + 1) * m;
    double* cs_s = cs + (size_t)s * m;
    double* sn_s = sn + (size_t)s * m;
    double* gs = g + (size_t)s * (m + 1);
    for (int i = 0; i < j; ++i) {
      const double a = Hs[i * m + j], b = Hs[(i + 1) * m + j];
      Hs[i * m + j] = cs_s[i] * a + sn_s[i] * b;
      Hs[(i + 1) * m + j] = -sn_s[i] * a + cs_s[i] * b;
    }
    const double a = Hs[j * m + j], b = Hs[(j + 1) * m + j];
    const double hnext = b;
    const double den = hypot(a, b);
    const double c = den != 0.0 ? a / den : 1.0;
    const double sgn = den != 0.0 ? b / den : 0.0;
    cs_s[j] = c;
    sn_s[j] = sgn;
    Hs[j * m + j] = den;
    Hs[(j + 1) * m + j] = 0.0;
    gs[j + 1] = -sgn * gs[j];
    gs[j] = c * gs[j];
    its[s] += 1;
    jend[s] = j + 1;
    const bool stop = fabs(gs[j + 1]) <= tol * bnorm[s] || its[s] >= maxit || hnext == 0.0 || !isfinite(gs[j + 1]);
    if (stop) act[s] = 0;
    mine += stop ? 0 : 1;
  }
  cnt[threadIdx.x] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < blockDim.x; ++k) t += cnt[k];
    *count = t;
  }
}

// x_s += Z y_s with H_s y_s = g_s (jend_s x jend_s triangle), every system
// that iterated in this cycle.
__global__ void __launch_bounds__(KB) k_bupdate(int nch, const int4* __restrict__ ch, const int* __restrict__ jend,
                                                const double* __restrict__ H, const double* __restrict__ g, int m,
                                                const double* __restrict__ Z, size_t N, double* __restrict__ x) {
  extern __shared__ double ys[];
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int4 d = ch[c];
    const int s = d.x;
    const int je = jend[s];
    if (je == 0) continue;
    const double* Hs = H + (size_t)s * (m + 1) * m;
    const double* gs = g + (size_t)s * (m + 1);
    if (threadIdx.x == 0) {
      for (int i = je - 1; i >= 0; --i) {
        double a = gs[i];
        for (int t = i + 1; t < je; ++t) a -= Hs[i * m + t] * ys[t];
        ys[i] = a / Hs[i * m + i];
      }
    }
    __syncthreads();
    for (int r = d.y + threadIdx.x; r < d.z; r += KB) {
      double a = x[r];
      for (int k = 0; k < je; ++k) a += ys[k] * Z[(size_t)k * N + r];
      x[r] = a;
    }
    __syncthreads();
  }
}

// out_r = in_r / scal_s for rows of active systems (scal_s != 0)
__global__ void __launch_bounds__(KB) k_bdivide(int nch, const int4* __restrict__ ch, const double* __restrict__ scal,
                                                const int* __restrict__ act, const double* in, double* out) {
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int4 d = ch[c];
    const int s = d.x;
    if (!act[s] || scal[s] == 0.0) continue;
    const double q = scal[s];
    for (int r = d.y + threadIdx.x; r < d.z; r += KB) out[r] = in[r] / q;
  }
}

}  // namespace

struct InnerGraph {
  int j = -1, mL = 0, mU = 0, precond = 0;
  int64_t gen = -1;  // launch configuration of the factors at capture
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
};

struct silu_batch_s {
  silu_ctx ctx = nullptr;
  int count = 0;
  std::vector<int64_t> offsets;  // count + 1
  silu_mat A = nullptr;          // concatenated block-diagonal matrix
  silu_ilu F = nullptr;          // concatenated factors
  // chunk tables (host and device)
  std::vector<int> chunks;  // 4 ints per chunk: system, first row, end row, 0
  std::vector<int> sys_chunk0;
  DBuf d_chunks, d_sys_chunk0;
  int nch = 0;
  // batched Krylov workspace
  int restart = 0;
  DBuf V, Z, w, H, cs, sn, g, part0, part1, bnorm, beta, relres, done, act, jend, its, counter;
  std::vector<InnerGraph> graphs;
  double graph_tol = -1.0;  // tol and maxit the captured iterations were made with
  int graph_maxit = -1;
  ~silu_batch_s() {
    for (InnerGraph& ig : graphs)
      if (ig.exec) cudaGraphExecDestroy(ig.exec);
    silu_ilu_destroy(F);
    silu_mat_destroy(A);
  }
};

namespace {

int grid_for(silu_batch B) {
  const int want = B->nch;
  const int cap = 8 * (B->ctx->env.sms > 0 ? B->ctx->env.sms : 1);
  return want < cap ? (want > 0 ? want : 1) : cap;
}

cudaError_t ensure_bkrylov(silu_batch B, int m) {
  if (B->restart >= m && B->V.p) return cudaSuccess;
  for (InnerGraph& ig : B->graphs)
    if (ig.exec) cudaGraphExecDestroy(ig.exec);
  B->graphs.clear();
  const size_t N = (size_t)B->offsets.back();
  const size_t ns = (size_t)B->count;
  cudaError_t e;
  if ((e = B->V.ensure(sizeof(double) * N * (m + 1))) != cudaSuccess) return e;
  if ((e = B->Z.ensure(sizeof(double) * N * m)) != cudaSuccess) return e;
  if ((e = B->w.ensure(sizeof(double) * N)) != cudaSuccess) return e;
  if ((e = B->H.ensure(sizeof(double) * ns * (m + 1) * m)) != cudaSuccess) return e;
  if ((e = B->cs.ensure(sizeof(double) * ns * m)) != cudaSuccess) return e;
  if ((e = B->sn.ensure(sizeof(double) * ns * m)) != cudaSuccess) return e;
  if ((e = B->g.ensure(sizeof(double) * ns * (m + 1))) != cudaSuccess) return e;
  if ((e = B->part0.ensure(sizeof(double) * (size_t)B->nch)) != cudaSuccess) return e;
  if ((e = B->part1.ensure(sizeof(double) * (size_t)B->nch)) != cudaSuccess) return e;
  if ((e = B->bnorm.ensure(sizeof(double) * ns)) != cudaSuccess) return e;
  if ((e = B->beta.ensure(sizeof(double) * ns)) != cudaSuccess) return e;
  if ((e = B->relres.ensure(sizeof(double) * ns)) != cudaSuccess) return e;
  if ((e = B->done.ensure(sizeof(int) * ns)) != cudaSuccess) return e;
  if ((e = B->act.ensure(sizeof(int) * ns)) != cudaSuccess) return e;
  if ((e = B->jend.ensure(sizeof(int) * ns)) != cudaSuccess) return e;
  if ((e = B->its.ensure(sizeof(int) * ns)) != cudaSuccess) return e;
  if ((e = B->counter.ensure(sizeof(int) * 4)) != cudaSuccess) return e;
  B->restart = m;
  return cudaSuccess;
}

// The fixed kernel sequence of inner iteration j (on the batch's buffers).
void inner_iteration(silu_batch B, int j, int m, int mL, int mU, int precond, double tol, int maxit) {
  silu_ilu F = B->F;
  silu_ctx ctx = B->ctx;
  cudaStream_t s = ctx->stream;
  const size_t N = (size_t)B->offsets.back();
  const int gA = lanes_of(F->lanesA, F->autoA);
  double* V = B->V.as<double>();
  double* Z = B->Z.as<double>();
  double* w = B->w.as<double>();
  double* part[2] = {B->part0.as<double>(), B->part1.as<double>()};
  const int4* ch = B->d_chunks.as<int4>();
  const int* sc0 = B->d_sys_chunk0.as<int>();
  const int* act = B->act.as<int>();
  const int grid = grid_for(B);
  double* vj = V + (size_t)j * N;
  double* zj = Z + (size_t)j * N;
  if (precond == SILU_PRECOND_SWEEPS)
    smooth_chunk(F, zj, vj, 1, 1, 0, mL, mU, true);
  else
    CK(cudaMemcpyAsync(zj, vj, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  LAUNCH(ctx, SILU_K_RESIDUAL,
         sweep_launch(F, F->A->d, MODE_D, 1, gA, 1, nullptr, zj, w, nullptr, nullptr, EPI_SPMV));
  LAUNCH(ctx, SILU_K_KRYLOV, (k_bdot<<<grid, KB, 0, s>>>(B->nch, ch, w, V, part[0]), cudaGetLastError()));
  int cur = 0;
  for (int i = 0; i <= j; ++i) {
    const double* vnext = (i < j) ? V + (size_t)(i + 1) * N : nullptr;
    LAUNCH(ctx, SILU_K_KRYLOV,
           (k_bmgs<<<grid, KB, 0, s>>>(B->nch, ch, sc0, part[cur], B->H.as<double>(), m, i, j, w, V + (size_t)i * N,
                                        vnext, part[cur ^ 1], act),
            cudaGetLastError()));
    cur ^= 1;
  }
  LAUNCH(ctx, SILU_K_KRYLOV,
         (k_bnormalize<<<grid, KB, 0, s>>>(B->nch, ch, sc0, part[cur], B->H.as<double>(), m, j, w,
                                           V + (size_t)(j + 1) * N, act),
          cudaGetLastError()));
  LAUNCH(ctx, SILU_K_KRYLOV,
         (k_bgivens<<<1, KB, 0, s>>>(B->count, j, m, B->H.as<double>(), B->cs.as<double>(), B->sn.as<double>(),
                                     B->g.as<double>(), B->bnorm.as<double>(), tol, maxit, B->act.as<int>(),
                                     B->its.as<int>(), B->jend.as<int>(), B->counter.as<int>() + 1),
          cudaGetLastError()));
}

// Run inner iteration j: replay its captured graph (capturing it first).
void run_inner(silu_batch B, int j, int m, int mL, int mU, int precond, double tol, int maxit) {
  silu_ctx ctx = B->ctx;
  for (InnerGraph& ig : B->graphs)
    if (ig.j == j && ig.mL == mL && ig.mU == mU && ig.precond == precond && ig.gen == B->F->config_gen) {
      ctx->launches += ig.kernels;
      CK(cudaGraphLaunch(ig.exec, ctx->stream));
      return;
    }
  // tol and maxit enter k_bgivens as kernel arguments: silu_batch_fgmres drops
  // the captured graphs when they change
  cudaStream_t cap = nullptr;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaStream_t saved = ctx->stream;
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  ctx->stream = cap;
  const int64_t l0 = ctx->launches;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    try {
      inner_iteration(B, j, m, mL, mU, precond, tol, maxit);
    } catch (const CudaFail& f) {
      e = f.e;
    }
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = e2;
  }
  ctx->stream = saved;
  ctx->profiling = prof;
  InnerGraph ig;
  ig.j = j;
  ig.mL = mL;
  ig.mU = mU;
  ig.precond = precond;
  ig.gen = B->F->config_gen;
  ig.kernels = ctx->launches - l0;
  ctx->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ig.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  CK(e);
  B->graphs.push_back(ig);
  ctx->launches += ig.kernels;
  CK(cudaGraphLaunch(ig.exec, ctx->stream));
}

}  // namespace

extern "C" {

silu_status silu_batch_setup(silu_ctx ctx, int count, const int64_t* n, const int64_t* const* row_ptr,
                             const int32_t* const* col_idx, const double* const* val, silu_kind kind, double tau,
                             int fill, silu_scale scale, silu_prec prec, silu_batch* out) {
  NvtxRange nvtx_("silu:silu_batch_setup");
  if (!ctx || !out || count < 1 || !n || !row_ptr || !col_idx || !val) return set_err(ctx, SILU_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  if (kind < SILU_ILU0 || kind > SILU_SGS || scale < SILU_SCALE_NONE || scale > SILU_SCALE_ROWCOL ||
      prec < SILU_FP64 || prec > SILU_FP32)
    return set_err(ctx, SILU_ERR_INVALID_ARG, "bad enum value");
  silu_batch B = nullptr;
  try {
    std::vector<Csr> As(count);
    std::vector<Factors> Fs(count);
    std::vector<int> st(count, H_OK);
    std::vector<std::string> msg(count);
    // independent host factorisations, in parallel
    const int nthreads = std::max(1, std::min<int>(count, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
      pool.emplace_back([&, t]() {
        set_setup_thread_budget(1);  // the systems are the parallelism here
        for (int k = t; k < count; k += nthreads) {
          const int64_t nk = n[k];
          if (nk < 0 || !row_ptr[k]) {
            st[k] = H_BADARG;
            msg[k] = "bad system size";
            continue;
          }
          st[k] = csr_canonical(nk, row_ptr[k][nk], row_ptr[k], col_idx[k], val[k], As[k], msg[k]);
          if (st[k] != H_OK) continue;
          st[k] = factor_kind(As[k], (int)kind, tau, fill, Fs[k], msg[k]);
        }
      });
    for (std::thread& th : pool) th.join();
    for (int k = 0; k < count; ++k)
      if (st[k] != H_OK) return set_err(ctx, (silu_status)st[k], "system " + std::to_string(k) + ": " + msg[k]);
    B = new silu_batch_s;
    B->ctx = ctx;
    B->count = count;
    B->offsets.assign(count + 1, 0);
    for (int k = 0; k < count; ++k) B->offsets[k + 1] = B->offsets[k] + As[k].n;
    const int64_t N = B->offsets.back();
    if (N >= INT32_MAX) {
      delete B;
      return set_err(ctx, SILU_ERR_INVALID_ARG, "batch has more than 2^31 - 1 rows");
    }
    // concatenate A, L and U block-diagonally
    auto concat = [&](auto pick, Csr& out) {
      out.n = N;
      out.rp.assign(N + 1, 0);
      int64_t nnz = 0;
      for (int k = 0; k < count; ++k) nnz += pick(k).nnz();
      out.ci.resize(nnz);
      out.va.resize(nnz);
      int64_t p = 0;
      for (int k = 0; k < count; ++k) {
        const Csr& T = pick(k);
        const int64_t off = B->offsets[k];
        for (int64_t i = 0; i < T.n; ++i) out.rp[off + i + 1] = out.rp[off] + T.rp[i + 1];
        for (int64_t q = 0; q < T.nnz(); ++q) {
          out.ci[p + q] = (int32_t)(T.ci[q] + off);
          out.va[p + q] = T.va[q];
        }
        p += T.nnz();
      }
    };
    silu_mat M = new silu_mat_s;
    M->ctx = ctx;
    concat([&](int k) -> const Csr& { return As[k]; }, M->A);
    B->A = M;
    silu_ilu F = new silu_ilu_s;
    F->ctx = ctx;
    F->A = M;
    F->kind = kind;
    F->scale = scale;
    F->prec = prec;
    F->tau = tau;
    F->fill = fill;
    B->F = F;
    concat([&](int k) -> const Csr& { return Fs[k].L; }, F->F.L);
    concat([&](int k) -> const Csr& { return Fs[k].U; }, F->F.U);
    As.clear();
    Fs.clear();
    if (ctx->device >= 0) {
      silu_status ds = device_ok(ctx);
      if (ds != SILU_OK) {
        delete B;
        return ds;
      }
      cudaError_t e = upload_csr(M->A, false, M->rp, M->ci, M->va, M->tiles, M->d, ctx->stream);
      if (e != cudaSuccess) {
        delete B;
        return cuda_err(ctx, e, "upload of the batch matrix");
      }
    }
    silu_status fs = finish_setup(F);
    if (fs != SILU_OK) {
      delete B;
      return fs;
    }
    // row chunks that never straddle two systems
    B->sys_chunk0.assign(count + 1, 0);
    for (int k = 0; k < count; ++k) {
      for (int64_t r = B->offsets[k]; r < B->offsets[k + 1]; r += kChunkRows) {
        B->chunks.push_back(k);
        B->chunks.push_back((int)r);
        B->chunks.push_back((int)std::min<int64_t>(r + kChunkRows, B->offsets[k + 1]));
        B->chunks.push_back(0);
      }
      B->sys_chunk0[k + 1] = (int)(B->chunks.size() / 4);
    }
    B->nch = (int)(B->chunks.size() / 4);
    if (ctx->device >= 0) {
      cudaError_t e = upload(B->d_chunks, B->chunks.data(), B->chunks.size(), ctx->stream);
      if (e == cudaSuccess) e = upload(B->d_sys_chunk0, B->sys_chunk0.data(), B->sys_chunk0.size(), ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) {
        delete B;
        return cuda_err(ctx, e, "upload of the batch tables");
      }
    }
  } catch (const std::bad_alloc&) {
    delete B;
    return set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  *out = B;
  return SILU_OK;
}

void silu_batch_destroy(silu_batch B) { delete B; }

silu_status silu_batch_info(silu_batch B, int* count, int64_t* offsets, silu_ilu* factors) {
  if (!B) return SILU_ERR_INVALID_ARG;
  if (count) *count = B->count;
  if (offsets) std::memcpy(offsets, B->offsets.data(), sizeof(int64_t) * B->offsets.size());
  if (factors) *factors = B->F;
  return SILU_OK;
}

silu_status silu_batch_smooth(silu_batch B, double* x, const double* b, int sweeps_L, int sweeps_U) {
  NvtxRange nvtx_("silu:silu_batch_smooth");
  if (!B) return SILU_ERR_INVALID_ARG;
  return ilu_smooth(B->F, x, b, 1, sweeps_L, sweeps_U);
}

silu_status silu_batch_fgmres(silu_batch B, double* x, const double* b, double tol, int restart, int maxit,
                              int sweeps_L, int sweeps_U, int precond, int* iters, double* relres) {
  NvtxRange nvtx_("silu:silu_batch_fgmres");
  if (!B) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = B->ctx;
  if (!x || !b || !(tol >= 0.0) || restart < 1 || maxit < 0 || sweeps_L < 0 || sweeps_U < 0 ||
      (precond != SILU_PRECOND_SWEEPS && precond != SILU_PRECOND_NONE))
    return set_err(ctx, SILU_ERR_INVALID_ARG, "silu_batch_fgmres: bad argument");
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  const int m = restart;
  const int ns = B->count;
  const size_t N = (size_t)B->offsets.back();
  cudaStream_t s = ctx->stream;
  silu_ilu F = B->F;
  int remaining = 0;
  try {
    CK(ensure_vectors(F, 1));
    CK(ensure_bkrylov(B, m));
    // captured iterations carry tol and maxit as kernel arguments
    if (tol != B->graph_tol || maxit != B->graph_maxit) {
      for (InnerGraph& ig : B->graphs)
        if (ig.exec) cudaGraphExecDestroy(ig.exec);
      B->graphs.clear();
      B->graph_tol = tol;
      B->graph_maxit = maxit;
    }
    const int grid = grid_for(B);
    const int4* ch = B->d_chunks.as<int4>();
    const int* sc0 = B->d_sys_chunk0.as<int>();
    double* V = B->V.as<double>();
    int* hp = (int*)ctx->pinned;
    const int gA = lanes_of(F->lanesA, F->autoA);
    CK(cudaMemsetAsync(B->its.p, 0, sizeof(int) * ns, s));
    LAUNCH(ctx, SILU_K_KRYLOV, (k_bdot<<<grid, KB, 0, s>>>(B->nch, ch, b, b, B->part0.as<double>()), cudaGetLastError()));
    LAUNCH(ctx, SILU_K_KRYLOV,
           (k_bsysnorm<<<(ns + 255) / 256, 256, 0, s>>>(ns, sc0, B->part0.as<double>(), B->bnorm.as<double>()),
            cudaGetLastError()));
    for (;;) {
      // true residual of every system, restart state
      LAUNCH(ctx, SILU_K_RESIDUAL, sweep_launch(F, F->A->d, MODE_D, 1, gA, 1, b, x, V, nullptr, nullptr, EPI_STORE));
      LAUNCH(ctx, SILU_K_KRYLOV, (k_bdot<<<grid, KB, 0, s>>>(B->nch, ch, V, V, B->part0.as<double>()), cudaGetLastError()));
      LAUNCH(ctx, SILU_K_KRYLOV,
             (k_bsysnorm<<<(ns + 255) / 256, 256, 0, s>>>(ns, sc0, B->part0.as<double>(), B->beta.as<double>()),
              cudaGetLastError()));
      LAUNCH(ctx, SILU_K_KRYLOV,
             (k_bstart<<<1, KB, 0, s>>>(ns, m, B->beta.as<double>(), B->bnorm.as<double>(), tol, maxit,
                                        B->its.as<int>(), B->done.as<int>(), B->act.as<int>(), B->jend.as<int>(),
                                        B->g.as<double>(), B->relres.as<double>(), B->counter.as<int>()),
              cudaGetLastError()));
      CK(cudaMemcpyAsync(hp, B->counter.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hp[0] == 0) break;
      LAUNCH(ctx, SILU_K_KRYLOV,
             (k_bdivide<<<grid, KB, 0, s>>>(B->nch, ch, B->beta.as<double>(), B->act.as<int>(), V, V),
              cudaGetLastError()));
      CK(cudaMemsetAsync(B->H.p, 0, B->H.bytes, s));
      for (int j = 0; j < m; ++j) {
        run_inner(B, j, m, sweeps_L, sweeps_U, precond, tol, maxit);
        CK(cudaMemcpyAsync(hp + 1, B->counter.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hp[1] == 0) break;
      }
      LAUNCH(ctx, SILU_K_KRYLOV,
             (k_bupdate<<<grid, KB, sizeof(double) * (size_t)m, s>>>(B->nch, ch, B->jend.as<int>(),
                                                                     B->H.as<double>(), B->g.as<double>(), m,
                                                                     B->Z.as<double>(), N, x),
              cudaGetLastError()));
    }
    std::vector<int> done(ns), its(ns);
    std::vector<double> rr(ns);
    CK(cudaMemcpyAsync(done.data(), B->done.p, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(its.data(), B->its.p, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(rr.data(), B->relres.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < ns; ++k) {
      if (iters) iters[k] = its[k];
      if (relres) relres[k] = rr[k];
      if (!done[k]) ++remaining;
    }
  } catch (const CudaFail& f) {
    return cuda_err(ctx, f.e, f.what);
  }
  silu_status cs = silu_ctx_check(ctx);
  if (cs != SILU_OK) return cs;
  if (remaining) return set_err(ctx, SILU_ERR_NOT_CONVERGED, std::to_string(remaining) + " systems above tol");
  return SILU_OK;
}

}  // extern "C"
