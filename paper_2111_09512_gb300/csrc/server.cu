// Solve server: continuous batching of pressure solves on one GPU.
//
// Requests (a host CSR system, a right-hand side and solve parameters)
// arrive at any time and wait in a FIFO queue.  A request is admitted when a
// worker slot is free and its device-memory estimate fits in what is left of
// the server's HBM budget; a request larger than the whole budget is refused
// at submission, and a full queue refuses new work (load shedding).  Each
// worker owns a CUDA stream and a context: it factors the admitted system on
// the host, uploads it, runs the flexible GMRES solve on its stream and
// copies the solution back, so several requests run on the device at once and
// a new one starts as soon as a slot and memory free up.  All kernels are
// deterministic and take no input from other requests, so a result is the
// same alone and in the mix.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "internal.h"

using namespace silu;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  Csr A;  // canonical copy
  std::vector<double> b;
  silu_request_params p{};
  int64_t bytes = 0;
  bool cancelled = false;
  silu_result res{};
  std::vector<double> x;
  bool finished = false;
};

}  // namespace

struct silu_server_s {
  int device = -1;
  int64_t budget = 0;
  int64_t used = 0;
  int max_queue = 0;
  int workers_count = 1;  // set before the workers start
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work;  // workers wait for admissible work
  std::condition_variable cv_done;  // waiters wait for results
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_ticket = 1;
  bool stopping = false;
  int running = 0;
  int64_t completed = 0, refused = 0;
  double t0 = 0.0;
};

namespace {

// Device bytes a request holds while it runs: the matrix, both factors,
// dinv, the staged-kernel tiles, the smoother's four work vectors, the
// Krylov basis and preconditioned vectors, x and b, and (for direct solves)
// FP64 copies of the factors and the level lists.
int64_t estimate_bytes(int64_t n, int64_t nnz, const silu_request_params& p) {
  const int64_t fnnz = std::max<int64_t>(nnz - n, 0);  // ILU(0): nnz(L_s) + nnz(U) = nnz(A)
  const int64_t vb = p.prec == SILU_FP32 ? 4 : 8;
  int64_t b = nnz * 12 + n * 4;
  b += fnnz * (vb + 4) + 2 * n * 4 + n * 8;
  b += 4 * n * 8;
  b += (int64_t)(2 * p.restart + 2) * n * 8;
  b += 2 * n * 8;
  if (p.precond == SILU_PRECOND_DIRECT || p.precond == SILU_PRECOND_AMG_DIRECT) b += fnnz * 12 + 4 * n;
  // AMG: coarse operators (operator complexity about 2.5 for these matrices),
  // P and R of every level, four vectors and the l1 diagonal per level
  if (p.precond == SILU_PRECOND_AMG || p.precond == SILU_PRECOND_AMG_DIRECT) b += nnz * 12 * 8 / 5 + n * 160;
  b += (b / 16) + (1 << 20);  // tiles, padding, small buffers
  return b;
}

void finish(silu_server S, const std::shared_ptr<Request>& r, int status) {
  std::lock_guard<std::mutex> lock(S->mu);
  r->res.status = status;
  r->res.t_done = now_s() - S->t0;
  r->finished = true;
  S->completed++;
  S->cv_done.notify_all();
}

void solve_one(silu_server S, silu_ctx ctx, const std::shared_ptr<Request>& r) {
  Request& q = *r;
  silu_mat M = nullptr;
  silu_ilu F = nullptr;
  double* dx = nullptr;
  double* db = nullptr;
  int status = SILU_OK;
  const int64_t n = q.A.n;
  do {
    status = silu_mat_create(ctx, n, q.A.nnz(), q.A.rp.data(), q.A.ci.data(), q.A.va.data(), &M);
    if (status != SILU_OK) break;
    status = ilu_setup(ctx, M, (silu_kind)q.p.kind, q.p.tau, q.p.fill, SILU_SCALE_ROW, (silu_prec)q.p.prec, &F);
    if (status != SILU_OK) break;
    if (q.p.precond == SILU_PRECOND_AMG || q.p.precond == SILU_PRECOND_AMG_DIRECT) {
      status = silu_amg_setup(F, nullptr);
      if (status != SILU_OK) break;
    }
    q.res.t_setup_done = now_s() - S->t0;
    if (ctx->device < 0) {
      status = SILU_ERR_NO_DEVICE;
      break;
    }
    if (n == 0) break;
    if (cudaMalloc(&dx, sizeof(double) * n) != cudaSuccess || cudaMalloc(&db, sizeof(double) * n) != cudaSuccess) {
      status = SILU_ERR_OOM;
      break;
    }
    if (cudaMemsetAsync(dx, 0, sizeof(double) * n, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(db, q.b.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
      status = SILU_ERR_CUDA;
      break;
    }
    int its = 0;
    double rel = 0.0;
    status = fgmres_solve(F, dx, db, q.p.tol, q.p.restart, q.p.maxit, q.p.sweeps_L, q.p.sweeps_U, q.p.precond,
                          &its, &rel);
    q.res.iterations = its;
    q.res.relres = rel;
    q.x.resize(n);
    if (cudaMemcpyAsync(q.x.data(), dx, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      status = SILU_ERR_CUDA;
  } while (false);
  if (dx) cudaFree(dx);
  if (db) cudaFree(db);
  silu_ilu_destroy(F);
  silu_mat_destroy(M);
  finish(S, r, status);
}

void worker_main(silu_server S, int index) {
  // requests are the parallelism here: each worker's setups share the host
  // cores with the other workers'
  {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    silu::set_setup_thread_budget(std::max(1, hw / std::max(1, (int)S->workers_count)));
  }
  silu_ctx ctx = nullptr;
  cudaStream_t stream = nullptr;
  if (S->device >= 0) {
    cudaSetDevice(S->device);
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  }
  if (silu_ctx_create(S->device, stream, &ctx) != SILU_OK) ctx = nullptr;
  (void)index;
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      // FIFO: the head is admitted once its memory fits in the budget
      S->cv_work.wait(lock, [&] {
        if (S->stopping) return true;
        while (!S->queue.empty() && S->queue.front()->cancelled) S->queue.pop_front();
        return !S->queue.empty() && S->used + S->queue.front()->bytes <= S->budget;
      });
      if (S->stopping && S->queue.empty()) break;
      if (S->stopping) {
        // drain: refuse what has not started
        for (auto& q : S->queue) {
          q->res.status = SILU_ERR_CANCELLED;
          q->finished = true;
        }
        S->queue.clear();
        S->cv_done.notify_all();
        break;
      }
      r = S->queue.front();
      S->queue.pop_front();
      S->used += r->bytes;
      S->running++;
      r->res.t_admit = now_s() - S->t0;
    }
    if (ctx)
      solve_one(S, ctx, r);
    else
      finish(S, r, SILU_ERR_CUDA);
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->used -= r->bytes;
      S->running--;
    }
    S->cv_work.notify_all();
  }
  silu_ctx_destroy(ctx);
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

silu_status silu_server_create(int device, int64_t hbm_budget_bytes, int workers, int max_queue,
                               silu_server* out) {
  if (!out || hbm_budget_bytes <= 0 || workers < 1 || workers > 64 || max_queue < 1) return SILU_ERR_INVALID_ARG;
  *out = nullptr;
  if (device >= 0) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device >= count) return SILU_ERR_NO_DEVICE;
  }
  silu_server S = new (std::nothrow) silu_server_s;
  if (!S) return SILU_ERR_OOM;
  S->device = device;
  S->budget = hbm_budget_bytes;
  S->max_queue = max_queue;
  S->t0 = now_s();
  S->workers_count = workers;
  for (int w = 0; w < workers; ++w) S->workers.emplace_back(worker_main, S, w);
  *out = S;
  return SILU_OK;
}

silu_status silu_server_submit(silu_server S, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                               const double* val, const double* b, const silu_request_params* params,
                               uint64_t* ticket) {
  if (!S || !params || !ticket || (n > 0 && !b)) return SILU_ERR_INVALID_ARG;
  const silu_request_params& p = *params;
  if (p.kind < SILU_ILU0 || p.kind > SILU_SGS || p.prec < SILU_FP64 || p.prec > SILU_FP32 || p.restart < 1 ||
      p.maxit < 0 || p.precond < 0 || p.precond > SILU_PRECOND_AMG_DIRECT || !(p.tol >= 0.0))
    return SILU_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  std::string msg;
  try {
    const int st = csr_canonical(n, n >= 0 && row_ptr ? row_ptr[n] : 0, row_ptr, col_idx, val, r->A, msg);
    if (st != H_OK) return (silu_status)st;
    r->b.assign(b, b + n);
    for (double v : r->b)
      if (!std::isfinite(v)) return SILU_ERR_INVALID_ARG;
  } catch (const std::bad_alloc&) {
    return SILU_ERR_OOM;
  }
  r->p = p;
  r->bytes = estimate_bytes(n, r->A.nnz(), p);
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->stopping) return SILU_ERR_CANCELLED;
  if (r->bytes > S->budget) {
    S->refused++;
    return SILU_ERR_OOM;
  }
  if ((int)S->queue.size() >= S->max_queue) {
    S->refused++;
    return SILU_ERR_BUSY;
  }
  r->ticket = S->next_ticket++;
  r->res.t_submit = now_s() - S->t0;
  r->res.device_bytes = r->bytes;
  S->queue.push_back(r);
  S->all[r->ticket] = r;
  *ticket = r->ticket;
  S->cv_work.notify_all();
  return SILU_OK;
}

silu_status silu_server_cancel(silu_server S, uint64_t ticket) {
  if (!S) return SILU_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return SILU_ERR_INVALID_ARG;
  Request& q = *it->second;
  if (q.finished || q.res.t_admit > 0.0) return SILU_ERR_BUSY;  // running or done
  for (auto qi = S->queue.begin(); qi != S->queue.end(); ++qi)
    if ((*qi)->ticket == ticket) {
      S->queue.erase(qi);
      break;
    }
  q.cancelled = true;
  q.finished = true;
  q.res.status = SILU_ERR_CANCELLED;
  q.res.t_done = now_s() - S->t0;
  S->cv_done.notify_all();
  S->cv_work.notify_all();
  return SILU_OK;
}

silu_status silu_server_poll(silu_server S, uint64_t ticket, int wait, int* done, silu_result* res, double* x) {
  if (!S) return SILU_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return SILU_ERR_INVALID_ARG;
  std::shared_ptr<Request> r = it->second;
  if (wait) S->cv_done.wait(lock, [&] { return r->finished; });
  if (done) *done = r->finished ? 1 : 0;
  if (!r->finished) return SILU_OK;
  if (res) *res = r->res;
  if (x && !r->x.empty()) std::memcpy(x, r->x.data(), sizeof(double) * r->x.size());
  S->all.erase(it);  // results are handed out once
  return SILU_OK;
}

silu_status silu_server_stats(silu_server S, int64_t* queued, int64_t* running, int64_t* completed,
                              int64_t* refused, int64_t* bytes_in_use) {
  if (!S) return SILU_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  if (queued) *queued = (int64_t)S->queue.size();
  if (running) *running = S->running;
  if (completed) *completed = S->completed;
  if (refused) *refused = S->refused;
  if (bytes_in_use) *bytes_in_use = S->used;
  return SILU_OK;
}

void silu_server_destroy(silu_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (std::thread& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
