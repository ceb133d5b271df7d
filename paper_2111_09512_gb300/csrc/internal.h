// Internal declarations shared by the C-ABI translation units of libsilu
// (api.cu, batch.cu): handle structures, device buffers, error plumbing,
// launch accounting and the smoother orchestration helpers.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "amg_setup.h"
#include "device.cuh"
#include "host_factor.h"
#include "krylov.cuh"
#include "silu.h"

namespace silu {

// Owning device buffer.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (b <= bytes && p) return cudaSuccess;
    release();
    if (b == 0) b = 16;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = b;
    return cudaSuccess;
  }
  template <class T>
  T* as() const {
    return (T*)p;
  }
};


}  // namespace silu

using silu::DBuf;
using silu::DevCsr;

struct silu_ctx_s {
  int device = -1;
  cudaStream_t stream = nullptr;
  std::string err;
  double* pinned = nullptr;  // small host buffer for scalar read-backs
  int64_t launches = 0;      // kernels launched on this context
  silu::LaunchEnv env;       // SM count and device error word
  // event timing of launches (silu_ctx_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> events;  // pool; records use pairs (2k, 2k+1)
  std::vector<int> rec_class;       // class of record k
  std::vector<int64_t> rec_count;   // launches covered by record k
  size_t nrec = 0;
  int run_class = -1;               // class of the open run of launches (ProfRun), or -1
  long run_rec = -1;                // its record once started
};

struct silu_mat_s {
  silu_ctx ctx = nullptr;
  silu::Csr A;
  DBuf rp, ci, va, tiles;
  DevCsr d;
  int64_t gen = 0;  // bumped when the launch shape of d changes (captured graphs that use A go stale)
};

// A captured level-scheduled solve on the workspace vectors of one column block.
struct LevelGraph {
  int R = 0, ldx = 0;
  size_t col = 0;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

// A captured FGMRES inner iteration (Arnoldi index j) on the Krylov workspace.
struct KrylovGraph {
  int j = -1, m = 0, mL = 0, mU = 0, precond = 0;
  int64_t gen = -1;   // launch configuration the graph was captured with
  int64_t agen = -1;  // and the matrix's
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
};

struct Workspace {
  size_t vec_bytes = 0;  // per buffer
  DBuf r, c, p0, p1;
  std::vector<LevelGraph> graphs;    // valid while r and c keep their addresses
  std::vector<KrylovGraph> kgraphs;  // valid while every workspace buffer keeps its address
  ~Workspace() { drop_graphs(); }
  void drop_graphs() {
    for (LevelGraph& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    graphs.clear();
    for (KrylovGraph& g : kgraphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    kgraphs.clear();
  }
  int restart = 0;
  DBuf V, Z, w, H, cs, sn, g, yk, part0, part1, scal;
};

// Device arrays of a length-sorted copy of a factor (staged kernel only).
struct SortedBufs {
  DBuf rp, ci, va, perm, tiles;
};

// Device copy of one AMG level (Sec. 3).  Level 0's operator is the
// silu_mat's; coarser levels keep their own.  P is stored negated so that the
// prolongation x += P v is the sweep kernel's x += c - (-P) v with c = 0.
struct AmgDevLevel {
  int64_t n = 0;
  DBuf A_rp, A_ci, A_va, A_tiles, P_rp, P_ci, P_va, P_tiles, R_rp, R_ci, R_va, R_tiles;
  DevCsr A, Pneg, R;
  DBuf l1inv, x, t, b, r;
  DBuf G_rp, G_ci, G_va, G_tiles, gdinv, y2;  // polynomial Gauss-Seidel: L D^{-1}, 1 / a_ii, a second sweep buffer
  DevCsr Lgs;
};

// An AMG hierarchy attached to a factor object: the factors smooth the
// finest level (and, with ilu_levels > 1, factors of their own the next
// levels), l1-Jacobi or polynomial Gauss-Seidel the coarser ones, the
// coarsest is solved directly.
struct AmgState {
  silu::AmgHost host;
  std::vector<std::unique_ptr<AmgDevLevel>> lev;
  DBuf cinv;  // dense inverse of the coarsest operator
  int nu = 1;  // smoothing steps before and after the correction on levels >= 1
  int coarse_kind = SILU_AMG_L1_JACOBI;
  int gs_terms = 2;
  int ilu_levels = 1;
  double theta = 0.25;
  int max_levels = 25;
  int64_t coarse_size = 400;
  // the ILU smoothers of levels 1 .. ilu_levels - 1 (silu_amg_params.ilu_levels):
  // A_l and its row-scaled factors as objects of their own, indexed by level
  // (owned; null at level 0, which F smooths, and below)
  std::vector<silu_mat> ilu_mat;
  std::vector<silu_ilu> ilu_fac;
  AmgState() = default;
  AmgState(const AmgState&) = delete;
  AmgState& operator=(const AmgState&) = delete;
  ~AmgState();
};

// The ILUT Schur complement smoother attached to a factor object (Sec. 3.1,
// Eq. schur): A permuted to [B E; F C] (interior rows first, interface rows
// last), B factored by ILUT and applied by the sweeps, one GMRES iteration
// on the interface system.
struct SchurState {
  int parts = 0;
  int64_t nI = 0, nG = 0;
  std::vector<int32_t> iface;  // 1 = interface row
  silu_mat Bmat = nullptr;     // B (owned)
  silu_ilu FB = nullptr;       // ILUT factors of B (owned)
  DBuf rowsI, rowsG;           // original row of each interior / interface unknown
  DBuf E_rp, E_ci, E_va, E_t, F_rp, F_ci, F_va, F_t, C_rp, C_ci, C_va, C_t;
  DevCsr E, F, C;
  DBuf f, u, t, xi, g, s, w, y, r, part0, part1;
  // the interface GMRES iteration's right preconditioner (silu_schur_set_interface_prec):
  // 0 none (the paper's iteration), 1 diag(C); 1 / c_kk and its scratch vector
  int iface_prec = 0;
  bool cdiag_ok = false;
  DBuf cdinv, q;
  ~SchurState();
};

struct silu_ilu_s {
  silu_ctx ctx = nullptr;
  silu_mat A = nullptr;
  silu_kind kind = SILU_ILU0;
  silu_scale scale = SILU_SCALE_ROW;
  silu_prec prec = SILU_FP64;
  double tau = 0.0;
  int fill = 0;
  silu::Factors F;
  silu::Csr Us;
  std::vector<double> dinv;  // D^{-1} (row scaling), or D_r (row/column scaling)
  std::vector<double> dcol;  // D_c (row/column scaling only)
  int ruiz_steps = 0;
  std::vector<int32_t> levL, levU, levLptr, levLrows, levUptr, levUrows;
  int32_t nlevL = 0, nlevU = 0;
  // device: sweep factors, and their length-sorted copies where those pay
  DBuf L_rp, L_ci, L_va, L_tiles, U_rp, U_ci, U_va, U_tiles, d_dinv, d_dcol;
  SortedBufs Lsort, Usort;
  bool sorted_ready = false;  // sorted copies built (where they pay) for the current values
  double pad_nat[2] = {0.0, 0.0}, pad_sorted[2] = {0.0, 0.0};  // L_s, upper sweep factor
  std::vector<double> tune_ms;  // per autotuner candidate, last tuning (-1: not run)
  DevCsr dL, dU;
  // device: FP64 L_s and Utilde_s for the direct path (aliases of dL/dU when possible)
  DBuf L64_va, S_rp, S_ci, S_va, S_tiles, levLrows_d, levUrows_d;
  DevCsr dL64, dS64;
  bool direct_ready = false;
  int level_overlap = -1;  // levels launched as programmatic dependents: -1 undecided, 0 no, 1 yes
  // persistent exact solves (kernels_trisolve.cu): level-ordered copies of L_s
  // and the scaled strict upper factor, the item list, and per column count
  // R = 1, 2, 4 the tagged vectors and the launch state
  int direct_mode = 0;  // 0 automatic, 1 one launch per level, 2 one persistent launch per application
  int fused_mode = 0;   // smoother in one cooperative launch: 0 for small systems, 1 never, 2 always
  int direct_choice[3] = {0, 0, 0};  // automatic: schedule kept per column count (0 undecided)
  DBuf tri_items, tri_lrp, tri_lci, tri_lva, tri_urp, tri_uci, tri_uva;
  DBuf tri_y[3], tri_v[3], tri_state[3];
  silu::TriPlan tri;
  int lanesL = 0, lanesU = 0, lanesA = 0;
  int64_t config_gen = 0;  // bumped whenever a launch shape changes (captured graphs go stale)
  int variant = 0;  // 0 auto, 1 plain lanes-per-row kernel, 2 staged kernel where possible
  int autoL = 4, autoU = 4, autoA = 8;
  Workspace ws;
  std::unique_ptr<AmgState> amg;  // silu_amg_setup
  std::unique_ptr<SchurState> schur;  // silu_schur_setup
};

// An NVTX range around a public call, so timeline profilers show the library's
// phases (no effect unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// The upper sweep factor is a unit-diagonal scaled copy (F->Us) rather than raw U.
inline bool scaled_upper(const silu_ilu_s* F) {
  return F->scale == SILU_SCALE_ROW || F->scale == SILU_SCALE_ROWCOL;
}

namespace silu {

inline silu_status set_err(silu_ctx ctx, silu_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

inline silu_status cuda_err(silu_ctx ctx, cudaError_t e, const char* what) {
  return set_err(ctx, e == cudaErrorMemoryAllocation ? SILU_ERR_OOM : SILU_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

struct CudaFail {
  cudaError_t e;
  const char* what;
};

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) throw CudaFail{e_, #call}; \
  } while (0)

// Counts a kernel launch and, while profiling, brackets it with events.
// Opens a record for a launch of class cls: its start event on the
// context's stream.  Returns the record index, or -1 if no event is free.
inline long prof_open(silu_ctx ctx, int cls) {
  const size_t k = ctx->nrec;
  if (ctx->events.size() < 2 * (k + 1)) {
    for (int t = 0; t < 2; ++t) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return -1;
      ctx->events.push_back(ev);
    }
  }
  if (ctx->rec_class.size() <= k) {
    ctx->rec_class.resize(k + 1);
    ctx->rec_count.resize(k + 1);
  }
  ctx->rec_class[k] = cls;
  ctx->rec_count[k] = 1;
  ctx->nrec = k + 1;
  cudaEventRecord(ctx->events[2 * k], ctx->stream);
  return (long)k;
}

// Times one launch (when profiling): start and end events around it, or,
// inside a ProfRun of the same class, one more launch of the run's record.
struct ProfScope {
  silu_ctx ctx;
  long k = -1;
  ProfScope(silu_ctx c, int cls) : ctx(c) {
    ctx->launches++;
    if (!ctx->profiling) return;
    if (ctx->run_class == cls) {
      if (ctx->run_rec >= 0)
        ctx->rec_count[(size_t)ctx->run_rec]++;
      else
        ctx->run_rec = prof_open(ctx, cls);
      return;
    }
    k = prof_open(ctx, cls);
  }
  ~ProfScope() {
    if (k >= 0) cudaEventRecord(ctx->events[2 * (size_t)k + 1], ctx->stream);
  }
};

// Consecutive launches of one class (the sweeps of one factor in one
// smoother application) timed as one record: events between them would stop
// each sweep from starting while the previous one drains.
struct ProfRun {
  silu_ctx ctx;
  ProfRun(silu_ctx c, int cls) : ctx(c) {
    ctx->run_class = cls;
    ctx->run_rec = -1;
  }
  ~ProfRun() {
    if (ctx->run_rec >= 0) cudaEventRecord(ctx->events[2 * (size_t)ctx->run_rec + 1], ctx->stream);
    ctx->run_class = -1;
    ctx->run_rec = -1;
  }
};

#define LAUNCH(ctx, cls, call)        \
  do {                                \
    ProfScope ps_((ctx), (cls));      \
    CK(call);                         \
  } while (0)


inline int pick_lanes(const silu::Csr& T) {
  const double avg = T.n ? (double)T.nnz() / (double)T.n : 0.0;
  int g = 1;
  while (g < 32 && g < avg) g <<= 1;
  return std::max(2, g);
}

template <class T>
cudaError_t upload(DBuf& b, const T* src, size_t count, cudaStream_t s) {
  cudaError_t e = b.ensure(sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  return cudaMemcpyAsync(b.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, s);
}

// Upload CSR (int64 row pointers narrowed to int32) with values as double or
// float.  Arrays get kCsrPad spare (zeroed) elements for the staged kernel's

cudaError_t upload_csr(const Csr& T, bool fp32, DBuf& rp, DBuf& ci, DBuf& va, DBuf& tiles, DevCsr& d,
                       cudaStream_t s);
// The tile entry limit of the automatic launch shape: narrow tiles for FP64
// values with one lane per row whose rows fit them (silu::narrow_fits).
int auto_tile_nnz(const Csr& T, bool fp32, int lanes, int passes);
// Length-sorted copy of T for the staged kernel (silu::make_sorted); clears
// the copy in d when it would not pay.
cudaError_t upload_sorted(const Csr& T, bool fp32, SortedBufs& b, DevCsr& d, cudaStream_t s);
// Upload L_s and the upper sweep factor of F with their sorted copies,
// keeping the launch shapes chosen earlier (autotuner, variant).
cudaError_t upload_factors(silu_ilu F);
// Build the length-sorted copies of the sweep factors (once; where they pay).
cudaError_t ensure_sorted(silu_ilu F);
silu_status device_ok(silu_ctx ctx);
cudaError_t ensure_vectors(silu_ilu F, int nrhs);
cudaError_t ensure_krylov(silu_ilu F, int m);
cudaError_t ensure_direct(silu_ilu F);
// The captured level-by-level exact solve of one column block (built and
// cached on first use; settles whether levels overlap).
cudaGraphExec_t level_graph(silu_ilu F, int R, int ldx, size_t col);
// Level-ordered factor copies and items of the persistent exact solves.
cudaError_t build_tri_plan(silu_ilu F);
// Tagged vectors and launch state of the persistent solve for R columns.
cudaError_t ensure_tri(silu_ilu F, int R);
int tri_slot(int R);
// Automatic schedule: time both on R columns once and keep the faster.
cudaError_t decide_direct(silu_ilu F, int R);
inline int lanes_of(int fixed, int autov) { return fixed > 0 ? fixed : autov; }
cudaError_t sweep_launch(silu_ilu F, const DevCsr& T, Mode mode, int R, int lanes, int ldx, const void* c,
                         const void* in, void* out, const double* dinv, double* x, int epi);
// One smoother application on columns [0, R) (leading dimension ldx, workspace
// column offset col); x_zero: zero initial guess, x is written, not updated.
void smooth_chunk(silu_ilu F, double* x, const double* b, int R, int ldx, size_t col, int mL, int mU, bool x_zero);
// The same update with level-scheduled exact solves.  `inline_levels`
// launches the level kernels directly instead of through the cached graph
// (used while a stream capture is recording).
void direct_chunk(silu_ilu F, double* x, const double* b, int R, int ldx, size_t col, bool x_zero,
                  bool inline_levels = false);
// One AMG V-cycle (Alg. mgcycle) on A x = b for one right-hand side, the
// finest level smoothed by m_L + m_U sweeps of F's smoother, by its exact
// triangular solves when mL < 0, or, with schur, by one application of F's
// Schur complement smoother (m_L + m_U sweeps in its blocks) before and after
// the coarse-grid correction (x_zero: x is an output, the cycle starts from
// zero; capturing: a stream capture is recording).  Requires F->amg (and
// F->schur with schur) and F's one-column workspace (and amg_prepare_direct
// for mL < 0).  Levels with an ILU smoother of their own are smoothed the way
// the finest level is (sweeps, or exact solves when mL < 0; sweeps under
// schur).
void amg_cycle(silu_ilu F, double* x, const double* b, int mL, int mU, bool x_zero, bool capturing,
               bool schur = false);
// Before a cycle with exact triangular solves (mL < 0) runs or is captured:
// F's and every ILU level's direct-solve data and launch form (ensure_direct).
cudaError_t amg_prepare_direct(silu_ilu F);
// z = M^{-1} r of F's Schur complement smoother (one right-hand side,
// device vectors of n entries; z is written).  Requires F->schur.
void schur_apply(silu_ilu F, const double* r, double* z, int mL, int mU);
// Systems of at most this many rows apply the smoother in one fused
// cooperative launch by default (silu_ilu_set_fused).
constexpr int64_t kFusedMaxRows = 131072;
// Ruiz equilibration limits for SILU_SCALE_ROWCOL.
constexpr int kRuizMaxit = 20;
constexpr double kRuizTol = 1e-2;
// Unit-diagonal copy of the upper factor (row or row/column scaling) into
// F->Us, F->dinv (and F->dcol); returns a silu::HostStatus.
int scale_upper(silu_ilu F, std::string& msg);
// Scale, level sets, launch shapes and upload for F->F already factored.
silu_status finish_setup(silu_ilu F);

}  // namespace silu
