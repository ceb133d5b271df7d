// Internal device-side declarations of libsilu: buffers, matrices in device
// memory, and the launchers of the sm_103a kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace silu {

// Epilogues of the sweep kernel.  Each computes, for row i and column r,
// s = sum_j T_ij in_j and then writes:
enum Epi : int {
  EPI_STORE = 0,       // out = c - s
  EPI_SCALE = 1,       // out = dinv_i (c - s)                       (last L sweep -> D^{-1} y)
  EPI_ADDX = 2,        // x += c - s                                 (last U sweep, fused update)
  EPI_SCALE_ADDX = 3,  // x += dinv_i (c - s)                        (last L sweep when m_U = 1)
  EPI_JAC = 4,         // out = in_i + dinv_i (c - s)                (Jacobi on raw U, Eq. LUiterMat)
  EPI_JAC_ADDX = 5,    // x += in_i + dinv_i (c - s)
  EPI_RICH = 6,        // out = c - s + in_i                         (plain Richardson on raw U)
  EPI_RICH_ADDX = 7,   // x += c - s + in_i
  EPI_SPMV = 8,        // out = s
  EPI_SCALE_SETX = 9,  // x = dinv_i (c - s)                         (zero initial guess)
  EPI_SETX = 10,       // x = c - s
  EPI_JAC_SETX = 11,   // x = in_i + dinv_i (c - s)
  EPI_RICH_SETX = 12   // x = c - s + in_i
};

// Arithmetic mode of a sweep launch.
enum Mode : int {
  MODE_D = 0,   // FP64 matrix, FP64 vectors
  MODE_F = 1,   // FP32 matrix, FP32 vectors, FP32 accumulation
  MODE_DF = 2   // FP64 matrix and input vectors, FP32 output (residual feeding FP32 sweeps)
};

// Staged-sweep tile limits (entries per warp tile; a tile has
// 32 * passes / lanes rows).  The CSR arrays of a tiled matrix are allocated with kCsrPad spare
// elements so that copies rounded out to 16-byte boundaries stay inside the
// allocation.
constexpr int kTileNnz = 424;
constexpr int kTileRows = 32;
constexpr int kCsrPad = 8;
// Narrow tiles (FP64 values, one lane per row, rows of at most
// kNarrowChunkRows entries and kNarrowMeanRow on average): at most
// kTileNnzNarrow - 8 entries per tile, swept by 24 warps per CTA with
// kNarrowChunkRows gathers in flight per lane.
constexpr int kTileNnzNarrow = 360;
constexpr int kNarrowChunkRows = 10;
constexpr double kNarrowMeanRow = 9.0;

struct DevCsr {
  int n = 0;
  int64_t nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  void* va = nullptr;   // double or float
  bool fp32 = false;
  // warp tiles for the staged sweep kernel: tile t is the descriptor
  // {r0, r1, p0, p1} of rows [r0, r1) and entries [p0, p1): at most
  // kTileRows rows (one per lane of a warp) and kTileNnz - 8 entries;
  // ntiles = 0 when some row is too long to stage (the lanes-per-row kernel
  // is used then)
  int4* tiles = nullptr;
  int ntiles = 0;
  // length-sorted copy for the staged kernel (rows of each kSortWindow-row
  // window in descending length, perm = their row numbers; nstiles = 0 when
  // there is none); swept instead of the natural order when use_sorted, with
  // one lane per row
  int* srp = nullptr;
  int* sci = nullptr;
  void* sva = nullptr;
  int* perm = nullptr;
  int4* stiles = nullptr;
  int nstiles = 0;
  bool use_sorted = false;
  int tile_lanes = 1;  // lanes per row in the staged kernel (1, 2 or 4)
  int tile_passes = 1; // rows per lane in a tile (1, 2 or 4; only with one lane per row)
  int chunk = 16;      // entries gathered per lane before the FMAs (8 or 16)
  int tile_nnz = kTileNnz;  // the entry limit the tiles were cut with (kTileNnzNarrow: narrow configuration)
};


// Lanes per row for the staged kernel from the mean row length: one lane per
// row up to 16 entries, two up to 32, four beyond (each warp-wide FMA then
// carries about as many useful entries as the longest row allows).
int staged_lanes(const int64_t* rp, int64_t n);
// Rows per lane with one lane per row: 4 for rows of about 3 entries, 2 up
// to about 6, else 1 (so that a tile's bulk copies stay a few KB).
int staged_passes(const int64_t* rp, int64_t n, int lanes);

// Rows of every kSortWindow consecutive rows are sorted by length for the
// sorted copy; it is made when tiles of consecutive rows would spend more
// than kSortPadMin FMA slots per entry and sorting removes at least
// kSortGain of them.
constexpr int kSortWindow = 512;
constexpr double kSortPadMin = 1.08;
constexpr double kSortGain = 0.05;

// FMA slots per stored entry of one-lane-per-row tiles of a row pointer: a
// tile costs 32 lanes times its longest row.  0 when some row is too long.
double tile_pad(const int64_t* rp, int64_t n);
// Rows of each kSortWindow-row window in descending length (stable): perm[s]
// is the original row of stored row s, srp the sorted row pointer.
void window_sort(const int64_t* rp, int64_t n, std::vector<int32_t>& perm, std::vector<int64_t>& srp);
// The sorted copy is made for tile_pad values natural -> sorted when this holds.
bool sorting_pays(double natural, double sorted);
// Length-sorted copy of a CSR matrix (host): returns false when it would not
// pay (see above).
bool make_sorted(const int64_t* rp, const int32_t* ci, const double* va, int64_t n, std::vector<int64_t>& srp,
                 std::vector<int32_t>& sci, std::vector<double>& sva, std::vector<int32_t>& perm);

// Build the warp-tile descriptors of a CSR row pointer (host), four ints per
// tile, for `lanes` lanes per row and `passes` rows per lane (32 * passes /
// lanes rows per tile).  Returns false if a row has more than kTileNnz - 8
// entries.
bool make_tiles(const int64_t* rp, int64_t n, int lanes, int passes, std::vector<int>& desc,
                int max_nnz = kTileNnz);
// Whether a row pointer suits the narrow configuration (see kTileNnzNarrow).
bool narrow_fits(const int64_t* rp, int64_t n);

// L2 flags of a staged sweep launch.  kFlagReverse: walk the tiles last to
// first (set on every other staged launch of a context when LaunchEnv::l2
// has it).
// kFlagFactorNormal: factor copies at normal L2 priority (else evict-first).
// kFlagVectorNormal: vector loads and stores at normal priority (else
// evict-last).  None of them changes a result bit.
constexpr int kFlagReverse = 1;
constexpr int kFlagFactorNormal = 2;
constexpr int kFlagVectorNormal = 4;
constexpr int kL2Default = kFlagReverse;

// Device-side state shared by launches on one context.
struct LaunchEnv {
  int sms = 0;          // multiprocessors of the device
  int* err = nullptr;   // err[0]: device error word (bit 0: a copy wait gave up,
                        // bit 1: the self-test wait gave up, bit 2: a wait of
                        // the persistent triangular solve gave up, bit 3: a
                        // grid barrier of the fused smoother gave up); err[1]:
                        // a flag that nothing sets (self-test); err[2..3]: the
                        // fused smoother's grid-barrier words
  bool overlap = true;  // staged sweeps launched as programmatic dependents of
                        // the kernel before them (prologue overlaps its tail)
  int l2 = kL2Default;  // L2 reuse flags of staged sweeps (kFlag* above)
  // staged launches made so far (host side): with alternating directions,
  // odd launches walk the tiles backwards
  mutable unsigned flips = 0;
};

#ifdef __CUDACC__
// Programmatic dependent launch: let the next kernel in the stream be
// scheduled now, and wait here until the kernel before this one has completed
// and its writes are visible.  Both are no-ops for a kernel not launched as a
// programmatic dependent.
__device__ __forceinline__ void grid_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_wait_prior() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Self-test of the bounded-wait error path (one thread, no fault).
cudaError_t launch_wait_flag(const int* flag, unsigned long long timeout_ns, int* err, cudaStream_t s);

// Launch out/x = epilogue(c - T in) over all rows.  Vectors are row-major
// with leading dimension ldx; the launch covers columns [0, R) of the
// pointers given (callers offset them).  lanes = threads per row.
cudaError_t launch_sweep(const DevCsr& T, Mode mode, int R, int lanes, int ldx, const void* c, const void* in,
                         void* out, const double* dinv, double* x, int epi, cudaStream_t s);

// Same result (one right-hand side), staged kernel: persistent CTAs stream
// row tiles of T into shared memory with bulk asynchronous copies.
cudaError_t launch_sweep_staged(const DevCsr& T, Mode mode, const LaunchEnv& env, const void* c, const void* in,
                                void* out, const double* dinv, double* x, int epi, cudaStream_t s);
// The staged sweep for R = 2 or 4 interleaved right-hand sides (leading
// dimension ldx >= R): each staged factor entry feeds R FMAs.  Needs a tile
// partition with one lane per row (staged_multi_ok); natural row order.
bool staged_multi_ok(const DevCsr& T, int R);
cudaError_t launch_sweep_staged_multi(const DevCsr& T, Mode mode, const LaunchEnv& env, int R, int ldx, const void* c,
                                      const void* in, void* out, const double* dinv, double* x, int epi,
                                      cudaStream_t s);
// Opt every staged-kernel instantiation into its shared-memory size on the
// current device (done once per context, before any stream capture).
cudaError_t staged_prepare();

// Level-scheduled substitution over the rows listed in rows[0..nrows).
//  lower:  y_i -= sum_j T_ij y_j ; if c_out: c_out_i = dinv_i y_i
//  upper:  y_i -= sum_j T_ij y_j ; if x: x_i += y_i
// overlap: launched as a programmatic dependent of the previous level.
cudaError_t launch_level(const DevCsr& T, const int* rows, int nrows, int R, int lanes, int ldx, double* y,
                         const double* dinv, double* c_out, double* x, bool overlap, cudaStream_t s);

// Both exact triangular solves of one application in one persistent launch
// (kernels_trisolve.cu).  Rows of L_s and of the scaled strict upper factor
// are stored in level order (row numbers in rowsL / rowsU, columns
// unchanged); items are runs of at most 32 level-ordered rows of one level,
// {first, last + 1, gate row or -1, gate in the upper solve}, the nitemsL
// lower items first, then the upper ones.
struct TriPlan {
  int nitemsL = 0, nitems = 0;
  int window = 0;  // items worth keeping in flight: the widest level's items times the gate distance + 1
  const int* items = nullptr;  // 4 ints per item
  const int* rowsL = nullptr;
  const int* lrp = nullptr;
  const int* lci = nullptr;
  const double* lva = nullptr;
  const int* rowsU = nullptr;
  const int* urp = nullptr;
  const int* uci = nullptr;
  const double* uva = nullptr;
};
// y = L^{-1} r, c = dinv (.) y, v = Utilde^{-1} c, x (+)= (dcol (.)) v for R
// right-hand sides (1, 2 or 4; r and x row-major with leading dimensions ldr
// and ldx).  y, v (n x R doubles) and state (4 unsigned) belong to this R for
// the factor object: zeroed once when allocated, then only this launch
// touches them.  A wait that gives up sets bit 2 (value 4) of *err.
cudaError_t launch_trisolve(const TriPlan& P, int R, const double* r, int ldr, const double* dinv, const double* dcol,
                            double* y, double* v, unsigned* state, double* x, int ldx, bool x_zero, int sms, int* err,
                            cudaStream_t s);

// One smoother application with row-scaled (rowcol: row/column scaled)
// factors in one cooperative launch (kernels_fused.cu): the residual, the
// sweeps on Ls and Us and the update of x, separated by grid-wide barriers
// on bar[0..1] (two words zeroed once; each barrier leaves them consistent).
// Same step sequence and vectors (r, c, p0, p1: the workspace, FP32 when
// f32) as the launch-per-sweep path.  A barrier wait that gives up sets bit
// 3 (value 8) of *err.
cudaError_t launch_smooth_fused(const DevCsr& A, const DevCsr& Ls, const DevCsr& Us, bool f32, int R, int ldx,
                                int mL, int mU, bool x_zero, bool rowcol, const double* dinv, const double* dcol,
                                const double* b, double* x, void* r, void* c, void* p0, void* p1, unsigned* bar,
                                int sms, int* err, cudaStream_t s);

// Elementwise helpers over n rows x R columns (leading dimension ldx).
//  out(float or double) = scale ? dinv_i in : in      (in: double or float)
cudaError_t launch_scale(int n, int R, int ldx, const void* in, bool in_f32, const double* dinv, void* out,
                         bool out_f32, cudaStream_t s);
//  x (+)= (dinv_i) in
cudaError_t launch_addx(int n, int R, int ldx, const void* in, bool in_f32, const double* dinv, double* x,
                        bool accumulate, cudaStream_t s);

}  // namespace silu
