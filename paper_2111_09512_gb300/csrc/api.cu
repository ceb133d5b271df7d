// C ABI of libsilu (declared in include/silu.h): handles, host setup and
// the stream-ordered orchestration of the device kernels.
#include <cstdio>

#include "internal.h"

using namespace silu;

namespace silu {

int auto_tile_nnz(const Csr& T, bool fp32, int lanes, int passes) {
  return (!fp32 && lanes == 1 && passes == 1 && silu::narrow_fits(T.rp.data(), T.n)) ? silu::kTileNnzNarrow
                                                                                      : silu::kTileNnz;
}

// Uploads T (row pointers, columns, values in FP64 or FP32) as
// 16-byte-rounded copies, and builds the row tiles of the staged kernel in
// the automatic launch shape.
cudaError_t upload_csr(const silu::Csr& T, bool fp32, DBuf& rp, DBuf& ci, DBuf& va, DBuf& tiles, DevCsr& d,
                       cudaStream_t s) {
  const size_t n = (size_t)T.n, nnz = (size_t)T.nnz();
  const size_t vs = fp32 ? sizeof(float) : sizeof(double);
  std::vector<int32_t> rp32(T.rp.begin(), T.rp.end());
  cudaError_t e = rp.ensure(sizeof(int32_t) * (n + 1 + silu::kCsrPad));
  if (e == cudaSuccess) e = ci.ensure(sizeof(int32_t) * (nnz + silu::kCsrPad));
  if (e == cudaSuccess) e = va.ensure(vs * (nnz + silu::kCsrPad));
  if (e == cudaSuccess) e = cudaMemsetAsync(rp.p, 0, rp.bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ci.p, 0, ci.bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(va.p, 0, va.bytes, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rp.p, rp32.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz)
    e = cudaMemcpyAsync(ci.p, T.ci.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s);
  std::vector<float> v32;
  if (e == cudaSuccess && nnz) {
    if (fp32) {
      v32.assign(T.va.begin(), T.va.end());
      e = cudaMemcpyAsync(va.p, v32.data(), sizeof(float) * nnz, cudaMemcpyHostToDevice, s);
    } else {
      e = cudaMemcpyAsync(va.p, T.va.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s);
    }
  }
  std::vector<int> tl;
  const int tlanes = silu::staged_lanes(T.rp.data(), T.n);
  const int tpasses = silu::staged_passes(T.rp.data(), T.n, tlanes);
  const int tnnz = auto_tile_nnz(T, fp32, tlanes, tpasses);
  const bool tiled = silu::make_tiles(T.rp.data(), T.n, tlanes, tpasses, tl, tnnz);
  if (e == cudaSuccess && tiled) e = upload(tiles, tl.data(), tl.size(), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging vectors die at return
  d.n = (int)T.n;
  d.nnz = T.nnz();
  d.rp = rp.as<int>();
  d.ci = ci.as<int>();
  d.va = va.p;
  d.fp32 = fp32;
  d.tiles = tiled ? tiles.as<int4>() : nullptr;
  d.ntiles = tiled ? (int)(tl.size() / 4) : 0;
  d.tile_lanes = tlanes;
  d.tile_passes = tpasses;
  d.tile_nnz = tnnz;
  return e;
}

cudaError_t upload_sorted(const Csr& T, bool fp32, SortedBufs& b, DevCsr& d, cudaStream_t s) {
  d.srp = nullptr;
  d.sci = nullptr;
  d.sva = nullptr;
  d.perm = nullptr;
  d.stiles = nullptr;
  d.nstiles = 0;
  d.use_sorted = false;
  std::vector<int64_t> srp;
  std::vector<int32_t> sci, perm;
  std::vector<double> sva;
  if (!silu::make_sorted(T.rp.data(), T.ci.data(), T.va.data(), T.n, srp, sci, sva, perm)) {
    b.rp.release();
    b.ci.release();
    b.va.release();
    b.perm.release();
    b.tiles.release();
    return cudaSuccess;
  }
  Csr S;
  S.n = T.n;
  S.rp.swap(srp);
  S.ci.swap(sci);
  S.va.swap(sva);
  DevCsr sd;
  cudaError_t e = upload_csr(S, fp32, b.rp, b.ci, b.va, b.tiles, sd, s);
  std::vector<int> tl;
  if (e == cudaSuccess && !silu::make_tiles(S.rp.data(), S.n, 1, 1, tl)) return cudaSuccess;
  if (e == cudaSuccess) e = upload(b.tiles, tl.data(), tl.size(), s);
  if (e == cudaSuccess) e = b.perm.ensure(sizeof(int32_t) * (perm.size() + silu::kCsrPad));
  if (e == cudaSuccess) e = cudaMemsetAsync(b.perm.p, 0, b.perm.bytes, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.perm.p, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  d.srp = sd.rp;
  d.sci = sd.ci;
  d.sva = sd.va;
  d.perm = b.perm.as<int>();
  d.stiles = b.tiles.as<int4>();
  d.nstiles = (int)(tl.size() / 4);
  return cudaSuccess;
}

namespace {

// Re-apply a launch shape kept from before an upload: tiles for g lanes per
// row and rl rows per lane, gather width.
cudaError_t keep_shape(const Csr& h, DBuf& tiles, DevCsr& T, const DevCsr& old, cudaStream_t s) {
  T.chunk = old.chunk;
  if (old.tile_lanes == T.tile_lanes && old.tile_passes == T.tile_passes && old.tile_nnz == T.tile_nnz)
    return cudaSuccess;
  // narrow tiles only where the new values' rows still fit them
  const int lim = (old.tile_nnz == silu::kTileNnzNarrow && !silu::narrow_fits(h.rp.data(), h.n)) ? silu::kTileNnz
                                                                                                 : old.tile_nnz;
  std::vector<int> tl;
  if (!silu::make_tiles(h.rp.data(), h.n, old.tile_lanes, old.tile_passes, tl, lim)) return cudaSuccess;
  cudaError_t e = upload(tiles, tl.data(), tl.size(), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    T.tiles = tiles.as<int4>();
    T.ntiles = (int)(tl.size() / 4);
    T.tile_lanes = old.tile_lanes;
    T.tile_passes = old.tile_passes;
    T.tile_nnz = lim;
  }
  return e;
}

}  // namespace

cudaError_t ensure_sorted(silu_ilu F) {
  if (F->sorted_ready) return cudaSuccess;
  cudaStream_t s = F->ctx->stream;
  const bool f32 = F->prec == SILU_FP32;
  const Csr& Ut = scaled_upper(F) ? F->Us : F->F.U;
  F->ws.drop_graphs();
  F->config_gen++;
  cudaError_t e = upload_sorted(F->F.L, f32, F->Lsort, F->dL, s);
  if (e == cudaSuccess) e = upload_sorted(Ut, f32, F->Usort, F->dU, s);
  if (e == cudaSuccess) F->sorted_ready = true;
  return e;
}

cudaError_t upload_factors(silu_ilu F) {
  cudaStream_t s = F->ctx->stream;
  const bool f32 = F->prec == SILU_FP32;
  const Csr& Ut = scaled_upper(F) ? F->Us : F->F.U;
  const bool had = F->dL.rp != nullptr;
  const DevCsr oldL = F->dL, oldU = F->dU;
  F->ws.drop_graphs();  // captured launches refer to the shapes and arrays replaced here
  F->config_gen++;
  cudaError_t e = upload_csr(F->F.L, f32, F->L_rp, F->L_ci, F->L_va, F->L_tiles, F->dL, s);
  if (e == cudaSuccess) e = upload_csr(Ut, f32, F->U_rp, F->U_ci, F->U_va, F->U_tiles, F->dU, s);
  if (e == cudaSuccess && F->sorted_ready) {  // sorted copies in use: rebuild them from the new values
    F->sorted_ready = false;
    e = ensure_sorted(F);
  }
  if (e == cudaSuccess && had) e = keep_shape(F->F.L, F->L_tiles, F->dL, oldL, s);
  if (e == cudaSuccess && had) e = keep_shape(Ut, F->U_tiles, F->dU, oldU, s);
  return e;
}

silu_status device_ok(silu_ctx ctx) {
  if (!ctx) return SILU_ERR_INVALID_ARG;
  if (ctx->device < 0) return set_err(ctx, SILU_ERR_NO_DEVICE, "host-only context");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  return SILU_OK;
}

cudaError_t ensure_vectors(silu_ilu F, int nrhs) {
  const size_t bytes = sizeof(double) * (size_t)F->F.L.n * (size_t)nrhs;
  Workspace& w = F->ws;
  if (bytes <= w.vec_bytes && w.r.p) return cudaSuccess;
  w.drop_graphs();
  cudaError_t e;
  if ((e = w.r.ensure(bytes)) != cudaSuccess) return e;
  if ((e = w.c.ensure(bytes)) != cudaSuccess) return e;
  if ((e = w.p0.ensure(bytes)) != cudaSuccess) return e;
  if ((e = w.p1.ensure(bytes)) != cudaSuccess) return e;
  w.vec_bytes = bytes;
  return cudaSuccess;
}

cudaError_t ensure_krylov(silu_ilu F, int m) {
  Workspace& w = F->ws;
  if (m <= w.restart && w.V.p) return cudaSuccess;
  w.drop_graphs();
  const size_t n = (size_t)F->F.L.n;
  cudaError_t e;
  if ((e = w.V.ensure(sizeof(double) * n * (size_t)(m + 1))) != cudaSuccess) return e;
  if ((e = w.Z.ensure(sizeof(double) * n * (size_t)m)) != cudaSuccess) return e;
  if ((e = w.w.ensure(sizeof(double) * n)) != cudaSuccess) return e;
  if ((e = w.H.ensure(sizeof(double) * (size_t)(m + 1) * (size_t)m)) != cudaSuccess) return e;
  if ((e = w.cs.ensure(sizeof(double) * (size_t)m)) != cudaSuccess) return e;
  if ((e = w.sn.ensure(sizeof(double) * (size_t)m)) != cudaSuccess) return e;
  if ((e = w.g.ensure(sizeof(double) * (size_t)(m + 1))) != cudaSuccess) return e;
  if ((e = w.yk.ensure(sizeof(double) * (size_t)m)) != cudaSuccess) return e;
  if ((e = w.part0.ensure(sizeof(double) * 1024)) != cudaSuccess) return e;
  if ((e = w.part1.ensure(sizeof(double) * 1024)) != cudaSuccess) return e;
  if ((e = w.scal.ensure(sizeof(double) * 8)) != cudaSuccess) return e;
  w.restart = m;
  return cudaSuccess;
}

namespace {

// Rows of T (strict triangle, FP64) in the order level_rows lists them: row
// pointers and columns as int32, values as FP64, each row's entries kept in
// column order.
void level_copy(const Csr& T, const std::vector<int32_t>& level_rows, std::vector<int32_t>& rp,
                std::vector<int32_t>& ci, std::vector<double>& va) {
  const int64_t n = T.n;
  rp.assign((size_t)n + 1, 0);
  for (int64_t k = 0; k < n; ++k) {
    const int32_t i = level_rows[(size_t)k];
    rp[(size_t)k + 1] = rp[(size_t)k] + (int32_t)(T.rp[i + 1] - T.rp[i]);
  }
  ci.resize((size_t)T.nnz());
  va.resize((size_t)T.nnz());
  for (int64_t k = 0; k < n; ++k) {
    const int32_t i = level_rows[(size_t)k];
    std::copy(T.ci.begin() + T.rp[i], T.ci.begin() + T.rp[i + 1], ci.begin() + rp[(size_t)k]);
    std::copy(T.va.begin() + T.rp[i], T.va.begin() + T.rp[i + 1], va.begin() + rp[(size_t)k]);
  }
}

// Levels between an item and the row it waits on before reading its entries.
constexpr int kTriGateLevels = 3;

// Items of at most 32 consecutive level-ordered rows of one level, four
// ints each: first and last + 1 level-ordered position, the gate row and
// whether the gate is a row of the upper solve.  The gate of the item at
// offset o within level l >= g (g = kTriGateLevels) is the first row of the
// item at offset min(o, items(l-g) - 1) of level l-g (items of one level
// spread their gates over that level); levels below g have none (-1).
int level_items(const std::vector<int32_t>& level_ptr, const std::vector<int32_t>& level_rows, int upper,
                std::vector<int32_t>& items) {
  std::vector<int32_t> lev_first;  // first item (local index) of each level, then the end
  const size_t base = items.size() / 4;
  size_t local = 0;
  for (size_t l = 0; l + 1 < level_ptr.size(); ++l) {
    lev_first.push_back((int32_t)local);
    local += (size_t)((level_ptr[l + 1] - level_ptr[l] + 31) / 32);
  }
  lev_first.push_back((int32_t)local);
  for (size_t l = 0; l + 1 < level_ptr.size(); ++l) {
    int32_t o = 0;
    for (int32_t b = level_ptr[l]; b < level_ptr[l + 1]; b += 32, ++o) {
      items.push_back(b);
      items.push_back(std::min(b + 32, level_ptr[l + 1]));
      int32_t gate = -1;
      if (l >= (size_t)kTriGateLevels) {
        const size_t g = l - (size_t)kTriGateLevels;
        const int32_t cnt = lev_first[g + 1] - lev_first[g];
        const int32_t gi = lev_first[g] + std::min(o, cnt - 1);  // local item of level l - kTriGateLevels
        gate = level_rows[(size_t)items[(base + (size_t)gi) * 4]];
      }
      items.push_back(gate);
      items.push_back(upper);
    }
  }
  int widest = 0;  // items of the widest level
  for (size_t l = 0; l + 1 < lev_first.size(); ++l) widest = std::max(widest, lev_first[l + 1] - lev_first[l]);
  return widest;
}

}  // namespace

// Level-ordered copies of L_s and of the scaled strict upper factor, and the
// item list of the persistent solve (Sec. 4's level sets, one launch).
cudaError_t build_tri_plan(silu_ilu F) {
  cudaStream_t s = F->ctx->stream;
  std::vector<int32_t> rp, ci, items;
  std::vector<double> va;
  const int wideL = level_items(F->levLptr, F->levLrows, 0, items);
  const int nitemsL = (int)(items.size() / 4);
  const int wideU = level_items(F->levUptr, F->levUrows, 1, items);
  cudaError_t e = upload(F->tri_items, items.data(), items.size(), s);
  // uploads are stream-ordered copies from these host vectors: wait before reusing them
  level_copy(F->F.L, F->levLrows, rp, ci, va);
  if (e == cudaSuccess) e = upload(F->tri_lrp, rp.data(), rp.size(), s);
  if (e == cudaSuccess) e = upload(F->tri_lci, ci.data(), ci.size(), s);
  if (e == cudaSuccess) e = upload(F->tri_lva, va.data(), va.size(), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  level_copy(F->Us, F->levUrows, rp, ci, va);
  e = upload(F->tri_urp, rp.data(), rp.size(), s);
  if (e == cudaSuccess) e = upload(F->tri_uci, ci.data(), ci.size(), s);
  if (e == cudaSuccess) e = upload(F->tri_uva, va.data(), va.size(), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  silu::TriPlan& P = F->tri;
  P.nitemsL = nitemsL;
  P.nitems = (int)(items.size() / 4);
  // more warps than the items of a few levels would only wait on their gates
  P.window = std::max(wideL, wideU) * (kTriGateLevels + 1);
  P.items = F->tri_items.as<int>();
  P.rowsL = F->levLrows_d.as<int>();
  P.lrp = F->tri_lrp.as<int>();
  P.lci = F->tri_lci.as<int>();
  P.lva = F->tri_lva.as<double>();
  P.rowsU = F->levUrows_d.as<int>();
  P.urp = F->tri_urp.as<int>();
  P.uci = F->tri_uci.as<int>();
  P.uva = F->tri_uva.as<double>();
  return cudaSuccess;
}

int tri_slot(int R) { return R == 1 ? 0 : (R == 2 ? 1 : 2); }

// The tagged vectors and launch state of the persistent solve for R columns
// (allocated and zeroed once per factor object; never during a capture).
cudaError_t ensure_tri(silu_ilu F, int R) {
  const int k = tri_slot(R);
  if (F->tri_state[k].p) return cudaSuccess;
  cudaStream_t s = F->ctx->stream;
  const size_t vb = sizeof(double) * (size_t)std::max<int64_t>(F->F.L.n, 1) * (size_t)R;
  cudaError_t e = F->tri_y[k].ensure(vb);
  if (e == cudaSuccess) e = F->tri_v[k].ensure(vb);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->tri_y[k].p, 0, vb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->tri_v[k].p, 0, vb, s);
  DBuf st;
  if (e == cudaSuccess) e = st.ensure(4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(st.p, 0, 4 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  std::swap(F->tri_state[k].p, st.p);
  std::swap(F->tri_state[k].bytes, st.bytes);
  return cudaSuccess;
}

// With the automatic schedule, time one direct application of R columns
// (from zero, on workspace vectors) under each schedule and keep the faster
// for R (same results either way up to the rounding of the tagged entries).
cudaError_t decide_direct(silu_ilu F, int R) {
  const int k = tri_slot(R);
  if (F->direct_mode != 0 || F->direct_choice[k] != 0) return cudaSuccess;
  cudaError_t e = ensure_vectors(F, R);
  if (e != cudaSuccess) return e;
  cudaStream_t s = F->ctx->stream;
  const size_t vb = sizeof(double) * (size_t)F->F.L.n * (size_t)R;
  double* bw = F->ws.p0.as<double>();
  double* xw = F->ws.p1.as<double>();
  e = cudaMemsetAsync(bw, 0, vb, s);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float ms[2] = {0.f, 0.f};
  const int64_t launches = F->ctx->launches;
  const bool prof = F->ctx->profiling;
  F->ctx->profiling = false;
  try {
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
      F->direct_choice[k] = c == 0 ? 2 : 1;
      direct_chunk(F, xw, bw, R, R, 0, true);  // warm-up (builds the level graph on first use)
      CK(cudaEventRecord(ev[0], s));
      direct_chunk(F, xw, bw, R, R, 0, true);
      CK(cudaEventRecord(ev[1], s));
      CK(cudaEventSynchronize(ev[1]));
      CK(cudaEventElapsedTime(&ms[c], ev[0], ev[1]));
    }
  } catch (const CudaFail& f) {
    e = f.e;
  }
  F->ctx->profiling = prof;
  F->ctx->launches = launches;
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  F->direct_choice[k] = e == cudaSuccess ? (ms[0] <= ms[1] ? 2 : 1) : 0;
  return e;
}

cudaError_t ensure_direct(silu_ilu F) {
  if (F->direct_ready) return cudaSuccess;
  F->ws.drop_graphs();  // captured solves refer to the arrays uploaded here
  cudaStream_t s = F->ctx->stream;
  cudaError_t e = cudaSuccess;
  // FP64 L_s: reuse the sweep copy when it is FP64
  if (F->prec == SILU_FP64) {
    F->dL64 = F->dL;
  } else {
    F->dL64 = F->dL;
    e = F->L64_va.ensure(sizeof(double) * (F->F.L.va.size() + silu::kCsrPad));
    if (e == cudaSuccess) e = cudaMemsetAsync(F->L64_va.p, 0, F->L64_va.bytes, s);
    if (e == cudaSuccess && !F->F.L.va.empty())
      e = cudaMemcpyAsync(F->L64_va.p, F->F.L.va.data(), sizeof(double) * F->F.L.va.size(),
                          cudaMemcpyHostToDevice, s);
    F->dL64.va = F->L64_va.p;
    F->dL64.fp32 = false;
  }
  if (e != cudaSuccess) return e;
  // FP64 Utilde_s: reuse when the sweeps use it in FP64
  if (F->prec == SILU_FP64 && scaled_upper(F)) {
    F->dS64 = F->dU;
  } else {
    e = upload_csr(F->Us, false, F->S_rp, F->S_ci, F->S_va, F->S_tiles, F->dS64, s);
    if (e != cudaSuccess) return e;
  }
  e = upload(F->levLrows_d, F->levLrows.data(), F->levLrows.size(), s);
  if (e == cudaSuccess) e = upload(F->levUrows_d, F->levUrows.data(), F->levUrows.size(), s);
  if (e == cudaSuccess) e = build_tri_plan(F);
  if (e == cudaSuccess) e = ensure_tri(F, 1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) F->direct_ready = true;
  for (int& c : F->direct_choice) c = 0;  // the factors changed: decide again
  if (e == cudaSuccess) e = decide_direct(F, 1);
  return e;
}


// One sweep-shaped launch: the staged kernel for a single right-hand side
// when the matrix has a tile partition (and the variant allows it), on the
// length-sorted copy when that is selected, else the lanes-per-row kernel.
cudaError_t sweep_launch(silu_ilu F, const DevCsr& T, silu::Mode mode, int R, int lanes, int ldx, const void* c,
                         const void* in, void* out, const double* dinv, double* x, int epi) {
  cudaStream_t s = F->ctx->stream;
  // several right-hand sides: the staged kernel reads each factor entry once
  // for all R columns; on small systems (fewer tiles than a grid of warps
  // has) its pipeline start costs more than it saves, unless a staged
  // variant was asked for explicitly
  if (R > 1 && F->variant != 1 && silu::staged_multi_ok(T, R) &&
      (F->variant >= 2 || T.ntiles >= F->ctx->env.sms * 16))
    return silu::launch_sweep_staged_multi(T, mode, F->ctx->env, R, ldx, c, in, out, dinv, x, epi, s);
  if (R == 1 && ldx == 1 && T.ntiles > 0 && F->variant != 1) {
    if (F->variant != 3 || T.nstiles == 0) return silu::launch_sweep_staged(T, mode, F->ctx->env, c, in, out, dinv, x, epi, s);
    DevCsr t = T;  // variant 3: the length-sorted copy
    t.use_sorted = true;
    return silu::launch_sweep_staged(t, mode, F->ctx->env, c, in, out, dinv, x, epi, s);
  }
  return silu::launch_sweep(T, mode, R, lanes, ldx, c, in, out, dinv, x, epi, s);
}

// ---------------------------------------------------------------------------
// One smoother application on columns [0, R) of x/b (leading dimension ldx),
// workspace pointers offset by the same column.  x_zero: x is an output only
// (zero initial guess, so r = b and the result is stored, not added).
// ---------------------------------------------------------------------------
// Whether one application of R columns runs as one fused cooperative launch:
// row-scaled factors (row or row/column scaling), R = 1, 2 or 4, and, in the
// automatic mode, several columns of a system small enough that launches
// dominate (with one column the staged sweeps, each launched as a
// programmatic dependent of the one before, are as fast on small systems).
bool use_fused(silu_ilu F, int R) {
  if (F->fused_mode == 1 || !scaled_upper(F) || (R != 1 && R != 2 && R != 4)) return false;
  return F->fused_mode == 2 || (R > 1 && F->F.L.n <= kFusedMaxRows);
}

void smooth_chunk(silu_ilu F, double* x, const double* b, int R, int ldx, size_t col, int mL, int mU, bool x_zero) {
  cudaStream_t s = F->ctx->stream;
  const bool f32 = F->prec == SILU_FP32;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const silu::Mode sm = f32 ? silu::MODE_F : silu::MODE_D;
  const int n = (int)F->F.L.n;
  const double* dinv = F->d_dinv.as<double>();
  const DevCsr& A = F->A->d;
  char* bufR = F->ws.r.as<char>() + col * es;
  char* bufC = F->ws.c.as<char>() + col * es;
  char* bufP0 = F->ws.p0.as<char>() + col * es;
  char* bufP1 = F->ws.p1.as<char>() + col * es;
  if (use_fused(F, R)) {
    const bool rc = F->scale == SILU_SCALE_ROWCOL;
    LAUNCH(F->ctx, SILU_K_FUSED,
           silu::launch_smooth_fused(A, F->dL, F->dU, f32, R, ldx, mL, mU, x_zero, rc, dinv,
                                     rc ? F->d_dcol.as<double>() : nullptr, b, x, bufR, bufC, bufP0, bufP1,
                                     (unsigned*)(F->ctx->env.err + 2), F->ctx->env.sms, F->ctx->env.err, s));
    return;
  }
  const int gL = lanes_of(F->lanesL, F->autoL), gU = lanes_of(F->lanesU, F->autoU), gA = lanes_of(F->lanesA, F->autoA);
  const bool rowscale = scaled_upper(F);
  const bool rowcol = F->scale == SILU_SCALE_ROWCOL;
  const double* dcol = F->d_dcol.as<double>();
  const bool jacobi = F->scale == SILU_SCALE_NONE;

  // What happens to y = L^{-1} r once it is known.
  //   FINAL_Y:   x (+)= y                        (m_U = 0, or m_U = 1 with plain Richardson)
  //   FINAL_DY:  x (+)= D^{-1} y                 (m_U = 1 with row scaling or Jacobi)
  //   NEED_C:    c = D^{-1} y (or D_r y) materialised  (m_U >= 2 with scaling; m_U = 1 with row/column scaling)
  //   NEED_Y:    y materialised                   (m_U >= 2, unscaled variants)
  enum { FINAL_Y, FINAL_DY, NEED_C, NEED_Y } after;
  if (mU == 0 || (mU == 1 && !rowscale && !jacobi))
    after = FINAL_Y;
  else if (mU == 1 && !rowcol)
    after = FINAL_DY;
  else if (rowscale)
    after = NEED_C;
  else
    after = NEED_Y;

  // ---- residual ----------------------------------------------------------
  const void* r = nullptr;
  bool r_fused_to_c = false;
  if (x_zero) {
    if (f32) {
      LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_scale(n, R, ldx, b, false, nullptr, bufR, true, s));
      r = bufR;
    } else {
      r = b;
    }
  } else if (mL <= 1 && after == NEED_C) {
    // r is only needed as D^{-1} r: fuse the scaling into the residual
    LAUNCH(F->ctx, SILU_K_RESIDUAL, sweep_launch(F, A, f32 ? silu::MODE_DF : silu::MODE_D, R, gA, ldx, b, x, bufC, dinv, nullptr,
                          silu::EPI_SCALE));
    r_fused_to_c = true;
  } else {
    LAUNCH(F->ctx, SILU_K_RESIDUAL, sweep_launch(F, A, f32 ? silu::MODE_DF : silu::MODE_D, R, gA, ldx, b, x, bufR, dinv, nullptr,
                          silu::EPI_STORE));
    r = bufR;
  }

  // ---- L sweeps: y^1 = r, y^{k} = r - L_s y^{k-1} -------------------------
  const void* y = r;  // current iterate
  const void* cvec = r_fused_to_c ? (const void*)bufC : nullptr;
  bool done = false;  // x already written
  if (mL >= 2) {
    ProfRun run(F->ctx, SILU_K_SWEEP_L);
    const void* in = r;
    char* pp[2] = {bufP0, bufP1};
    for (int k = 2; k <= mL; ++k) {
      const bool last = (k == mL);
      char* out = pp[k & 1];
      int epi = silu::EPI_STORE;
      void* o = out;
      if (last) {
        if (after == FINAL_Y) {
          epi = x_zero ? silu::EPI_SETX : silu::EPI_ADDX;
          o = nullptr;
        } else if (after == FINAL_DY) {
          epi = x_zero ? silu::EPI_SCALE_SETX : silu::EPI_SCALE_ADDX;
          o = nullptr;
        } else if (after == NEED_C) {
          epi = silu::EPI_SCALE;
          o = bufC;
        }
      }
      LAUNCH(F->ctx, SILU_K_SWEEP_L, sweep_launch(F, F->dL, sm, R, gL, ldx, r, in, o, dinv, x, epi));
      in = out;
      if (last) {
        if (after == FINAL_Y || after == FINAL_DY) done = true;
        if (after == NEED_C) cvec = bufC;
        if (after == NEED_Y) y = out;
      }
    }
  }
  if (!done && after == FINAL_Y) {
    LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_addx(n, R, ldx, y, f32, nullptr, x, !x_zero, s));
    done = true;
  }
  if (!done && after == FINAL_DY) {
    LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_addx(n, R, ldx, y, f32, dinv, x, !x_zero, s));
    done = true;
  }
  if (done) return;

  // ---- U sweeps -----------------------------------------------------------
  if (after == NEED_C) {
    if (!cvec) {  // y = r came without a fused scaling (x_zero, m_L <= 1)
      LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_scale(n, R, ldx, y, f32, dinv, bufC, f32, s));
      cvec = bufC;
    }
    // v^1 = c; v^k = c - Utilde_s v^{k-1}; with row/column scaling the
    // update is x (+)= D_c v (the dcol vector takes dinv's place in the epilogue)
    if (rowcol && mU == 1) {
      LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_addx(n, R, ldx, cvec, f32, dcol, x, !x_zero, s));
      return;
    }
    ProfRun run(F->ctx, SILU_K_SWEEP_U);
    const void* in = cvec;
    char* pp[2] = {bufP0, bufP1};
    for (int k = 2; k <= mU; ++k) {
      const bool last = (k == mU);
      char* out = pp[k & 1];
      int epi = last ? (x_zero ? silu::EPI_SETX : silu::EPI_ADDX) : silu::EPI_STORE;
      if (last && rowcol) epi = x_zero ? silu::EPI_SCALE_SETX : silu::EPI_SCALE_ADDX;
      LAUNCH(F->ctx, SILU_K_SWEEP_U, sweep_launch(F, F->dU, sm, R, gU, ldx, cvec, in, last ? nullptr : out,
                                                  last && rowcol ? dcol : dinv, x, epi));
      in = out;
    }
    return;
  }
  // unscaled variants: c = y (unscaled), two ping-pong buffers distinct from y
  char* cand[4] = {bufC, bufP0, bufP1, bufR};
  char* q[2] = {nullptr, nullptr};
  int nq = 0;
  for (int t = 0; t < 4 && nq < 2; ++t)
    if ((const void*)cand[t] != y) q[nq++] = cand[t];
  const void* in;
  if (jacobi) {
    // v^1 = D^{-1} y
    LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_scale(n, R, ldx, y, f32, dinv, q[0], f32, s));
    in = q[0];
  } else {
    in = y;  // v^1 = y
  }
  ProfRun run(F->ctx, SILU_K_SWEEP_U);
  for (int k = 2; k <= mU; ++k) {
    const bool last = (k == mU);
    char* out = (in == q[0]) ? q[1] : q[0];
    int epi;
    if (jacobi)
      epi = last ? (x_zero ? silu::EPI_JAC_SETX : silu::EPI_JAC_ADDX) : silu::EPI_JAC;
    else
      epi = last ? (x_zero ? silu::EPI_RICH_SETX : silu::EPI_RICH_ADDX) : silu::EPI_RICH;
    LAUNCH(F->ctx, SILU_K_SWEEP_U, sweep_launch(F, F->dU, sm, R, gU, ldx, y, in, last ? nullptr : out, dinv, x, epi));
    in = out;
  }
}

// The level-scheduled substitutions of one column block captured into a CUDA
// graph: one kernel node per level, each depending on the previous one
// (Sec. 4: rows of a level are independent, levels are ordered).  The graph
// works on the workspace vectors only: y (holding r on entry) becomes
// L^{-1} r, c becomes Utilde^{-1} D^{-1} y.  overlap: each level launched as
// a programmatic dependent of the one before.
cudaGraphExec_t capture_levels(silu_ilu F, int R, int ldx, size_t col, bool overlap) {
  cudaStream_t cap = nullptr;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const double* dinv = F->d_dinv.as<double>();
  double* y = F->ws.r.as<double>() + col;
  double* c = F->ws.c.as<double>() + col;
  const int gL = lanes_of(F->lanesL, F->autoL), gU = lanes_of(F->lanesU, F->autoU);
  const int* rowsL = F->levLrows_d.as<int>();
  const int* rowsU = F->levUrows_d.as<int>();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  for (int l = 0; e == cudaSuccess && l < F->nlevL; ++l) {
    const int b0 = F->levLptr[l], b1 = F->levLptr[l + 1];
    e = silu::launch_level(F->dL64, rowsL + b0, b1 - b0, R, gL, ldx, y, dinv, c, nullptr, overlap, cap);
  }
  for (int l = 0; e == cudaSuccess && l < F->nlevU; ++l) {
    const int b0 = F->levUptr[l], b1 = F->levUptr[l + 1];
    e = silu::launch_level(F->dS64, rowsU + b0, b1 - b0, R, gU, ldx, c, dinv, nullptr, nullptr, overlap, cap);
  }
  const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  if (e == cudaSuccess) e = e2;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  CK(e);
  return exec;
}

// Event-timed duration of one launch of a level graph (after one untimed
// launch); it overwrites the workspace vectors y and c of its column block.
float time_levels(silu_ilu F, cudaGraphExec_t exec) {
  cudaStream_t s = F->ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  CK(e);
  return t;
}

// The level graph of one column block (cached).  Whether levels overlap is
// decided once per factor object by timing both captures of the first graph
// built: overlapping helps when levels are small and launch-bound, and can
// cost when they are large; both give the same bits.  Building a graph
// overwrites the workspace vectors y and c of its column block.
cudaGraphExec_t level_graph(silu_ilu F, int R, int ldx, size_t col) {
  for (const LevelGraph& g : F->ws.graphs)
    if (g.R == R && g.ldx == ldx && g.col == col) return g.exec;
  cudaGraphExec_t exec = nullptr;
  if (F->ctx->env.overlap && F->level_overlap < 0) {
    cudaGraphExec_t on = capture_levels(F, R, ldx, col, true);
    cudaGraphExec_t off = nullptr;
    float t_on = 0.f, t_off = 0.f;
    try {
      off = capture_levels(F, R, ldx, col, false);
      t_on = time_levels(F, on);
      t_off = time_levels(F, off);
    } catch (const CudaFail&) {
      cudaGraphExecDestroy(on);
      if (off) cudaGraphExecDestroy(off);
      throw;
    }
    F->level_overlap = t_on < t_off ? 1 : 0;
    exec = F->level_overlap ? on : off;
    cudaGraphExecDestroy(F->level_overlap ? off : on);
  } else {
    exec = capture_levels(F, R, ldx, col, F->ctx->env.overlap && F->level_overlap != 0);
  }
  LevelGraph g;
  g.R = R;
  g.ldx = ldx;
  g.col = col;
  g.exec = exec;
  g.kernels = F->nlevL + F->nlevU;
  F->ws.graphs.push_back(g);
  return exec;
}

// Direct application on columns [0, R): x (+)= Utilde^{-1} D^{-1} L^{-1} (b - A x).
void direct_chunk(silu_ilu F, double* x, const double* b, int R, int ldx, size_t col, bool x_zero,
                  bool inline_levels) {
  cudaStream_t s = F->ctx->stream;
  const int n = (int)F->F.L.n;
  double* y = F->ws.r.as<double>() + col;
  double* c = F->ws.c.as<double>() + col;
  const int gA = lanes_of(F->lanesA, F->autoA);
  const int k = tri_slot(R);
  const int schedule = F->direct_mode != 0 ? F->direct_mode : (F->direct_choice[k] != 0 ? F->direct_choice[k] : 2);
  if (schedule == 2) {
    // both solves and the update of x in one persistent launch
    if (!F->tri_state[k].p) CK(cudaErrorNotReady);  // ensure_tri(F, R) runs before any capture
    const double* r = b;
    if (!x_zero) {
      LAUNCH(F->ctx, SILU_K_RESIDUAL, sweep_launch(F, F->A->d, silu::MODE_D, R, gA, ldx, b, x, y, nullptr, nullptr,
                                                    silu::EPI_STORE));
      r = y;
    }
    const double* dcol = F->scale == SILU_SCALE_ROWCOL ? F->d_dcol.as<double>() : nullptr;  // x += D_c v
    LAUNCH(F->ctx, SILU_K_LEVEL, silu::launch_trisolve(F->tri, R, r, ldx, F->d_dinv.as<double>(), dcol,
                                                       F->tri_y[k].as<double>(), F->tri_v[k].as<double>(),
                                                       F->tri_state[k].as<unsigned>(), x, ldx, x_zero,
                                                       F->ctx->env.sms, F->ctx->env.err, s));
    return;
  }
  // built before y is written: building may run the graph on the workspace
  cudaGraphExec_t exec = inline_levels ? nullptr : level_graph(F, R, ldx, col);
  const bool overlap = F->ctx->env.overlap && F->level_overlap != 0;
  if (x_zero)
    LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_scale(n, R, ldx, b, false, nullptr, y, false, s));
  else
    LAUNCH(F->ctx, SILU_K_RESIDUAL, sweep_launch(F, F->A->d, silu::MODE_D, R, gA, ldx, b, x, y, nullptr, nullptr, silu::EPI_STORE));
  if (inline_levels) {
    const double* dinv = F->d_dinv.as<double>();
    const int gL = lanes_of(F->lanesL, F->autoL), gU = lanes_of(F->lanesU, F->autoU);
    const int* rowsL = F->levLrows_d.as<int>();
    const int* rowsU = F->levUrows_d.as<int>();
    for (int l = 0; l < F->nlevL; ++l) {
      const int b0 = F->levLptr[l], b1 = F->levLptr[l + 1];
      LAUNCH(F->ctx, SILU_K_LEVEL, silu::launch_level(F->dL64, rowsL + b0, b1 - b0, R, gL, ldx, y, dinv, c, nullptr,
                                                        overlap, s));
    }
    for (int l = 0; l < F->nlevU; ++l) {
      const int b0 = F->levUptr[l], b1 = F->levUptr[l + 1];
      LAUNCH(F->ctx, SILU_K_LEVEL, silu::launch_level(F->dS64, rowsU + b0, b1 - b0, R, gU, ldx, c, dinv, nullptr, nullptr,
                                                        overlap, s));
    }
  } else {
    ProfScope ps(F->ctx, SILU_K_LEVEL);
    F->ctx->launches += F->nlevL + F->nlevU - 1;  // one count came from ProfScope
    CK(cudaGraphLaunch(exec, s));
  }
  const double* dcol = F->scale == SILU_SCALE_ROWCOL ? F->d_dcol.as<double>() : nullptr;  // x += D_c v
  LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_addx(n, R, ldx, c, false, dcol, x, !x_zero, s));
}

int chunk_width(int left) { return left >= 4 ? 4 : (left >= 2 ? 2 : 1); }


namespace {

// The fixed kernel sequence of FGMRES inner iteration j on the workspace:
// z_j = M^{-1} v_j, w = A z_j, modified Gram-Schmidt against v_0..v_j,
// h_{j+1,j} and v_{j+1}, then the Givens update of column j, which leaves
// |g_{j+1}| and h_{j+1,j} in scal[1], scal[2].
void fgmres_inner(silu_ilu F, int j, int m, int mL, int mU, int precond, bool capturing) {
  cudaStream_t s = F->ctx->stream;
  Workspace& W = F->ws;
  const int n = (int)F->F.L.n;
  const int gA = lanes_of(F->lanesA, F->autoA);
  double* V = W.V.as<double>();
  double* Z = W.Z.as<double>();
  double* w = W.w.as<double>();
  double* H = W.H.as<double>();
  double* part[2] = {W.part0.as<double>(), W.part1.as<double>()};
  auto vec = [&](double* base, int k) { return base + (size_t)k * (size_t)n; };
  double* vj = vec(V, j);
  double* zj = vec(Z, j);
  if (precond == SILU_PRECOND_SWEEPS)
    smooth_chunk(F, zj, vj, 1, 1, 0, mL, mU, true);
  else if (precond == SILU_PRECOND_DIRECT)
    direct_chunk(F, zj, vj, 1, 1, 0, true, capturing);
  else if (precond == SILU_PRECOND_AMG)
    amg_cycle(F, zj, vj, mL, mU, true, capturing, false);
  else if (precond == SILU_PRECOND_AMG_DIRECT)
    amg_cycle(F, zj, vj, -1, -1, true, capturing, false);
  else if (precond == SILU_PRECOND_AMG_SCHUR)
    amg_cycle(F, zj, vj, mL, mU, true, capturing, true);
  else if (precond == SILU_PRECOND_SCHUR)
    schur_apply(F, vj, zj, mL, mU);
  else
    CK(cudaMemcpyAsync(zj, vj, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  LAUNCH(F->ctx, SILU_K_RESIDUAL, sweep_launch(F, F->A->d, silu::MODE_D, 1, gA, 1, nullptr, zj, w, nullptr, nullptr, silu::EPI_SPMV));
  LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_dot_part(n, w, V, part[0], s));
  int cur = 0;
  for (int i = 0; i <= j; ++i) {
    const double* vnext = (i < j) ? vec(V, i + 1) : nullptr;
    LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_mgs_step(n, part[cur], H + (size_t)i * m + j, w, vec(V, i), vnext, part[cur ^ 1], s));
    cur ^= 1;
  }
  LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_normalize(n, part[cur], H + (size_t)(j + 1) * m + j, w, vec(V, j + 1), s));
  LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_givens(j, m, H, W.cs.as<double>(), W.sn.as<double>(), W.g.as<double>(), W.scal.as<double>() + 1, s));
}

// Run inner iteration j from its captured graph (capturing it on first use).
void fgmres_inner_graph(silu_ilu F, int j, int m, int mL, int mU, int precond) {
  silu_ctx ctx = F->ctx;
  for (KrylovGraph& kg : F->ws.kgraphs)
    if (kg.j == j && kg.m == m && kg.mL == mL && kg.mU == mU && kg.precond == precond && kg.gen == F->config_gen &&
        kg.agen == F->A->gen) {
      ctx->launches += kg.kernels;
      CK(cudaGraphLaunch(kg.exec, ctx->stream));
      return;
    }
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
      fgmres_inner(F, j, m, mL, mU, precond, true);
    } catch (const CudaFail& f) {
      e = f.e;
    }
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = e2;
  }
  ctx->stream = saved;
  ctx->profiling = prof;
  KrylovGraph kg;
  kg.j = j;
  kg.m = m;
  kg.mL = mL;
  kg.mU = mU;
  kg.precond = precond;
  kg.gen = F->config_gen;
  kg.agen = F->A->gen;
  kg.kernels = ctx->launches - l0;
  ctx->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&kg.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  CK(e);
  F->ws.kgraphs.push_back(kg);
  ctx->launches += kg.kernels;
  CK(cudaGraphLaunch(kg.exec, ctx->stream));
}

}  // namespace

// Unit-diagonal copy of the upper factor: row scaling (Eq. newD) or, for
// SILU_SCALE_ROWCOL, row/column scaling (Eq. rowcolScale).
int scale_upper(silu_ilu F, std::string& msg) {
  if (F->scale == SILU_SCALE_ROWCOL)
    return silu::rowcol_scale(F->F.U, kRuizMaxit, kRuizTol, F->Us, F->dinv, F->dcol, F->ruiz_steps, msg);
  F->dcol.clear();
  return silu::row_scale(F->F.U, F->Us, F->dinv, msg);
}

silu_status finish_setup(silu_ilu F) {
  silu_ctx ctx = F->ctx;
  std::string msg;
  int st = scale_upper(F, msg);
  if (st != silu::H_OK) return set_err(ctx, (silu_status)st, msg);
  F->nlevL = silu::levels_lower(F->F.L, F->levL);
  F->nlevU = silu::levels_upper(F->F.U, true, F->levU);
  silu::group_levels(F->levL, F->nlevL, F->levLptr, F->levLrows);
  silu::group_levels(F->levU, F->nlevU, F->levUptr, F->levUrows);
  const silu::Csr& Ut = scaled_upper(F) ? F->Us : F->F.U;
  F->autoL = pick_lanes(F->F.L);
  F->autoU = pick_lanes(Ut);
  F->autoA = pick_lanes(F->A->A);
  {
    const Csr* fac[2] = {&F->F.L, &Ut};
    std::vector<int32_t> perm;
    std::vector<int64_t> srp;
    for (int k = 0; k < 2; ++k) {
      F->pad_nat[k] = silu::tile_pad(fac[k]->rp.data(), fac[k]->n);
      silu::window_sort(fac[k]->rp.data(), fac[k]->n, perm, srp);
      F->pad_sorted[k] = silu::tile_pad(srp.data(), fac[k]->n);
    }
  }
  if (ctx->device >= 0) {
    silu_status ds = device_ok(ctx);
    if (ds != SILU_OK) return ds;
    cudaStream_t s = ctx->stream;
    cudaError_t e = upload_factors(F);
    if (e == cudaSuccess) e = upload(F->d_dinv, F->dinv.data(), F->dinv.size(), s);
    if (e == cudaSuccess && !F->dcol.empty()) e = upload(F->d_dcol, F->dcol.data(), F->dcol.size(), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "upload of the factors");
  }
  return SILU_OK;
}

}  // namespace silu

// ===========================================================================
extern "C" {

const char* silu_version(void) { return "silu 0.1 (sm_103a)"; }

silu_status silu_ctx_create(int device, void* cuda_stream, silu_ctx* out) {
  if (!out) return SILU_ERR_INVALID_ARG;
  *out = nullptr;
  silu_ctx c = new (std::nothrow) silu_ctx_s;
  if (!c) return SILU_ERR_OOM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (device >= 0) {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device >= count) {
      delete c;
      return SILU_ERR_NO_DEVICE;
    }
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->pinned, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->env.sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->env.err, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->env.err, 0, 4 * sizeof(int));
    if (e == cudaSuccess) e = silu::staged_prepare();
    if (e != cudaSuccess) {
      delete c;
      return SILU_ERR_CUDA;
    }
  }
  *out = c;
  return SILU_OK;
}

void silu_ctx_destroy(silu_ctx ctx) {
  if (!ctx) return;
  if (ctx->device >= 0) cudaSetDevice(ctx->device);
  for (cudaEvent_t ev : ctx->events) cudaEventDestroy(ev);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->env.err) cudaFree(ctx->env.err);
  delete ctx;
}

silu_status silu_ctx_profile(silu_ctx ctx, int enable) {
  if (!ctx) return SILU_ERR_INVALID_ARG;
  if (enable) {
    silu_status ds = device_ok(ctx);
    if (ds != SILU_OK) return ds;
    ctx->nrec = 0;
  }
  ctx->profiling = enable != 0;
  return SILU_OK;
}

silu_status silu_ctx_set_overlap(silu_ctx ctx, int enable) {
  if (!ctx) return SILU_ERR_INVALID_ARG;
  ctx->env.overlap = enable != 0;
  return SILU_OK;
}

silu_status silu_ctx_set_l2_reuse(silu_ctx ctx, int flags) {
  if (!ctx) return SILU_ERR_INVALID_ARG;
  if (flags < 0 || flags > 7) return set_err(ctx, SILU_ERR_INVALID_ARG, "L2 reuse flags must be in [0, 7]");
  ctx->env.l2 = flags;
  return SILU_OK;
}

silu_status silu_ctx_profile_read(silu_ctx ctx, int kclass, int64_t* launches, double* total_ms) {
  if (!ctx || kclass < 0 || kclass >= SILU_K_NCLASS) return SILU_ERR_INVALID_ARG;
  int64_t cnt = 0;
  double ms = 0.0;
  if (ctx->nrec > 0) {
    silu_status ds = device_ok(ctx);
    if (ds != SILU_OK) return ds;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamSynchronize");
    for (size_t k = 0; k < ctx->nrec; ++k) {
      if (ctx->rec_class[k] != kclass) continue;
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ctx->events[2 * k], ctx->events[2 * k + 1]);
      if (e != cudaSuccess) return cuda_err(ctx, e, "cudaEventElapsedTime");
      ms += t;
      cnt += ctx->rec_count[k];
    }
  }
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = ms;
  return SILU_OK;
}

silu_status silu_ctx_check(silu_ctx ctx) {
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamSynchronize");
  int flag = 0;
  e = cudaMemcpy(&flag, ctx->env.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemset(ctx->env.err, 0, sizeof(int));
  // a fused application that gave up at a grid barrier may have left the
  // barrier's arrival count behind: start the next one from a clean state
  if (e == cudaSuccess && (flag & 8)) e = cudaMemset(ctx->env.err + 2, 0, 2 * sizeof(int));
  if (e != cudaSuccess) return cuda_err(ctx, e, "error word read-back");
  if (flag) return set_err(ctx, SILU_ERR_TIMEOUT, "a bounded device wait gave up; results of the affected calls are invalid");
  return SILU_OK;
}

namespace {

// Rebuild the staged-kernel tiles of T (host CSR h) for g lanes per row and
// rl rows per lane.
cudaError_t retile(const Csr& h, DBuf& tiles, DevCsr& T, int g, int rl, cudaStream_t s, int max_nnz) {
  std::vector<int> tl;
  if (!silu::make_tiles(h.rp.data(), h.n, g, rl, tl, max_nnz)) return cudaSuccess;  // keeps the current tiles
  cudaError_t e = upload(tiles, tl.data(), tl.size(), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    T.tiles = tiles.as<int4>();
    T.ntiles = (int)(tl.size() / 4);
    T.tile_lanes = g;
    T.tile_passes = rl;
    T.tile_nnz = max_nnz;
  }
  return e;
}

// Tile limit of an autotuner candidate's gather width: 0 automatic (narrow
// tiles where they fit), 10 narrow tiles where they fit, else the default.
int candidate_tile_nnz(const Csr& h, bool fp32, int g, int rl, int chunk) {
  if (chunk == 0) return auto_tile_nnz(h, fp32, g, rl);
  if (chunk == silu::kNarrowChunkRows) return auto_tile_nnz(h, fp32, g, rl);
  return silu::kTileNnz;
}

// variant 2: staged kernel with `lanes` lanes per row (0 = from the mean row
// length) and `passes` rows per lane (0 = automatic), gather width `chunk`;
// variant 3: staged kernel on the length-sorted copies (where they exist;
// one lane per row), gather width `chunk`;
// variant 1: lanes-per-row kernel with `lanes` lanes.
struct TuneCandidate {
  int variant, lanes, passes, chunk;
};

// chunk 0: the automatic configuration (narrow tiles with 10 gathers in
// flight where the rows fit them, else 16); chunk 10: the narrow
// configuration where it fits.
const TuneCandidate kTune[] = {{2, 0, 0, 0},  {2, 0, 0, 16}, {2, 0, 0, 8},  {2, 1, 1, 16}, {2, 1, 2, 16},
                               {2, 1, 4, 16}, {2, 1, 4, 8},  {2, 2, 1, 16}, {2, 4, 1, 16}, {1, 2, 0, 16},
                               {1, 4, 0, 16}, {1, 8, 0, 16}, {3, 1, 1, 16}, {3, 1, 1, 8}};

}  // namespace

silu_status silu_ilu_autotune(silu_ilu F, int sweeps_L, int sweeps_U, int* choice, double* ms_out) {
  NvtxRange nvtx_("silu:silu_ilu_autotune");
  if (!F || sweeps_L < 0 || sweeps_U < 0) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  const size_t n = (size_t)F->F.L.n;
  if (n == 0) return SILU_OK;
  cudaStream_t s = ctx->stream;
  const Csr& Ut = scaled_upper(F) ? F->Us : F->F.U;
  const int autoL = silu::staged_lanes(F->F.L.rp.data(), F->F.L.n);
  const int autoU = silu::staged_lanes(Ut.rp.data(), Ut.n);
  DBuf x, b;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = 0;
  double best_ms = 1e300;
  try {
    CK(x.ensure(sizeof(double) * n));
    CK(b.ensure(sizeof(double) * n));
    CK(cudaMemsetAsync(b.p, 0, sizeof(double) * n, s));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(ensure_vectors(F, 1));
    const int ncand = (int)(sizeof(kTune) / sizeof(kTune[0]));
    bool have_sorted = false;
    for (int k = 0; k < 2; ++k) have_sorted = have_sorted || silu::sorting_pays(F->pad_nat[k], F->pad_sorted[k]);
    if (have_sorted) CK(ensure_sorted(F));
    have_sorted = F->dL.nstiles > 0 || F->dU.nstiles > 0;
    auto apply = [&](const TuneCandidate& c) {
      F->variant = c.variant;
      if (c.variant == 1) {
        F->lanesL = F->lanesU = c.lanes;
      } else {
        F->lanesL = F->lanesU = 0;
        const int gL = c.lanes ? c.lanes : autoL, gU = c.lanes ? c.lanes : autoU;
        const int pL = c.passes ? c.passes : silu::staged_passes(F->F.L.rp.data(), F->F.L.n, gL);
        const int pU = c.passes ? c.passes : silu::staged_passes(Ut.rp.data(), Ut.n, gU);
        const bool f32 = F->prec == SILU_FP32;
        const int rlL = gL == 1 ? pL : 1, rlU = gU == 1 ? pU : 1;
        CK(retile(F->F.L, F->L_tiles, F->dL, gL, rlL, s, candidate_tile_nnz(F->F.L, f32, gL, rlL, c.chunk)));
        CK(retile(Ut, F->U_tiles, F->dU, gU, rlU, s, candidate_tile_nnz(Ut, f32, gU, rlU, c.chunk)));
        F->dL.chunk = F->dU.chunk = (c.chunk == 8) ? 8 : 16;
      }
    };
    F->tune_ms.assign((size_t)ncand, -1.0);
    for (int k = 0; k < ncand; ++k) {
      if (kTune[k].variant == 3 && !have_sorted) continue;
      apply(kTune[k]);
      CK(cudaMemsetAsync(x.p, 0, sizeof(double) * n, s));
      smooth_chunk(F, x.as<double>(), b.as<double>(), 1, 1, 0, sweeps_L, sweeps_U, false);
      CK(cudaEventRecord(e0, s));
      const int reps = 5;
      for (int r = 0; r < reps; ++r) smooth_chunk(F, x.as<double>(), b.as<double>(), 1, 1, 0, sweeps_L, sweeps_U, false);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      const double per = (double)t / reps;
      F->tune_ms[(size_t)k] = per;
      if (per < best_ms) {
        best_ms = per;
        best = k;
      }
    }
    apply(kTune[best]);
    F->ws.drop_graphs();
    F->config_gen++;
  } catch (const CudaFail& f) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return cuda_err(ctx, f.e, f.what);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (choice) *choice = best;
  if (ms_out) *ms_out = best_ms;
  return silu_ctx_check(ctx);
}

silu_status silu_ilu_tune_table(silu_ilu F, int cap, int32_t* shape, double* ms, int* count) {
  if (!F || cap < 0 || !count) return SILU_ERR_INVALID_ARG;
  const int nc = (int)F->tune_ms.size();
  *count = nc;
  for (int k = 0; k < nc && k < cap; ++k) {
    if (shape) {
      shape[4 * k] = kTune[k].variant;
      shape[4 * k + 1] = kTune[k].lanes;
      shape[4 * k + 2] = kTune[k].passes;
      shape[4 * k + 3] = kTune[k].chunk;
    }
    if (ms) ms[k] = F->tune_ms[(size_t)k];
  }
  return SILU_OK;
}

silu_status silu_ctx_selftest_timeout(silu_ctx ctx, int timeout_ms) {
  if (!ctx || timeout_ms < 1 || timeout_ms > 10000) return SILU_ERR_INVALID_ARG;
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  try {
    LAUNCH(ctx, SILU_K_ELEMENTWISE,
           silu::launch_wait_flag(ctx->env.err + 1, (unsigned long long)timeout_ms * 1000000ull, ctx->env.err,
                                  ctx->stream));
  } catch (const CudaFail& f) {
    return cuda_err(ctx, f.e, f.what);
  }
  return SILU_OK;
}

silu_status silu_ilu_set_kernel(silu_ilu F, int variant) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (variant < 0 || variant > 3) return set_err(F->ctx, SILU_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  if (variant == 3 && F->ctx->device >= 0) {
    silu_status ds = device_ok(F->ctx);
    if (ds != SILU_OK) return ds;
    cudaError_t e = ensure_sorted(F);
    if (e != cudaSuccess) return cuda_err(F->ctx, e, "upload of the sorted factor copies");
  }
  F->variant = variant;
  F->ws.drop_graphs();
  F->config_gen++;
  return SILU_OK;
}

silu_status silu_ilu_set_fused(silu_ilu F, int mode) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2) return set_err(F->ctx, SILU_ERR_INVALID_ARG, "fused mode must be 0, 1 or 2");
  F->fused_mode = mode;
  F->ws.drop_graphs();
  F->config_gen++;
  return SILU_OK;
}

silu_status silu_ilu_set_direct(silu_ilu F, int mode) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2) return set_err(F->ctx, SILU_ERR_INVALID_ARG, "direct mode must be 0, 1 or 2");
  F->direct_mode = mode;
  F->ws.drop_graphs();
  F->config_gen++;
  return SILU_OK;
}

silu_status silu_ilu_layout(silu_ilu F, double* pad_natural, double* pad_sorted, int32_t* in_use) {
  if (!F) return SILU_ERR_INVALID_ARG;
  const DevCsr* d[2] = {&F->dL, &F->dU};
  for (int k = 0; k < 2; ++k) {
    if (pad_natural) pad_natural[k] = F->pad_nat[k];
    if (pad_sorted) pad_sorted[k] = F->pad_sorted[k];
    if (in_use) {
      in_use[k] = F->ctx->device >= 0 && d[k]->nstiles > 0 && F->variant == 3 ? 1 : 0;
    }
  }
  return SILU_OK;
}

silu_status silu_ctx_launch_count(silu_ctx ctx, int64_t* launches) {
  if (!ctx || !launches) return SILU_ERR_INVALID_ARG;
  *launches = ctx->launches;
  return SILU_OK;
}

const char* silu_last_error(silu_ctx ctx) { return ctx ? ctx->err.c_str() : "null context"; }

silu_status silu_mat_create(silu_ctx ctx, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                            const double* val, silu_mat* out) {
  if (!ctx || !out) return SILU_ERR_INVALID_ARG;
  *out = nullptr;
  silu_mat M = new (std::nothrow) silu_mat_s;
  if (!M) return set_err(ctx, SILU_ERR_OOM, "out of host memory");
  M->ctx = ctx;
  std::string msg;
  try {
    int st = silu::csr_canonical(n, nnz, row_ptr, col_idx, val, M->A, msg);
    if (st != silu::H_OK) {
      delete M;
      return set_err(ctx, (silu_status)st, msg);
    }
    if (ctx->device >= 0) {
      silu_status ds = device_ok(ctx);
      if (ds != SILU_OK) {
        delete M;
        return ds;
      }
      cudaError_t e = upload_csr(M->A, false, M->rp, M->ci, M->va, M->tiles, M->d, ctx->stream);
      if (e != cudaSuccess) {
        delete M;
        return cuda_err(ctx, e, "upload of A");
      }
    }
  } catch (const std::bad_alloc&) {
    delete M;
    return set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  *out = M;
  return SILU_OK;
}

void silu_mat_destroy(silu_mat A) { delete A; }

silu_status silu_mat_set_shape(silu_mat A, int lanes, int passes, int chunk) {
  if (!A) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = A->ctx;
  if (!(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4) || !(passes == 0 || passes == 1 || passes == 2 ||
                                                                   passes == 4) ||
      !(chunk == 0 || chunk == 8 || chunk == 10 || chunk == 16) || (lanes != 1 && passes > 1))
    return set_err(ctx, SILU_ERR_INVALID_ARG,
                   "lanes 0/1/2/4, passes 0/1/2/4 (more than 1 only with one lane), chunk 0/8/10/16");
  if (ctx->device < 0 || A->A.n == 0) return SILU_OK;
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  const int g = lanes ? lanes : silu::staged_lanes(A->A.rp.data(), A->A.n);
  const int rl = g == 1 ? (passes ? passes : silu::staged_passes(A->A.rp.data(), A->A.n, g)) : 1;
  const int lim = candidate_tile_nnz(A->A, false, g, rl, chunk);
  if (chunk == silu::kNarrowChunkRows && lim != silu::kTileNnzNarrow)
    return set_err(ctx, SILU_ERR_INVALID_ARG, "the narrow configuration needs one lane per row and short rows");
  std::vector<int> tl;
  if (!silu::make_tiles(A->A.rp.data(), A->A.n, g, rl, tl, lim))
    return set_err(ctx, SILU_ERR_INVALID_ARG, "a row is too long for the staged kernel");
  // new tiles in a new buffer (the old one may still be read by queued work)
  DBuf nt;
  cudaError_t e = upload(nt, tl.data(), tl.size(), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "upload of the tiles");
  std::swap(A->tiles.p, nt.p);
  std::swap(A->tiles.bytes, nt.bytes);
  A->d.tiles = A->tiles.as<int4>();
  A->d.ntiles = (int)(tl.size() / 4);
  A->d.tile_lanes = g;
  A->d.tile_passes = rl;
  A->d.tile_nnz = lim;
  A->d.chunk = (chunk == 8) ? 8 : 16;
  A->gen++;
  return SILU_OK;
}

silu_status silu_mat_autotune(silu_mat A, int* lanes, int* passes, int* chunk, double* ms_out) {
  NvtxRange nvtx_("silu:silu_mat_autotune");
  if (!A) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = A->ctx;
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  const size_t n = (size_t)A->A.n;
  // candidates: {lanes, passes, chunk}, the automatic choice first
  static const int kShapes[][3] = {{0, 0, 0},  {0, 0, 16}, {0, 0, 8}, {1, 1, 10}, {1, 1, 16}, {1, 1, 8}, {1, 2, 16},
                                   {1, 2, 8},  {1, 4, 16}, {1, 4, 8}, {2, 1, 16}, {2, 1, 8},  {4, 1, 16}, {4, 1, 8}};
  int best = -1;
  double best_ms = 1e300;
  if (n > 0) {
    cudaStream_t s = ctx->stream;
    DBuf x, b, r;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
      CK(x.ensure(sizeof(double) * n));
      CK(b.ensure(sizeof(double) * n));
      CK(r.ensure(sizeof(double) * n));
      CK(cudaMemsetAsync(x.p, 0, sizeof(double) * n, s));
      CK(cudaMemsetAsync(b.p, 0, sizeof(double) * n, s));
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      for (int k = 0; k < (int)(sizeof(kShapes) / sizeof(kShapes[0])); ++k) {
        // shapes a row does not fit are skipped
        if (silu_mat_set_shape(A, kShapes[k][0], kShapes[k][1], kShapes[k][2]) != SILU_OK) continue;
        silu_status st = silu_mat_residual(A, r.as<double>(), x.as<double>(), b.as<double>(), 1);
        CK(cudaEventRecord(e0, s));
        const int reps = 5;
        for (int q = 0; q < reps && st == SILU_OK; ++q)
          st = silu_mat_residual(A, r.as<double>(), x.as<double>(), b.as<double>(), 1);
        if (st != SILU_OK) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return st;
        }
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        if ((double)t / reps < best_ms) {
          best_ms = (double)t / reps;
          best = k;
        }
      }
    } catch (const CudaFail& f) {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      return cuda_err(ctx, f.e, f.what);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (best < 0) best = 0;
  silu_status st = silu_mat_set_shape(A, kShapes[best][0], kShapes[best][1], kShapes[best][2]);
  if (st != SILU_OK) return st;
  if (lanes) *lanes = A->d.tile_lanes;
  if (passes) *passes = A->d.tile_passes;
  if (chunk) *chunk = A->d.tile_nnz == silu::kTileNnzNarrow ? silu::kNarrowChunkRows : A->d.chunk;
  if (ms_out) *ms_out = best < 0 || n == 0 ? 0.0 : best_ms;
  return silu_ctx_check(ctx);
}

silu_status silu_mat_residual(silu_mat A, double* r, const double* x, const double* b, int nrhs) {
  NvtxRange nvtx_("silu:silu_mat_residual");
  if (!A || !r || !x || !b || nrhs < 1) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = A->ctx;
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  if (A->A.n == 0) return SILU_OK;
  cudaStream_t s = ctx->stream;
  try {
    if (nrhs == 1 && A->d.ntiles > 0) {
      LAUNCH(ctx, SILU_K_RESIDUAL, silu::launch_sweep_staged(A->d, silu::MODE_D, ctx->env, b, x, r, nullptr, nullptr,
                                                             silu::EPI_STORE, s));
    } else {
      // column blocks of at most 4 right-hand sides, as the smoother's residual
      for (int c0 = 0; c0 < nrhs;) {
        const int w = chunk_width(nrhs - c0);
        LAUNCH(ctx, SILU_K_RESIDUAL, silu::launch_sweep(A->d, silu::MODE_D, w, pick_lanes(A->A), nrhs, b + c0, x + c0,
                                                        r + c0, nullptr, nullptr, silu::EPI_STORE, s));
        c0 += w;
      }
    }
  } catch (const silu::CudaFail& f) {
    return cuda_err(ctx, f.e, f.what);
  }
  return SILU_OK;
}

silu_status ilu_setup(silu_ctx ctx, silu_mat A, silu_kind kind, double tau, int fill, silu_scale scale,
                      silu_prec prec, silu_ilu* out) {
  NvtxRange nvtx_("silu:ilu_setup");
  if (!ctx || !A || !out || A->ctx != ctx) return set_err(ctx, SILU_ERR_INVALID_ARG, "bad handle");
  *out = nullptr;
  if (kind < SILU_ILU0 || kind > SILU_SGS || scale < SILU_SCALE_NONE || scale > SILU_SCALE_ROWCOL ||
      prec < SILU_FP64 || prec > SILU_FP32)
    return set_err(ctx, SILU_ERR_INVALID_ARG, "bad enum value");
  silu_ilu F = new (std::nothrow) silu_ilu_s;
  if (!F) return set_err(ctx, SILU_ERR_OOM, "out of host memory");
  F->ctx = ctx;
  F->A = A;
  F->kind = kind;
  F->scale = scale;
  F->prec = prec;
  F->tau = tau;
  F->fill = fill;
  std::string msg;
  try {
    const int st = silu::factor_kind(A->A, (int)kind, tau, fill, F->F, msg);
    if (st != silu::H_OK) {
      delete F;
      return set_err(ctx, (silu_status)st, msg);
    }
    const silu_status fs = finish_setup(F);
    if (fs != SILU_OK) {
      delete F;
      return fs;
    }
  } catch (const std::bad_alloc&) {
    delete F;
    return set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  *out = F;
  return SILU_OK;
}

namespace {

// Factor file: a fixed header (magic "SILUFAC1", then kind, scale, prec,
// fill as int32, tau as double, n, nnz(L_s), nnz(U) as int64) followed by
// L_s and U as CSR (int64 row pointers, int32 columns, double values), all
// little-endian as the host stores them.
constexpr char kFacMagic[8] = {'S', 'I', 'L', 'U', 'F', 'A', 'C', '1'};

bool write_csr(FILE* f, const Csr& T) {
  return fwrite(T.rp.data(), sizeof(int64_t), T.rp.size(), f) == T.rp.size() &&
         fwrite(T.ci.data(), sizeof(int32_t), T.ci.size(), f) == T.ci.size() &&
         fwrite(T.va.data(), sizeof(double), T.va.size(), f) == T.va.size();
}

bool read_csr(FILE* f, int64_t n, int64_t nnz, Csr& T) {
  T.n = n;
  T.rp.resize(n + 1);
  T.ci.resize(nnz);
  T.va.resize(nnz);
  if (fread(T.rp.data(), sizeof(int64_t), T.rp.size(), f) != T.rp.size() ||
      fread(T.ci.data(), sizeof(int32_t), T.ci.size(), f) != T.ci.size() ||
      fread(T.va.data(), sizeof(double), T.va.size(), f) != T.va.size())
    return false;
  if (T.rp[0] != 0 || T.rp[n] != nnz) return false;
  for (int64_t i = 0; i < n; ++i)
    if (T.rp[i + 1] < T.rp[i]) return false;
  for (int32_t c : T.ci)
    if (c < 0 || c >= n) return false;
  for (double v : T.va)
    if (!std::isfinite(v)) return false;
  return true;
}

}  // namespace

silu_status silu_ilu_save(silu_ilu F, const char* path) {
  if (!F || !path) return SILU_ERR_INVALID_ARG;
  FILE* f = fopen(path, "wb");
  if (!f) return set_err(F->ctx, SILU_ERR_INVALID_ARG, std::string("cannot open ") + path);
  const int32_t hdr32[4] = {(int32_t)F->kind, (int32_t)F->scale, (int32_t)F->prec, (int32_t)F->fill};
  const int64_t hdr64[3] = {F->F.L.n, F->F.L.nnz(), F->F.U.nnz()};
  bool ok = fwrite(kFacMagic, 1, 8, f) == 8 && fwrite(hdr32, sizeof(int32_t), 4, f) == 4 &&
            fwrite(&F->tau, sizeof(double), 1, f) == 1 && fwrite(hdr64, sizeof(int64_t), 3, f) == 3 &&
            write_csr(f, F->F.L) && write_csr(f, F->F.U);
  ok = (fclose(f) == 0) && ok;
  if (!ok) return set_err(F->ctx, SILU_ERR_INVALID_ARG, std::string("cannot write ") + path);
  return SILU_OK;
}

silu_status silu_ilu_load(silu_ctx ctx, silu_mat A, const char* path, silu_ilu* out) {
  NvtxRange nvtx_("silu:silu_ilu_load");
  if (!ctx || !A || !path || !out || A->ctx != ctx) return set_err(ctx, SILU_ERR_INVALID_ARG, "bad handle");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return set_err(ctx, SILU_ERR_INVALID_ARG, std::string("cannot open ") + path);
  silu_ilu F = nullptr;
  silu_status st = SILU_OK;
  try {
    char magic[8];
    int32_t hdr32[4];
    double tau = 0.0;
    int64_t hdr64[3];
    if (fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kFacMagic, 8) != 0 || fread(hdr32, sizeof(int32_t), 4, f) != 4 ||
        fread(&tau, sizeof(double), 1, f) != 1 || fread(hdr64, sizeof(int64_t), 3, f) != 3) {
      st = set_err(ctx, SILU_ERR_INVALID_ARG, "not a factor file");
    } else if (hdr64[0] != A->A.n || hdr64[1] < 0 || hdr64[2] < hdr64[0] || hdr32[0] < SILU_ILU0 ||
               hdr32[0] > SILU_SGS || hdr32[1] < SILU_SCALE_NONE || hdr32[1] > SILU_SCALE_ROWCOL ||
               hdr32[2] < SILU_FP64 || hdr32[2] > SILU_FP32) {
      st = set_err(ctx, SILU_ERR_INVALID_ARG, "factor file does not fit the matrix");
    } else {
      F = new silu_ilu_s;
      F->ctx = ctx;
      F->A = A;
      F->kind = (silu_kind)hdr32[0];
      F->scale = (silu_scale)hdr32[1];
      F->prec = (silu_prec)hdr32[2];
      F->fill = hdr32[3];
      F->tau = tau;
      if (!read_csr(f, hdr64[0], hdr64[1], F->F.L) || !read_csr(f, hdr64[0], hdr64[2], F->F.U))
        st = set_err(ctx, SILU_ERR_INVALID_ARG, "corrupt factor file");
      for (int64_t i = 0; st == SILU_OK && i < F->F.L.n; ++i)  // L strictly lower, U with its diagonal first
        for (int64_t p = F->F.L.rp[i]; p < F->F.L.rp[i + 1]; ++p)
          if (F->F.L.ci[p] >= i) st = set_err(ctx, SILU_ERR_INVALID_ARG, "corrupt factor file (L)");
      for (int64_t i = 0; st == SILU_OK && i < F->F.U.n; ++i) {
        const int64_t b = F->F.U.rp[i], e = F->F.U.rp[i + 1];
        if (e <= b || F->F.U.ci[b] != i) st = set_err(ctx, SILU_ERR_INVALID_ARG, "corrupt factor file (U)");
        for (int64_t p = b + 1; st == SILU_OK && p < e; ++p)
          if (F->F.U.ci[p] <= i) st = set_err(ctx, SILU_ERR_INVALID_ARG, "corrupt factor file (U)");
      }
      if (st == SILU_OK) st = finish_setup(F);
    }
  } catch (const std::bad_alloc&) {
    st = set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  fclose(f);
  if (st != SILU_OK) {
    delete F;
    return st;
  }
  *out = F;
  return SILU_OK;
}

silu_status ilu_refactor(silu_ilu F, const double* new_val) {
  NvtxRange nvtx_("silu:ilu_refactor");
  if (!F || !new_val) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (F->kind == SILU_ILUT) return set_err(ctx, SILU_ERR_INVALID_ARG, "ILUT has no reusable symbolic phase");
  std::string msg;
  try {
    silu::Csr& A = F->A->A;
    for (int64_t p = 0; p < A.nnz(); ++p)
      if (!std::isfinite(new_val[p])) return set_err(ctx, SILU_ERR_INVALID_ARG, "non-finite value");
    std::copy(new_val, new_val + A.nnz(), A.va.begin());
    int st = (F->kind == SILU_GS || F->kind == SILU_SGS) ? silu::factor_gs(A, F->kind == SILU_SGS, F->F, msg)
                                                          : silu::refactor_numeric(A, F->F, msg);
    if (st == silu::H_OK) st = silu::scale_upper(F, msg);
    if (st != silu::H_OK) return set_err(ctx, (silu_status)st, msg);
    if (ctx->device >= 0) {
      silu_status ds = device_ok(ctx);
      if (ds != SILU_OK) return ds;
      cudaStream_t s = ctx->stream;
      cudaError_t e = upload(F->A->va, A.va.data(), A.va.size(), s);
      if (e == cudaSuccess) e = upload_factors(F);
      if (e == cudaSuccess) e = upload(F->d_dinv, F->dinv.data(), F->dinv.size(), s);
      if (e == cudaSuccess && !F->dcol.empty()) e = upload(F->d_dcol, F->dcol.data(), F->dcol.size(), s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_err(ctx, e, "upload of the refactored factors");
      F->A->d.va = F->A->va.p;
      F->direct_ready = false;
    }
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  return SILU_OK;
}

silu_status silu_ilu_reserve(silu_ilu F, int nrhs, int restart) {
  if (!F || nrhs < 1 || restart < 0) return SILU_ERR_INVALID_ARG;
  silu_status ds = device_ok(F->ctx);
  if (ds != SILU_OK) return ds;
  cudaError_t e = ensure_vectors(F, nrhs);
  if (e == cudaSuccess && restart > 0) e = ensure_krylov(F, restart);
  if (e != cudaSuccess) return cuda_err(F->ctx, e, "workspace");
  return SILU_OK;
}

silu_status ilu_smooth(silu_ilu F, double* x, const double* b, int nrhs, int sweeps_L, int sweeps_U) {
  NvtxRange nvtx_("silu:ilu_smooth");
  if (!F) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (!x || !b || nrhs < 1 || sweeps_L < 0 || sweeps_U < 0)
    return set_err(ctx, SILU_ERR_INVALID_ARG, "ilu_smooth: bad argument");
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  if (F->F.L.n == 0) return SILU_OK;
  try {
    CK(ensure_vectors(F, nrhs));
    for (int c0 = 0; c0 < nrhs;) {
      const int R = chunk_width(nrhs - c0);
      smooth_chunk(F, x + c0, b + c0, R, nrhs, (size_t)c0, sweeps_L, sweeps_U, false);
      c0 += R;
    }
  } catch (const CudaFail& f) {
    return cuda_err(ctx, f.e, f.what);
  }
  return SILU_OK;
}

silu_status direct_trisolve(silu_ilu F, double* x, const double* b, int nrhs) {
  NvtxRange nvtx_("silu:direct_trisolve");
  if (!F) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (!x || !b || nrhs < 1) return set_err(ctx, SILU_ERR_INVALID_ARG, "direct_trisolve: bad argument");
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  if (F->F.L.n == 0) return SILU_OK;
  try {
    CK(ensure_vectors(F, nrhs));
    CK(ensure_direct(F));
    for (int c0 = 0; c0 < nrhs;) {
      const int R = chunk_width(nrhs - c0);
      CK(ensure_tri(F, R));
      CK(decide_direct(F, R));
      direct_chunk(F, x + c0, b + c0, R, nrhs, (size_t)c0, false);
      c0 += R;
    }
  } catch (const CudaFail& f) {
    return cuda_err(ctx, f.e, f.what);
  }
  return SILU_OK;
}

silu_status fgmres_solve(silu_ilu F, double* x, const double* b, double tol, int restart, int maxit, int sweeps_L,
                         int sweeps_U, int precond, int* iters_out, double* relres_out) {
  NvtxRange nvtx_("silu:fgmres_solve");
  if (!F) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (iters_out) *iters_out = 0;
  if (relres_out) *relres_out = 0.0;
  if (!x || !b || !(tol >= 0.0) || restart < 1 || maxit < 0 || sweeps_L < 0 || sweeps_U < 0 || precond < 0 ||
      precond > 6 ||
      ((precond == SILU_PRECOND_AMG || precond == SILU_PRECOND_AMG_DIRECT || precond == SILU_PRECOND_AMG_SCHUR) &&
       !F->amg) ||
      ((precond == SILU_PRECOND_SCHUR || precond == SILU_PRECOND_AMG_SCHUR) && !F->schur))
    return set_err(ctx, SILU_ERR_INVALID_ARG, "fgmres_solve: bad argument");
  silu_status ds = device_ok(ctx);
  if (ds != SILU_OK) return ds;
  const int n = (int)F->F.L.n;
  const int m = restart;
  cudaStream_t s = ctx->stream;
  int its = 0;
  double relres = 0.0;
  silu_status result = SILU_OK;
  struct Events {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t v : e)
        if (v) cudaEventDestroy(v);
    }
    cudaEvent_t& operator[](int k) { return e[k]; }
  } it_done;
  try {
    CK(ensure_vectors(F, 1));
    CK(ensure_krylov(F, m));
    if (precond == SILU_PRECOND_DIRECT || precond == SILU_PRECOND_AMG_DIRECT) {
      CK(ensure_direct(F));
      level_graph(F, 1, 1, 0);  // settles the level launch form before iterations are captured
      if (precond == SILU_PRECOND_AMG_DIRECT) CK(amg_prepare_direct(F));  // and the ILU levels'
    }
    Workspace& W = F->ws;
    double* V = W.V.as<double>();
    double* Z = W.Z.as<double>();
    double* w = W.w.as<double>();
    double* H = W.H.as<double>();
    double* g = W.g.as<double>();
    double* part[2] = {W.part0.as<double>(), W.part1.as<double>()};
    double* scal = W.scal.as<double>();
    double* hp = ctx->pinned;
    const int gA = lanes_of(F->lanesA, F->autoA);
    CK(cudaEventCreateWithFlags(&it_done[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&it_done[1], cudaEventDisableTiming));
    // ||b||
    LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_dot_part(n, b, b, part[0], s));
    LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_norm_final(n, part[0], scal, s));
    CK(cudaMemcpyAsync(hp, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bnorm = hp[0];
    if (n == 0 || bnorm == 0.0) {
      if (n > 0) CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, s));
      CK(cudaStreamSynchronize(s));
      return SILU_OK;
    }
    for (;;) {
      // true residual r = b - A x into V_0, beta = ||r||
      LAUNCH(F->ctx, SILU_K_RESIDUAL, sweep_launch(F, F->A->d, silu::MODE_D, 1, gA, 1, b, x, V, nullptr, nullptr, silu::EPI_STORE));
      LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_dot_part(n, V, V, part[0], s));
      LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_norm_final(n, part[0], scal, s));
      CK(cudaMemcpyAsync(hp, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      relres = hp[0] / bnorm;
      if (relres <= tol) {
        result = SILU_OK;
        break;
      }
      if (its >= maxit) {
        result = SILU_ERR_NOT_CONVERGED;
        break;
      }
      CK(cudaMemsetAsync(g, 0, sizeof(double) * (size_t)(m + 1), s));
      CK(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)(m + 1) * (size_t)m, s));
      LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_normalize(n, part[0], g, V, V, s));
      // Inner iterations run one ahead of the host: iteration j + 1 is queued
      // before the host reads |g_{j+1}| and h_{j+1,j} of iteration j (copied
      // to their own pinned slot), so the device does not wait for the host's
      // decision.  An iteration queued after the one that ends the cycle only
      // writes column j + 1 of H, g_{j+1}, g_{j+2}, V_{j+2} and Z_{j+1}, none
      // of which the update of x with the first j + 1 columns reads, and the
      // next cycle rewrites them before reading them.
      auto queue_inner = [&](int j) {
        if (F->ctx->profiling)
          fgmres_inner(F, j, m, sweeps_L, sweeps_U, precond, false);  // per-kernel events need eager launches
        else
          fgmres_inner_graph(F, j, m, sweeps_L, sweeps_U, precond);
        CK(cudaMemcpyAsync(hp + 4 + 2 * (j & 1), scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(it_done[j & 1], s));
      };
      int jend = 0;
      queue_inner(0);
      for (int j = 0; j < m; ++j) {
        if (j + 1 < m && its + 2 <= maxit) queue_inner(j + 1);
        CK(cudaEventSynchronize(it_done[j & 1]));
        ++its;
        jend = j + 1;
        const double res = hp[4 + 2 * (j & 1)], hn = hp[5 + 2 * (j & 1)];
        if (!std::isfinite(res)) {
          result = SILU_WARN_DIVERGED;
          break;
        }
        if (res <= tol * bnorm || its >= maxit || hn == 0.0) break;
      }
      LAUNCH(F->ctx, SILU_K_KRYLOV, silu::launch_update_x(n, jend, m, H, g, W.yk.as<double>(), Z, x, s));
      if (result == SILU_WARN_DIVERGED) {
        CK(cudaStreamSynchronize(s));
        relres = NAN;
        break;
      }
    }
  } catch (const CudaFail& f) {
    return cuda_err(ctx, f.e, f.what);
  }
  if (iters_out) *iters_out = its;
  if (relres_out) *relres_out = relres;
  {
    silu_status cs = silu_ctx_check(ctx);
    if (cs != SILU_OK) return cs;
  }
  if (result == SILU_ERR_NOT_CONVERGED) set_err(ctx, result, "fgmres_solve: maxit reached above tol");
  if (result == SILU_WARN_DIVERGED) set_err(ctx, result, "fgmres_solve: non-finite residual estimate");
  return result;
}

silu_status silu_ilu_stats(silu_ilu F, int64_t* n, int64_t* nnz_L, int64_t* nnz_U, int32_t* levels_L,
                           int32_t* levels_U) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (n) *n = F->F.L.n;
  if (nnz_L) *nnz_L = F->F.L.nnz();
  if (nnz_U) *nnz_U = scaled_upper(F) ? F->Us.nnz() : F->F.U.nnz();
  if (levels_L) *levels_L = F->nlevL;
  if (levels_U) *levels_U = F->nlevU;
  return SILU_OK;
}

silu_status silu_ilu_export_sizes(silu_ilu F, int64_t* nnz_L, int64_t* nnz_Ufull, int64_t* nnz_Us) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (nnz_L) *nnz_L = F->F.L.nnz();
  if (nnz_Ufull) *nnz_Ufull = F->F.U.nnz();
  if (nnz_Us) *nnz_Us = F->Us.nnz();
  return SILU_OK;
}

silu_status silu_ilu_export(silu_ilu F, int64_t* Lp, int32_t* Lc, double* Lv, int64_t* Up, int32_t* Uc, double* Uv,
                            int64_t* Sp, int32_t* Sc, double* Sv, double* dinv, int32_t* levL, int32_t* levU) {
  if (!F) return SILU_ERR_INVALID_ARG;
  auto cp = [](auto* dst, const auto& src) {
    if (dst && !src.empty()) std::memcpy(dst, src.data(), sizeof(src[0]) * src.size());
  };
  cp(Lp, F->F.L.rp);
  cp(Lc, F->F.L.ci);
  cp(Lv, F->F.L.va);
  cp(Up, F->F.U.rp);
  cp(Uc, F->F.U.ci);
  cp(Uv, F->F.U.va);
  cp(Sp, F->Us.rp);
  cp(Sc, F->Us.ci);
  cp(Sv, F->Us.va);
  cp(dinv, F->dinv);
  cp(levL, F->levL);
  cp(levU, F->levU);
  return SILU_OK;
}

silu_status silu_ilu_export_colscale(silu_ilu F, double* dcol, int32_t* ruiz_steps) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (F->scale != SILU_SCALE_ROWCOL) return set_err(F->ctx, SILU_ERR_INVALID_ARG, "factor is not row/column scaled");
  if (dcol && !F->dcol.empty()) std::memcpy(dcol, F->dcol.data(), sizeof(double) * F->dcol.size());
  if (ruiz_steps) *ruiz_steps = F->ruiz_steps;
  return SILU_OK;
}

silu_status silu_ilu_dep(silu_ilu F, double* dep_L, double* dep_U, double* dep_scaled) {
  if (!F) return SILU_ERR_INVALID_ARG;
  // dep(T) of a triangular T (Eq. depB): its eigenvalues are its diagonal, so
  // dep(T)^2 is the sum of the squares of the off-diagonal entries
  auto offdiag = [](const Csr& T) {
    double s = 0.0;
    for (int64_t i = 0; i < T.n; ++i)
      for (int64_t p = T.rp[i]; p < T.rp[i + 1]; ++p)
        if (T.ci[p] != i) s += T.va[p] * T.va[p];
    return std::sqrt(s);
  };
  if (dep_L) *dep_L = offdiag(F->F.L);
  if (dep_U) *dep_U = offdiag(F->F.U);
  if (dep_scaled) *dep_scaled = offdiag(F->Us);
  return SILU_OK;
}

void silu_ilu_destroy(silu_ilu F) { delete F; }

silu_status silu_ilu_set_lanes(silu_ilu F, int lanes_L, int lanes_U, int lanes_A) {
  if (!F) return SILU_ERR_INVALID_ARG;
  auto ok = [](int g) { return g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32; };
  if (!ok(lanes_L) || !ok(lanes_U) || !ok(lanes_A))
    return set_err(F->ctx, SILU_ERR_INVALID_ARG, "lanes must be 0 or a power of two up to 32");
  F->lanesL = lanes_L;
  F->lanesU = lanes_U;
  F->lanesA = lanes_A;
  F->ws.drop_graphs();
  F->config_gen++;
  return SILU_OK;
}

}  // extern "C"
