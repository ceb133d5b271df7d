// Algebraic multigrid on the device (Sec. 3 of the paper, Alg. mgcycle): the
// V-cycle that the paper's solvers wrap around the scaled-ILU smoother.  The
// hierarchy is built on the host (amg_setup.cpp); every level's operator,
// restriction R = P^T and (negated) prolongation P are swept by the same
// sweep kernels as the smoother, the finest level is smoothed by the
// factor object's ILU smoother (optionally the next levels by ILU smoothers
// of their own, Sec. 6), coarser levels by l1-Jacobi or polynomial
// Gauss-Seidel, and the coarsest level is solved by a dense inverse.
#include <cstring>

#include "internal.h"

using silu::CudaFail;
using silu::DevCsr;
using silu::ProfScope;

namespace {

// x = Minv b for the dense m x m row-major inverse: one warp per row.
__global__ void k_dense_gemv(int m, const double* __restrict__ Minv, const double* __restrict__ b,
                             double* __restrict__ x) {
  const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  const double* row = Minv + (size_t)warp * (size_t)m;
  double s = 0.0;
  for (int j = lane; j < m; j += 32) s = fma(row[j], b[j], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) x[warp] = s;
}

cudaError_t launch_dense_gemv(int m, const double* Minv, const double* b, double* x, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)(((long long)m * 32 + threads - 1) / threads);
  k_dense_gemv<<<blocks, threads, 0, s>>>(m, Minv, b, x);
  return cudaGetLastError();
}

silu::Csr negated(const silu::Csr& P) {
  silu::Csr N = P;
  for (double& v : N.va) v = -v;
  return N;
}

// One sweep-kernel launch on a hierarchy operator (FP64 vectors, one column).
void op(silu_ilu F, const DevCsr& T, int cls, const double* c, const double* in, double* out, const double* dinv,
        double* x, int epi) {
  LAUNCH(F->ctx, cls, silu::sweep_launch(F, T, silu::MODE_D, 1, 4, 1, c, in, out, dinv, x, epi));
}

// nu sweeps of l1-Jacobi on level l, x <- x + D^{-1} (b - A x), ping-ponging
// between the level's x and t buffers; x_zero: start from x = 0 (the first
// sweep is then D^{-1} b).  Returns the buffer holding the result.
double* l1_jacobi(silu_ilu F, AmgDevLevel& L, double* cur, const double* b, int nu, bool x_zero) {
  cudaStream_t s = F->ctx->stream;
  const double* dinv = L.l1inv.as<double>();
  int k = 0;
  if (x_zero && nu == 0) CK(cudaMemsetAsync(cur, 0, sizeof(double) * (size_t)L.n, s));
  if (x_zero && nu > 0) {
    LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_scale((int)L.n, 1, 1, b, false, dinv, cur, false, s));
    k = 1;
  }
  for (; k < nu; ++k) {
    double* nxt = (cur == L.x.as<double>()) ? L.t.as<double>() : L.x.as<double>();
    op(F, L.A, SILU_K_RESIDUAL, b, cur, nxt, dinv, nullptr, silu::EPI_JAC);
    cur = nxt;
  }
  return cur;
}

// nu steps of polynomial Gauss-Seidel on level l (Sec. 3.1),
// x <- x + D^{-1} y with y = sum_{j<terms} (-L D^{-1})^j (b - A x), the
// Neumann series run as Richardson sweeps on L D^{-1} with the last one fused
// into the update of x (in place: x is not read by that launch).
double* poly_gs(silu_ilu F, AmgDevLevel& L, double* x, const double* b, int nu, int terms, bool x_zero) {
  cudaStream_t s = F->ctx->stream;
  const double* dinv = L.gdinv.as<double>();
  if (x_zero && nu == 0) CK(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)L.n, s));
  for (int step = 0; step < nu; ++step) {
    const bool set = x_zero && step == 0;  // x is still zero: write, do not add
    const double* r = b;
    if (!set) {
      op(F, L.A, SILU_K_RESIDUAL, b, x, L.r.as<double>(), nullptr, nullptr, silu::EPI_STORE);
      r = L.r.as<double>();
    }
    if (terms <= 1) {
      LAUNCH(F->ctx, SILU_K_ELEMENTWISE, silu::launch_addx((int)L.n, 1, 1, r, false, dinv, x, !set, s));
      continue;
    }
    const double* in = r;
    double* pp[2] = {L.t.as<double>(), L.y2.as<double>()};
    for (int k = 2; k <= terms; ++k) {
      const bool last = k == terms;
      const int epi = last ? (set ? silu::EPI_SCALE_SETX : silu::EPI_SCALE_ADDX) : silu::EPI_STORE;
      op(F, L.Lgs, SILU_K_SWEEP_L, r, in, last ? nullptr : pp[k & 1], dinv, x, epi);
      in = pp[k & 1];
    }
  }
  return x;
}

// The configured smoother of a level below the finest: the level's own ILU
// smoother where it has one (m_L + m_U sweeps, or its exact triangular
// solves when mL < 0; x is updated in place), else the coarse smoother.
double* coarse_smooth(silu_ilu F, int l, double* x, const double* b, bool x_zero, int mL, int mU, bool capturing) {
  const AmgState& G = *F->amg;
  AmgDevLevel& L = *G.lev[l];
  if (silu_ilu FL = G.ilu_fac[l]) {
    if (mL < 0)
      silu::direct_chunk(FL, x, b, 1, 1, 0, x_zero, capturing);
    else
      silu::smooth_chunk(FL, x, b, 1, 1, 0, mL, mU, x_zero);
    return x;
  }
  if (G.coarse_kind == SILU_AMG_POLY_GS) return poly_gs(F, L, x, b, G.nu, G.gs_terms, x_zero);
  return l1_jacobi(F, L, x, b, G.nu, x_zero);
}

// Multilevel(A_l, b, x, l) of Alg. mgcycle for l >= 1, from x = 0; returns
// the buffer that holds x_l.
double* level_cycle(silu_ilu F, int l, int mL, int mU, bool capturing) {
  AmgState& G = *F->amg;
  AmgDevLevel& L = *G.lev[l];
  const int last = (int)G.lev.size() - 1;
  double* b = L.b.as<double>();
  if (l == last) {  // coarsest level: direct solve
    LAUNCH(F->ctx, SILU_K_KRYLOV, launch_dense_gemv((int)L.n, G.cinv.as<double>(), b, L.x.as<double>(),
                                                    F->ctx->stream));
    return L.x.as<double>();
  }
  double* x = coarse_smooth(F, l, L.x.as<double>(), b, true, mL, mU, capturing);
  AmgDevLevel& C = *G.lev[l + 1];
  op(F, L.A, SILU_K_RESIDUAL, b, x, L.r.as<double>(), nullptr, nullptr, silu::EPI_STORE);       // r = b - A x
  op(F, L.R, SILU_K_RESIDUAL, nullptr, L.r.as<double>(), C.b.as<double>(), nullptr, nullptr, silu::EPI_SPMV);
  const double* v = level_cycle(F, l + 1, mL, mU, capturing);
  op(F, L.Pneg, SILU_K_RESIDUAL, nullptr, v, nullptr, nullptr, x, silu::EPI_ADDX);             // x += P v
  return coarse_smooth(F, l, x, b, false, mL, mU, capturing);
}

cudaError_t upload_level(const silu::AmgLevel& H, AmgDevLevel& D, bool own_a, bool coarsest, bool gs,
                         cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  D.n = H.A.n;
  if (own_a) e = silu::upload_csr(H.A, false, D.A_rp, D.A_ci, D.A_va, D.A_tiles, D.A, s);
  if (e == cudaSuccess && !coarsest) {
    e = silu::upload_csr(negated(H.P), false, D.P_rp, D.P_ci, D.P_va, D.P_tiles, D.Pneg, s);
    if (e == cudaSuccess) e = silu::upload_csr(H.R, false, D.R_rp, D.R_ci, D.R_va, D.R_tiles, D.R, s);
  }
  if (e == cudaSuccess) e = silu::upload(D.l1inv, H.l1inv.data(), H.l1inv.size(), s);
  if (e == cudaSuccess && gs && own_a) {
    e = silu::upload_csr(H.Lgs, false, D.G_rp, D.G_ci, D.G_va, D.G_tiles, D.Lgs, s);
    if (e == cudaSuccess) e = silu::upload(D.gdinv, H.dinv.data(), H.dinv.size(), s);
  }
  const size_t vb = sizeof(double) * (size_t)std::max<int64_t>(D.n, 1);
  if (e == cudaSuccess) e = D.y2.ensure(vb);
  if (e == cudaSuccess) e = D.x.ensure(vb);
  if (e == cudaSuccess) e = D.t.ensure(vb);
  if (e == cudaSuccess) e = D.b.ensure(vb);
  if (e == cudaSuccess) e = D.r.ensure(vb);
  return e;
}

}  // namespace

AmgState::~AmgState() {
  for (silu_ilu f : ilu_fac)
    if (f) silu_ilu_destroy(f);
  for (silu_mat m : ilu_mat)
    if (m) silu_mat_destroy(m);
}

namespace silu {

cudaError_t amg_prepare_direct(silu_ilu F) {
  cudaError_t e = ensure_direct(F);
  if (e != cudaSuccess || !F->amg) return e;
  for (silu_ilu FL : F->amg->ilu_fac) {
    if (!FL) continue;
    e = ensure_direct(FL);
    if (e != cudaSuccess) return e;
    try {
      level_graph(FL, 1, 1, 0);  // settles the level launch form before a capture records the cycle
    } catch (const CudaFail& f) {
      return f.e;
    }
  }
  return cudaSuccess;
}

void amg_cycle(silu_ilu F, double* x, const double* b, int mL, int mU, bool x_zero, bool capturing, bool schur) {
  AmgState& G = *F->amg;
  AmgDevLevel& L0 = *G.lev[0];
  if (G.lev.size() == 1) {  // a single level: the direct solve
    CK(cudaMemcpyAsync(L0.b.p, b, sizeof(double) * (size_t)L0.n, cudaMemcpyDeviceToDevice, F->ctx->stream));
    LAUNCH(F->ctx, SILU_K_KRYLOV, launch_dense_gemv((int)L0.n, G.cinv.as<double>(), L0.b.as<double>(), x,
                                                    F->ctx->stream));
    return;
  }
  const DevCsr& A = F->A->d;
  AmgDevLevel& C = *G.lev[1];
  // finest-level smoother: Richardson sweeps, the exact triangular solves
  // when mL < 0, or one application of the ILUT Schur complement smoother
  // (Sec. 3.1; m_L + m_U sweeps in each block): x (+)= M^{-1} (b - A x)
  auto smooth = [&](bool xz) {
    if (schur) {
      if (xz) {
        schur_apply(F, b, x, mL, mU);  // x = M^{-1} b (every row written)
      } else {
        double* r = F->schur->r.as<double>();
        double* z = F->ws.r.as<double>();
        op(F, A, SILU_K_RESIDUAL, b, x, r, nullptr, nullptr, EPI_STORE);
        schur_apply(F, r, z, mL, mU);
        LAUNCH(F->ctx, SILU_K_ELEMENTWISE, launch_addx((int)L0.n, 1, 1, z, false, nullptr, x, true, F->ctx->stream));
      }
    } else if (mL < 0) {
      direct_chunk(F, x, b, 1, 1, 0, xz, capturing);
    } else {
      smooth_chunk(F, x, b, 1, 1, 0, mL, mU, xz);
    }
  };
  smooth(x_zero);                                                                   // pre-smoothing
  op(F, A, SILU_K_RESIDUAL, b, x, L0.r.as<double>(), nullptr, nullptr, EPI_STORE);  // r = b - A x
  op(F, L0.R, SILU_K_RESIDUAL, nullptr, L0.r.as<double>(), C.b.as<double>(), nullptr, nullptr, EPI_SPMV);
  const double* v = level_cycle(F, 1, mL, mU, capturing);
  op(F, L0.Pneg, SILU_K_RESIDUAL, nullptr, v, nullptr, nullptr, x, EPI_ADDX);        // x += P v
  smooth(false);                                                                    // post-smoothing
}

}  // namespace silu

extern "C" {

silu_status silu_amg_setup(silu_ilu F, const silu_amg_params* params) {
  NvtxRange nvtx_("silu:silu_amg_setup");
  if (!F) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  silu_amg_params p = {0.25, 25, 400, 1, SILU_AMG_L1_JACOBI, 2, 1};
  if (params) p = *params;
  if (p.jacobi_sweeps < 0) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "jacobi_sweeps must be >= 0");
  if ((p.coarse_smoother != SILU_AMG_L1_JACOBI && p.coarse_smoother != SILU_AMG_POLY_GS) || p.gs_terms < 1)
    return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "bad coarse smoother or gs_terms");
  if (p.ilu_levels < 0) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "ilu_levels must be >= 0");
  if (p.ilu_levels > 1 && F->kind != SILU_ILU0 && F->kind != SILU_ILUK && F->kind != SILU_ILUT)
    return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "ILU smoothing below the finest level needs an ILU kind");
  std::unique_ptr<AmgState> G;
  try {
    G.reset(new AmgState);
    G->theta = p.theta;
    G->max_levels = p.max_levels;
    G->coarse_size = p.coarse_size;
    G->nu = p.jacobi_sweeps;
    G->coarse_kind = p.coarse_smoother;
    G->gs_terms = p.gs_terms;
    std::string msg;
    int st = silu::amg_build(F->A->A, p.theta, p.max_levels, p.coarse_size, G->host, msg);
    if (st == silu::H_OK && p.coarse_smoother == SILU_AMG_POLY_GS) st = silu::amg_gs_factors(G->host, msg);
    if (st != silu::H_OK) return silu::set_err(ctx, (silu_status)st, msg);
    // levels 1 .. ilu_levels - 1 above the coarsest: an incomplete
    // factorisation of A_l of F's kind, row-scaled, as a factor object
    const int nlev = (int)G->host.lev.size();
    G->ilu_levels = std::max(1, std::min(p.ilu_levels, nlev - 1));
    G->ilu_mat.assign(nlev, nullptr);
    G->ilu_fac.assign(nlev, nullptr);
    for (int l = 1; l < G->ilu_levels; ++l) {
      const silu::Csr& Al = G->host.lev[l].A;
      silu_status sl = silu_mat_create(ctx, Al.n, Al.nnz(), Al.rp.data(), Al.ci.data(), Al.va.data(), &G->ilu_mat[l]);
      if (sl == SILU_OK)
        sl = ilu_setup(ctx, G->ilu_mat[l], F->kind, F->tau, F->fill, SILU_SCALE_ROW, F->prec, &G->ilu_fac[l]);
      if (sl != SILU_OK) return sl;  // the context's message names the failure
    }
    if (ctx->device >= 0) {
      silu_status ds = silu::device_ok(ctx);
      if (ds != SILU_OK) return ds;
      cudaStream_t s = ctx->stream;
      const size_t nl = G->host.lev.size();
      cudaError_t e = silu::ensure_vectors(F, 1);
      for (size_t l = 0; e == cudaSuccess && l < nl; ++l) {
        G->lev.emplace_back(new AmgDevLevel);
        e = upload_level(G->host.lev[l], *G->lev[l], l > 0, l + 1 == nl, p.coarse_smoother == SILU_AMG_POLY_GS, s);
      }
      if (e == cudaSuccess)
        e = silu::upload(G->cinv, G->host.coarse_inv.data(), G->host.coarse_inv.size(), s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return silu::cuda_err(ctx, e, "upload of the AMG hierarchy");
      for (silu_ilu FL : G->ilu_fac) {
        if (!FL) continue;
        e = silu::ensure_vectors(FL, 1);
        if (e != cudaSuccess) return silu::cuda_err(ctx, e, "workspace of an AMG level's ILU smoother");
      }
    }
  } catch (const std::bad_alloc&) {
    return silu::set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  F->ws.drop_graphs();  // captured FGMRES iterations may refer to an older hierarchy
  F->config_gen++;
  F->amg = std::move(G);
  return SILU_OK;
}

silu_status silu_amg_vcycle(silu_ilu F, double* x, const double* b, int sweeps_L, int sweeps_U) {
  NvtxRange nvtx_("silu:silu_amg_vcycle");
  if (!F || !x || !b || (sweeps_L < 0) != (sweeps_U < 0)) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (!F->amg) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "no AMG hierarchy (silu_amg_setup)");
  silu_status ds = silu::device_ok(ctx);
  if (ds != SILU_OK) return ds;
  if (F->F.L.n == 0) return SILU_OK;
  try {
    CK(silu::ensure_vectors(F, 1));
    if (sweeps_L < 0) CK(silu::amg_prepare_direct(F));
    silu::amg_cycle(F, x, b, sweeps_L, sweeps_U, false, false, false);
  } catch (const CudaFail& f) {
    return silu::cuda_err(ctx, f.e, f.what);
  }
  return SILU_OK;
}

silu_status silu_amg_vcycle_schur(silu_ilu F, double* x, const double* b, int sweeps_L, int sweeps_U) {
  NvtxRange nvtx_("silu:silu_amg_vcycle_schur");
  if (!F || !x || !b || sweeps_L < 0 || sweeps_U < 0) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (!F->amg) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "no AMG hierarchy (silu_amg_setup)");
  if (!F->schur) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "no Schur complement smoother (silu_schur_setup)");
  silu_status ds = silu::device_ok(ctx);
  if (ds != SILU_OK) return ds;
  if (F->F.L.n == 0) return SILU_OK;
  try {
    CK(silu::ensure_vectors(F, 1));
    silu::amg_cycle(F, x, b, sweeps_L, sweeps_U, false, false, true);
  } catch (const CudaFail& f) {
    return silu::cuda_err(ctx, f.e, f.what);
  }
  return SILU_OK;
}

silu_status silu_amg_level_ilu(silu_ilu F, int level, silu_ilu* out) {
  if (!F || !out) return SILU_ERR_INVALID_ARG;
  *out = nullptr;
  if (!F->amg) return silu::set_err(F->ctx, SILU_ERR_INVALID_ARG, "no AMG hierarchy (silu_amg_setup)");
  const int nlev = (int)F->amg->host.lev.size();
  if (level < 0 || level >= nlev) return silu::set_err(F->ctx, SILU_ERR_INVALID_ARG, "no such level");
  if (level == 0) {
    *out = F;
    return SILU_OK;
  }
  if (!F->amg->ilu_fac[level])
    return silu::set_err(F->ctx, SILU_ERR_INVALID_ARG, "this level has no ILU smoother (silu_amg_params.ilu_levels)");
  *out = F->amg->ilu_fac[level];
  return SILU_OK;
}

silu_status silu_amg_stats(silu_ilu F, int cap, int* levels, int64_t* rows, int64_t* nnz_A, int64_t* nnz_P) {
  if (!F || cap < 0) return SILU_ERR_INVALID_ARG;
  if (!F->amg) return silu::set_err(F->ctx, SILU_ERR_INVALID_ARG, "no AMG hierarchy (silu_amg_setup)");
  const auto& H = F->amg->host.lev;
  if (levels) *levels = (int)H.size();
  for (int l = 0; l < cap && l < (int)H.size(); ++l) {
    if (rows) rows[l] = H[l].A.n;
    if (nnz_A) nnz_A[l] = H[l].A.nnz();
    if (nnz_P) nnz_P[l] = H[l].P.nnz();
  }
  return SILU_OK;
}

silu_status silu_amg_export_level(silu_ilu F, int level, int64_t* Ap, int32_t* Ac, double* Av, int64_t* Pp,
                                  int32_t* Pc, double* Pv, int32_t* cf) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (!F->amg) return silu::set_err(F->ctx, SILU_ERR_INVALID_ARG, "no AMG hierarchy (silu_amg_setup)");
  const auto& H = F->amg->host.lev;
  if (level < 0 || level >= (int)H.size()) return silu::set_err(F->ctx, SILU_ERR_INVALID_ARG, "no such level");
  const silu::AmgLevel& L = H[level];
  auto cp = [](auto* dst, const auto& src) {
    if (dst && !src.empty()) std::memcpy(dst, src.data(), sizeof(src[0]) * src.size());
  };
  cp(Ap, L.A.rp);
  cp(Ac, L.A.ci);
  cp(Av, L.A.va);
  cp(Pp, L.P.rp);
  cp(Pc, L.P.ci);
  cp(Pv, L.P.va);
  cp(cf, L.cf);
  return SILU_OK;
}

}  // extern "C"
