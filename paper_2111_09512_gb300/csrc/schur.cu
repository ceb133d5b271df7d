// The ILUT Schur complement smoother (Sec. 3.1 of the paper, Eq. schur).
//
// The unknowns are split as the paper's subdomain / interface partition:
// `parts` contiguous row blocks stand in for the MPI ranks, a row with an
// entry in another block is an interface row, and A permuted to interior
// rows first is [B E; F C] with B block diagonal.  One application
// z = M^{-1} r:
//   f = r_I, g = r_G;  s = g - F B^{-1} f;
//   one GMRES iteration on S y = s (S = C - F B^{-1} E) from y = 0, which is
//   the minimal-residual step y = ((S s).s / (S s).(S s)) s, so no residual
//   of the full system is formed (the saving the paper points out); with the
//   optional right preconditioner M = diag(C) (not in the paper) the step is
//   y = ((S q).s / (S q).(S q)) q with q = M^{-1} s;
//   x_I = B^{-1} (f - E y);  z = [x_I; y] in the original order.
// Every B^{-1} is the row-scaled ILUT smoother of B from zero: m_L + m_U
// Richardson sweeps on the sweep kernels.
#include <cstring>

#include "internal.h"

using silu::CudaFail;
using silu::Csr;
using silu::DevCsr;
using silu::ProfScope;

namespace {

constexpr int kT = 256;

__global__ void k_gather(int n, const int* __restrict__ rows, const double* __restrict__ in, double* __restrict__ out) {
  const int k = blockIdx.x * kT + threadIdx.x;
  if (k < n) out[k] = in[rows[k]];
}

__global__ void k_scatter(int n, const int* __restrict__ rows, const double* __restrict__ in, double* __restrict__ out) {
  const int k = blockIdx.x * kT + threadIdx.x;
  if (k < n) out[rows[k]] = in[k];
}

cudaError_t gather(int n, const int* rows, const double* in, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<(n + kT - 1) / kT, kT, 0, s>>>(n, rows, in, out);
  return cudaGetLastError();
}

cudaError_t scatter(int n, const int* rows, const double* in, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scatter<<<(n + kT - 1) / kT, kT, 0, s>>>(n, rows, in, out);
  return cudaGetLastError();
}

void op(silu_ilu F, const DevCsr& T, const double* c, const double* in, double* out, int epi) {
  LAUNCH(F->ctx, SILU_K_RESIDUAL, silu::sweep_launch(F, T, silu::MODE_D, 1, 4, 1, c, in, out, nullptr, nullptr, epi));
}

// rows `rows` of A with columns renumbered by cmap (-1: dropped)
void submatrix(const Csr& A, const std::vector<int32_t>& rows, const std::vector<int32_t>& cmap, Csr& S) {
  S.n = (int64_t)rows.size();
  S.rp.assign(S.n + 1, 0);
  S.ci.clear();
  S.va.clear();
  for (size_t t = 0; t < rows.size(); ++t) {
    for (int64_t p = A.rp[rows[t]]; p < A.rp[rows[t] + 1]; ++p)
      if (cmap[A.ci[p]] >= 0) {
        S.ci.push_back(cmap[A.ci[p]]);
        S.va.push_back(A.va[p]);
      }
    S.rp[t + 1] = (int64_t)S.ci.size();
  }
}

}  // namespace

SchurState::~SchurState() {
  if (FB) silu_ilu_destroy(FB);
  if (Bmat) silu_mat_destroy(Bmat);
}

namespace silu {

void schur_apply(silu_ilu F, const double* r, double* z, int mL, int mU) {
  SchurState& S = *F->schur;
  cudaStream_t st = F->ctx->stream;
  silu_ilu FB = S.FB;
  const int nI = (int)S.nI, nG = (int)S.nG;
  double *f = S.f.as<double>(), *u = S.u.as<double>(), *t = S.t.as<double>(), *xi = S.xi.as<double>();
  double *g = S.g.as<double>(), *s = S.s.as<double>(), *w = S.w.as<double>(), *y = S.y.as<double>();
  const int* rI = S.rowsI.as<int>();
  const int* rG = S.rowsG.as<int>();
  LAUNCH(F->ctx, SILU_K_ELEMENTWISE, gather(nI, rI, r, f, st));
  LAUNCH(F->ctx, SILU_K_ELEMENTWISE, gather(nG, rG, r, g, st));
  if (nG > 0) {
    if (nI > 0) {
      smooth_chunk(FB, u, f, 1, 1, 0, mL, mU, true);  // u = B^{-1} f
      op(F, S.F, g, u, s, EPI_STORE);                  // s = g - F u
    } else {
      CK(cudaMemcpyAsync(s, g, sizeof(double) * (size_t)nG, cudaMemcpyDeviceToDevice, st));
    }
    // the direction q: s, or M^{-1} s with M = diag(C)
    double* q = s;
    if (S.iface_prec == 1) {
      q = S.q.as<double>();
      LAUNCH(F->ctx, SILU_K_ELEMENTWISE, launch_scale(nG, 1, 1, s, false, S.cdinv.as<double>(), q, false, st));
    }
    // w = S q = C q - F B^{-1} E q
    op(F, S.C, nullptr, q, w, EPI_SPMV);
    if (nI > 0) {
      op(F, S.E, nullptr, q, t, EPI_SPMV);
      smooth_chunk(FB, u, t, 1, 1, 0, mL, mU, true);
      op(F, S.F, w, u, g, EPI_STORE);  // g is free now: g = C q - F u
      std::swap(g, w);
    }
    LAUNCH(F->ctx, SILU_K_KRYLOV, launch_dot_part(nG, w, s, S.part0.as<double>(), st));
    LAUNCH(F->ctx, SILU_K_KRYLOV, launch_dot_part(nG, w, w, S.part1.as<double>(), st));
    LAUNCH(F->ctx, SILU_K_KRYLOV, launch_mr_step(nG, S.part0.as<double>(), S.part1.as<double>(), q, y, st));
  }
  if (nI > 0) {
    if (nG > 0)
      op(F, S.E, f, y, t, EPI_STORE);  // t = f - E y
    else
      CK(cudaMemcpyAsync(t, f, sizeof(double) * (size_t)nI, cudaMemcpyDeviceToDevice, st));
    smooth_chunk(FB, xi, t, 1, 1, 0, mL, mU, true);  // x_I = B^{-1} (f - E y)
    LAUNCH(F->ctx, SILU_K_ELEMENTWISE, scatter(nI, rI, xi, z, st));
  }
  LAUNCH(F->ctx, SILU_K_ELEMENTWISE, scatter(nG, rG, y, z, st));
}

}  // namespace silu

extern "C" {

silu_status silu_schur_setup(silu_ilu F, int parts, double tau, int fill) {
  NvtxRange nvtx_("silu:silu_schur_setup");
  if (!F || parts < 1 || !(tau >= 0.0) || fill < 0) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  const Csr& A = F->A->A;
  const int64_t n = A.n;
  std::unique_ptr<SchurState> S;
  try {
    S.reset(new SchurState);
    S->parts = parts;
    // block of each row: the k with k n / parts <= i < (k+1) n / parts
    std::vector<int32_t> blk(n);
    for (int k = 0, i = 0; k < parts; ++k)
      for (const int64_t e = ((int64_t)k + 1) * n / parts; i < e; ++i) blk[i] = k;
    S->iface.assign(n, 0);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
        if (blk[A.ci[p]] != blk[i]) {
          S->iface[i] = 1;
          break;
        }
    std::vector<int32_t> rowsI, rowsG, mapI(n, -1), mapG(n, -1);
    for (int64_t i = 0; i < n; ++i) {
      if (S->iface[i]) {
        mapG[i] = (int32_t)rowsG.size();
        rowsG.push_back((int32_t)i);
      } else {
        mapI[i] = (int32_t)rowsI.size();
        rowsI.push_back((int32_t)i);
      }
    }
    S->nI = (int64_t)rowsI.size();
    S->nG = (int64_t)rowsG.size();
    Csr B, E, Fm, C;
    submatrix(A, rowsI, mapI, B);
    submatrix(A, rowsI, mapG, E);
    submatrix(A, rowsG, mapI, Fm);
    submatrix(A, rowsG, mapG, C);
    // 1 / c_kk for the optional diag(C) preconditioner of the interface iteration
    std::vector<double> cdinv((size_t)S->nG, 0.0);
    S->cdiag_ok = true;
    for (int64_t k = 0; k < S->nG; ++k) {
      double d = 0.0;
      for (int64_t p = C.rp[k]; p < C.rp[k + 1]; ++p)
        if (C.ci[p] == k) d = C.va[p];
      if (d == 0.0) S->cdiag_ok = false;
      cdinv[(size_t)k] = d != 0.0 ? 1.0 / d : 0.0;
    }
    silu_status st = silu_mat_create(ctx, B.n, B.nnz(), B.rp.data(), B.ci.data(), B.va.data(), &S->Bmat);
    if (st == SILU_OK) st = ilu_setup(ctx, S->Bmat, SILU_ILUT, tau, fill, SILU_SCALE_ROW, F->prec, &S->FB);
    if (st != SILU_OK) return st;
    if (ctx->device >= 0) {
      silu_status ds = silu::device_ok(ctx);
      if (ds != SILU_OK) return ds;
      cudaStream_t s = ctx->stream;
      cudaError_t e = silu::ensure_vectors(S->FB, 1);
      if (e == cudaSuccess) e = silu::upload_csr(E, false, S->E_rp, S->E_ci, S->E_va, S->E_t, S->E, s);
      if (e == cudaSuccess) e = silu::upload_csr(Fm, false, S->F_rp, S->F_ci, S->F_va, S->F_t, S->F, s);
      if (e == cudaSuccess) e = silu::upload_csr(C, false, S->C_rp, S->C_ci, S->C_va, S->C_t, S->C, s);
      if (e == cudaSuccess) e = silu::upload(S->rowsI, rowsI.data(), rowsI.size(), s);
      if (e == cudaSuccess) e = silu::upload(S->rowsG, rowsG.data(), rowsG.size(), s);
      const size_t bi = sizeof(double) * (size_t)std::max<int64_t>(S->nI, 1);
      const size_t bg = sizeof(double) * (size_t)std::max<int64_t>(S->nG, 1);
      for (DBuf* d : {&S->f, &S->u, &S->t, &S->xi})
        if (e == cudaSuccess) e = d->ensure(bi);
      for (DBuf* d : {&S->g, &S->s, &S->w, &S->y, &S->q})
        if (e == cudaSuccess) e = d->ensure(bg);
      if (e == cudaSuccess && S->nG > 0) e = silu::upload(S->cdinv, cdinv.data(), cdinv.size(), s);
      if (e == cudaSuccess) e = S->r.ensure(sizeof(double) * (size_t)std::max<int64_t>(n, 1));
      if (e == cudaSuccess) e = S->part0.ensure(sizeof(double) * 1024);
      if (e == cudaSuccess) e = S->part1.ensure(sizeof(double) * 1024);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return silu::cuda_err(ctx, e, "upload of the Schur complement smoother");
    }
  } catch (const std::bad_alloc&) {
    return silu::set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  F->ws.drop_graphs();
  F->config_gen++;
  F->schur = std::move(S);
  return SILU_OK;
}

silu_status silu_schur_smooth(silu_ilu F, double* x, const double* b, int sweeps_L, int sweeps_U) {
  NvtxRange nvtx_("silu:silu_schur_smooth");
  if (!F || !x || !b || sweeps_L < 0 || sweeps_U < 0) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (!F->schur) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "no Schur complement smoother (silu_schur_setup)");
  silu_status ds = silu::device_ok(ctx);
  if (ds != SILU_OK) return ds;
  const int n = (int)F->F.L.n;
  if (n == 0) return SILU_OK;
  cudaStream_t s = ctx->stream;
  try {
    SchurState& S = *F->schur;
    double* r = S.r.as<double>();
    LAUNCH(ctx, SILU_K_RESIDUAL, silu::sweep_launch(F, F->A->d, silu::MODE_D, 1, 4, 1, b, x, r, nullptr, nullptr,
                                                    silu::EPI_STORE));
    CK(silu::ensure_vectors(F, 1));
    double* z = F->ws.r.as<double>();
    silu::schur_apply(F, r, z, sweeps_L, sweeps_U);
    LAUNCH(ctx, SILU_K_ELEMENTWISE, silu::launch_addx(n, 1, 1, z, false, nullptr, x, true, s));
  } catch (const CudaFail& f) {
    return silu::cuda_err(ctx, f.e, f.what);
  }
  return SILU_OK;
}

silu_status silu_schur_set_interface_prec(silu_ilu F, int mode) {
  if (!F) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  if (!F->schur) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "no Schur complement smoother (silu_schur_setup)");
  if (mode != 0 && mode != 1) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "mode must be 0 or 1");
  if (mode == 1 && !F->schur->cdiag_ok)
    return silu::set_err(ctx, SILU_ERR_ZERO_PIVOT, "an interface row has a zero diagonal entry");
  if (F->schur->iface_prec != mode) {
    F->schur->iface_prec = mode;
    F->ws.drop_graphs();  // captured FGMRES iterations hold the other form
    F->config_gen++;
  }
  return SILU_OK;
}

silu_status silu_schur_stats(silu_ilu F, int64_t* n_interior, int64_t* n_interface, int32_t* iface) {
  if (!F) return SILU_ERR_INVALID_ARG;
  if (!F->schur) return silu::set_err(F->ctx, SILU_ERR_INVALID_ARG, "no Schur complement smoother (silu_schur_setup)");
  if (n_interior) *n_interior = F->schur->nI;
  if (n_interface) *n_interface = F->schur->nG;
  if (iface && !F->schur->iface.empty())
    std::memcpy(iface, F->schur->iface.data(), sizeof(int32_t) * F->schur->iface.size());
  return SILU_OK;
}

}  // extern "C"
