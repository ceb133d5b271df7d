// Diagnostics of the sweep factors on the device.
//
// silu_ilu_power_norms: the numerical nilpotence of Sec. 5.2 (Fig. Up).  The
// Neumann series of the Richardson sweeps may be truncated after p terms
// once ||T^p||_2 is small, long before the guaranteed nilpotence index; the
// paper plots ||U_s^p||_2 against p.  Here each ||T^p||_2 is estimated by
// power iteration on (T^p)^T T^p, with every product an SpMV of the sweep
// kernels (T) or of T's transpose (built on the host for the call), and the
// norms by the deterministic block-partial reductions of the Krylov kernels.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

using silu::Csr;
using silu::CudaFail;
using silu::ProfScope;
using silu::DevCsr;

namespace {

// CSR of the transpose (rows of T^T = columns of T), columns ascending.
void transpose(const Csr& T, Csr& Tt) {
  const int64_t n = T.n;
  Tt.n = n;
  Tt.rp.assign(n + 1, 0);
  for (int32_t c : T.ci) Tt.rp[c + 1]++;
  for (int64_t i = 0; i < n; ++i) Tt.rp[i + 1] += Tt.rp[i];
  Tt.ci.resize(T.ci.size());
  Tt.va.resize(T.va.size());
  std::vector<int64_t> fill(Tt.rp.begin(), Tt.rp.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = T.rp[i]; p < T.rp[i + 1]; ++p) {
      const int64_t q = fill[T.ci[p]]++;
      Tt.ci[q] = (int32_t)i;
      Tt.va[q] = T.va[p];
    }
}

}  // namespace

extern "C" silu_status silu_ilu_power_norms(silu_ilu F, int which, int pmax, int iters, const double* v0,
                                            double* out) {
  NvtxRange nvtx_("silu:silu_ilu_power_norms");
  if (!F || !v0 || !out || (which != 0 && which != 1) || pmax < 1 || iters < 1) return SILU_ERR_INVALID_ARG;
  silu_ctx ctx = F->ctx;
  silu_status ds = silu::device_ok(ctx);
  if (ds != SILU_OK) return ds;
  const Csr& T = which == 0 ? F->F.L : F->Us;
  const int n = (int)T.n;
  if (n == 0) {
    std::fill(out, out + pmax, 0.0);
    return SILU_OK;
  }
  double v0n = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(v0[i])) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "non-finite start vector");
    v0n += v0[i] * v0[i];
  }
  if (v0n == 0.0) return silu::set_err(ctx, SILU_ERR_INVALID_ARG, "zero start vector");
  cudaStream_t s = ctx->stream;
  try {
    Csr Tt;
    transpose(T, Tt);
    DBuf rp, ci, va, tiles, trp, tci, tva, ttiles, dv0, dv, da, db, part, dout, dz;
    DevCsr dT, dTt;
    CK(silu::upload_csr(T, false, rp, ci, va, tiles, dT, s));
    CK(silu::upload_csr(Tt, false, trp, tci, tva, ttiles, dTt, s));
    CK(silu::upload(dv0, v0, (size_t)n, s));
    CK(dv.ensure(sizeof(double) * n));
    CK(da.ensure(sizeof(double) * n));
    CK(db.ensure(sizeof(double) * n));
    CK(part.ensure(sizeof(double) * 1024));
    CK(dout.ensure(sizeof(double) * (size_t)pmax));
    CK(dz.ensure(sizeof(double)));
    double* v = dv.as<double>();
    double* a = da.as<double>();
    double* b = db.as<double>();
    double* pt = part.as<double>();
    double* o = dout.as<double>();
    const int lT = pick_lanes(T), lTt = pick_lanes(Tt);
    // one product: dst = M src (EPI_SPMV), through the same launcher as the sweeps
    auto spmv = [&](const DevCsr& M, int lanes, const double* src, double* dst) {
      LAUNCH(ctx, SILU_K_SWEEP_U, silu::sweep_launch(F, M, silu::MODE_D, 1, lanes, 1, nullptr, src, dst, nullptr,
                                                     nullptr, silu::EPI_SPMV));
    };
    for (int p = 1; p <= pmax; ++p) {
      // v = v0 / ||v0||
      LAUNCH(ctx, SILU_K_KRYLOV, silu::launch_dot_part(n, dv0.as<double>(), dv0.as<double>(), pt, s));
      LAUNCH(ctx, SILU_K_KRYLOV, silu::launch_normalize(n, pt, o + (p - 1), dv0.as<double>(), v, s));
      for (int it = 0; it < iters; ++it) {
        const double* src = v;
        double* pp[2] = {a, b};
        for (int k = 0; k < p; ++k) {  // a = T^p v
          spmv(dT, lT, src, pp[k & 1]);
          src = pp[k & 1];
        }
        LAUNCH(ctx, SILU_K_KRYLOV, silu::launch_dot_part(n, src, src, pt, s));
        LAUNCH(ctx, SILU_K_KRYLOV, silu::launch_norm_final(n, pt, o + (p - 1), s));  // s_p = ||T^p v||
        const int base = p & 1;  // the buffer src points at is pp[(p - 1) & 1]
        for (int k = 0; k < p; ++k) {  // (T^T)^p T^p v
          double* dst = pp[(base + k) & 1];
          spmv(dTt, lTt, src, dst);
          src = dst;
        }
        LAUNCH(ctx, SILU_K_KRYLOV, silu::launch_dot_part(n, src, src, pt, s));
        // v = z / ||z|| (left unchanged when z = 0, where s_p is 0 as well)
        LAUNCH(ctx, SILU_K_KRYLOV, silu::launch_normalize(n, pt, dz.as<double>(), src, v, s));
      }
    }
    CK(cudaMemcpyAsync(out, o, sizeof(double) * (size_t)pmax, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } catch (const silu::CudaFail& f) {
    return silu::cuda_err(ctx, f.e, f.what);
  } catch (const std::bad_alloc&) {
    return silu::set_err(ctx, SILU_ERR_OOM, "out of host memory");
  }
  return SILU_OK;
}
