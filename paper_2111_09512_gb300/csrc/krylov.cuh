// Launchers of the FP64 Krylov kernels (flexible GMRES, reductions, the
// minimal-residual step of the Schur complement smoother).
#pragma once

#include <cuda_runtime.h>

namespace silu {

// ---- Krylov (FP64, one right-hand side) --------------------------------
// Block partial sums are written to part[0..nparts); every consumer reduces
// them in the same fixed order, so results are bitwise reproducible.
int krylov_parts(int n);
cudaError_t launch_dot_part(int n, const double* a, const double* b, double* part, cudaStream_t s);
// h = sum(part_in); if hout: *hout = h; w -= h vi; part_out = partials of w.vnext (or |w|^2 if vnext null)
cudaError_t launch_mgs_step(int n, const double* part_in, double* hout, double* w, const double* vi,
                            const double* vnext, double* part_out, cudaStream_t s);
// h = sqrt(sum(part_in)); *hout = h; vout = w / h (skipped if h == 0)
cudaError_t launch_normalize(int n, const double* part_in, double* hout, const double* w, double* vout,
                             cudaStream_t s);
// Givens on column j of H (row-major (m+1) x m, leading dim m); writes
// res[0] = |g_{j+1}| and res[1] = h_{j+1,j}
cudaError_t launch_givens(int j, int m, double* H, double* cs, double* sn, double* g, double* res, cudaStream_t s);
// solve the jend x jend triangle, then x += sum_k y_k Z_k
cudaError_t launch_update_x(int n, int jend, int m, const double* H, const double* g, double* y, const double* Z,
                            double* x, cudaStream_t s);
// y = (sum(part_num) / sum(part_den)) s (0 when the denominator sums to 0); both
// partial arrays written by launch_dot_part over n rows
cudaError_t launch_mr_step(int n, const double* part_num, const double* part_den, const double* sv, double* y,
                           cudaStream_t s);
// *out = sqrt(sum(part_in)) for partials written by a launch over n rows
cudaError_t launch_norm_final(int n, const double* part_in, double* out, cudaStream_t s);

}  // namespace silu
