// adjoint.cu -- transposed FMM: gradients of a loss through Eq. 1 with
// respect to star positions, masses, kappa_s and gamma (not in the paper).
#include "cx.cuh"
#include "lens_internal.h"

namespace lens {

void adjoint(Plan& P, const double* rays, int64_t m, const double* gy, double* gxy, double* gm,
             double* gkg, cudaStream_t s) {
  (void)P; (void)rays; (void)m; (void)gy; (void)gxy; (void)gm; (void)gkg; (void)s;
  fail(LENS_EINVAL, "lens_deflect_adjoint: not available in this build");
}

}  // namespace lens
