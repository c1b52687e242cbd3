// images.h -- images of a point source and the lensed Gaussian source on a
// deflected ray grid (images.cu).
#pragma once
#include "lens_internal.h"

namespace lens {
// Image cells of the point source (b1, b2) on the (ny+1) x (nx+1) corner
// grid y; writes at most max_out entries, returns the number found.
int64_t find_images(const double* y, int64_t nx, int64_t ny, double x0, double y0, double h,
                    double b1, double b2, int64_t max_out, double* out, int64_t* cells,
                    DeviceAlloc& da, cudaStream_t s);
// out[r] = exp(-|y_r - beta|^2 / 2 sigma^2)
void source_image(const double* y, int64_t m, double b1, double b2, double sigma, double* out,
                  cudaStream_t s);
}  // namespace lens
