// potential.h -- the lensing potential through the plan's expansions
// (potential.cu).
#pragma once
#include "lens_internal.h"

namespace lens {
// psi at m rays (dev m x 2) into psi (dev m); the plan's expansions must be
// complete (waits for them on `s`).
void evaluate_potential(Plan& P, const double* rays, int64_t m, double* psi, cudaStream_t s);
}  // namespace lens
