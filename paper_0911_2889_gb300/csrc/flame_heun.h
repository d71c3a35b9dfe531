// Heun's second-order step of eq. (SivCurv1c) from two Euler steps: the
// combining launch (flame_heun.cu).
#pragma once
#include <cuda_runtime.h>

namespace flame {
// s0: Phi_n (n complex entries); s: the state after two Euler steps, in
// place -> (Phi_n + s)/2; sc[0], sc[1]: Phi_0 and t at t_n (device);
// mean, t: the caller's device scalars -> the averaged mean mode and t_{n+1}.
cudaError_t heun_combine(const float2 *s0, float2 *s, long n, const double *sc, double *mean, double *t, double t0,
                         double dt, cudaStream_t st);
cudaError_t heun_combine(const double2 *s0, double2 *s, long n, const double *sc, double *mean, double *t, double t0,
                         double dt, cudaStream_t st);
}  // namespace flame
