// Heun's second-order step (the explicit two-stage Runge-Kutta method) of
// eq. (SivCurv1c), composed from the Euler step: with Phi* = E(Phi_n) and
// E(Phi*) = Phi* + dt F(Phi*, t_{n+1}), the update
// Phi_n + (dt/2) (F(Phi_n, t_n) + F(Phi*, t_{n+1})) is (Phi_n + E(Phi*))/2.
#include "flame_heun.h"
#include "flame_ops.cuh"

namespace flame {

// s0: Phi_n (n entries), s: E(Phi*) in place; sc[0], sc[1]: Phi_0 and t at
// t_n; mean, t: the caller's, after the two Euler steps (t = t_{n+2}), set
// to the averaged mean mode and t_{n+1}.
template <class R>
__global__ void k_heun_combine(const CplxT<R> *__restrict__ s0, CplxT<R> *__restrict__ s, long n,
                               const double *__restrict__ sc, double *mean, double *t, double t0, double dt) {
    using C = CplxT<R>;
    const R half = (R)0.5;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const C a = s0[i], b = s[i];
        s[i] = C{(a.x + b.x) * half, (a.y + b.y) * half};
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *mean = 0.5 * (sc[0] + *mean);
        const long k = __double2ll_rn((sc[1] - t0) / dt);
        *t = t0 + (double)(k + 1) * dt;
    }
}

template <class R>
static cudaError_t launch_heun(const CplxT<R> *s0, CplxT<R> *s, long n, const double *sc, double *mean, double *t,
                               double t0, double dt, cudaStream_t st) {
    const int blocks = (int)std::max<long>(1, std::min<long>((n + 255) / 256, 8L * sm_count()));
    return launch_cl(k_heun_combine<R>, dim3(blocks), 256, 0, st, 1, s0, s, n, sc, mean, t, t0, dt);
}

cudaError_t heun_combine(const float2 *s0, float2 *s, long n, const double *sc, double *mean, double *t, double t0,
                         double dt, cudaStream_t st) {
    return launch_heun<float>(s0, s, n, sc, mean, t, t0, dt, st);
}

cudaError_t heun_combine(const double2 *s0, double2 *s, long n, const double *sc, double *mean, double *t, double t0,
                         double dt, cudaStream_t st) {
    return launch_heun<double>(s0, s, n, sc, mean, t, t0, dt, st);
}

}  // namespace flame
