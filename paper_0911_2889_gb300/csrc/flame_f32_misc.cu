// FP32 (FLAME_FP32_MIXED) twiddle tables, standalone 2-D FFT launchers and
// geometry helpers.
#include "flame_ops.cuh"

namespace flame {
template cudaError_t Ops<float>::init_twiddles(float2 *, int, cudaStream_t);
template cudaError_t Ops<float>::rows_r2c(const float *, float2 *, int, int, const float2 *, cudaStream_t, int *);
template cudaError_t Ops<float>::rows_c2r(const float2 *, float *, int, int, const float2 *, cudaStream_t, int *);
template cudaError_t Ops<float>::cols(const float2 *, float2 *, int, int, int, int, const float2 *, cudaStream_t, int *);
template cudaError_t Ops<float>::box_from_spec(const float2 *, float2 *, double *, int, int, int, int, cudaStream_t, int *);
template Geom Ops<float>::geom_cols(int, int, int);
template Geom Ops<float>::geom_rows(int, int, int);
template void Ops<float>::tiles(const StepArgs &, int, int *, int *, int *);

#ifdef FLAME_DEBUG_BOUNDS
static __global__ void k_bounds_probe(int *status, int i, int n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        [[maybe_unused]] const bool ok = FLAME_IN(status, i, n, kSiteProbe);
    }
}
cudaError_t bounds_probe(int *status, int i, int n, cudaStream_t s) {
    k_bounds_probe<<<1, 32, 0, s>>>(status, i, n);
    return cudaGetLastError();
}
#else
cudaError_t bounds_probe(int *, int, int, cudaStream_t) { return cudaErrorNotSupported; }
#endif
}  // namespace flame
