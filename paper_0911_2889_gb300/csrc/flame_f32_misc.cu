// FP32 (FLAME_FP32_MIXED) twiddle tables, standalone 2-D FFT launchers and
// geometry helpers.
#include "flame_ops.cuh"

namespace flame {
template cudaError_t Ops<float>::init_twiddles(float2 *, int, cudaStream_t);
template cudaError_t Ops<float>::rows_r2c(const float *, float2 *, int, int, const float2 *, cudaStream_t);
template cudaError_t Ops<float>::rows_c2r(const float2 *, float *, int, int, const float2 *, cudaStream_t);
template cudaError_t Ops<float>::cols(const float2 *, float2 *, int, int, int, int, const float2 *, cudaStream_t);
template cudaError_t Ops<float>::box_from_spec(const float2 *, float2 *, double *, int, int, int, int, cudaStream_t);
template Geom Ops<float>::geom_cols(int, int, int);
template Geom Ops<float>::geom_rows(int, int, int);
template void Ops<float>::tiles(const StepArgs &, int, int *, int *, int *);
}  // namespace flame
