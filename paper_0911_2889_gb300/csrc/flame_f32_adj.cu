// FP32 (FLAME_FP32_MIXED) launchers of the area objective and the adjoint
// step and their kernels (the adjoint's pass A is the one of flame_f32_a.cu).
#include "flame_ops.cuh"

namespace flame {
extern template cudaError_t Ops<float>::passA(const FlameDesc &, cudaStream_t, int, const CUtensorMap *);
template cudaError_t Ops<float>::area(const AdjDesc &, cudaStream_t);
template cudaError_t Ops<float>::adj_step(const AdjDesc &, cudaStream_t);
}  // namespace flame
