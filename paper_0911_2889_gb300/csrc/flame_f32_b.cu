// FP32 (FLAME_FP32_MIXED) launchers of pass B and their kernels.
#include "flame_ops.cuh"

namespace flame {
template cudaError_t Ops<float>::passB(const FlameDesc &, cudaStream_t, int, const CUtensorMap *);
template cudaError_t Ops<float>::passB_area(const FlameDesc &, cudaStream_t);
template cudaError_t Ops<float>::passB_batch(const FlameDesc *, int, const StepArgs &, cudaStream_t, int,
                                             const CUtensorMap *);
}  // namespace flame
