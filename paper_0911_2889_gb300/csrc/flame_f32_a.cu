// FP32 (FLAME_FP32_MIXED) launchers of pass A and their kernels.
#include "flame_ops.cuh"

namespace flame {
template cudaError_t Ops<float>::passA(const FlameDesc &, cudaStream_t, int, const CUtensorMap *);
template cudaError_t Ops<float>::passA_batch(const FlameDesc *, int, const StepArgs &, cudaStream_t, int,
                                             const CUtensorMap *);
}  // namespace flame
