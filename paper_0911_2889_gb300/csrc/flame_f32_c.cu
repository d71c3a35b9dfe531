// FP32 (FLAME_FP32_MIXED) launchers of pass C (alone and fused with the next
// pass A) and their kernels.
#include "flame_ops.cuh"

namespace flame {
template cudaError_t Ops<float>::passC(const FlameDesc &, cudaStream_t);
template cudaError_t Ops<float>::passCA(const FlameDesc &, cudaStream_t, const CUtensorMap *);
template cudaError_t Ops<float>::passC_batch(const FlameDesc *, int, const StepArgs &, cudaStream_t, bool);
}  // namespace flame
