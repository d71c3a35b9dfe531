// FP32 instantiation of the kernels and launchers (FLAME_FP32_MIXED).
#include "flame_ops.cuh"
template struct flame::Ops<float>;
