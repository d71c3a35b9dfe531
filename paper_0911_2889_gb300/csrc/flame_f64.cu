// FP64 instantiation of the kernels and launchers (FLAME_FP64).
#include "flame_ops.cuh"
template struct flame::Ops<double>;
