// flame_peak.cu -- measured FMA throughput of this GPU in FP64 and FP32
// (flame_fma_peak), the denominator the FP64 step is reported against: the
// FP64 path of the step is bound by GB300's narrow FP64 units, not by HBM.
//
// Every thread runs 8 independent FMA chains (x <- x * a + b) for `iters`
// iterations, so the FMA pipe sees enough independent work to stay full; the
// grid is 8 CTAs of 256 threads per SM.  The chains' results are folded
// into one store per thread, so nothing is optimised away.
#include <cuda_runtime.h>

#include "flame.h"
#include "flame_internal.h"

namespace {

template <class R>
__global__ void __launch_bounds__(256) k_fma_chains(R *sink, int iters, R a, R b) {
    R x0 = (R)threadIdx.x, x1 = x0 + (R)1, x2 = x0 + (R)2, x3 = x0 + (R)3;
    R x4 = x0 + (R)4, x5 = x0 + (R)5, x6 = x0 + (R)6, x7 = x0 + (R)7;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <class R> cudaError_t run(int iters, R *sink, int blocks, cudaStream_t s) {
    k_fma_chains<R><<<blocks, 256, 0, s>>>(sink, iters, (R)0.999999, (R)1e-7);
    return cudaGetLastError();
}

}  // namespace

extern "C" flame_status flame_fma_peak(int prec, double *flops_per_s) {
    if (!flops_per_s || (prec != FLAME_FP64 && prec != FLAME_FP32_MIXED)) {
        flame::set_last_error("flame_fma_peak: bad argument");
        return FLAME_EINVAL;
    }
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 8 * nsm, threads = 256;
    const int iters = prec == FLAME_FP64 ? 2048 : 65536;
    void *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)blocks * threads * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run is the warm-up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess)
            e = prec == FLAME_FP64 ? run<double>(iters, static_cast<double *>(sink), blocks, s)
                                   : run<float>(iters, static_cast<float *>(sink), blocks, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    if (e != cudaSuccess) {
        flame::set_last_error(cudaGetErrorString(e));
        return FLAME_ECUDA;
    }
    const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads;
    *flops_per_s = flops / (best * 1e-3);
    return FLAME_OK;
}
