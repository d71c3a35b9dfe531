// flame_noalloc.cu -- flame_step_noalloc: the explicit step for callers that
// may not allocate device memory.
//
// Who needs this: code that runs where a cudaMalloc is not allowed or not
// safe -- for example inside a host callback or another library's hook that
// forbids allocation, under a memory manager that owns every byte of the
// device, or in a process whose allocator must never be re-entered.  Such a
// caller still owns and passes its state, mean mode and time; this entry
// point brings its own scratch (twiddle tables, the two step workspaces and
// the status word) in one statically sized device array, so it never calls
// cudaMalloc, cudaFree, a graph instantiation or any other allocating routine.
//
// The scratch array below is part of the library image: every GPU that loads
// libflame.so holds its kNoAllocScratchBytes until the process exits.  All
// calls on a device share it, and it keeps whatever the last call left in it,
// so two calls whose work overlaps on the GPU (different streams, no ordering
// between them) race on it and give wrong results.  Each call rewrites all of
// the scratch it reads (tables, workspaces) and clears the status word, so
// ordered calls of different sizes do not see each other's data.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "flame.h"
#include "flame_internal.h"
#include "fft_engine.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;  // 8 MiB per device

// The scratch itself.  In host code this name is only a stand-in for the
// symbol, never a usable address: the device address is obtained with
// cudaGetSymbolAddress once per device (see scratch_on_device).
static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
// Device address per device, set on the first call made on that device.
// Calls may come from several host threads: the lookup is done once per
// device under a mutex and published through an atomic.
std::atomic<void *> g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mu;

// Errors are reported through flame_last_error(), like every other call.
flame_status nfail(flame_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    flame::set_last_error(buf);
    return s;
}

// Device address of g_scratch on the current device, looked up on the first
// call made on that device (with the device current).
flame_status scratch_on_device(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(FLAME_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(FLAME_EUNSUPPORTED, "device %d out of range", dev);
    void *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        p = g_scratch_ptr[dev].load(std::memory_order_relaxed);
        if (!p) {
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p)
                return nfail(FLAME_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            g_scratch_ptr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return FLAME_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }
int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

template <class R>
flame_status run_steps(const flame::StepArgs &a, unsigned char *base, size_t off_tw1, size_t off_twm,
                       size_t off_uv, size_t off_gk, size_t off_sc, void *state, double *mean, double *t,
                       int nsteps, cudaStream_t s) {
    using C = typename flame::Ops<R>::C;
    cudaError_t e = flame::Ops<R>::init_twiddles(reinterpret_cast<C *>(base + off_tw1), a.logn1, s);
    if (e == cudaSuccess) e = flame::Ops<R>::init_twiddles(reinterpret_cast<C *>(base + off_twm), a.logm, s);
    double *dscal = reinterpret_cast<double *>(base + off_sc);
    int *status = reinterpret_cast<int *>(base + off_sc + 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);  // must start at zero
    if (e != cudaSuccess) return nfail(FLAME_ECUDA, "flame_step_noalloc set-up: %s", cudaGetErrorString(e));
    flame::FlameDesc d;
    memset(&d, 0, sizeof d);
    d.a = a;
    d.state = state;
    d.uv = base + off_uv;
    d.gk = base + off_gk;
    d.tw1 = base + off_tw1;
    d.twm = base + off_twm;
    d.t_in = t;
    d.coef = dscal + 8;  // 48 bytes at off_sc + 64 (the arena keeps 256 bytes there)
    d.mean = mean;
    d.t_out = t;
    d.status = status;
    for (int i = 0; i < nsteps; ++i) {
        e = flame::Ops<R>::passA(d, s);
        if (e == cudaSuccess) e = flame::Ops<R>::passB(d, s);
        if (e == cudaSuccess) e = flame::Ops<R>::passC(d, s);
        if (e != cudaSuccess) return nfail(FLAME_ECUDA, "flame_step_noalloc launch: %s", cudaGetErrorString(e));
    }
    return FLAME_OK;
}

}  // namespace

extern "C" {

flame_status flame_step_noalloc(const flame_params *params, void *state, double *mean_mode, double *t,
                                int nsteps, void *stream) {
    if (!params || !state || !mean_mode || !t) return nfail(FLAME_EINVAL, "flame_step_noalloc: null pointer");
    if (nsteps < 0) return nfail(FLAME_EINVAL, "flame_step_noalloc: nsteps=%d < 0", nsteps);
    flame_params p = *params;
    if (p.prec != FLAME_FP64 && p.prec != FLAME_FP32_MIXED)
        return nfail(FLAME_EINVAL, "flame_step_noalloc: unknown precision %d", (int)p.prec);
    if (!pow2_in(p.n_theta, 16, 4096) || !pow2_in(p.n_phi, 32, 8192))
        return nfail(FLAME_EUNSUPPORTED, "flame_step_noalloc: grid %dx%d not supported", p.n_theta, p.n_phi);
    if (p.K1 < 0 || p.K2 < 0) return nfail(FLAME_EINVAL, "flame_step_noalloc: negative K");
    if (p.K1 == 0) p.K1 = (p.n_theta - 1) / 4;
    if (p.K2 == 0) p.K2 = (p.n_phi - 1) / 4;
    if (4 * p.K1 + 1 > p.n_theta || 4 * p.K2 + 1 > p.n_phi)
        return nfail(FLAME_EINVAL, "flame_step_noalloc: need 4K+1 <= N");
    if (!std::isfinite(p.gamma) || !(p.theta_pi > 0) || !std::isfinite(p.theta_pi) || !(p.s1 >= 0) ||
        !(p.s2 >= 0) || !std::isfinite(p.s1) || !std::isfinite(p.s2) || !(p.t0 > 0) || !(p.dt > 0) ||
        !std::isfinite(p.t0) || !std::isfinite(p.dt) || (p.flags & ~3u) || p.flags == 3u)
        return nfail(FLAME_EINVAL, "flame_step_noalloc: invalid model parameters");
    if (p.s1 == 0) p.s1 = p.theta_pi;
    if (p.s2 == 0) p.s2 = p.theta_pi;

    flame::StepArgs a;
    memset(&a, 0, sizeof a);
    a.n1 = p.n_theta;
    a.n2 = p.n_phi;
    a.logn1 = ilog2(p.n_theta);
    a.logm = ilog2(p.n_phi / 2);
    a.K1 = p.K1;
    a.K2 = p.K2;
    a.ldk = p.K2 + 1;
    a.s1 = p.s1;
    a.s2 = p.s2;
    a.s1f = (float)p.s1;
    a.s2f = (float)p.s2;
    a.gamma = p.gamma;
    a.t0 = p.t0;
    a.dt = p.dt;
    a.flags = p.flags;

    // scratch layout: twiddles (N1), twiddles (N2/2), (U,V), G, scalars
    const size_t csz = p.prec == FLAME_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t off_tw1 = 0;
    const size_t off_twm = off_tw1 + align256(flame::tw_alloc_len(a.logn1) * csz);
    const size_t off_uv = off_twm + align256(flame::tw_alloc_len(a.logm) * csz);
    const size_t off_gk = off_uv + align256((size_t)a.n1 * a.ldk * 2 * csz);
    // gk holds column pairs: an even number of columns
    const size_t off_sc = off_gk + align256((size_t)a.n1 * ((a.ldk + 1) & ~1) * csz);
    const size_t need = off_sc + 256;
    if (need > kNoAllocScratchBytes)
        return nfail(FLAME_EUNSUPPORTED,
                     "flame_step_noalloc: grid %dx%d needs %zu bytes of scratch, the static maximum is %zu",
                     p.n_theta, p.n_phi, need, kNoAllocScratchBytes);
    if (nsteps == 0) return FLAME_OK;

    void *scratch = nullptr;
    flame_status st = scratch_on_device(&scratch);
    if (st != FLAME_OK) return st;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p.prec == FLAME_FP64)
        return run_steps<double>(a, base, off_tw1, off_twm, off_uv, off_gk, off_sc, state, mean_mode, t, nsteps, s);
    return run_steps<float>(a, base, off_tw1, off_twm, off_uv, off_gk, off_sc, state, mean_mode, t, nsteps, s);
}

}  // extern "C"
