// flame_kernels.cuh -- the kernels of the spectral flame step and of the
// standalone 2-D real FFTs, templated on the working precision R.
//
// Step of eq. (SivCurv1c) (Sec. 2) with the FFT evaluation of the quadratic
// term (Sec. 3), in three passes over HBM:
//   pass A (columns): i kappa_1 Phi and Phi -> zero-padded inverse FFT along
//                     k1 (the first index, Sec. 3) -> U(j1,k2), V(j1,k2)
//   pass B (rows):    inverse FFT along k2 of U + iV -> u + iv on the grid,
//                     g = u^2 + v^2 = |grad Phi|^2, forward real FFT of g
//                     along j2, keep k2 <= K2 -> G(j1,k2)
//   pass C (columns): forward FFT along j1, keep |k1| <= K1, scale,
//                     Euler update with the linear operator, symmetrization
//                     of the k2 = 0 column (Sec. 3), FP64 mean mode and time.
// The transposition the paper performs with MPI_ALLTOALL between the column
// and row transforms (Sec. 3) is the change of access direction between
// passes: each pass reads and writes whole tiles, and the reordering inside a
// transform goes through shared memory.
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>  // CUtensorMap

#include "fft_engine.cuh"
#include "flame_internal.h"

namespace flame {

template <class R> using CplxT = typename VecOf<R>::c;  // float2 / double2

// Index checks of the index-checking build (-DFLAME_DEBUG_BOUNDS).
// FLAME_IN(status, i, n, site) is true when 0 <= i < n.  Otherwise it sets
// kStatusBounds in the status word, records the first failure (site, index,
// extent) in the three words after it, and is false: the caller then skips
// the access, so a bad index is reported instead of touching memory outside
// its array.  In the normal build it is the constant true and the index
// expression is not evaluated.
#ifdef FLAME_DEBUG_BOUNDS
static __device__ __noinline__ bool bounds_fail(int *status, int site, long long i, long long n) {
    if (status) {
        atomicOr(status, 1 << kStatusBounds);
        if (atomicCAS(status + 1, 0, site) == 0) {
            status[2] = (int)i;
            status[3] = (int)n;
        }
    }
    return false;
}
#define FLAME_IN(status, i, n, site)                                                     \
    ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n) ||          \
     ::flame::bounds_fail((status), (site), (long long)(i), (long long)(n)))
#else
#define FLAME_IN(status, i, n, site) true
#endif
// Extents (complex entries) of the step's arrays: the compact box (state,
// forcing, stage buffer), the (U, V) workspace and the G workspace (column
// pairs: an even number of columns).
__host__ __device__ __forceinline__ long long box_len(const StepArgs &a) { return (long long)(2 * a.K1 + 1) * a.ldk; }
__host__ __device__ __forceinline__ long long uv_len(const StepArgs &a) { return 2LL * a.n1 * a.ldk; }
__host__ __device__ __forceinline__ long long gk_len(const StepArgs &a) { return (long long)a.n1 * ((a.ldk + 1) & ~1); }
static_assert(sizeof(float2) == sizeof(VecOf<float>::type) && sizeof(double2) == sizeof(VecOf<double>::type), "C and V sizes");

// s1, s2 in the kernel's precision (the FP32 copies are rounded on the host)
template <class R> __device__ __forceinline__ R scale1(const StepArgs &s) {
    if constexpr (std::is_same<R, float>::value) return s.s1f;
    else return s.s1;
}
template <class R> __device__ __forceinline__ R scale2(const StepArgs &s) {
    if constexpr (std::is_same<R, float>::value) return s.s2f;
    else return s.s2;
}

// FP32 kernels fit 128 registers (two CTAs of 256 threads per SM); FP64
// kernels need up to 255 (one CTA per SM).
template <class R> constexpr int kMinBlocks = sizeof(R) == 4 ? 2 : 1;

// Element of the interleaved (U, V) workspace: two complex numbers.
template <class R> struct UV { CplxT<R> u, v; };

// Index (in complex units) of element (j1, k2) of the gk workspace: column
// pairs interleaved, ((k2/2) N1 + j1) * 2 + k2 % 2, so that a column pair is
// one contiguous block read 16 bytes per row (pass C) and the two rows of a
// row pair at two adjacent k2 fill one 32-byte sector (pass B).
__host__ __device__ __forceinline__ size_t gk_index(int j1, int k2, int n1) {
    return (((size_t)(k2 >> 1) * n1 + j1) << 1) + (k2 & 1);
}

// Index (in complex units) of element (j1, k2) of the uv workspace: row pairs
// are interleaved, ((j1/2) ldk + k2) * 2 + j1 % 2 pairs of (U, V), so that a
// row pair is one contiguous block (pass B) and a column's row pair is one
// 32-byte sector (pass A).
__host__ __device__ __forceinline__ size_t uv_index(int j1, int k2, int ldk) {
    return 2 * ((((size_t)(j1 >> 1) * ldk + k2) << 1) + (j1 & 1));
}

template <class R> __device__ __forceinline__ UV<R> ld_uv(const CplxT<R> *p) {
    if constexpr (std::is_same<R, float>::value) {
        float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
    } else {
        return {__ldg(p), __ldg(p + 1)};
    }
}
// (U, V) in shared memory (16-byte aligned slots)
template <class R> __device__ __forceinline__ UV<R> ld_uv_s(const UV<R> *p) {
    if constexpr (std::is_same<R, float>::value) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
    } else {
        const double2 *d = reinterpret_cast<const double2 *>(p);
        return {d[0], d[1]};
    }
}
template <class R> __device__ __forceinline__ void st_uv_s(UV<R> *p, UV<R> e) {
    if constexpr (std::is_same<R, float>::value) {
        *reinterpret_cast<float4 *>(p) = make_float4(e.u.x, e.u.y, e.v.x, e.v.y);
    } else {
        double2 *d = reinterpret_cast<double2 *>(p);
        d[0] = e.u;
        d[1] = e.v;
    }
}
template <class R> __device__ __forceinline__ void st_uv(CplxT<R> *p, CplxT<R> u, CplxT<R> v) {
    if constexpr (std::is_same<R, float>::value) {
        *reinterpret_cast<float4 *>(p) = make_float4(u.x, u.y, v.x, v.y);
    } else {
        p[0] = u;
        p[1] = v;
    }
}

template <class R> __device__ __forceinline__ CV<typename VecOf<R>::type> pack2(CplxT<R> a, CplxT<R> b) {
    using V = typename VecOf<R>::type;
    return {V{a.x, b.x}, V{a.y, b.y}};
}
template <class R> __device__ __forceinline__ CplxT<R> lane0(CV<typename VecOf<R>::type> z) {
    return CplxT<R>{z.re.x, z.im.x};
}
template <class R> __device__ __forceinline__ CplxT<R> lane1(CV<typename VecOf<R>::type> z) {
    return CplxT<R>{z.re.y, z.im.y};
}

// ----------------------------------------------------------------------------
// The retained modes of a 2-D real field (Sec. 2's physical-space initial
// perturbation): spec is the field's unnormalised r2c, N1 x (N2/2+1)
// row-major; box entry (k1, k2), ABI index k2 (2K1+1) + k1 + K1, is
// spec[k1 mod N1][k2] / (N1 N2).  On k2 = 0 the k1 < 0 entries are the
// conjugates of the k1 > 0 ones, the k = 0 slot is 0, and the field's mean
// (FP64) goes to *mean.
template <class R>
__global__ void k_box_from_spec(const CplxT<R> *__restrict__ spec, CplxT<R> *__restrict__ state, double *mean,
                                int n1, int n2, int K1, int K2, int *status) {
    using C = CplxT<R>;
    const int ld1 = 2 * K1 + 1, ldm = n2 / 2 + 1;
    const long total = (long)ld1 * (K2 + 1);
    const double inv = 1.0 / ((double)n1 * (double)n2);
    const R rinv = (R)inv;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int k2 = (int)(i / ld1), k1 = (int)(i % ld1) - K1;
        C v{0, 0};
        if (k1 == 0 && k2 == 0) {
            *mean = (double)spec[0].x * inv;
        } else {
            const bool mirror = k2 == 0 && k1 < 0;
            const int row = mirror ? -k1 : (k1 < 0 ? k1 + n1 : k1);
            const long long si = (long long)row * ldm + k2;
            const C s = FLAME_IN(status, si, (long long)n1 * ldm, kSiteBoxSpec) ? spec[si] : C{0, 0};
            v = C{s.x * rinv, (mirror ? -s.y : s.y) * rinv};
        }
        if (FLAME_IN(status, i, total, kSiteBoxSpec)) state[i] = v;
    }
}

// ----------------------------------------------------------------------------
// Twiddle table generation (FP64 sincospi, rounded once)
// ----------------------------------------------------------------------------
template <class R> __global__ void k_twiddles(CplxT<R> *tab, int logN, int LE) {
    const int N = 1 << logN, E = 1 << LE;
    const int len = tw_table_len(logN, LE);
    const int fin = tw_final_offset(logN, LE);
    const int real = tw_real_offset(logN, LE);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        long num, den;  // angle = 2 pi num / den
        if (i < fin) {
            int off = 0, ns = E;
            while (i >= off + (E - 1) * ns) { off += (E - 1) * ns; ns <<= LE; }
            int r = (i - off) / ns + 1, m = (i - off) % ns;
            num = (long)r * m;
            den = (long)E * ns;
        } else if (i < real) {
            int rho = 1 << (logN % LE), ns = N / rho;
            int q = (i - fin) / ns + 1, m = (i - fin) % ns;
            num = (long)q * m;
            den = N;
        } else {
            num = i - real;
            den = 2L * N;
        }
        double s, c;
        sincospi(2.0 * (double)(num % den) / (double)den, &s, &c);
        tab[i] = CplxT<R>{(R)c, (R)s};
    }
}

// ----------------------------------------------------------------------------
// Standalone 2-D real FFT passes
// ----------------------------------------------------------------------------
// Row pass of r2c: two rows per thread group (row 2p, 2p+1), half-length
// complex FFT of h[m] = x[2m] + i x[2m+1] followed by the real-input
// post-processing  Y[k] = E[k] + exp(-2 pi i k/N2) O[k],
// E = (H[k] + conj H[M-k])/2, O = (H[k] - conj H[M-k])/(2i).
// LOG > 0: half length 2^LOG fixed at compile time; LOG = 0: any length.
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_rows_r2c(const R *__restrict__ in, CplxT<R> *__restrict__ out, int n1,
                                                  int logm, const CplxT<R> *__restrict__ tw, int *status) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = LOG > 0 ? 1 << LOG : 1 << logm, T = M >> 4, ldo = M + 1;
    const int g = threadIdx.x / T, t = threadIdx.x % T, G = blockDim.x / T;
    const int pair = blockIdx.x * G + g;
    const bool valid = pair < (n1 >> 1);
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len(M);
    auto sm = make_planes(base, M);
    const C *ra = reinterpret_cast<const C *>(in) + (size_t)(2 * pair) * M;
    const C *rb = ra + M;
    CV<V> x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const bool in = valid && FLAME_IN(status, (long long)(2 * pair + 1) * M + t + r * T, (long long)n1 * M, kSiteFftIn);
        C a = in ? __ldg(ra + t + r * T) : C{0, 0};
        C b = in ? __ldg(rb + t + r * T) : C{0, 0};
        x[r] = pack2<R>(a, b);
    }
    fft_line<-1, LOG>(x, logm, t, sm, tw);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) sm.st(t + r * T, x[r]);
    __syncthreads();
    const C *P = tw + tw_real_offset(LOG > 0 ? LOG : logm);
    C *oa = out + (size_t)(2 * pair) * ldo, *ob = oa + ldo;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = t + r * T;
        CV<V> h = x[r], hc = sm.ld((M - k) & (M - 1));
        const R hf = (R)0.5;
        CV<V> E{vmul(vadd(h.re, hc.re), vbc(hf)), vmul(vsub(h.im, hc.im), vbc(hf))};
        // O = (h - conj hc) / (2i) = (D.im/2, -D.re/2), D = (h.re - hc.re, h.im + hc.im)
        CV<V> O{vmul(vadd(h.im, hc.im), vbc(hf)), vmul(vsub(hc.re, h.re), vbc(hf))};
        C w = __ldg(P + k);  // exp(+2 pi i k/N2); forward uses the conjugate
        CV<V> Y = cadd(E, cmul_s(O, w.x, -w.y));
        if (valid && FLAME_IN(status, (long long)(2 * pair + 1) * ldo + k, (long long)n1 * ldo, kSiteFftOut)) {
            oa[k] = lane0<R>(Y);
            ob[k] = lane1<R>(Y);
        }
    }
    if (valid && t == 0 && FLAME_IN(status, (long long)(2 * pair + 1) * ldo + M, (long long)n1 * ldo, kSiteFftOut)) {
        CV<V> h0 = x[0];
        oa[M] = C{h0.re.x - h0.im.x, 0};
        ob[M] = C{h0.re.y - h0.im.y, 0};
    }
}

// Row pass of c2r: pre-processing H[k] = (Y[k] + conj Y[M-k]) +
// i exp(+2 pi i k/N2) (Y[k] - conj Y[M-k]), half-length inverse FFT, then
// x[2m] = Re h[m], x[2m+1] = Im h[m].
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_rows_c2r(const CplxT<R> *__restrict__ in, R *__restrict__ out, int n1,
                                                  int logm, const CplxT<R> *__restrict__ tw, int *status) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = LOG > 0 ? 1 << LOG : 1 << logm, T = M >> 4, ldi = M + 1;
    const int g = threadIdx.x / T, t = threadIdx.x % T, G = blockDim.x / T;
    const int pair = blockIdx.x * G + g;
    const bool valid = pair < (n1 >> 1);
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len(M);
    auto sm = make_planes(base, M);
    const C *ia = in + (size_t)(2 * pair) * ldi, *ib = ia + ldi;
    const C *P = tw + tw_real_offset(LOG > 0 ? LOG : logm);
    CV<V> x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = t + r * T;
        const bool in = valid && FLAME_IN(status, (long long)(2 * pair + 1) * ldi + M - k, (long long)n1 * ldi, kSiteFftIn) &&
                        FLAME_IN(status, (long long)(2 * pair + 1) * ldi + k, (long long)n1 * ldi, kSiteFftIn);
        C a = in ? __ldg(ia + k) : C{0, 0};
        C b = in ? __ldg(ib + k) : C{0, 0};
        C ac = in ? __ldg(ia + M - k) : C{0, 0};
        C bc = in ? __ldg(ib + M - k) : C{0, 0};
        CV<V> y = pack2<R>(a, b), yc = pack2<R>(ac, bc);
        CV<V> S{vadd(y.re, yc.re), vsub(y.im, yc.im)};
        CV<V> D{vsub(y.re, yc.re), vadd(y.im, yc.im)};
        C w = __ldg(P + k);
        CV<V> wD = cmul_s(D, w.x, w.y);
        x[r] = cadd_rot<1>(S, wD);
    }
    fft_line<1, LOG>(x, logm, t, sm, tw);
    if (valid) {
        C *oa = reinterpret_cast<C *>(out) + (size_t)(2 * pair) * M, *ob = oa + M;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (!FLAME_IN(status, (long long)(2 * pair + 1) * M + t + r * T, (long long)n1 * M, kSiteFftOut)) continue;
            oa[t + r * T] = lane0<R>(x[r]);
            ob[t + r * T] = lane1<R>(x[r]);
        }
    }
}

// Column FFT of length n = 2^logn over ncols columns of a row-major array
// with row stride ld (complex units); columns 2p, 2p+1 form one thread
// group; in may equal out.  The G groups of a CTA take adjacent column
// pairs and interleave their threads (group = thread mod G), so that one
// warp's access to a row covers G adjacent column pairs: NT = 512 threads
// (FP32, 2^10 .. 2^12 points) widens that from 16 to 32 bytes and more.
template <class R, int DIR, int LOG, int NT = 256>
__global__ void __launch_bounds__(NT, NT == 256 ? kMinBlocks<R> : 1)
    k_cols(const CplxT<R> *in, CplxT<R> *out, int logn, int ncols, int ld, const CplxT<R> *__restrict__ tw, int *status) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = LOG > 0 ? 1 << LOG : 1 << logn, T = n >> 4;
    const int G = blockDim.x / T, g = threadIdx.x % G, t = threadIdx.x / G;
    const int c0 = 2 * (blockIdx.x * G + g);
    const bool va = c0 < ncols, vb = c0 + 1 < ncols;
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len(n);
    auto sm = make_planes(base, n);
    CV<V> x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const size_t row = (size_t)(t + r * T) * ld;
        const long long len = (long long)n * ld;
        C a = va && FLAME_IN(status, row + c0, len, kSiteFftIn) ? in[row + c0] : C{0, 0};
        C b = vb && FLAME_IN(status, row + c0 + 1, len, kSiteFftIn) ? in[row + c0 + 1] : C{0, 0};
        x[r] = pack2<R>(a, b);
    }
    fft_line<DIR, LOG>(x, logn, t, sm, tw);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const size_t row = (size_t)(t + r * T) * ld;
        const long long len = (long long)n * ld;
        if (va && FLAME_IN(status, row + c0, len, kSiteFftOut)) out[row + c0] = lane0<R>(x[r]);
        if (vb && FLAME_IN(status, row + c0 + 1, len, kSiteFftOut)) out[row + c0 + 1] = lane1<R>(x[r]);
    }
}

// ----------------------------------------------------------------------------
// Step passes
// ----------------------------------------------------------------------------
// Bulk prefetch of a contiguous range into L2 (no register or shared-memory
// cost): the next wave's input streams from HBM while this wave computes.
// The bulk prefetch needs a 16-byte aligned start and a size that is a
// multiple of 16: the range is shrunk to [align_up(begin), align_down(end)),
// so it never reaches outside [begin, end).
__device__ __forceinline__ void l2_prefetch(const void *begin, size_t bytes) {
    const size_t b = (reinterpret_cast<size_t>(begin) + 15) & ~(size_t)15;
    const size_t e = (reinterpret_cast<size_t>(begin) + bytes) & ~(size_t)15;
    if (e > b)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b), "r"((unsigned)(e - b)) : "memory");
}

// Programmatic dependent launch: wait until the previous kernel on the
// stream has completed and its memory is visible (a no-op when the launch is
// an ordinary one), and let the next kernel's CTAs be scheduled.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Tensor stores (TMA) from shared memory.  The writing threads fence their
// shared-memory stores towards the async proxy, the CTA synchronises, then one
// thread issues the copies, commits them as a bulk group and waits until they
// have read shared memory (a hardware wait on the copy engine, no spinning).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *tm, const void *smem, int x, int y, int z) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<unsigned long long>(tm)),
                 "r"(sa), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
// A tensor map read from global memory (one per flame of an ensemble) is
// made visible to the tensor-map proxy before its first use.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *tm) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<unsigned long long>(tm))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait_read() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Compile-time CTA shape of the FP32 step kernels (LOG > 0): G line groups of
// T = 2^LOG / 16 threads, and, for pass A, clusters of CL CTAs (CL G = 8
// columns) that write their transposed output cooperatively through
// distributed shared memory, one 128-byte line per row.
template <int LOG> struct Shape {
    static constexpr int T = (1 << LOG) >> 4;
    static constexpr int G = T >= 256 ? 1 : 256 / T;
    static constexpr int CL = (LOG > 0 && G <= 8) ? 8 / G : 1;
};
template <> struct Shape<0> {
    static constexpr int T = 0, G = 0, CL = 1;
};

// E points per thread: 16 (runtime-length kernels, FP64) or 8 (compile-time
// FP32 kernels: 512-thread CTAs at 64 registers, two CTAs per SM).
template <int DIR, int LOG, int E, class V, class C>
__device__ __forceinline__ void fft_line_e(CV<V> (&x)[E], int logn, int t, const Planes<V> &sm, const C *tw) {
    if constexpr (E == 8) line_fft_ct<DIR, LOG, 8>(x, t, sm, tw + tw_table_len(LOG, 4), CtaBarrier{});
    else if constexpr (E == 4)
        line_fft_ct<DIR, LOG, 4>(x, t, sm, tw + tw_table_len(LOG, 4) + tw_table_len(LOG, 3), CtaBarrier{});
    else fft_line<DIR, LOG>(x, logn, t, sm, tw);
}

// Shared-memory twiddles of the compile-time FP32 pass-B kernels (E = 16,
// 2^8..2^12; pass B's ~100 KB of shared memory per CTA leaves too little L1
// for its 64 KB of global twiddle tables):
// the 480 factor entries of TwShared, then (pass B) the factors of the real
// post-processing table P[k] = exp(2 pi i k / 2M): Plo[k mod 64], Phi[k / 64].
constexpr int kTwSmemBytes = 6144;  // >= (480 + 64 + 4096/64) * 8
template <class R, int LOG, int E> constexpr bool kSharedTw = std::is_same<R, float>::value && LOG >= 8 && E == 16;

// cos and sin of k pi / 16, k = 0..15: the factors exp(i pi r / E) (E = 16,
// or E = 8 at every second k) that relate the real-transform twiddles of
// the E points of one thread (see passB_body).
struct Roots32 {
    static constexpr double c[16] = {1.0, 0.980785280403230449126182236134239037, 0.923879532511286756128183189396788933,
                                     0.831469612302545237078788377617905756, 0.707106781186547524400844362104849039,
                                     0.555570233019602224742830813948532874, 0.382683432365089771728459984030398866,
                                     0.195090322016128267848284868477022240, 0.0, -0.195090322016128267848284868477022240,
                                     -0.382683432365089771728459984030398866, -0.555570233019602224742830813948532874,
                                     -0.707106781186547524400844362104849039, -0.831469612302545237078788377617905756,
                                     -0.923879532511286756128183189396788933, -0.980785280403230449126182236134239037};
    static constexpr double s[16] = {0.0, 0.195090322016128267848284868477022240, 0.382683432365089771728459984030398866,
                                     0.555570233019602224742830813948532874, 0.707106781186547524400844362104849039,
                                     0.831469612302545237078788377617905756, 0.923879532511286756128183189396788933,
                                     0.980785280403230449126182236134239037, 1.0, 0.980785280403230449126182236134239037,
                                     0.923879532511286756128183189396788933, 0.831469612302545237078788377617905756,
                                     0.707106781186547524400844362104849039, 0.555570233019602224742830813948532874,
                                     0.382683432365089771728459984030398866, 0.195090322016128267848284868477022240};
};

// a * b + c with one rounding, in the precision of the arguments (explicit,
// so that every kernel built from the same body rounds alike)
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// 1/x and sqrt(x) (x > 0) for the area terms: FP32 within a few ulp from the
// hardware reciprocal and reciprocal square root, FP64 correctly rounded
__device__ __forceinline__ float rcp_r(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_r(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }

// b * exp(i pi r / E) * sgn with the factor a compile-time constant
template <int R_, int E, int SGN, class C> __device__ __forceinline__ C mul_root(C b) {
    using Real = decltype(C::x);
    constexpr int k = R_ * (16 / E);
    constexpr Real cr = (Real)(SGN * Roots32::c[k]), ci = (Real)(SGN * Roots32::s[k]);
    if constexpr (k == 0) return SGN > 0 ? b : C{-b.x, -b.y};
    else if constexpr (k == 8) return C{-ci * b.y, ci * b.x};
    else return C{fma_rn(b.x, cr, -(b.y * ci)), fma_rn(b.x, ci, b.y * cr)};
}

template <class C> struct RealTw {
    const C *lo, *hi;
    __device__ __forceinline__ C operator()(int k) const {
        const C a = lo[k & 63], b = hi[k >> 6];
        return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
    }
    // P = exp(2 pi i k / 2M), k < M = 2^LOGM
    template <int LOGM> __device__ __forceinline__ static void fill(C *lo_dst, C *hi_dst, const C *P) {
        for (int i = threadIdx.x; i < 64 + (1 << LOGM) / 64; i += blockDim.x) {
            if (i < 64) lo_dst[i] = __ldg(P + i);
            else hi_dst[i - 64] = __ldg(P + 64 * (i - 64));
        }
    }
};

// CTA shape of the compile-time kernels with E points per thread: G line
// groups of T = 2^LOG / E threads (256 threads for E = 16, 512 for E = 8) and
// clusters of CL CTAs holding 8 line groups (pass A's write-out).
template <int LOG, int E> struct ShapeE {
    static constexpr int T = (1 << LOG) / E;
    static constexpr int THREADS = E == 16 ? 256 : 512;
    static constexpr int G = T >= THREADS ? 1 : THREADS / T;
    static constexpr int CL = (G <= 8) ? 8 / G : 1;
};
template <int E> struct ShapeE<0, E> {  // runtime-length kernels: no clusters
    static constexpr int T = 0, THREADS = 256, G = 0, CL = 1;
};

// Memory layouts (the state's is also documented in include/flame.h):
//   state  column-major compact box: element (k1, k2) at k2 * ld1 + (k1 + K1),
//          ld1 = 2 K1 + 1
//   uv     N1 x (K2+1) pairs (U, V), row pairs interleaved: element (j1, k2)
//          at uv_index(j1, k2, ldk) = 2 (((j1/2) ldk + k2) 2 + j1 % 2), ldk = K2 + 1
//   gk     N1 x (K2+1), column pairs interleaved: element (j1, k2) at
//          gk_index(j1, k2, N1) = ((k2/2) N1 + j1) 2 + k2 % 2
// Every pass reads whole contiguous blocks (state columns, uv rows, gk
// columns); the transposition between the column and row passes is done by
// the scattered stores of passes A and B.

// Pass A (a1 + a2): column k2 of the compact box -> inverse FFT along k1 of
// a = i s1 k1 Phi and b = Phi (one pair of lines), zero padded outside
// |k1| <= K1 (positions K1 < n < N1 - K1; with N1 >= 4 K1 + 1 the registers
// r = 4..11 of the first pass are always zero and are dropped at compile
// time).  Writes uv[j1][k2] = (U, V) with U = synthesis of a, V = i s2 k2 x
// synthesis of b.
template <class R, int LOG, int E, bool CLU = true, bool TMA = false, bool GMAP = false>
__device__ __forceinline__ void passA_body(const FlameDesc &d, int tile, int ntiles, int pf,
                                           const CUtensorMap *tm = nullptr) {
    griddep_wait();
    griddep_launch();
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    const C *__restrict__ state = static_cast<const C *>(d.state);
    C *__restrict__ uv = static_cast<C *>(d.uv);
    const C *__restrict__ tw1 = static_cast<const C *>(d.tw1);
    const int N1 = LOG > 0 ? (1 << LOG) : (1 << a.logn1), T = N1 / E;
    const int G = blockDim.x / T, g = threadIdx.x / T, t = threadIdx.x % T;
    const int ld1 = 2 * a.K1 + 1;
    if (threadIdx.x == 0 && pf > 0 && tile + pf < ntiles) {
        const int c = (tile + pf) * G, nc = min(G, a.K2 + 1 - c);
        if (nc > 0) l2_prefetch(state + (size_t)c * ld1, (size_t)nc * ld1 * sizeof(C));
    }
    const int k2 = tile * G + g;
    const bool valid = k2 <= a.K2;
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len_e<E>(N1);
    auto sm = make_planes_e<E>(base, N1);
    constexpr bool STW = false;  // pass A's twiddles stay in L1 (measured faster)
    C *stw = reinterpret_cast<C *>(reinterpret_cast<V *>(smraw) + (size_t)G * 2 * plane_len_e<E>(N1));
    if constexpr (STW) TwShared<C>::template fill<(STW ? LOG : 8)>(stw, tw1);  // synced by the transform
    const R s1 = scale1<R>(a), s2k2 = scale2<R>(a) * (R)k2;
    const C *col = state + (size_t)k2 * ld1 + a.K1;  // col[k1], k1 = -K1..K1
    // band rows: r < E/4 (k1 = n <= K1) and r >= 3E/4 (k1 = n - N1 >= -K1);
    // the middle half of the registers is zero padding, dropped at compile time
    CV<V> x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        x[r] = CV<V>{vzero(V{}), vzero(V{})};
        if (r < E / 4 || r >= 3 * E / 4) {
            const int n = t + r * T;
            const int k1 = (r < E / 4) ? n : n - N1;
            const bool in_box = valid && ((r < E / 4) ? (n <= a.K1) : (k1 >= -a.K1));
            if (in_box && FLAME_IN(d.status, (long long)k2 * ld1 + a.K1 + k1, box_len(a), kSiteAState)) {
                C phi = __ldg(col + k1);
                if (k1 == 0 && k2 == 0) phi = C{0, 0};
                const R f = s1 * (R)k1;
                C da{-f * phi.y, f * phi.x};  // i s1 k1 Phi
                x[r] = pack2<R>(da, phi);
            }
        }
    }
    if constexpr (STW) {
        __syncthreads();
        fft_line_s<1, (STW ? LOG : 8)>(x, t, sm, tw1, stw);
    } else {
        fft_line_e<1, LOG, E>(x, a.logn1, t, sm, tw1);
    }
    constexpr int CL = CLU ? ShapeE<LOG, E>::CL : 1;
    if constexpr (CL > 1 && std::is_same<R, float>::value) {
        // Park (U, V) of this column at its natural row index, then the CL
        // CTAs of the cluster (CL G adjacent columns) write rows: CTA q takes
        // rows [q N1/CL, (q+1) N1/CL), consecutive threads consecutive columns
        // of one row (CL G x 16 bytes = 128 contiguous bytes per row).
        namespace cg = cooperative_groups;
        cg::cluster_group cluster = cg::this_cluster();
        constexpr int GG = ShapeE<LOG, E>::G, NC = CL * GG, NN = 1 << LOG, ROWS = NN / CL;
        constexpr int NT = ShapeE<LOG, E>::THREADS;
        float4 *park = reinterpret_cast<float4 *>(base);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int n = t + r * T;
            C U = lane0<R>(x[r]);
            C Vb = lane1<R>(x[r]);
            park[spad(n)] = make_float4(U.x, U.y, -s2k2 * Vb.y, s2k2 * Vb.x);
        }
        cluster.sync();
        const int q = (int)cluster.block_rank();
        const int col0 = (tile / CL) * NC;
        static_assert((ROWS * NC) % NT == 0, "threads per CTA");
        // element e: row parity e % 2, column (e / 2) % NC, row pair e / (2 NC);
        // consecutive threads cover one row pair's NC columns x 2 rows
        // (NC x 32 contiguous bytes of the interleaved uv)
#pragma unroll
        for (int i = 0; i < ROWS * NC / NT; ++i) {
            const int e = (int)threadIdx.x + NT * i;
            const int c = (e >> 1) % NC, n = q * ROWS + 2 * (e / (2 * NC)) + (e & 1);
            const int kc = col0 + c;
            const float4 *rb = cluster.map_shared_rank(
                reinterpret_cast<const float4 *>(reinterpret_cast<V *>(smraw) + (size_t)(c % GG) * 2 * plane_len_e<E>(NN)),
                c / GG);
            const float4 v = rb[spad(n)];
            if (kc <= a.K2 && FLAME_IN(d.status, uv_index(n, kc, a.ldk) + 1, uv_len(a), kSiteAUv))
                *reinterpret_cast<float4 *>(uv + uv_index(n, kc, a.ldk)) = v;
        }
        cluster.sync();
    } else if constexpr (TMA && std::is_same<R, float>::value && LOG > 0) {
        // Park (U, V) of this column at row n (16 bytes per row: the order of
        // a column of the interleaved uv, row pair by row pair), then the
        // first thread of the group writes the column with tensor stores of
        // uv_box_pairs(N1) row pairs (32 bytes each, one uv sector per row
        // pair).  The copy engine, not the load/store unit, then issues the
        // scattered sector writes of a column.
        __syncthreads();  // the transform's last exchange has been read
        float4 *park = reinterpret_cast<float4 *>(base);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int n = t + r * T;
            C U = lane0<R>(x[r]);
            C Vb = lane1<R>(x[r]);
            park[n] = make_float4(U.x, U.y, -s2k2 * Vb.y, s2k2 * Vb.x);
        }
        fence_async_smem();
        __syncthreads();
        // a tensor copy needs a 128-byte aligned shared address: any other
        // placement of the dynamic shared memory takes the direct stores
        const bool aligned = (__cvta_generic_to_shared(smraw) & 127) == 0;
        if (!aligned && valid) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int n = t + r * T;
                if (FLAME_IN(d.status, uv_index(n, k2, a.ldk) + 1, uv_len(a), kSiteAUv))
                    *reinterpret_cast<float4 *>(uv + uv_index(n, k2, a.ldk)) = park[n];
            }
        }
        if (aligned && t == 0 && valid) {
            constexpr int BP = uv_box_pairs(1 << LOG);
            if constexpr (GMAP) tensormap_acquire(tm);
#pragma unroll 1
            for (int p0 = 0; p0 < (N1 >> 1); p0 += BP)
                if (FLAME_IN(d.status, k2, a.ldk, kSiteATma) && FLAME_IN(d.status, p0, a.n1 >> 1, kSiteATma))
                    tma_store_3d(tm, park + 2 * p0, 0, k2, p0);
            bulk_commit_and_wait_read();
        }
    } else if (valid) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int n = t + r * T;
            C U = lane0<R>(x[r]);
            C Vb = lane1<R>(x[r]);
            C Vv{-s2k2 * Vb.y, s2k2 * Vb.x};  // i s2 k2 (synthesis of Phi)
            if (FLAME_IN(d.status, uv_index(n, k2, a.ldk) + 1, uv_len(a), kSiteAUv))
                st_uv<R>(uv + uv_index(n, k2, a.ldk), U, Vv);
        }
    }
}

// Step coefficients at t_n, evaluated in FP64 (then rounded for FP32).
// The integrating factor of the linear part over [t_n, t_{n+1}] (r0 = t) is
//   E_k = exp(int omega_k) = exp(-|kappa|^2 ia + |kappa| ib),
//   ia = 1/t_n - 1/t_{n+1} = d/(t_n t_{n+1}),  ib = (gamma/2) ln(1 + d/t_n),
// with d = t_{n+1} - t_n (exact in FP64), written without cancellation.
struct Coef {
    double tn, a, b, c;  // a = 1/r0^2, b = gamma/(2 r0), c = 1/(2 r0^2)
    double ia, ib;       // integrating-factor exponent coefficients
};
// (ia, ib are derived only for the integrating-factor stage: the FP64 log
// costs the deriving thread microseconds on GB300's narrow FP64 pipe.)
__device__ __forceinline__ Coef step_coef(const StepArgs &s, double t, bool if_stage) {
    long n = __double2ll_rn((t - s.t0) / s.dt);
    double tn = s.t0 + (double)n * s.dt;
    Coef k;
    k.tn = tn;
    k.a = 1.0 / (tn * tn);
    k.b = s.gamma / (2.0 * tn);
    k.c = 0.5 * k.a;
    k.ia = k.ib = 0.0;
    if (if_stage) {
        const double tn1 = s.t0 + (double)(n + 1) * s.dt;
        const double dd = tn1 - tn;
        k.ia = dd / (tn * tn1);
        k.ib = 0.5 * s.gamma * log1p(dd / tn);
    }
    return k;
}

// The step coefficients in the kernel's precision: 1/r0^2, gamma/(2 r0),
// c/(N1 N2) (c = 1/(2 r0^2) with the inverse transform's scale folded in),
// dt and the integrating-factor coefficients.  One thread of pass B derives
// them in FP64 for the whole step and pass C loads them: GB300's FP64 pipe
// is narrow, and the divisions cost a column-pass CTA more than its loads
// when every CTA derives them.
template <class R> struct CoefR {
    R a, b, cs, dt, ia, ib;
};
template <class R> __device__ __forceinline__ CoefR<R> coef_r(const Coef &cf, const StepArgs &s) {
    const double inv = 1.0 / ((double)s.n1 * (double)s.n2);
    return CoefR<R>{(R)cf.a, (R)cf.b, (R)(cf.c * inv), (R)s.dt, (R)cf.ia, (R)cf.ib};
}
// Layout of FlameDesc::coef: t_n, c, then CoefR<R> from byte 16 (64 bytes
// in all for FP64).
template <class R> __device__ __forceinline__ void store_coef(double *coef, const StepArgs &s, double t,
                                                              bool if_stage) {
    const Coef cf = step_coef(s, t, if_stage);
    coef[0] = cf.tn;
    coef[1] = cf.c;
    *reinterpret_cast<CoefR<R> *>(coef + 2) = coef_r<R>(cf, s);
}
template <class R> __device__ __forceinline__ CoefR<R> load_coef(const double *coef) {
    return *reinterpret_cast<const CoefR<R> *>(coef + 2);
}

// Pass B (a3..a6): rows 2p and 2p+1 of uv.  For each row the full spectrum
// Z[k] = U[k] + i V[k] (k = -K2..K2, U[-k] = conj U[k]) is transformed by
// two half-length inverse FFTs (even and odd grid points:
// z[2m+q] = sum_k Z[k] exp(2 pi i k q/N2) exp(2 pi i k m/M)), giving
// u + iv; then g = u^2 + v^2 and h[m] = g[2m] + i g[2m+1] is transformed
// forward with the real-input post-processing; G[k], k <= K2, is written
// (column-major gk).  G[j1][0] is the row sum of g used for the FP64 mean mode.
// Sum over the T threads of one line group (T a power of two; groups are
// aligned to T threads).  Groups of up to 32 threads reduce by shuffles;
// larger ones add one CTA barrier and `scratch` (one slot per warp of the
// CTA).  Every thread of the CTA calls it; the group's sum is returned to
// all its threads.
template <class F> __device__ __forceinline__ F group_sum(F v, int T, F *scratch) {
    const int w = min(T, 32);
    for (int o = w >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (T <= 32) return v;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // the scratch's previous use has been read
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    const int first = (threadIdx.x / T) * (T >> 5);
    F s = 0;
    for (int i = 0; i < (T >> 5); ++i) s += scratch[first + i];
    return s;
}

template <class R, int LOG, int E, bool TMA = false, bool GMAP = false, bool AREA = false, bool WL = false>
__device__ __forceinline__ void passB_body(const FlameDesc &d, int tile, int ntiles, int pf,
                                           const CUtensorMap *tm = nullptr) {
    griddep_wait();
    griddep_launch();
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    const C *__restrict__ uv = static_cast<const C *>(d.uv);
    C *__restrict__ gk = static_cast<C *>(d.gk);
    const C *__restrict__ twm = static_cast<const C *>(d.twm);
    const int M = LOG > 0 ? (1 << LOG) : (1 << a.logm), T = M / E;
    const int g = threadIdx.x / T, t = threadIdx.x % T, G = blockDim.x / T;
    if (threadIdx.x == 0 && pf > 0 && tile + pf < ntiles) {
        const int p0 = (tile + pf) * G, np = min(G, (a.n1 >> 1) - p0);
        if (np > 0) l2_prefetch(uv + 2 * (size_t)(2 * p0) * a.ldk, (size_t)np * 2 * a.ldk * 2 * sizeof(C));
    }
    const int pair = tile * G + g;
    const bool valid = pair < (a.n1 >> 1);
    // per group: the exchange buffer, then M entries of C (sizeof(C) ==
    // sizeof(V) in both precisions); the area variant adds the synthesis of
    // Phi on the two rows (M two-line points) and its own staging of row 2p
    // (M/2 (U, V) entries)
    const int gstride = 2 * plane_len_e<E>(M) + M + (AREA ? 3 * M : 0);
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * gstride;
    auto sm = make_planes_e<E>(base, M);  // (E = 8 pads one slot every 8: st_raw/ld_raw)
    const C *P = twm + tw_real_offset(a.logm);  // exp(+2 pi i k/N2), k < M
    if (tile == 0 && threadIdx.x == 0) store_coef<R>(d.coef, a, *d.t_in, d.stage == kStageIF1);
    constexpr bool STW = kSharedTw<R, LOG, E>;
    constexpr int LS = STW ? LOG : 8;
    C *stw = reinterpret_cast<C *>(reinterpret_cast<V *>(smraw) + (size_t)G * gstride);
    RealTw<C> Pt{stw + 480, stw + 544};
    if constexpr (STW) {
        TwShared<C>::template fill<LS>(stw, twm);
        RealTw<C>::template fill<LS>(stw + 480, stw + 544, P);
        __syncthreads();
    }
    auto realtw = [&](int k) -> C {
        if constexpr (STW) return Pt(k);
        else return __ldg(P + k);
    };
    // WL: 4096-point rows with the warp-local exchanges of line_fft4096_wl;
    // the inverse transforms take natural order and leave the points in
    // digit-swapped order, which the pointwise |z|^2 and the forward
    // transform (digit-swapped in, natural out) take as they are
    static_assert(!WL || (STW && LOG == 12 && !AREA), "warp-local exchanges: FP32 4096-point rows");
    auto fft = [&](auto dirc, CV<V>(&x)[E]) {
        constexpr int DIR = decltype(dirc)::value;
        if constexpr (WL) line_fft4096_wl<DIR, (DIR > 0)>(x, t, sm, TwShared<C>{stw, stw + 240});
        else if constexpr (STW) fft_line_s<DIR, LS>(x, t, sm, twm, stw);
        else fft_line_e<DIR, LOG, E>(x, a.logm, t, sm, twm);
    };

    // Input staging.  Thread t loads, for k = t + r T (r < E/2: each k in
    // [0, M/2) once; K2 < M/2), the (U, V) of both rows: one 32-byte sector
    // of the row-pair interleave.  Row 2p's entries are staged in the
    // exchange buffer (idle until the first transform's first exchange) and
    // row 2p+1's in the h region (idle until the first row's |z|^2 is
    // parked), so the negative frequencies -k, which other threads need,
    // are read from shared memory instead of being loaded a second time.
    // After row 2p's transform, |z|^2 of row 2p is parked in the h region
    // (M entries per group) while row 2p+1 is transformed; row 2p+1's stays
    // in registers.
    C *h_first = reinterpret_cast<C *>(base + 2 * plane_len_e<E>(M));
    CV<V> *phi_park = reinterpret_cast<CV<V> *>(base + 2 * plane_len_e<E>(M) + M);  // area variant
    UV<R> *stage0 = AREA ? reinterpret_cast<UV<R> *>(base + 2 * plane_len_e<E>(M) + 3 * M)
                         : reinterpret_cast<UV<R> *>(base),
          *stage1 = reinterpret_cast<UV<R> *>(h_first);
    const int half = M >> 1;
    UV<R> e0[E / 2];
    {
        const C *src = uv + uv_index(2 * pair, 0, a.ldk);  // k: row 2p at src + 4k, row 2p+1 at src + 4k + 2
#pragma unroll
        for (int r = 0; r < E / 2; ++r) {
            const int k = t + r * T;
            UV<R> e1{C{0, 0}, C{0, 0}};
            e0[r] = e1;
            if (valid && k <= a.K2 &&
                FLAME_IN(d.status, uv_index(2 * pair, 0, a.ldk) + 4 * (long long)k + 3, uv_len(a), kSiteBUv)) {
                e0[r] = ld_uv<R>(src + 4 * (size_t)k);
                e1 = ld_uv<R>(src + 4 * (size_t)k + 2);
            }
            st_uv_s<R>(stage0 + k, e0[r]);
            st_uv_s<R>(stage1 + k, e1);
        }
    }
    __syncthreads();
    // the full spectrum Z of one row (Z[k] = U[k] + i V[k], U[-k] = conj
    // U[k]) split into the inputs of the two half-length inverse FFTs:
    // lane 0 Z[k], lane 1 Z[k] exp(2 pi i k/N2)
    // Real-transform twiddles of this thread's points: w^k, w = exp(2 pi i /
    // N2), for k = n = t + r T (r < E/2) and k = n - M (r >= E/2) are
    // w^t exp(i pi r / E) and -conj(w^t exp(i pi r / E)) (w^M = -1, T = M/E):
    // one table entry per thread, the rest compile-time roots.
    const C wt = realtw(t);
    auto build = [&](auto own, const UV<R> *stage, CV<V>(&x)[E]) {
        static_for<0, E>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            const int n = t + r * T;
            // r < E/2: k = n >= 0 (n < M/2); r >= E/2: k = n - M < 0
            const int kk = (r < E / 2) ? n : M - n;
            UV<R> e{C{0, 0}, C{0, 0}};
            if constexpr (decltype(own)::value) {
                if (r < E / 2) e = e0[r];
                else if (kk < half) e = ld_uv_s<R>(stage + kk);
            } else {
                if (kk < half) e = ld_uv_s<R>(stage + kk);
            }
            C z = (r < E / 2) ? C{e.u.x - e.v.y, e.u.y + e.v.x}     // U + iV
                              : C{e.u.x + e.v.y, e.v.x - e.u.y};    // conj U + i conj V
            // exp(2 pi i k/N2) for this point's signed k
            const C w = mul_root<r, E, (r < E / 2 ? 1 : -1)>(wt);
            C z1 = C{fma_rn(z.x, w.x, -(z.y * w.y)), fma_rn(z.x, w.y, z.y * w.x)};
            x[r] = pack2<R>(z, z1);
        });
    };
    CV<V> x[E];
    // Area variant: Phi on rows 2p, 2p+1 (without the mean mode), as the
    // inverse row transform of S[k] = P_2p[k] + i P_2p+1[k], P the column
    // synthesis of Phi: for k2 >= 1, P = V / (i s2 k2) (pass A wrote V =
    // i s2 k2 P); for k2 = 0, P(j1) = 2 Re sum_{k1 = 1..K1} Phi_{k1,0}
    // exp(2 pi i k1 j1 / N1), summed here.  Parked for the area terms.
    __shared__ R ared[32];
    R apart = 0;  // this thread's share of the rows' area sums
    R rr = 0;     // r0 + Phi_0
    if constexpr (AREA) {
        rr = (R)(*d.t_in + *d.mean);
        const C *st0 = static_cast<const C *>(d.state) + a.K1;  // column k2 = 0, index k1
        const C *t1r = static_cast<const C *>(d.tw1) + tw_real_offset(a.logn1);  // exp(2 pi i k / 2 N1), k < N1
        R p0[2] = {0, 0};
        for (int k1 = 1 + t; k1 <= a.K1; k1 += T) {
            if (!FLAME_IN(d.status, a.K1 + k1, box_len(a), kSiteBArow)) continue;
            const C ph = st0[k1];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int m = (k1 * (2 * pair + q)) & (a.n1 - 1);  // N1 a power of two
                C w = __ldg(t1r + ((2 * m < a.n1) ? 2 * m : 2 * m - a.n1));
                if (2 * m >= a.n1) w = C{-w.x, -w.y};
                p0[q] += 2 * (ph.x * w.x - ph.y * w.y);
            }
        }
        p0[0] = group_sum<R>(p0[0], T, ared);
        p0[1] = group_sum<R>(p0[1], T, ared);
        const R is2 = (R)1 / scale2<R>(a);
        static_for<0, E>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            const int n = t + r * T;
            const int kk = (r < E / 2) ? n : M - n;
            C P0{0, 0}, P1{0, 0};
            if (kk == 0) {
                P0 = C{p0[0], 0};
                P1 = C{p0[1], 0};
            } else if (kk < half) {
                const C v0 = ld_uv_s<R>(stage0 + kk).v, v1 = ld_uv_s<R>(stage1 + kk).v;
                const R f = is2 * rcp_r((R)kk);  // P = V / (i s2 k) = (V.y, -V.x) / (s2 k)
                P0 = C{v0.y * f, -v0.x * f};
                P1 = C{v1.y * f, -v1.x * f};
            }
            // S[k] (r < E/2, k = kk) or S[-kk] = conj P0 + i conj P1
            const C S = (r < E / 2) ? C{P0.x - P1.y, P0.y + P1.x} : C{P0.x + P1.y, P1.x - P0.y};
            const C w = mul_root<r, E, (r < E / 2 ? 1 : -1)>(wt);
            x[r] = pack2<R>(S, C{fma_rn(S.x, w.x, -(S.y * w.y)), fma_rn(S.x, w.y, S.y * w.x)});
        });
        fft(std::integral_constant<int, 1>{}, x);
#pragma unroll
        for (int r = 0; r < E; ++r) phi_park[t + r * T] = x[r];
    }
    // area terms R sqrt(R^2 + g), R = r0 + Phi_0 + phi, at the points 2m + q of
    // one row (q = 0, 1 the lanes), phi from the parked synthesis (re: row 2p,
    // im: row 2p+1)
    auto area_terms = [&](const V(&gv)[E], bool second) {
        if constexpr (AREA) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const CV<V> ph = phi_park[t + r * T];
                const V pv = second ? ph.im : ph.re;
                const R R0 = rr + pv.x, R1 = rr + pv.y;
                apart += R0 * sqrt_r(fma_rn(R0, R0, gv[r].x)) + R1 * sqrt_r(fma_rn(R1, R1, gv[r].y));
            }
        }
    };
    build(std::true_type{}, stage0, x);
    fft(std::integral_constant<int, 1>{}, x);
    V sq0[E];
#pragma unroll
    for (int r = 0; r < E; ++r) sq0[r] = vfma(x[r].re, x[r].re, vmul(x[r].im, x[r].im));  // g at 2m, 2m+1
    area_terms(sq0, false);
    build(std::false_type{}, stage1, x);
    __syncthreads();  // stage1 fully read: the h region takes row 2p's g
#pragma unroll
    for (int r = 0; r < E; ++r) h_first[t + r * T] = C{sq0[r].x, sq0[r].y};
    fft(std::integral_constant<int, 1>{}, x);
    if constexpr (AREA) {
        V sq1[E];
#pragma unroll
        for (int r = 0; r < E; ++r) sq1[r] = vfma(x[r].re, x[r].re, vmul(x[r].im, x[r].im));
        area_terms(sq1, true);
        // the row pair's area sum (FP64 across the group's threads)
        const double tot = group_sum<double>((double)apart, T, reinterpret_cast<double *>(phi_park));
        if (t == 0 && valid && FLAME_IN(d.status, pair, a.n1 >> 1, kSiteBArow)) d.arow[pair] = tot;
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
        V sq = vfma(x[r].re, x[r].re, vmul(x[r].im, x[r].im));
        x[r] = pack2<R>(h_first[t + r * T], C{sq.x, sq.y});
    }
    fft(std::integral_constant<int, -1>{}, x);
    __syncthreads();
    // the post-processing of k in [0, M/2) reads H[M - k]: only H[0] and the
    // upper half (registers r >= E/2) go to shared memory
#pragma unroll
    for (int r = E / 2; r < E; ++r) sm.st_raw(spad_e<E>(t + r * T), x[r]);
    if (t == 0) sm.st_raw(0, x[0]);
    __syncthreads();
    // Tensor-store write-out (FP32, compile-time lengths): G of the row pair
    // is staged in the h region (free again: the forward transform has read
    // it) in the order of the column-pair interleaved gk, complex index
    // 4 (k/2) + k%2 for row 2p and + 2 for row 2p+1, and the first thread of
    // the group writes it with tensor stores of gk_box_pairs(ldk) column
    // pairs.  Other cases store directly.
    constexpr bool kTma = TMA && std::is_same<R, float>::value && LOG > 0;
    const bool staged = kTma && (__cvta_generic_to_shared(smraw) & 127) == 0;
    static_for<0, E / 2>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        const int k = t + r * T;
        if (valid && k <= a.K2) {
            CV<V> h = x[r], hc = sm.ld_raw(spad_e<E>((M - k) & (M - 1)));
            const R hf = (R)0.5;
            const C w = mul_root<r, E, 1>(wt);  // exp(2 pi i k/N2)
            CV<V> Ev{vmul(vadd(h.re, hc.re), vbc(hf)), vmul(vsub(h.im, hc.im), vbc(hf))};
            CV<V> Ov{vmul(vadd(h.im, hc.im), vbc(hf)), vmul(vsub(hc.re, h.re), vbc(hf))};
            CV<V> Y = cadd(Ev, cmul_s(Ov, w.x, -w.y));
            C *dst = staged ? h_first + 4 * (k >> 1) + (k & 1)
                            : gk + gk_index(2 * pair, k, a.n1);  // row 2p+1 two slots further
            if (staged || FLAME_IN(d.status, gk_index(2 * pair, k, a.n1) + 2, gk_len(a), kSiteBGk)) {
                dst[0] = lane0<R>(Y);
                dst[2] = lane1<R>(Y);
            }
        }
    });
    if constexpr (kTma) {
        if (staged) {
            fence_async_smem();
            __syncthreads();
            if (t == 0 && valid) {
                const int nq = (a.ldk + 1) >> 1, BQ = gk_box_pairs(a.ldk);
                if constexpr (GMAP) tensormap_acquire(tm);
#pragma unroll 1
                for (int q0 = 0; q0 < nq; q0 += BQ)
                    if (FLAME_IN(d.status, pair, a.n1 >> 1, kSiteBTma) && FLAME_IN(d.status, q0, (gk_len(a) / a.n1) >> 1, kSiteBTma))
                        tma_store_3d(tm, h_first + 4 * q0, 0, pair, q0);
                bulk_commit_and_wait_read();
            }
        }
    }
}

// Explicitly rounded scalar arithmetic: the update of pass C is compiled in
// several kernels (plain and general epilogues, single flames and
// ensembles) that must give identical bits, so no product may be left to
// the compiler's choice of contraction.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// |kappa| = sqrt((s1 k1)^2 + (s2 k2)^2) for (k1, k2) != 0.  FP32: x times the
// hardware reciprocal square root (within a few ulp, far inside the FP32
// path's per-step tolerance); FP64: the correctly rounded square root.
template <class R> __device__ __forceinline__ R kappa_norm(R s1k1, R s2k2) {
    if constexpr (std::is_same<R, float>::value) {
        const float x = fmaf(s1k1, s1k1, s2k2 * s2k2);
        return x * rsqrtf(x);
    } else {
        return sqrt(fma(s1k1, s1k1, s2k2 * s2k2));
    }
}

// Pass C's epilogue, shared by its kernels: the update of one box entry
// (a8..a10), the area of the state entering the step for the record, and
// the mean mode, time and record written by thread 0 of tile 0.
template <class R> struct EpiArgs {
    CoefR<R> cf;
    R s1, s2;
    int stage;  // kStage*, uniform over the launch
    bool lin, nl;
};

// Entry (k1, k2) of the box, k = (k1, k2) != (0, 0) updated from the scaled
// transform gh = c-free ghat and the entry ph entering the step:
// Phi <- Phi + dt (omega Phi + c ghat + f) for the Euler stage and the
// combinations of the two-stage schemes (see kStage*).  col, fcol and scol
// point at k1 = 0 of column k2 of the state, the forcing (or null) and the
// stage buffer (or null); the k2 = 0 column also gets the conjugate mirror
// at -k1.  nw returns the new entry (0 for k = 0); bad collects non-finite
// results.
template <class R, bool GEN>
__device__ __forceinline__ void update_entry(const FlameDesc &d, const EpiArgs<R> &e, int k1, int k2, CplxT<R> gh,
                                             CplxT<R> ph, CplxT<R> *col, const CplxT<R> *fcol, CplxT<R> *scol,
                                             CplxT<R> &nw, int &bad) {
    using C = CplxT<R>;
    const StepArgs &a = d.a;
    nw = C{0, 0};
    [[maybe_unused]] const long long bi = (long long)k2 * (2 * a.K1 + 1) + a.K1 + k1;  // box index of (k1, k2)
    if (!FLAME_IN(d.status, bi, box_len(a), kSiteCState)) return;
    if (k1 == 0 && k2 == 0) {
        col[0] = C{0, 0};
        return;
    }
    const R rdt = e.cf.dt;
    const R kap = kappa_norm<R>(rmul(e.s1, (R)k1), rmul(e.s2, (R)k2));
    const R om = e.lin ? rmul(kap, rfma(-kap, e.cf.a, e.cf.b)) : (R)0;
    const R cn = e.nl ? e.cf.cs : (R)0;
    // the non-stiff part: c ghat (+ the forcing f_k)
    C nt{rmul(cn, gh.x), rmul(cn, gh.y)};
    if (GEN && fcol && FLAME_IN(d.status, bi, box_len(a), kSiteCForcing)) {
        const C f = fcol[k1];
        nt = C{radd(nt.x, f.x), radd(nt.y, f.y)};
    }
    // dt F = dt (omega Phi + nt)
    const C df{rmul(rdt, rfma(om, ph.x, nt.x)), rmul(rdt, rfma(om, ph.y, nt.y))};
    const int stage = GEN ? e.stage : kStageEuler;
    if (stage != kStageEuler && !FLAME_IN(d.status, bi, box_len(a), kSiteCSave)) return;
    C v;
    if (stage == kStageEuler || stage == kStageHeun1) {
        v = C{radd(ph.x, df.x), radd(ph.y, df.y)};
        if (stage == kStageHeun1) scol[k1] = ph;
    } else if (stage == kStageHeun2) {
        const C sv = scol[k1];
        const R h = (R)0.5;
        v = C{rmul(h, radd(radd(sv.x, ph.x), df.x)), rmul(h, radd(radd(sv.y, ph.y), df.y))};
    } else if (stage == kStageIF1) {
        // exact propagator of the linear part over the step
        R ef = (R)1;
        if (e.lin) {
            const R ex = rmul(kap, rfma(-kap, e.cf.ia, e.cf.ib));
            if constexpr (std::is_same<R, float>::value) ef = expf(ex);
            else ef = exp(ex);
        }
        const R hdt = rmul((R)0.5, rdt);
        v = C{rmul(ef, rfma(rdt, nt.x, ph.x)), rmul(ef, rfma(rdt, nt.y, ph.y))};
        scol[k1] = C{rmul(ef, rfma(hdt, nt.x, ph.x)), rmul(ef, rfma(hdt, nt.y, ph.y))};
    } else {  // kStageIF2
        const C sv = scol[k1];
        const R hdt = rmul((R)0.5, rdt);
        v = C{rfma(hdt, nt.x, sv.x), rfma(hdt, nt.y, sv.y)};
    }
    bad |= !(isfinite(v.x) && isfinite(v.y));
    col[k1] = v;
    nw = v;
    if (k2 == 0 && FLAME_IN(d.status, a.K1 - k1, box_len(a), kSiteCState)) col[-k1] = C{v.x, -v.y};
}

// The surface area of the state entering the step, for the record: the
// area variant of pass B left one FP64 sum per row pair (summed here by
// tile 0's threads, all of which call this), or the separate area kernels
// left the total; NaN when the step records no area.
template <bool GEN> __device__ __forceinline__ double record_area(const FlameDesc &d, int tile, int stage, int N1) {
    const StepArgs &a = d.a;
    double area = __longlong_as_double(0x7ff8000000000000LL);
    if (GEN && tile == 0 && d.rec && stage != kStageHeun2 && stage != kStageIF2) {
        if (d.rec_area == 1) {
            __shared__ double asum[32];
            double v = 0.0;
            for (int i = threadIdx.x; i < (a.n1 >> 1); i += blockDim.x)
                if (FLAME_IN(d.status, i, a.n1 >> 1, kSiteCRec)) v += d.arow[i];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) asum[threadIdx.x >> 5] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot += asum[w];
                const double two_pi = 6.283185307179586476925286766559;
                area = tot * (two_pi * two_pi / ((double)N1 * (double)a.n2 * a.s1 * a.s2));
            }
        } else if (d.rec_area == 2) {
            area = *d.aval;
        }
    }
    return area;
}

// Thread 0 of tile 0: the mean mode's update from rs, the FP64 sum of column
// k2 = 0 of gk (N1 N2 times the mean of |grad Phi|^2), the time, and the
// record entry of the step.
template <bool GEN>
__device__ __forceinline__ void finish_step(const FlameDesc &d, int stage, bool nl, int N1, double rs, double area) {
    const StepArgs &a = d.a;
    const double mg = rs / ((double)N1 * (double)a.n2);  // mean of |grad Phi|^2
    // dt times the mean mode's right-hand side (omega_0 = 0): c mg + f_0
    double inc = nl ? a.dt * d.coef[1] * mg : 0.0;
    if (GEN && d.forcing0 != 0.0) inc += a.dt * d.forcing0;
    const double m = *d.mean;
    long n = __double2ll_rn((d.coef[0] - a.t0) / a.dt);
    const long ri = ((n % max(d.rec_cap, 1)) + d.rec_cap) % max(d.rec_cap, 1);
    if (GEN && d.rec && stage != kStageHeun2 && stage != kStageIF2 && FLAME_IN(d.status, ri, d.rec_cap, kSiteCRec)) {
        double *e = d.rec + 4 * (size_t)ri;
        e[0] = d.coef[0];
        e[1] = m;
        e[2] = (nl ? d.coef[1] * mg : 0.0) + (GEN ? d.forcing0 : 0.0);
        e[3] = area;
    }
    if (stage == kStageEuler || stage == kStageHeun1 || stage == kStageIF1) {
        if (stage == kStageHeun1) *d.save_mean = m;
        if (stage == kStageIF1) *d.save_mean = m + 0.5 * inc;
        *d.mean = m + inc;
        *d.t_out = a.t0 + (double)(n + 1) * a.dt;
    } else {
        // second stages are evaluated at t_{n+1} and leave t there
        *d.mean = stage == kStageHeun2 ? 0.5 * (*d.save_mean + m + inc) : *d.save_mean + 0.5 * inc;
        *d.t_out = a.t0 + (double)n * a.dt;
    }
}

// Pass C (a7..a10): columns k2, k2+1 of gk -> forward FFT along j1 (outputs
// outside |k1| <= K1 unused and dropped at compile time), scaled by
// 1/(N1 N2) -> ghat; Phi <- Phi + dt (omega Phi + c ghat); the k2 = 0 column
// is written from its k1 > 0 half and its conjugate mirror; the block owning
// column 0 sums G[j1][0] in FP64 for the mean mode and advances t.  The state
// entries of the epilogue are loaded after the transform.
// GEN = false compiles the plain Euler step without forcing or record (the
// hot path); GEN = true reads the stage, forcing and record from the
// descriptor.
template <class R, int LOG, bool FUSE_A = false, int E = 16, bool GEN = true>
__device__ __forceinline__ void passC_body(const FlameDesc &d, int tile, int ntiles, int pf,
                                           const CUtensorMap *tm = nullptr) {
    griddep_wait();
    griddep_launch();
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    static_assert(E == 16 || ((E == 8 || E == 4) && !FUSE_A),
                  "E points per thread: 16, or 8 and 4 without the fused pass A");
    constexpr int QE = E / 4;  // band registers: r < QE (k1 >= 0) and r >= E - QE (k1 < 0)
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[256];  // one per thread (blockDim <= 256)
    const StepArgs &a = d.a;
    const C *__restrict__ gk = static_cast<const C *>(d.gk);
    C *__restrict__ state = static_cast<C *>(d.state);
    const C *__restrict__ tw1 = static_cast<const C *>(d.tw1);
    const int N1 = LOG > 0 ? (1 << LOG) : (1 << a.logn1), T = N1 / E;
    const int G = blockDim.x / T, g = threadIdx.x / T, t = threadIdx.x % T;
    const int ld1 = 2 * a.K1 + 1;
    if (threadIdx.x == 0 && pf > 0 && tile + pf < ntiles) {
        const int c = 2 * (tile + pf) * G, nc = min(2 * G, a.K2 + 1 - c);
        if (nc > 0) {
            l2_prefetch(gk + (size_t)c * N1, (size_t)nc * N1 * sizeof(C));
            l2_prefetch(state + (size_t)c * ld1, (size_t)nc * ld1 * sizeof(C));
        }
    }
    const CoefR<R> cfs = load_coef<R>(d.coef);  // derived by pass B
    const int c0 = 2 * (tile * G + g);
    const bool va = c0 <= a.K2, vb = c0 + 1 <= a.K2;
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len_e<E>(N1);
    auto sm = make_planes_e<E>(base, N1);
    constexpr bool STW = false;  // pass C's twiddles stay in L1 (measured faster)
    C *stw = reinterpret_cast<C *>(reinterpret_cast<V *>(smraw) + (size_t)G * 2 * plane_len_e<E>(N1));
    if constexpr (STW) TwShared<C>::template fill<(STW ? LOG : 8)>(stw, tw1);  // synced below
    const C *gp = gk + gk_index(0, c0, N1);  // row n: columns c0, c0+1 at gp[2n], gp[2n+1]
    CV<V> x[E];
    double colsum = 0.0;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int n = t + r * T;
        C p, q;
        const bool in = va && FLAME_IN(d.status, gk_index(0, c0, N1) + 2 * (long long)n + 1, gk_len(a), kSiteCGk);
        if constexpr (std::is_same<R, float>::value) {
            const float4 pq = in ? __ldg(reinterpret_cast<const float4 *>(gp) + n) : make_float4(0.f, 0.f, 0.f, 0.f);
            p = C{pq.x, pq.y};
            q = vb ? C{pq.z, pq.w} : C{0, 0};
        } else {
            p = in ? __ldg(gp + 2 * n) : C{0, 0};
            q = (in && vb) ? __ldg(gp + 2 * n + 1) : C{0, 0};
        }
        if (c0 == 0) colsum += (double)p.x;
        x[r] = pack2<R>(p, q);
    }
    // state entries this thread updates: rows r < QE (k1 = n) and r >= E - QE
    // (k1 = n - N1) of columns c0 and c0 + 1
    C *sa = state + (size_t)c0 * ld1 + a.K1, *sb = sa + ld1;
    // block-uniform: FP64 row sum of column 0, in spans of up to 32 threads
    // (power-of-two blocks) summed by each span's first thread in parallel
    const int span = min((int)blockDim.x, 32);
    if (tile == 0) {
        red[threadIdx.x] = colsum;
        __syncthreads();
        if (threadIdx.x % span == 0) {
            double s = 0.0;
            for (int w = 0; w < span; ++w) s += red[threadIdx.x + w];
            red[threadIdx.x] = s;  // the span's own slots: no other thread touches them
        }
        // the span sums are read by thread 0 after the transform's barriers
    }
    if constexpr (STW) {
        __syncthreads();
        fft_line_s<-1, (STW ? LOG : 8)>(x, t, sm, tw1, stw);
    } else {
        fft_line_e<-1, LOG, E>(x, a.logn1, t, sm, tw1);
    }

    __syncthreads();  // block 0's span sums (the transform may have no CTA barrier)
    // the state entries, read after the transform (they are L2-resident in
    // the persisting window; holding them across the transform cost more)
    C phi[E / 2][2];
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
        const int r = i < QE ? i : i + E / 2;
        const int n = t + r * T;
        const int k1 = (r < QE) ? n : n - N1;
        const bool in_box = (r < QE) ? (n <= a.K1) : (k1 >= -a.K1);
        [[maybe_unused]] const long long ia = (long long)c0 * ld1 + a.K1 + k1;
        phi[i][0] = (in_box && va && FLAME_IN(d.status, ia, box_len(a), kSiteCState)) ? sa[k1] : C{0, 0};
        phi[i][1] = (in_box && vb && FLAME_IN(d.status, ia + ld1, box_len(a), kSiteCState)) ? sb[k1] : C{0, 0};
    }
    const bool lin = !(a.flags & kNonlinearOnly), nl = !(a.flags & kLinearOnly);
    const int stage = GEN ? d.stage : kStageEuler;  // block-uniform
    const EpiArgs<R> ea{cfs, scale1<R>(a), scale2<R>(a), stage, lin, nl};
    const C *fa = GEN && d.forcing ? static_cast<const C *>(d.forcing) + (size_t)c0 * ld1 + a.K1 : nullptr;
    C *va_save = GEN && d.save ? static_cast<C *>(d.save) + (size_t)c0 * ld1 + a.K1 : nullptr;
    int bad = 0;
    C nphi[E / 2][2];  // the updated entries (kept for the fused pass A of the next step)
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
        const int r = i < QE ? i : i + E / 2;
        const int n = t + r * T;
        const int k1 = (r < QE) ? n : n - N1;
        const bool in_box = (r < QE) ? (n <= a.K1) : (k1 >= -a.K1);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int k2 = c0 + side;
            nphi[i][side] = C{0, 0};
            const bool ok = in_box && (side == 0 ? va : vb);
            if (!ok) continue;
            if (k2 == 0 && k1 < 0) continue;  // written as the mirror of +k1
            const int off = side ? ld1 : 0;
            update_entry<R, GEN>(d, ea, k1, k2, side == 0 ? lane0<R>(x[r]) : lane1<R>(x[r]), phi[i][side],
                                 (side == 0 ? sa : sb), fa ? fa + off : nullptr, va_save ? va_save + off : nullptr,
                                 nphi[i][side], bad);
        }
    }
    if (bad) atomicOr(d.status, 1 << kStatusNonfinite);
    const double area = record_area<GEN>(d, tile, stage, N1);
    if (tile == 0 && threadIdx.x == 0) {
        double rs = 0.0;
        for (int w = 0; w < (int)blockDim.x; w += span) rs += red[w];
        finish_step<GEN>(d, stage, nl, N1, rs, area);
    }
    if constexpr (FUSE_A && std::is_same<R, float>::value && LOG > 0) {
        // Pass A of the next step (a1, a2) on the two updated columns, from
        // registers: the same prologue, transform and tensor-store write-out
        // as k_passAt.  The k2 = 0 column's k1 < 0 half was written by other
        // threads (the conjugate mirror) and is read back after the barrier,
        // which also frees the exchange buffer.
        __syncthreads();
        const R s1 = ea.s1, s2 = ea.s2;
        if (c0 == 0) {
#pragma unroll
            for (int i = 4; i < 8; ++i) {
                const int k1 = t + (i + 8) * T - N1;
                if (k1 >= -a.K1 && FLAME_IN(d.status, a.K1 + k1, box_len(a), kSiteCState)) nphi[i][0] = sa[k1];
            }
        }
        const C *__restrict__ tw1a = static_cast<const C *>(d.tw1);
        float4 *park = reinterpret_cast<float4 *>(base);
        const bool aligned = (__cvta_generic_to_shared(smraw) & 127) == 0;
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            const int k2 = c0 + side;
            const bool valid = side == 0 ? va : vb;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                x[r] = CV<V>{vzero(V{}), vzero(V{})};
                if (r < 4 || r >= 12) {
                    const int i = r < 4 ? r : r - 8;
                    const int n = t + r * T;
                    const int k1 = (r < 4) ? n : n - N1;
                    if (!(valid && ((r < 4) ? (n <= a.K1) : (k1 >= -a.K1)))) continue;
                    C phi = side == 0 ? nphi[i][0] : nphi[i][1];
                    if (k1 == 0 && k2 == 0) phi = C{0, 0};
                    const R f = s1 * (R)k1;
                    x[r] = pack2<R>(C{-f * phi.y, f * phi.x}, phi);  // (i s1 k1 Phi, Phi)
                }
            }
            fft_line<1, LOG>(x, a.logn1, t, sm, tw1a);
            const R s2k2 = s2 * (R)k2;
            __syncthreads();  // the transform's last exchange has been read
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int n = t + r * T;
                C U = lane0<R>(x[r]);
                C Vb = lane1<R>(x[r]);
                park[n] = make_float4(U.x, U.y, -s2k2 * Vb.y, s2k2 * Vb.x);
            }
            fence_async_smem();
            __syncthreads();
            if (!aligned && valid) {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int n = t + r * T;
                    if (FLAME_IN(d.status, uv_index(n, k2, a.ldk) + 1, uv_len(a), kSiteCAUv))
                        *reinterpret_cast<float4 *>(static_cast<C *>(d.uv) + uv_index(n, k2, a.ldk)) = park[n];
                }
            }
            if (aligned && t == 0 && valid) {
                constexpr int BP = uv_box_pairs(1 << LOG);
#pragma unroll 1
                for (int p0 = 0; p0 < (N1 >> 1); p0 += BP)
                    if (FLAME_IN(d.status, k2, a.ldk, kSiteCAUv) && FLAME_IN(d.status, p0, a.n1 >> 1, kSiteCAUv))
                        tma_store_3d(tm, park + 2 * p0, 0, k2, p0);
                bulk_commit_and_wait_read();
            }
            __syncthreads();  // the park may be overwritten by the next transform
        }
    }
}

// ----------------------------------------------------------------------------
// One-line step passes: each line is transformed by its own group of
// T = 2^LOG / E threads (one real per point and component: V = D1 or F1),
// and a CTA holds the groups of one column (pass A: the two fields), one
// row pair (pass B: two rows x even/odd points) or one column pair (pass
// C).  Used for the FP64 short lines (2^4 .. 2^7 points, E = 4 or 8: the
// FP64 parity and trajectory grids) and, as an autotuned variant, for FP32
// lines of 2^8 .. 2^11 points (E = 16).  A small grid has too few line
// pairs to give every SM sub-partition a warp; with one line per group its
// work spreads over two to four times as many warps.
// ----------------------------------------------------------------------------
// offset of the radix-E table (E = 16, 8 or 4) in a line's twiddle allocation
template <int E> __host__ __device__ constexpr int tw_offset_e(int log) {
    return E == 16 ? 0 : E == 8 ? tw_table_len(log, 4) : tw_table_len(log, 4) + tw_table_len(log, 3);
}

// Pass A (a1, a2) on column k2: group 0 synthesises i s1 k1 Phi (-> U), group
// 1 synthesises Phi (-> V = i s2 k2 times it); each writes its half of the
// (U, V) entries of the column.
template <class R, int LOG, int E> __device__ __forceinline__ void passA1_body(const FlameDesc &d, int k2) {
    griddep_wait();
    griddep_launch();
    using C = CplxT<R>;
    using V1 = typename OneOf<R>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    constexpr int N1 = 1 << LOG, T = N1 / E, PL = plane_len_e<E>(N1);
    const int f = threadIdx.x / T, t = threadIdx.x % T;
    const int ld1 = 2 * a.K1 + 1;
    const bool valid = k2 <= a.K2;
    const Planes<V1> sm(reinterpret_cast<R *>(smraw) + (size_t)f * 2 * PL, PL);
    const C *tw = static_cast<const C *>(d.tw1) + tw_offset_e<E>(LOG);
    const C *col = static_cast<const C *>(d.state) + (size_t)k2 * ld1 + a.K1;  // col[k1], k1 = -K1..K1
    CV<V1> x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        x[r] = CV<V1>{{(R)0}, {(R)0}};
        // band rows r < E/4 (k1 = n >= 0) and r >= 3E/4 (k1 = n - N1 < 0); the rest is padding
        if (r < E / 4 || r >= 3 * E / 4) {
            const int n = t + r * T;
            const int k1 = (r < E / 4) ? n : n - N1;
            const bool in_box = valid && ((r < E / 4) ? (n <= a.K1) : (k1 >= -a.K1));
            if (in_box && FLAME_IN(d.status, (long long)k2 * ld1 + a.K1 + k1, box_len(a), kSiteAState)) {
                C phi = __ldg(col + k1);
                if (k1 == 0 && k2 == 0) phi = C{0, 0};
                const R fk = scale1<R>(a) * (R)k1;
                x[r] = f == 0 ? CV<V1>{{-fk * phi.y}, {fk * phi.x}} : CV<V1>{{phi.x}, {phi.y}};
            }
        }
    }
    line_fft_ct<1, LOG, E>(x, t, sm, tw, CtaBarrier{});
    if (!valid) return;
    C *uv = static_cast<C *>(d.uv);
    const R s2k2 = scale2<R>(a) * (R)k2;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const size_t i = uv_index(t + r * T, k2, a.ldk) + f;  // U, or V one slot further
        if (FLAME_IN(d.status, i, uv_len(a), kSiteAUv))
            uv[i] = f == 0 ? C{x[r].re.x, x[r].im.x} : C{-s2k2 * x[r].im.x, s2k2 * x[r].re.x};
    }
}

// Pass B (a3..a6) on row pair p: group 2q + s takes the grid points 2m + s
// of row 2p + q (the half-length inverse FFT of Z[k] exp(2 pi i k s / N2),
// Z = U + iV) and parks g = u^2 + v^2 there; then group q transforms
// h[m] = g[2m] + i g[2m+1] of row 2p + q forward and writes G[k], k <= K2,
// after the real-input post-processing.  Groups 2 and 3 transform zeros in
// the forward step, so that every group meets the same barriers.
template <class R, int LOG, int E> __device__ __forceinline__ void passB1_body(const FlameDesc &d, int pair) {
    griddep_wait();
    griddep_launch();
    using C = CplxT<R>;
    using V1 = typename OneOf<R>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    constexpr int M = 1 << LOG, T = M / E, PL = plane_len_e<E>(M);
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    const int q = g >> 1, s = g & 1;
    const bool valid = pair < (a.n1 >> 1);
    R *smd = reinterpret_cast<R *>(smraw);
    const Planes<V1> sm(smd + (size_t)g * 2 * PL, PL);
    R *h = smd + 8 * (size_t)PL;  // g of row 2p + q at h[2M q + j], j the grid point
    const C *tw = static_cast<const C *>(d.twm) + tw_offset_e<E>(LOG);
    const C *P = static_cast<const C *>(d.twm) + tw_real_offset(LOG);  // exp(2 pi i k / N2), k < M
    if (pair == 0 && threadIdx.x == 0) store_coef<R>(d.coef, a, *d.t_in, d.stage == kStageIF1);
    const size_t base = uv_index(2 * pair + q, 0, a.ldk);  // (U, V) of k at base + 4k
    const C *src = static_cast<const C *>(d.uv) + base;
    CV<V1> x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int n = t + r * T;
        const int kk = (r < E / 2) ? n : M - n;  // |k|: k = n (r < E/2) or n - M
        C z{0, 0};
        if (valid && kk <= a.K2 && kk < M / 2 && FLAME_IN(d.status, base + 4LL * kk + 1, uv_len(a), kSiteBUv)) {
            const C u = __ldg(src + 4 * (size_t)kk), v = __ldg(src + 4 * (size_t)kk + 1);
            // U[-k] = conj U[k], V[-k] = conj V[k]
            z = (r < E / 2) ? C{u.x - v.y, u.y + v.x} : C{u.x + v.y, v.x - u.y};
        }
        if (s == 1) {
            C w = __ldg(P + kk);  // exp(2 pi i k / N2) for the signed k
            if (r >= E / 2) w.y = -w.y;
            z = C{fma_rn(z.x, w.x, -(z.y * w.y)), fma_rn(z.x, w.y, z.y * w.x)};
        }
        x[r] = CV<V1>{{z.x}, {z.y}};
    }
    line_fft_ct<1, LOG, E>(x, t, sm, tw, CtaBarrier{});
#pragma unroll
    for (int r = 0; r < E; ++r) h[2 * M * q + 2 * (t + r * T) + s] = fma_rn(x[r].re.x, x[r].re.x, x[r].im.x * x[r].im.x);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int m = t + r * T;
        x[r] = g < 2 ? CV<V1>{{h[2 * M * g + 2 * m]}, {h[2 * M * g + 2 * m + 1]}} : CV<V1>{{(R)0}, {(R)0}};
    }
    line_fft_ct<-1, LOG, E>(x, t, sm, tw, CtaBarrier{});
    __syncthreads();
    // the post-processing of k in [0, M/2) reads H[M - k]: H[0] and the upper half go to shared memory
#pragma unroll
    for (int r = E / 2; r < E; ++r) sm.st_raw(spad_e<E>(t + r * T), x[r]);
    if (t == 0) sm.st_raw(0, x[0]);
    __syncthreads();
    if (g >= 2 || !valid) return;
    C *gk = static_cast<C *>(d.gk);
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
        const int k = t + r * T;
        if (k > a.K2) continue;
        const CV<V1> hk = x[r], hc = sm.ld_raw(spad_e<E>((M - k) & (M - 1)));
        const R hf = (R)0.5;
        const R ex = hf * (hk.re.x + hc.re.x), ey = hf * (hk.im.x - hc.im.x);
        const R ox = hf * (hk.im.x + hc.im.x), oy = hf * (hc.re.x - hk.re.x);
        const C w = __ldg(P + k);  // G = E + O conj(w)
        const C y{ex + fma_rn(ox, w.x, oy * w.y), ey + fma_rn(oy, w.x, -(ox * w.y))};
        const size_t i = gk_index(2 * pair + g, k, a.n1);
        if (FLAME_IN(d.status, i, gk_len(a), kSiteBGk)) gk[i] = y;
    }
}

// Pass C (a7..a10) on columns k2 = 2 tile + f (group f = 0, 1): the forward
// transform of column k2 of gk and the update of its box entries; tile 0
// sums column 0 in FP64 and finishes the step (mean mode, time, record).
template <class R, int LOG, int E, bool GEN> __device__ __forceinline__ void passC1_body(const FlameDesc &d, int tile) {
    griddep_wait();
    griddep_launch();
    using C = CplxT<R>;
    using V1 = typename OneOf<R>::type;
    constexpr int QE = E / 4;  // band registers: r < QE (k1 >= 0) and r >= E - QE (k1 < 0)
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    constexpr int N1 = 1 << LOG, T = N1 / E, PL = plane_len_e<E>(N1);
    const int f = threadIdx.x / T, t = threadIdx.x % T;
    const int k2 = 2 * tile + f;
    const bool valid = k2 <= a.K2;
    const int ld1 = 2 * a.K1 + 1;
    const CoefR<R> cfs = load_coef<R>(d.coef);  // derived by pass B
    const Planes<V1> sm(reinterpret_cast<R *>(smraw) + (size_t)f * 2 * PL, PL);
    const C *tw = static_cast<const C *>(d.tw1) + tw_offset_e<E>(LOG);
    const C *gk = static_cast<const C *>(d.gk);
    CV<V1> x[E];
    double colsum = 0.0;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const size_t i = gk_index(t + r * T, k2, N1);
        C p{0, 0};
        if (valid && FLAME_IN(d.status, i, gk_len(a), kSiteCGk)) p = __ldg(gk + i);
        if (k2 == 0) colsum += p.x;
        x[r] = CV<V1>{{p.x}, {p.y}};
    }
    // tile 0: the FP64 sum of column 0 over group 0 (its T threads) by
    // shuffles within each warp, then across the group's warps
    if (tile == 0) {
        if constexpr (T <= 32) {
            if (threadIdx.x < 32) {
                const unsigned lanes = blockDim.x >= 32 ? 0xffffffffu : (1u << blockDim.x) - 1u;
                for (int o = T >> 1; o > 0; o >>= 1) colsum += __shfl_xor_sync(lanes, colsum, o);
            }
        } else {
            __shared__ double wsum[T / 32];
            for (int o = 16; o > 0; o >>= 1) colsum += __shfl_xor_sync(0xffffffffu, colsum, o);
            if (f == 0 && (t & 31) == 0) wsum[t >> 5] = colsum;
            __syncthreads();
            if (threadIdx.x == 0)
                for (int w = 1; w < T / 32; ++w) colsum += wsum[w];
        }
    }
    line_fft_ct<-1, LOG, E>(x, t, sm, tw, CtaBarrier{});
    const bool lin = !(a.flags & kNonlinearOnly), nl = !(a.flags & kLinearOnly);
    const int stage = GEN ? d.stage : kStageEuler;
    const EpiArgs<R> ea{cfs, scale1<R>(a), scale2<R>(a), stage, lin, nl};
    C *col = static_cast<C *>(d.state) + (size_t)k2 * ld1 + a.K1;
    const C *fcol = GEN && d.forcing ? static_cast<const C *>(d.forcing) + (size_t)k2 * ld1 + a.K1 : nullptr;
    C *scol = GEN && d.save ? static_cast<C *>(d.save) + (size_t)k2 * ld1 + a.K1 : nullptr;
    int bad = 0;
    if (valid) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (!(r < QE || r >= E - QE)) continue;
            const int n = t + r * T;
            const int k1 = (r < QE) ? n : n - N1;
            const bool in_box = (r < QE) ? (n <= a.K1) : (k1 >= -a.K1);
            if (!in_box || (k2 == 0 && k1 < 0)) continue;  // k2 = 0, k1 < 0: the mirror of +k1
            const long long bi = (long long)k2 * ld1 + a.K1 + k1;
            const C ph = FLAME_IN(d.status, bi, box_len(a), kSiteCState) ? col[k1] : C{0, 0};
            C nw;
            update_entry<R, GEN>(d, ea, k1, k2, C{x[r].re.x, x[r].im.x}, ph, col, fcol, scol, nw, bad);
        }
    }
    if (bad) atomicOr(d.status, 1 << kStatusNonfinite);
    const double area = record_area<GEN>(d, tile, stage, N1);
    if (tile == 0 && threadIdx.x == 0) finish_step<GEN>(d, stage, nl, N1, colsum, area);
}

// Kernel entry points: one flame (descriptor by value) or an ensemble of
// equal-size flames (descriptor array, flame = blockIdx.y).  LOG > 0: line
// length 2^LOG fixed at compile time; LOG = 0: any length.
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_passA(FlameDesc d, int pf) {
    passA_body<R, LOG, 16>(d, blockIdx.x + d.tile0, gridDim.x + d.tile0, pf);
}
// compile-time length, direct (scattered) stores instead of the cluster write-out
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_passAd(FlameDesc d, int pf) {
    passA_body<R, LOG, 16, false>(d, blockIdx.x + d.tile0, gridDim.x + d.tile0, pf);
}
// compile-time length, column written out by tensor stores (FP32); the
// tensor map describes uv as (8 floats of a row pair) x k2 x row pair
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passAt(FlameDesc d, int pf, const __grid_constant__ CUtensorMap tm) {
    passA_body<R, LOG, 16, false, true>(d, blockIdx.x + d.tile0, gridDim.x + d.tile0, pf, &tm);
}
// One line per thread group (the passes above): CTAs of 2 (A, C) or 4 (B)
// groups of 2^LOG / E threads; pass C with the general epilogue (these
// kernels serve small grids, where the plain one would save nothing
// measurable).  MAXT: the largest CTA of the precision's line lengths.
template <class R> constexpr int kOneLineThreads = sizeof(R) == 8 ? 128 : 512;
template <class R, int LOG, int E>
__global__ void __launch_bounds__(kOneLineThreads<R>, 1) k_passA1(FlameDesc d, int pf) {
    passA1_body<R, LOG, E>(d, blockIdx.x + d.tile0);
}
template <class R, int LOG, int E>
__global__ void __launch_bounds__(kOneLineThreads<R>, 1) k_passB1(FlameDesc d, int pf) {
    passB1_body<R, LOG, E>(d, blockIdx.x);
}
template <class R, int LOG, int E>
__global__ void __launch_bounds__(kOneLineThreads<R>, 1) k_passC1(FlameDesc d, int pf) {
    passC1_body<R, LOG, E, true>(d, blockIdx.x + d.tile0);
}
template <class R, int LOG, int E>
__global__ void __launch_bounds__(kOneLineThreads<R>, 1) k_passC1_n(const FlameDesc *__restrict__ ds, int pf) {
    passC1_body<R, LOG, E, true>(ds[blockIdx.y], blockIdx.x);
}
template <class R, int LOG, int E>
__global__ void __launch_bounds__(kOneLineThreads<R>, 1) k_passA1_n(const FlameDesc *__restrict__ ds, int pf) {
    passA1_body<R, LOG, E>(ds[blockIdx.y], blockIdx.x);
}
template <class R, int LOG, int E>
__global__ void __launch_bounds__(kOneLineThreads<R>, 1) k_passB1_n(const FlameDesc *__restrict__ ds, int pf) {
    passB1_body<R, LOG, E>(ds[blockIdx.y], blockIdx.x);
}
// 8 points per thread, 512-thread CTAs (compile-time FP32 lengths)
template <class R, int LOG> __global__ void __launch_bounds__(512, 2) k_passA8(FlameDesc d, int pf) {
    passA_body<R, LOG, 8>(d, blockIdx.x + d.tile0, gridDim.x + d.tile0, pf);
}
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_passB(FlameDesc d, int pf) {
    passB_body<R, LOG, 16>(d, blockIdx.x, gridDim.x, pf);
}
// compile-time length, G written out by tensor stores (FP32); the tensor map
// describes gk as (8 floats of a row pair and column pair) x row pair x
// column pair
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passBt(FlameDesc d, int pf, const __grid_constant__ CUtensorMap tm) {
    passB_body<R, LOG, 16, true>(d, blockIdx.x, gridDim.x, pf, &tm);
}
// pass B that also sums the rows' surface area (the per-step record); its
// shared memory (three more row-length buffers) allows one CTA per SM
template <class R, int LOG, int E, int NT>
__global__ void __launch_bounds__(NT, 1) k_passB_area(FlameDesc d) {
    passB_body<R, LOG, E, false, false, true>(d, blockIdx.x, gridDim.x, 0);
}
// 8 points per thread, 512-thread CTAs (compile-time FP32 lengths)
template <class R, int LOG> __global__ void __launch_bounds__(512, 2) k_passB8(FlameDesc d, int pf) {
    passB_body<R, LOG, 8>(d, blockIdx.x, gridDim.x, pf);
}
template <class R, int LOG, bool GEN = true>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passC(FlameDesc d, int pf) {
    passC_body<R, LOG, false, 16, GEN>(d, blockIdx.x + d.tile0, gridDim.x + d.tile0, pf);
}
// pass C of one step fused with pass A of the next (FP32, compile-time
// lengths): the updated column pair is transformed back and written to uv
// by tensor stores (the uv map of k_passAt)
template <class R, int LOG, bool GEN = true>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passCA(FlameDesc d, int pf, const __grid_constant__ CUtensorMap tm) {
    passC_body<R, LOG, true, 16, GEN>(d, blockIdx.x, gridDim.x, pf, &tm);
}
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passA_n(const FlameDesc *__restrict__ ds, int pf) {
    passA_body<R, LOG, 16>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf);
}
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passAd_n(const FlameDesc *__restrict__ ds, int pf) {
    passA_body<R, LOG, 16, false>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf);
}
template <class R, int LOG>
__global__ void __launch_bounds__(512, 2) k_passA8_n(const FlameDesc *__restrict__ ds, int pf) {
    passA_body<R, LOG, 8>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf);
}
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passB_n(const FlameDesc *__restrict__ ds, int pf) {
    passB_body<R, LOG, 16>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf);
}
// ensembles with the tensor-store write-outs: maps[flame] is the flame's
// uv map (pass A) or gk map (pass B), in global memory
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passAt_n(const FlameDesc *__restrict__ ds, int pf,
                                                               const CUtensorMap *maps) {
    passA_body<R, LOG, 16, false, true, true>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf, maps + blockIdx.y);
}
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passBt_n(const FlameDesc *__restrict__ ds, int pf,
                                                               const CUtensorMap *maps) {
    passB_body<R, LOG, 16, true, true>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf, maps + blockIdx.y);
}
// 4096-point rows with warp-local exchanges (line_fft4096_wl), G written out
// by tensor stores
template <class R>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passBw(FlameDesc d, int pf, const __grid_constant__ CUtensorMap tm) {
    passB_body<R, 12, 16, true, false, false, true>(d, blockIdx.x, gridDim.x, pf, &tm);
}
template <class R>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passBw_n(const FlameDesc *__restrict__ ds, int pf,
                                                                 const CUtensorMap *maps) {
    passB_body<R, 12, 16, true, true, false, true>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf, maps + blockIdx.y);
}
// the same transforms with G written by direct stores (no tensor map): the
// arithmetic, and so the bits, of k_passBw
template <class R> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_passBwd(FlameDesc d, int pf) {
    passB_body<R, 12, 16, false, false, false, true>(d, blockIdx.x, gridDim.x, pf);
}
template <class R>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passBwd_n(const FlameDesc *__restrict__ ds, int pf) {
    passB_body<R, 12, 16, false, false, false, true>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf);
}
template <class R, int LOG>
__global__ void __launch_bounds__(512, 2) k_passB8_n(const FlameDesc *__restrict__ ds, int pf) {
    passB_body<R, LOG, 8>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf);
}
template <class R, int LOG>
__global__ void __launch_bounds__(256, kMinBlocks<R>) k_passC_n(const FlameDesc *__restrict__ ds, int pf) {
    passC_body<R, LOG>(ds[blockIdx.y], blockIdx.x, gridDim.x, pf);
}

}  // namespace flame
