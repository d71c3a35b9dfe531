// fft_engine.cuh -- device-side FFT building blocks for sm_103a.
//
// A "line" is one 1-D transform (a row or a column of the 2-D grid, Sec. 2:
// the 2-D FFT is the tensor product of 1-D ones).  Every thread carries TWO
// independent lines in lock step (the two halves of a V = float2 / double2):
// the FP32 path then runs on the paired FP32 instructions of sm_100+
// (__fadd2_rn / __fmul2_rn / __ffma2_rn), which halves the issue slots of
// the butterflies.
//
// Layout of a length-N line (N = 2^logN, 16 <= N <= 8192) over T = N/16
// threads: thread t holds x[r] = element t + r*T, r = 0..15.  A transform is
// a sequence of radix-16 Stockham passes (stride Ns = 16^s) followed, when
// logN is not a multiple of 4, by one radix-2/4/8 pass.  Between passes the
// line is exchanged through shared memory (two planes, re and im, padded by
// one slot every 16 to keep stores bank-conflict free).  The input of the
// first pass and the output of the last pass are both in the t + r*T layout,
// so global loads and stores of consecutive t are coalesced.
//
// Twiddles come from a per-length table generated in FP64 on the device
// (sincospi) and rounded once to the working precision.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>
#include <utility>

namespace flame {

// ----------------------------------------------------------------------------
// Two-line vector arithmetic
// ----------------------------------------------------------------------------
template <class R> struct VecOf;
template <> struct VecOf<float> { using type = float2; using c = float2; };
template <> struct VecOf<double> { using type = double2; using c = double2; };

// A negated operand of the paired instructions is free on sm_100+ (it is an
// operand modifier): vsub and the complex multiply below use it instead of
// a multiplication by a {-1, -1} constant.
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vbc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 vzero(float2) { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double2 vneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vbc(double s) { return make_double2(s, s); }
__device__ __forceinline__ double2 vzero(double2) { return make_double2(0.0, 0.0); }

// One line per thread (the one-line step kernels): a V of one double or one
// float, so that the two lines of a pair run in different warps.  GB300's
// FP64 units serve each SM sub-partition separately, and a line pair per
// warp leaves the other sub-partitions' units idle; small FP32 grids have
// too few line pairs to fill the SMs' warp slots.
struct D1 {
    double x;
};
struct F1 {
    float x;
};
__device__ __forceinline__ F1 vneg(F1 a) { return {-a.x}; }
__device__ __forceinline__ F1 vadd(F1 a, F1 b) { return {a.x + b.x}; }
__device__ __forceinline__ F1 vsub(F1 a, F1 b) { return {a.x - b.x}; }
__device__ __forceinline__ F1 vmul(F1 a, F1 b) { return {a.x * b.x}; }
__device__ __forceinline__ F1 vfma(F1 a, F1 b, F1 c) { return {fmaf(a.x, b.x, c.x)}; }
__device__ __forceinline__ F1 vzero(F1) { return {0.f}; }
__device__ __forceinline__ D1 vneg(D1 a) { return {-a.x}; }
__device__ __forceinline__ D1 vadd(D1 a, D1 b) { return {a.x + b.x}; }
__device__ __forceinline__ D1 vsub(D1 a, D1 b) { return {a.x - b.x}; }
__device__ __forceinline__ D1 vmul(D1 a, D1 b) { return {a.x * b.x}; }
__device__ __forceinline__ D1 vfma(D1 a, D1 b, D1 c) { return {fma(a.x, b.x, c.x)}; }
__device__ __forceinline__ D1 vzero(D1) { return {0.0}; }
// broadcast of a scalar to the V type of the tag
__device__ __forceinline__ float2 vbc_as(float s, float2) { return make_float2(s, s); }
__device__ __forceinline__ double2 vbc_as(double s, double2) { return make_double2(s, s); }
__device__ __forceinline__ D1 vbc_as(double s, D1) { return {s}; }
__device__ __forceinline__ F1 vbc_as(float s, F1) { return {s}; }
// the one-line V of a precision
template <class R> struct OneOf;
template <> struct OneOf<float> { using type = F1; };
template <> struct OneOf<double> { using type = D1; };

// Complex number whose re and im each hold the two lines (or one, for D1).
template <class V> struct CV { V re, im; };

template <class V> __device__ __forceinline__ CV<V> cadd(CV<V> a, CV<V> b) {
    return {vadd(a.re, b.re), vadd(a.im, b.im)};
}
template <class V> __device__ __forceinline__ CV<V> csub(CV<V> a, CV<V> b) {
    return {vsub(a.re, b.re), vsub(a.im, b.im)};
}
// a + s*i*b and a - s*i*b for s = +-1 (no explicit negation needed)
template <int S, class V> __device__ __forceinline__ CV<V> cadd_rot(CV<V> a, CV<V> b) {
    if constexpr (S > 0) return {vsub(a.re, b.im), vadd(a.im, b.re)};
    else return {vadd(a.re, b.im), vsub(a.im, b.re)};
}
template <int S, class V> __device__ __forceinline__ CV<V> csub_rot(CV<V> a, CV<V> b) {
    return cadd_rot<-S>(a, b);
}
// a * (wr + i wi) with the same scalar twiddle on both lines: two paired
// multiplies and two paired FMAs (the subtraction is a negated addend)
template <class V, class R> __device__ __forceinline__ CV<V> cmul_s(CV<V> a, R wr, R wi) {
    V vr = vbc_as(wr, V{}), vi = vbc_as(wi, V{});
    return {vfma(a.re, vr, vneg(vmul(a.im, vi))), vfma(a.re, vi, vmul(a.im, vr))};
}
template <class V, class R> __device__ __forceinline__ CV<V> cscale(CV<V> a, R s) {
    V v = vbc_as(s, V{});
    return {vmul(a.re, v), vmul(a.im, v)};
}

// compile-time loop
template <int B, int E, class F> __host__ __device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// cos / sin of 2 pi e / 16
struct Roots16 {
    static constexpr double C1 = 0.923879532511286756128183189396788933;  // cos(pi/8)
    static constexpr double S1 = 0.382683432365089771728459984030398866;  // sin(pi/8)
    static constexpr double H = 0.707106781186547524400844362104849039;   // sqrt(2)/2
    static constexpr double c[16] = {1.0, C1, H, S1, 0.0, -S1, -H, -C1,
                                     -1.0, -C1, -H, -S1, 0.0, S1, H, C1};
    static constexpr double s[16] = {0.0, S1, H, C1, 1.0, C1, H, S1,
                                     0.0, -S1, -H, -C1, -1.0, -C1, -H, -S1};
};

// a * exp(DIR 2 pi i E / R), R | 16, everything decided at compile time
template <int E, int R, int DIR, class V> __device__ __forceinline__ CV<V> tw_const(CV<V> a) {
    using Real = decltype(a.re.x);
    constexpr int e = ((E % R) * (16 / R)) & 15;
    constexpr double cr = Roots16::c[e];
    constexpr double ci = DIR * Roots16::s[e];
    if constexpr (ci == 0.0) {
        if constexpr (cr > 0) return a;
        else return {vneg(a.re), vneg(a.im)};  // folds into the consumer
    } else if constexpr (cr == 0.0) {
        // multiply by +-i
        if constexpr (ci > 0) return {vneg(a.im), a.re};
        else return {a.im, vneg(a.re)};
    } else if constexpr (cr == ci || cr == -ci) {
        // (cr + i ci) a = cr (a + i (ci/cr) a)
        constexpr int sg = (cr == ci) ? 1 : -1;
        CV<V> b = cadd_rot<sg>(a, a);
        return cscale(b, (Real)cr);
    } else {
        return cmul_s(a, (Real)cr, (Real)ci);
    }
}

// ----------------------------------------------------------------------------
// In-register DFTs, natural order in and out.  DIR = -1 forward, +1 inverse.
// ----------------------------------------------------------------------------
template <int R, int DIR, class V> __device__ __forceinline__ void dft(CV<V> *x);

template <int DIR, class V> __device__ __forceinline__ void dft2(CV<V> *x) {
    CV<V> a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
}
template <int DIR, class V> __device__ __forceinline__ void dft4(CV<V> *x) {
    CV<V> s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    CV<V> s13 = cadd(x[1], x[3]), d13 = csub(x[1], x[3]);
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd_rot<DIR>(d02, d13);
    x[3] = csub_rot<DIR>(d02, d13);
}

// R = R1 * R2: R2 DFTs of size R1 over n = R2 n1 + n2, twiddles
// w_R^(n2 k1), then R1 DFTs of size R2 over n2; output index k1 + R1 k2.
template <int R1, int R2, int DIR, class V> __device__ __forceinline__ void dft_split(CV<V> *x) {
    constexpr int R = R1 * R2;
    CV<V> y[R];
    static_for<0, R2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        CV<V> s[R1];
        static_for<0, R1>([&](auto n1c) {
            constexpr int n1 = decltype(n1c)::value;
            s[n1] = x[R2 * n1 + n2];
        });
        dft<R1, DIR>(s);
        static_for<0, R1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            y[n2 * R1 + k1] = tw_const<n2 * k1, R, DIR>(s[k1]);
        });
    });
    static_for<0, R1>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        CV<V> s[R2];
        static_for<0, R2>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            s[n2] = y[n2 * R1 + k1];
        });
        dft<R2, DIR>(s);
        static_for<0, R2>([&](auto k2c) {
            constexpr int k2 = decltype(k2c)::value;
            x[k1 + R1 * k2] = s[k2];
        });
    });
}

template <int R, int DIR, class V> __device__ __forceinline__ void dft(CV<V> *x) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) dft2<DIR>(x);
    else if constexpr (R == 4) dft4<DIR>(x);
    else if constexpr (R == 8) dft_split<4, 2, DIR>(x);
    else if constexpr (R == 16) dft_split<4, 4, DIR>(x);
    else static_assert(R <= 16, "radix");
}

// ----------------------------------------------------------------------------
// Twiddle tables.  For a line of length N = 2^logN the table holds, in order:
//   for each radix-16 pass s >= 1 (stride Ns = 16^s):
//       w[(r-1) Ns + m] = exp(2 pi i r m / (16 Ns)),  r = 1..15, m < Ns
//   for the final radix-rho pass (rho = 2^(logN mod 4) > 1, Ns = N / rho):
//       w[(q-1) Ns + m] = exp(2 pi i q m / N),        q = 1..rho-1, m < Ns
//   real-transform table (used when N is the half length of a 2N real FFT):
//       w[k] = exp(2 pi i k / (2N)),                  k < N
// Stored with the + sign; forward transforms use the conjugate.
// ----------------------------------------------------------------------------
__host__ __device__ constexpr int tw_pass_offset(int s, int LE = 4) {  // offset of pass s >= 1
    int off = 0, ns = 1 << LE;
    for (int q = 1; q < s; ++q) { off += ((1 << LE) - 1) * ns; ns <<= LE; }
    return off;
}
__host__ __device__ constexpr int tw_final_offset(int logN, int LE = 4) { return tw_pass_offset(logN / LE, LE); }
__host__ __device__ constexpr int tw_real_offset(int logN, int LE = 4) {
    return tw_final_offset(logN, LE) + ((1 << (logN % LE)) - 1) * ((1 << logN) >> (logN % LE));
}
__host__ __device__ constexpr int tw_table_len(int logN, int LE = 4) { return tw_real_offset(logN, LE) + (1 << logN); }
// A line's twiddle allocation: the radix-16 table, then the radix-8 table
// (8-point-per-thread kernels), then the radix-4 table (4 points per thread,
// the FP64 short-line kernels).
__host__ __device__ constexpr int tw_alloc_len(int logN) {
    return tw_table_len(logN, 4) + tw_table_len(logN, 3) + tw_table_len(logN, 2);
}
// log2 of the points per thread E (16, 8 or 4)
template <int E> __host__ __device__ constexpr int log2_e() { return E == 16 ? 4 : E == 8 ? 3 : 2; }

// ----------------------------------------------------------------------------
// Shared-memory exchange
// ----------------------------------------------------------------------------
__host__ __device__ constexpr int spad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int plane_len(int N) { return N + (N >> 4); }
// radix-E exchanges pad one slot every E (E = 8 or 16)
template <int E> __host__ __device__ constexpr int spad_e(int i) { return i + (i >> log2_e<E>()); }
template <int E> __host__ __device__ constexpr int plane_len_e(int N) { return N + (N >> log2_e<E>()); }

// Barrier over the threads that share the exchange buffers.
struct CtaBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Exchange buffer of one pair of lines: plane_len(N) slots of CV<V>.  FP32:
// one plane of 16-byte slots (one 128-bit access per point, conflict-free for
// the Stockham store pattern thanks to the padding); FP64: separate re and im
// planes of 16-byte slots.  Both take plane_len(N) * 2 * sizeof(V) bytes.
template <class V> struct Planes;
template <> struct Planes<float2> {
    float4 *p;
    __device__ __forceinline__ explicit Planes(float2 *base) : p(reinterpret_cast<float4 *>(base)) {}
    __device__ __forceinline__ void st(int i, CV<float2> v) const {
        p[spad(i)] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
    }
    __device__ __forceinline__ CV<float2> ld(int i) const {
        float4 q = p[spad(i)];
        return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
    }
    // slot index already padded
    __device__ __forceinline__ void st_raw(int j, CV<float2> v) const {
        p[j] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
    }
    __device__ __forceinline__ CV<float2> ld_raw(int j) const {
        float4 q = p[j];
        return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
    }
};
template <> struct Planes<double2> {
    double2 *re, *im;
    int len;
    __device__ __forceinline__ Planes(double2 *base, int n) : re(base), im(base + plane_len(n)) {}
    // planes of `plane` slots each (the radix-8 padding needs plane_len_e<8>)
    __device__ __forceinline__ Planes(double2 *base, int n, int plane) : re(base), im(base + plane) {}
    __device__ __forceinline__ void st(int i, CV<double2> v) const { re[spad(i)] = v.re; im[spad(i)] = v.im; }
    __device__ __forceinline__ CV<double2> ld(int i) const { return {re[spad(i)], im[spad(i)]}; }
    __device__ __forceinline__ void st_raw(int j, CV<double2> v) const { re[j] = v.re; im[j] = v.im; }
    __device__ __forceinline__ CV<double2> ld_raw(int j) const { return {re[j], im[j]}; }
};
// One-line exchange buffer: separate re and im planes of `plane` reals each.
template <class V1> struct Planes1 {
    using Real = decltype(V1::x);
    Real *re, *im;
    __device__ __forceinline__ Planes1(Real *base, int plane) : re(base), im(base + plane) {}
    __device__ __forceinline__ void st(int i, CV<V1> v) const { re[spad(i)] = v.re.x; im[spad(i)] = v.im.x; }
    __device__ __forceinline__ CV<V1> ld(int i) const { return {{re[spad(i)]}, {im[spad(i)]}}; }
    __device__ __forceinline__ void st_raw(int j, CV<V1> v) const { re[j] = v.re.x; im[j] = v.im.x; }
    __device__ __forceinline__ CV<V1> ld_raw(int j) const { return {{re[j]}, {im[j]}}; }
};
template <> struct Planes<D1> : Planes1<D1> {
    using Planes1<D1>::Planes1;
};
template <> struct Planes<F1> : Planes1<F1> {
    using Planes1<F1>::Planes1;
};
// Exchange buffer of a group: `base` points at 2 * plane_len(n) V slots.
__device__ __forceinline__ Planes<float2> make_planes(float2 *base, int n) { return Planes<float2>(base); }
__device__ __forceinline__ Planes<double2> make_planes(double2 *base, int n) { return Planes<double2>(base, n); }
// exchange buffer of a radix-E transform (E = 8 pads one slot every 8)
template <int E> __device__ __forceinline__ Planes<float2> make_planes_e(float2 *base, int n) {
    return Planes<float2>(base);
}
template <int E> __device__ __forceinline__ Planes<double2> make_planes_e(double2 *base, int n) {
    return Planes<double2>(base, n, plane_len_e<E>(n));
}

// Loads the twiddle of a table entry (stored with + sign) for direction DIR.
template <int DIR, class C> __device__ __forceinline__ void load_tw(const C *tab, int i, decltype(C::x) &wr,
                                                                    decltype(C::x) &wi) {
    C w = __ldg(tab + i);
    wr = w.x;
    wi = (DIR > 0) ? w.y : -w.y;
}

// Full transform of one pair of lines of length N = 2^logN held as x[16].
// tw: twiddle table of this length (see above).  All threads of the barrier
// must call this with the same logN.  On return the result is in x in the
// same t + r*T layout; shared memory may still be read by other threads, so
// callers synchronise before reusing it.
template <int DIR, class V, class C, class Bar>
__device__ __forceinline__ void line_fft(CV<V> (&x)[16], int logN, int t, const Planes<V> &sm,
                                         const C *__restrict__ tw, Bar bar) {
    using Real = decltype(C::x);
    const int N = 1 << logN;
    const int T = N >> 4;
    const int P16 = logN >> 2;
    const int lr = logN & 3;
    const C *twp = tw;
#pragma unroll 1
    for (int s = 0; s < P16; ++s) {
        const int Ns = 1 << (4 * s);
        if (s > 0) {
            const int m = t & (Ns - 1);
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                Real wr, wi;
                load_tw<DIR>(twp, (r - 1) * Ns + m, wr, wi);
                x[r] = cmul_s(x[r], wr, wi);
            }
            twp += 15 * Ns;
        }
        dft<16, DIR>(x);
        const bool last = (s == P16 - 1) && (lr == 0);
        if (!last) {
            const int idxD = ((t >> (4 * s)) << (4 * s + 4)) + (t & (Ns - 1));
            bar();
#pragma unroll
            for (int r = 0; r < 16; ++r) sm.st(idxD + r * Ns, x[r]);
            bar();
#pragma unroll
            for (int r = 0; r < 16; ++r) x[r] = sm.ld(t + r * T);
        }
    }
    if (lr > 0) {
        auto final_pass = [&](auto rhoc) {
            constexpr int rho = decltype(rhoc)::value;
            constexpr int B = 16 / rho;  // butterflies per thread
            const int Ns = N / rho;
            const C *twf = tw + tw_final_offset(logN);
#pragma unroll
            for (int mm = 0; mm < B; ++mm) {
                const int j = t + mm * T;
                CV<V> y[rho];
#pragma unroll
                for (int q = 0; q < rho; ++q) y[q] = x[mm + q * B];
#pragma unroll
                for (int q = 1; q < rho; ++q) {
                    Real wr, wi;
                    load_tw<DIR>(twf, (q - 1) * Ns + j, wr, wi);
                    y[q] = cmul_s(y[q], wr, wi);
                }
                dft<rho, DIR>(y);
#pragma unroll
                for (int q = 0; q < rho; ++q) x[mm + q * B] = y[q];
            }
        };
        if (lr == 1) final_pass(std::integral_constant<int, 2>{});
        else if (lr == 2) final_pass(std::integral_constant<int, 4>{});
        else final_pass(std::integral_constant<int, 8>{});
    }
}

// Twiddle sources of the compile-time transform.  TwGlobal reads the
// per-length table; TwShared reads a factorised copy in shared memory: the
// pass-1 section (w_256^(r m), 15 x 16 entries) and the first 16 entries of
// each pass-2 row (w_4096^(r m), m < 16), so that for m = m_lo + 16 m_hi
//   w_4096^(r m) = w_4096^(r m_lo) * w_256^(r m_hi),
// 480 entries (3.75 KB in FP32) instead of 4080.
template <class C> struct TwGlobal {
    const C *tw;
    template <int S, int LE>
    __device__ __forceinline__ C get(int r, int m) const {
        constexpr int Ns = 1 << (LE * S);
        return __ldg(tw + tw_pass_offset(S, LE) + (r - 1) * Ns + m);
    }
};
template <class C> struct TwShared {
    const C *t1;   // [15][16]: w_256^(r m)
    const C *t2;   // [15][16]: w_4096^(r m), m < 16
    template <int S, int LE>
    __device__ __forceinline__ C get(int r, int m) const {
        static_assert(LE == 4 && S <= 2, "radix-16 passes 1 and 2 only");
        if constexpr (S == 1) return t1[(r - 1) * 16 + m];
        else {
            const C a = t2[(r - 1) * 16 + (m & 15)], b = t1[(r - 1) * 16 + (m >> 4)];
            return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
        }
    }
    // copies the factor tables of the radix-16 global table of a line of
    // length 2^LOG into smem: pass 1 always (LOG >= 8), pass 2 when it
    // exists (LOG >= 12); the caller synchronises before use
    template <int LOG> __device__ __forceinline__ static void fill(C *dst, const C *tw) {
        static_assert(LOG >= 8, "pass 1 needs N >= 256");
        constexpr int n = LOG >= 12 ? 480 : 240;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int h = i / 240, j = i % 240, r = j / 16, m = j % 16;
            dst[i] = h == 0 ? __ldg(tw + tw_pass_offset(1, 4) + r * 16 + m)
                            : __ldg(tw + tw_pass_offset(2, 4) + r * 256 + m);
        }
    }
};

// Same transform with the length known at compile time (LOGN) and E points
// per thread (radix-E passes, E = 16 or 8; T = N/E threads per line): pass
// strides, twiddle-table offsets and padded exchange addresses fold into
// immediates.  With one pad slot every E slots, padded addresses are
// base + r * stride because the strides are multiples of E:
//   store of pass s:  spad(idxD + r Ns) = spad(idxD) + r (Ns == 1 ? 1 : Ns + Ns/E)
//   load:             spad(t + r T)     = spad(t) + r (T + T/E)      (T >= E)
// `tw` is the radix-E table of this length.
template <int DIR, int LOGN, int E, class V, class C, class Bar, class TW = TwGlobal<C>>
__device__ __forceinline__ void line_fft_ct(CV<V> (&x)[E], int t, const Planes<V> &sm,
                                            const C *__restrict__ tw, Bar bar, TW twp = TW{nullptr}) {
    using Real = decltype(C::x);
    constexpr int LE = log2_e<E>();
    constexpr int N = 1 << LOGN, T = N / E, P = LOGN / LE, LR = LOGN % LE;
    static_for<0, P>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        constexpr int Ns = 1 << (LE * s);
        if constexpr (s > 0) {
            const int m = t & (Ns - 1);
            TW src = twp;
            if constexpr (std::is_same<TW, TwGlobal<C>>::value) src.tw = tw;
#pragma unroll
            for (int r = 1; r < E; ++r) {
                const C w = src.template get<s, LE>(r, m);
                x[r] = cmul_s(x[r], w.x, DIR > 0 ? w.y : -w.y);
            }
        }
        dft<E, DIR>(x);
        constexpr bool last = (s == P - 1) && (LR == 0);
        if constexpr (!last) {
            const int idxD = ((t >> (LE * s)) << (LE * s + LE)) + (t & (Ns - 1));
            const int wb = spad_e<E>(idxD);
            constexpr int ws = (Ns == 1) ? 1 : Ns + Ns / E;
            bar();
#pragma unroll
            for (int r = 0; r < E; ++r) sm.st_raw(wb + r * ws, x[r]);
            bar();
            if constexpr (T >= E) {
                const int rb = spad_e<E>(t);
                constexpr int rs = T + T / E;
#pragma unroll
                for (int r = 0; r < E; ++r) x[r] = sm.ld_raw(rb + r * rs);
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) x[r] = sm.ld_raw(spad_e<E>(t + r * T));
            }
        }
    });
    if constexpr (LR > 0) {
        constexpr int rho = 1 << LR, B = E / rho, Ns = N / rho;
        const C *twf = tw + tw_final_offset(LOGN, LE);
#pragma unroll
        for (int mm = 0; mm < B; ++mm) {
            const int j = t + mm * T;
            CV<V> y[rho];
#pragma unroll
            for (int q = 0; q < rho; ++q) y[q] = x[mm + q * B];
#pragma unroll
            for (int q = 1; q < rho; ++q) {
                Real wr, wi;
                load_tw<DIR>(twf, (q - 1) * Ns + j, wr, wi);
                y[q] = cmul_s(y[q], wr, wi);
            }
            dft<rho, DIR>(y);
#pragma unroll
            for (int q = 0; q < rho; ++q) x[mm + q * B] = y[q];
        }
    }
}

// Compile-time length when LOG > 0, runtime length otherwise.
template <int DIR, int LOG, class V, class C>
__device__ __forceinline__ void fft_line(CV<V> (&x)[16], int logn, int t, const Planes<V> &sm,
                                         const C *__restrict__ tw) {
    if constexpr (LOG > 0) line_fft_ct<DIR, LOG, 16>(x, t, sm, tw, CtaBarrier{});
    else line_fft<DIR>(x, logn, t, sm, tw, CtaBarrier{});
}
// Compile-time length (8 <= LOG <= 12) with the radix-16 pass twiddles taken
// from the shared-memory factors `stw` (see TwShared); the final-pass
// twiddles still come from `tw`.
template <int DIR, int LOG, class V, class C>
__device__ __forceinline__ void fft_line_s(CV<V> (&x)[16], int t, const Planes<V> &sm, const C *__restrict__ tw,
                                           const C *stw) {
    static_assert(LOG >= 8 && LOG <= 12, "shared twiddles cover passes 1 and 2");
    line_fft_ct<DIR, LOG, 16>(x, t, sm, tw, CtaBarrier{}, TwShared<C>{stw, stw + 240});
}

// 4096-point transform of a line pair over T = 256 threads with one of its
// two exchanges inside a warp.  With n = 256 a + 16 b + c and
// k = k_a + 16 k_b + 256 k_c (a, b, c, k_* < 16),
//   W^(n k) = W16^(a k_a) W4096^((16 b + c) k_a) W16^(b k_b) W256^(c k_b) W16^(c k_c),
// so the line is three radix-16 passes (over a, b, c) with the twiddles
// W4096^((16 b + c) k_a) and W256^(c k_b) between them.  Thread t = 16 hi + lo
// (hi = t / 16, lo = t mod 16) holds 16 values of one digit in registers and
// the other two digits by its index:
//   NAT_IN  (natural in, digit-swapped out):
//     pass 1 (b, c) = (hi, lo), input n = t + 256 r;
//     pass 2 (k_a, c) = (hi, lo): the first exchange crosses warps;
//     pass 3 (k_a, k_b) = (hi, lo): the second stays within the 16 threads of
//     one hi, output k = swap(t) + 256 r, swap(t) = 16 lo + hi.
//   !NAT_IN (digit-swapped in, natural out):
//     pass 1 (b, c) = (lo, hi), input n = swap(t) + 256 r;
//     pass 2 (k_a, c) = (lo, hi): the first exchange stays within the 16
//     threads of one hi;
//     pass 3 (k_a, k_b) = (lo, hi): the second crosses warps, output
//     k = t + 256 r.
// An inverse transform with NAT_IN followed, after pointwise work, by a
// forward one without it needs no exchange between the two and gives
// natural order at both ends.  A warp-local exchange reads and writes only
// the slots [256 hi, 256 hi + 256) (before padding) of its own 16 threads,
// so it is ordered by __syncwarp; the cross-warp one by the CTA barrier.
// Every exchange is bank-conflict free with the one-slot-in-16 padding.
template <int DIR, bool NAT_IN, class V, class C>
__device__ __forceinline__ void line_fft4096_wl(CV<V> (&x)[16], int t, const Planes<V> &sm, const TwShared<C> &tw) {
    const int hi = t >> 4, lo = t & 15;
    // W4096^(m r) for m = m_lo + 16 m_hi (the factors of TwShared), or
    // W256^(m_lo r) when m_hi < 0
    auto twiddle = [&](int m_lo, int m_hi) {
        const C *t1 = tw.t1 + m_lo, *t2 = tw.t2 + m_lo, *t1h = tw.t1 + m_hi;
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            C w;
            if (m_hi < 0) w = t1[(r - 1) * 16];
            else {
                const C a = t2[(r - 1) * 16], b = t1h[(r - 1) * 16];
                w = C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
            }
            x[r] = cmul_s(x[r], w.x, DIR > 0 ? w.y : -w.y);
        }
    };
    // padded slots: spad(base + r stride) = spad(base) + r (stride + stride / 16)
    // for strides that are multiples of 16, and spad(base) + r for stride 1
    // from a multiple of 16 (the only forms used below)
    auto store = [&](int base, auto sc) {
        constexpr int stride = decltype(sc)::value, ps = stride == 1 ? 1 : stride + stride / 16;
        const int b = spad(base);
#pragma unroll
        for (int r = 0; r < 16; ++r) sm.st_raw(b + r * ps, x[r]);
    };
    auto load = [&](int base, auto sc) {
        constexpr int stride = decltype(sc)::value, ps = stride == 1 ? 1 : stride + stride / 16;
        const int b = spad(base);
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = sm.ld_raw(b + r * ps);
    };
    using S1 = std::integral_constant<int, 1>;
    using S16 = std::integral_constant<int, 16>;
    using S256 = std::integral_constant<int, 256>;
    dft<16, DIR>(x);                                                          // over a
    twiddle(NAT_IN ? lo : hi, NAT_IN ? hi : lo);                             // W4096^((16 b + c) k_a)
    if constexpr (NAT_IN) {
        __syncthreads();
        store(t, S256{});             // slot 256 k_a + 16 b + c
        __syncthreads();
        load(256 * hi + lo, S16{});   // (k_a, c) = (hi, lo), b = r
    } else {
        __syncwarp();
        store(256 * hi + lo, S16{});  // slot 256 c + 16 k_a + b
        __syncwarp();
        load(256 * hi + 16 * lo, S1{});  // (k_a, c) = (lo, hi), b = r
    }
    dft<16, DIR>(x);                                                          // over b
    twiddle(NAT_IN ? lo : hi, -1);                                           // W256^(c k_b)
    if constexpr (NAT_IN) {
        __syncwarp();
        store(256 * hi + lo, S16{});     // slot 256 k_a + 16 k_b + c
        __syncwarp();
        load(256 * hi + 16 * lo, S1{});  // (k_a, k_b) = (hi, lo), c = r
    } else {
        __syncthreads();
        store(256 * hi + lo, S16{});  // slot 256 c + 16 k_b + k_a
        __syncthreads();
        load(t, S256{});              // (k_a, k_b) = (lo, hi), c = r
    }
    dft<16, DIR>(x);                                                          // over c
}

}  // namespace flame
