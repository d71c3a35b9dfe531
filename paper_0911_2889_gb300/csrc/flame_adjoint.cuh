// flame_adjoint.cuh -- kernels of the area objective and of the discrete
// adjoint of the explicit step (project-added; the paper has neither).
//
// Conventions (inner product on spectra: <X, Y> = Re sum over the full
// spectrum of conj(X_k) Y_k; synthesis  phi(x) = sum_k Phi_k e^{ik.x};
// analysis  hat(a)_k = sum_x a(x) e^{-ik.x}):
//
//   area   A = sum_x w R sqrt(R^2 + |grad phi|^2),  R = r0 + phi,
//          w = (2 pi)^2 / (N1 N2 s1 s2);
//          dA/dPhi_k = hat(a)_k - i kappa_1 hat(b1)_k - i kappa_2 hat(b2)_k with
//          a = w (S + R^2/S), b_i = w R d_i phi / S, S = sqrt(R^2 + |grad phi|^2).
//   adjoint of one Euler step at (Phi_n, t_n), lambda = lambda_{n+1}:
//          lambda_n = lambda + dt (omega_k lambda + c P_k)   (k != 0),
//          P = (1/(N1 N2)) [ -i kappa_1 hat(q1) - i kappa_2 hat(q2) ],
//          q_i = 2 ell d_i phi_n,  ell = synthesis of lambda (with lambda_0),
//          lambda_0 unchanged; dL/dgamma += <lambda, dt |kappa|/(2 r0) Phi_n>.
#pragma once

#include "flame_kernels.cuh"

namespace flame {

template <class R> __device__ __forceinline__ CplxT<R> cmulc(CplxT<R> a, CplxT<R> b) {
    return CplxT<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// --- area, pass A: columns of (i s1 k1 Phi, Phi with the mean mode) ---------
// writes uv[j1][k2] = (U, P) with U = synthesis of i s1 k1 Phi and P the
// column synthesis of Phi (the mean mode at k = 0).
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_areaA(AdjDesc d) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    const C *state = static_cast<const C *>(d.state);
    C *uv = static_cast<C *>(d.uv);
    const int N1 = 1 << a.logn1, T = N1 >> 4;
    const int G = blockDim.x / T, g = threadIdx.x / T, t = threadIdx.x % T;
    const int ld1 = 2 * a.K1 + 1;
    const int k2 = blockIdx.x * G + g;
    const bool valid = k2 <= a.K2;
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len(N1);
    auto sm = make_planes(base, N1);
    const C *col = state + (size_t)k2 * ld1 + a.K1;
    const double mean0 = *d.mean;
    CV<V> x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        x[r] = CV<V>{vzero(V{}), vzero(V{})};
        if (r < 4 || r >= 12) {
            const int n = t + r * T;
            const int k1 = (r < 4) ? n : n - N1;
            const bool in_box = valid && ((r < 4) ? (n <= a.K1) : (k1 >= -a.K1));
            if (in_box) {
                C phi = col[k1];
                if (k1 == 0 && k2 == 0) phi = C{(R)mean0, 0};
                const R f = scale1<R>(a) * (R)k1;
                x[r] = pack2<R>(C{-f * phi.y, f * phi.x}, phi);
            }
        }
    }
    fft_line<1, LOG>(x, a.logn1, t, sm, static_cast<const C *>(d.tw1));
    if (valid) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int n = t + r * T;
            st_uv<R>(uv + uv_index(n, k2, a.ldk), lane0<R>(x[r]), lane1<R>(x[r]));
        }
    }
}

// Half-band inverse of one row: from the row spectrum S[k] (k = -K2..K2,
// S[-k] = conj S[k] unless `full`) builds the lanes Y_q[k mod M] =
// S[k] e^{2 pi i k q / N2} (q = 0, 1) and transforms them; lane q of x[r]
// is then the synthesis at grid point 2m + q, m = t + r T.
template <class R, int LOG, class Get>
__device__ __forceinline__ void halfband_ifft(CV<typename VecOf<R>::type> (&x)[16], const StepArgs &a, int t,
                                              const CplxT<R> *P, const CplxT<R> *twm, Get get, bool valid,
                                              void *smbase) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    const int M = 1 << a.logm, T = M >> 4;
    auto sm = make_planes(static_cast<V *>(smbase), M);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = t + r * T;
        const int kk = (r < 8) ? n : M - n;
        C z{0, 0};
        if (valid && kk <= a.K2) z = get(kk, r < 8);
        C w = __ldg(P + kk);
        C z1 = (r < 8) ? C{z.x * w.x - z.y * w.y, z.x * w.y + z.y * w.x}
                       : C{z.x * w.x + z.y * w.y, z.y * w.x - z.x * w.y};
        x[r] = pack2<R>(z, z1);
    }
    fft_line<1, LOG>(x, a.logm, t, sm, twm);
}

// Forward real transform of two real rows given as h_q[m] = f_q[2m] + i
// f_q[2m+1] in the lanes of x (q = 0, 1); on return out(k, Y) is called for
// k = 0..K2 (r < 8) with Y the pair of analyses (lane 0: f_0, lane 1: f_1).
template <class R, int LOG, class Out>
__device__ __forceinline__ void real_fwd(CV<typename VecOf<R>::type> (&x)[16], const StepArgs &a, int t,
                                         const CplxT<R> *P, const CplxT<R> *twm, void *smbase, bool valid,
                                         Out out) {
    using V = typename VecOf<R>::type;
    const int M = 1 << a.logm, T = M >> 4;
    auto sm = make_planes(static_cast<V *>(smbase), M);
    fft_line<-1, LOG>(x, a.logm, t, sm, twm);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) sm.st(t + r * T, x[r]);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int k = t + r * T;
        if (valid && k <= a.K2) {
            CV<V> h = x[r], hc = sm.ld((M - k) & (M - 1));
            const R hf = (R)0.5;
            CV<V> E{vmul(vadd(h.re, hc.re), vbc(hf)), vmul(vsub(h.im, hc.im), vbc(hf))};
            CV<V> O{vmul(vadd(h.im, hc.im), vbc(hf)), vmul(vsub(hc.re, h.re), vbc(hf))};
            auto w = __ldg(P + k);
            out(k, cadd(E, cmul_s(O, w.x, -w.y)));
        }
    }
    __syncthreads();
}

// --- area, pass B: one row per group ----------------------------------------
// u + iv from U, V = i s2 k2 P; phi from P; pointwise area terms; forward
// real transforms of a, b1, b2.  Writes aw[k2][j1] = (hat a, hat b1) and
// gk[k2][j1] = hat b2 (column-major), rowsum[j1] = sum_x of w R S over the row.
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_areaB(AdjDesc d) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[256];  // one per thread (blockDim = N2/32 <= 256)
    const StepArgs &a = d.a;
    const C *uv = static_cast<const C *>(d.uv);
    const C *twm = static_cast<const C *>(d.twm);
    const int M = 1 << a.logm, T = M >> 4;
    const int t = threadIdx.x;  // one group per CTA
    const int row = blockIdx.x;
    const bool valid = row < a.n1;
    V *base = reinterpret_cast<V *>(smraw);
    C *park = reinterpret_cast<C *>(base + 2 * plane_len(M));  // M entries
    const C *P = twm + tw_real_offset(a.logm);
    const C *src = uv + uv_index(valid ? row : 0, 0, a.ldk);  // element kk at src + 4 kk
    const R s2 = scale2<R>(a);
    // phi at 2m, 2m+1 (real parts of the two lanes), parked
    CV<V> x[16];
    halfband_ifft<R, LOG>(x, a, t, P, twm,
                     [&](int kk, bool pos) {
                         UV<R> e = ld_uv<R>(src + 4 * (size_t)kk);
                         return pos ? e.v : C{e.v.x, -e.v.y};
                     },
                     valid, base);
#pragma unroll
    for (int r = 0; r < 16; ++r) park[t + r * T] = C{x[r].re.x, x[r].re.y};
    // u + iv at 2m, 2m+1
    halfband_ifft<R, LOG>(x, a, t, P, twm,
                     [&](int kk, bool pos) {
                         UV<R> e = ld_uv<R>(src + 4 * (size_t)kk);
                         const R f = s2 * (R)kk;
                         C Vv{-f * e.v.y, f * e.v.x};  // i s2 k2 P
                         if (pos) return C{e.u.x - Vv.y, e.u.y + Vv.x};
                         return C{e.u.x + Vv.y, Vv.x - e.u.y};
                     },
                     valid, base);
    const double r0 = *d.t;
    const R w = (R)((2.0 * 3.14159265358979323846) * (2.0 * 3.14159265358979323846) /
                    ((double)a.n1 * (double)a.n2 * a.s1 * a.s2));
    double part = 0.0;
    C hb2[16];
    CV<V> y[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        C ph = park[t + r * T];
        R av[2], b1[2], b2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const R u = q == 0 ? x[r].re.x : x[r].re.y;
            const R v = q == 0 ? x[r].im.x : x[r].im.y;
            const R Rr = (R)r0 + (q == 0 ? ph.x : ph.y);
            const R S = sqrt(Rr * Rr + u * u + v * v);
            part += (double)(w * Rr * S);
            av[q] = w * (S + Rr * Rr / S);
            b1[q] = w * Rr * u / S;
            b2[q] = w * Rr * v / S;
        }
        y[r] = pack2<R>(C{av[0], av[1]}, C{b1[0], b1[1]});
        hb2[r] = C{b2[0], b2[1]};
    }
    if (!valid) part = 0.0;
    red[t] = part;  // summed by thread 0 after the barriers of real_fwd
    C *aw = static_cast<C *>(d.aw);
    C *gk = static_cast<C *>(d.gk);
    real_fwd<R, LOG>(y, a, t, P, twm, base, valid, [&](int k, CV<V> Y) {
        C *dst = aw + 2 * ((size_t)k * a.n1 + row);
        st_uv<R>(dst, lane0<R>(Y), lane1<R>(Y));
    });
#pragma unroll
    for (int r = 0; r < 16; ++r) y[r] = pack2<R>(hb2[r], C{0, 0});
    real_fwd<R, LOG>(y, a, t, P, twm, base, valid, [&](int k, CV<V> Y) { gk[(size_t)k * a.n1 + row] = lane0<R>(Y); });
    if (t == 0 && valid) {
        double s = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) s += red[i];
        d.rowsum[row] = s;
    }
}

// --- area, pass C: one column per group -------------------------------------
// forward column transforms of (hat a, hat b1) and hat b2, combination
// grad = A - i s1 k1 B1 - i s2 k2 B2 on the box; block 0 also reduces the
// row sums into the area and writes dA/dPhi_0.
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_areaC(AdjDesc d) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    const int N1 = 1 << a.logn1, T = N1 >> 4;
    const int G = blockDim.x / T, g = threadIdx.x / T, t = threadIdx.x % T;
    const int ld1 = 2 * a.K1 + 1;
    const int k2 = blockIdx.x * G + g;
    const bool valid = k2 <= a.K2;
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len(N1);
    auto sm = make_planes(base, N1);
    const C *tw1 = static_cast<const C *>(d.tw1);
    const C *aw = static_cast<const C *>(d.aw) + 2 * (size_t)(valid ? k2 : 0) * N1;
    const C *gk = static_cast<const C *>(d.gk) + (size_t)(valid ? k2 : 0) * N1;
    // hat b2 first (only the box rows are kept), then (hat a, hat b1)
    CV<V> x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = t + r * T;
        x[r] = pack2<R>(valid ? gk[n] : C{0, 0}, C{0, 0});
    }
    fft_line<-1, LOG>(x, a.logn1, t, sm, tw1);
    C B2[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) B2[i] = lane0<R>(x[i < 4 ? i : i + 8]);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = t + r * T;
        UV<R> e = valid ? ld_uv<R>(aw + 2 * n) : UV<R>{C{0, 0}, C{0, 0}};
        x[r] = pack2<R>(e.u, e.v);
    }
    fft_line<-1, LOG>(x, a.logn1, t, sm, tw1);
    C *grad = static_cast<C *>(d.grad);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = i < 4 ? i : i + 8;
        const int n = t + r * T;
        const int k1 = (r < 4) ? n : n - N1;
        const bool in_box = valid && ((r < 4) ? (n <= a.K1) : (k1 >= -a.K1));
        if (in_box) {
            C A = lane0<R>(x[r]), B1 = lane1<R>(x[r]);
            const R f1 = scale1<R>(a) * (R)k1, f2 = scale2<R>(a) * (R)k2;
            // A - i f1 B1 - i f2 B2
            C gr{A.x + f1 * B1.y + f2 * B2[i].y, A.y - f1 * B1.x - f2 * B2[i].x};
            if (k1 == 0 && k2 == 0) {
                *d.dmean = (double)A.x;
                gr = C{0, 0};
            }
            if (grad) grad[(size_t)k2 * ld1 + k1 + a.K1] = gr;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < a.n1; ++i) s += d.rowsum[i];
        *d.area = s;
    }
}

// --- adjoint: column synthesis of lambda (two columns per group) -------------
// gk[j1][k2] (row-major) = column synthesis of lambda, lambda_0 at k = 0.
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_adjL(AdjDesc d) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    const int N1 = 1 << a.logn1, T = N1 >> 4;
    const int G = blockDim.x / T, g = threadIdx.x / T, t = threadIdx.x % T;
    const int ld1 = 2 * a.K1 + 1;
    const int c0 = 2 * (blockIdx.x * G + g);
    const bool va = c0 <= a.K2, vb = c0 + 1 <= a.K2;
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len(N1);
    auto sm = make_planes(base, N1);
    const C *lam = static_cast<const C *>(d.lam);
    const C *la = lam + (size_t)c0 * ld1 + a.K1, *lb = la + ld1;
    const double l0 = *d.lam0;
    CV<V> x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        x[r] = CV<V>{vzero(V{}), vzero(V{})};
        if (r < 4 || r >= 12) {
            const int n = t + r * T;
            const int k1 = (r < 4) ? n : n - N1;
            const bool in_box = (r < 4) ? (n <= a.K1) : (k1 >= -a.K1);
            C p = (in_box && va) ? la[k1] : C{0, 0};
            C q = (in_box && vb) ? lb[k1] : C{0, 0};
            if (c0 == 0 && k1 == 0) p = C{(R)l0, 0};
            x[r] = pack2<R>(p, q);
        }
    }
    fft_line<1, LOG>(x, a.logn1, t, sm, static_cast<const C *>(d.tw1));
    C *gk = static_cast<C *>(d.gk);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const size_t row = (size_t)(t + r * T) * a.ldk;
        if (va) gk[row + c0] = lane0<R>(x[r]);
        if (vb) gk[row + c0 + 1] = lane1<R>(x[r]);
    }
}

// --- adjoint, pass B: one row per group -------------------------------------
// ell from the lambda row (gk), u + iv from uv; q_i = 2 ell d_i phi;
// forward real transforms of q1 and q2 (paired); writes
// aw[k2][j1] = (hat q1, -i s2 k2 hat q2) column-major.
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_adjB(AdjDesc d) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const StepArgs &a = d.a;
    const C *uv = static_cast<const C *>(d.uv);
    const C *lrow = static_cast<const C *>(d.gk);
    const C *twm = static_cast<const C *>(d.twm);
    const int M = 1 << a.logm, T = M >> 4;
    const int t = threadIdx.x;
    const int row = blockIdx.x;
    const bool valid = row < a.n1;
    V *base = reinterpret_cast<V *>(smraw);
    C *park = reinterpret_cast<C *>(base + 2 * plane_len(M));
    const C *P = twm + tw_real_offset(a.logm);
    const C *src = uv + uv_index(valid ? row : 0, 0, a.ldk);  // element kk at src + 4 kk
    const C *lsrc = lrow + (size_t)(valid ? row : 0) * a.ldk;
    CV<V> x[16];
    halfband_ifft<R, LOG>(x, a, t, P, twm,
                     [&](int kk, bool pos) {
                         C e = lsrc[kk];
                         return pos ? e : C{e.x, -e.y};
                     },
                     valid, base);
#pragma unroll
    for (int r = 0; r < 16; ++r) park[t + r * T] = C{x[r].re.x, x[r].re.y};  // ell(2m), ell(2m+1)
    halfband_ifft<R, LOG>(x, a, t, P, twm,
                     [&](int kk, bool pos) {
                         UV<R> e = ld_uv<R>(src + 4 * (size_t)kk);
                         if (pos) return C{e.u.x - e.v.y, e.u.y + e.v.x};
                         return C{e.u.x + e.v.y, e.v.x - e.u.y};
                     },
                     valid, base);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        C l = park[t + r * T];
        const R l0 = (R)2 * l.x, l1 = (R)2 * l.y;
        // lanes: q1 = 2 ell u at (2m, 2m+1), q2 = 2 ell v at (2m, 2m+1)
        C h1{l0 * x[r].re.x, l1 * x[r].re.y};
        C h2{l0 * x[r].im.x, l1 * x[r].im.y};
        x[r] = pack2<R>(h1, h2);
    }
    C *aw = static_cast<C *>(d.aw);
    const R s2 = scale2<R>(a);
    real_fwd<R, LOG>(x, a, t, P, twm, base, valid, [&](int k, CV<V> Y) {
        C q1 = lane0<R>(Y), q2 = lane1<R>(Y);
        const R f = s2 * (R)k;
        st_uv<R>(aw + 2 * ((size_t)k * a.n1 + row), q1, C{f * q2.y, -f * q2.x});  // -i f q2
    });
}

// --- adjoint, pass C: one column per group ----------------------------------
// forward column transforms of (hat q1, -i k2 hat q2), P = (-i s1 k1 Q1 + Q2)
// / (N1 N2), lambda update on the box, k2 = 0 column from its k1 > 0 half,
// dL/dgamma contribution (FP64, one atomic per block).
template <class R, int LOG> __global__ void __launch_bounds__(256, kMinBlocks<R>) k_adjC(AdjDesc d) {
    using V = typename VecOf<R>::type;
    using C = CplxT<R>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[256];  // one per thread (blockDim <= 256)
    const StepArgs &a = d.a;
    const int N1 = 1 << a.logn1, T = N1 >> 4;
    const int G = blockDim.x / T, g = threadIdx.x / T, t = threadIdx.x % T;
    const int ld1 = 2 * a.K1 + 1;
    const int k2 = blockIdx.x * G + g;
    const bool valid = k2 <= a.K2;
    V *base = reinterpret_cast<V *>(smraw) + (size_t)g * 2 * plane_len(N1);
    auto sm = make_planes(base, N1);
    const C *aw = static_cast<const C *>(d.aw) + 2 * (size_t)(valid ? k2 : 0) * N1;
    CV<V> x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int n = t + r * T;
        UV<R> e = valid ? ld_uv<R>(aw + 2 * n) : UV<R>{C{0, 0}, C{0, 0}};
        x[r] = pack2<R>(e.u, e.v);
    }
    __shared__ CoefR<R> cfs;
    Coef cf{};  // thread 0 only
    if (threadIdx.x == 0) {
        cf = step_coef(a, *d.t, false);
        cfs = coef_r<R>(cf, a);
    }
    fft_line<-1, LOG>(x, a.logn1, t, sm, static_cast<const C *>(d.tw1));
    __syncthreads();  // cfs
    const bool lin = !(a.flags & kNonlinearOnly), nl = !(a.flags & kLinearOnly);
    const R ra = cfs.a, rb = cfs.b, rcs = cfs.cs, rdt = cfs.dt;
    const R s1 = scale1<R>(a), s2 = scale2<R>(a);
    const C *lam = static_cast<const C *>(d.lam) + (size_t)k2 * ld1 + a.K1;
    C *lout = static_cast<C *>(d.lam_out) + (size_t)k2 * ld1 + a.K1;
    const C *phi = static_cast<const C *>(d.state) + (size_t)k2 * ld1 + a.K1;
    double dg = 0.0;  // sum of 2 kappa (lambda . Phi); times dt / (2 r0) at the end
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        if (r < 4 || r >= 12) {
            const int n = t + r * T;
            const int k1 = (r < 4) ? n : n - N1;
            const bool in_box = valid && ((r < 4) ? (n <= a.K1) : (k1 >= -a.K1));
            // k2 = 0, k1 < 0: conjugate mirror of +k1, written (and counted in
            // the gamma gradient, with the same value) by the owner of +k1
            if (!in_box || (k1 == 0 && k2 == 0) || (k2 == 0 && k1 < 0)) continue;
            const R f1 = s1 * (R)k1;
            C Q1 = lane0<R>(x[r]), Q2 = lane1<R>(x[r]);
            C Pk{f1 * Q1.y + Q2.x, -f1 * Q1.x + Q2.y};  // -i f1 Q1 + Q2
            C l = lam[k1];
            const R kap = kappa_norm<R>(f1, s2 * (R)k2);
            if (lin) {
                C ph = phi[k1];
                // weight 2: k2 > 0 stands for +-k; k2 = 0 here counts +k1 and -k1
                dg += 2.0 * (double)kap * ((double)l.x * ph.x + (double)l.y * ph.y);
            }
            const R om = lin ? kap * (rb - kap * ra) : (R)0;
            const R cn = nl ? rcs : (R)0;
            C nw{l.x + rdt * (om * l.x + cn * Pk.x), l.y + rdt * (om * l.y + cn * Pk.y)};
            lout[k1] = nw;
            if (k2 == 0) lout[-k1] = C{nw.x, -nw.y};
        }
    }
    red[threadIdx.x] = dg;  // any block size
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) s += red[i];
        if (s != 0.0) atomicAdd(d.dgamma, s * (a.dt / (2.0 * cf.tn)));
    }
}

}  // namespace flame
