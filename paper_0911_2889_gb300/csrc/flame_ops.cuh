// flame_ops.cuh -- launch geometry and launchers of the kernels.  FP64 is
// instantiated whole by flame_f64.cu; the FP32 launchers are split over
// flame_f32_*.cu so that their kernels compile in parallel.
#pragma once

#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "flame_adjoint.cuh"

namespace flame {

constexpr size_t kSmemBudget = 200 * 1024;  // what one CTA may take here
constexpr int kThreadsTarget = 256;
constexpr int kMaxThreads = 256;  // launch bound of every line-FFT kernel

template <class R> static size_t group_smem(int logn) {
    return 2 * (size_t)plane_len(1 << logn) * sizeof(typename VecOf<R>::type);
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 148;
    }
    return n;
}

// G line groups of T = 2^logn / 16 threads per CTA: up to 256 threads and
// the shared-memory budget, but no more groups than keep at least two CTAs
// per SM busy (small grids spread over the whole GPU).  hint > 0 fixes G.
template <class R> static Geom make_geom(int logn, int nlines, int hint, size_t extra = 0) {
    const int T = (1 << logn) >> 4;
    int G = hint > 0 ? hint : (T >= kThreadsTarget ? 1 : kThreadsTarget / T);
    const size_t per = group_smem<R>(logn) + extra;
    while (G > 1 && (G * per > kSmemBudget || G * T > kMaxThreads)) G >>= 1;
    if (hint <= 0)
        while (G > 1 && (nlines + G - 1) / G < 2 * sm_count()) G >>= 1;

    Geom g;
    g.threads = G * T;
    g.blocks = (nlines + G - 1) / G;
    g.smem = G * per;
    return g;
}

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum (less its static shared memory), once per kernel and device,
// before its first launch.
static cudaError_t opt_in(const void *kernel) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({kernel, dev})) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.insert({kernel, dev});
    return e;
}

// CTAs of one kernel resident at once on the current device: a tile that
// starts now is followed, one wave later, by tile + resident_ctas.
static int resident_ctas(const void *kernel, const Geom &g) {
    if (opt_in(kernel) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int nsm = sm_count();
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, g.threads, g.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per * nsm;
}

// Line lengths with compile-time step kernels: FP32 2^8 .. 2^12 (the
// benchmark, ensemble and adjoint grids); everything else (and FP64) runs the
// runtime-length kernels (LOG = 0).
template <class R, class F> static void for_each_log(F &&f) {
    f(std::integral_constant<int, 0>{});
    if constexpr (sizeof(R) == 4) static_for<8, 13>(f);
}
template <class R, class F> static void with_log(int logn, F &&f) {
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        static_for<8, 13>([&](auto lc) {
            if (!done && logn == decltype(lc)::value) {
                f(lc);
                done = true;
            }
        });
    }
    if (!done) f(std::integral_constant<int, 0>{});
}

// Launch with a thread-block cluster of `cl` CTAs along x (grid.x must be a
// multiple of cl; cl <= 1: none) and, when w.bytes > 0, an L2 persisting
// access window over [w.base, w.base + w.bytes) (a fraction w.hit of its
// accesses persisting, the rest streaming).
// With pdl, the launch is a programmatic dependent launch: its CTAs may be
// scheduled while the previous kernel on the stream drains, and wait in
// hardware (griddepcontrol.wait, the first statement of every step pass's
// body) until that kernel has completed and its memory is visible.  Only
// the step passes, whose bodies begin with that wait, are launched so.
// Opt-in (FLAME_PDL=1): at 4096 x 8192 the graph-captured steps measured
// 0.2026 ms per step with it against 0.1967 ms without.
static bool pdl_on() {
    const char *v = getenv("FLAME_PDL");
    return v && strcmp(v, "1") == 0;
}
template <class... KArgs, class... Args>
static cudaError_t launch_x(const L2Window &w, bool pdl, void (*kernel)(KArgs...), dim3 grid, int threads,
                            size_t smem, cudaStream_t s, int cl, Args... args) {
    const cudaError_t oe = opt_in((const void *)kernel);
    if (oe != cudaSuccess) return oe;
    if (cl <= 1 && w.bytes == 0 && !pdl) {
        kernel<<<grid, threads, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[3];
    unsigned n = 0;
    if (pdl) {
        attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    if (cl > 1) {
        attr[n].id = cudaLaunchAttributeClusterDimension;
        attr[n].val.clusterDim.x = cl;
        attr[n].val.clusterDim.y = 1;
        attr[n].val.clusterDim.z = 1;
        ++n;
    }
    if (w.bytes > 0) {
        attr[n].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[n].val.accessPolicyWindow.base_ptr = const_cast<void *>(w.base);
        attr[n].val.accessPolicyWindow.num_bytes = w.bytes;
        attr[n].val.accessPolicyWindow.hitRatio = w.hit;
        attr[n].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[n].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <class... KArgs, class... Args>
static cudaError_t launch_w(const L2Window &w, void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem,
                            cudaStream_t s, int cl, Args... args) {
    return launch_x(w, false, kernel, grid, threads, smem, s, cl, args...);
}
// a step pass of one flame: L2 window and programmatic dependent launch
template <class... KArgs, class... Args>
static cudaError_t launch_s(const L2Window &w, void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem,
                            cudaStream_t s, int cl, Args... args) {
    return launch_x(w, pdl_on(), kernel, grid, threads, smem, s, cl, args...);
}
template <class... KArgs, class... Args>
static cudaError_t launch_cl(void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t s, int cl,
                             Args... args) {
    return launch_w(L2Window{nullptr, 0, 0.f}, kernel, grid, threads, smem, s, cl, args...);
}
template <class R, int L> static constexpr int cluster_of() {
    return (sizeof(R) == 4 && L > 0) ? Shape<L>::CL : 1;
}
static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Whether pass C needs its general epilogue (a two-stage scheme's stage,
// forcing or the per-step record) or the plain Euler one.
static bool general_epilogue(const FlameDesc &d) {
    return d.stage != kStageEuler || d.forcing != nullptr || d.forcing0 != 0.0 || d.rec != nullptr;
}

template <class R> Geom Ops<R>::geom_cols(int logn, int nlines, int hint) { return make_geom<R>(logn, nlines, hint); }
template <class R> Geom Ops<R>::geom_rows(int logm, int nlines, int hint) { return make_geom<R>(logm, nlines, hint); }

template <class R> cudaError_t Ops<R>::init_twiddles(C *tab, int logN, cudaStream_t s) {
    // radix-16 table, then the radix-8 and radix-4 tables (tw_alloc_len entries in all)
    const int len16 = tw_table_len(logN, 4), len8 = tw_table_len(logN, 3), len4 = tw_table_len(logN, 2);
    cudaError_t e = launch_cl(k_twiddles<R>, dim3((len16 + 255) / 256), 256, 0, s, 1, tab, logN, 4);
    if (e == cudaSuccess) e = launch_cl(k_twiddles<R>, dim3((len8 + 255) / 256), 256, 0, s, 1, tab + len16, logN, 3);
    if (e == cudaSuccess)
        e = launch_cl(k_twiddles<R>, dim3((len4 + 255) / 256), 256, 0, s, 1, tab + len16 + len8, logN, 2);
    return e;
}

template <class R>
cudaError_t Ops<R>::box_from_spec(const C *spec, C *state, double *mean, int n1, int n2, int K1, int K2,
                                  cudaStream_t s, int *status) {
    const long total = (long)(2 * K1 + 1) * (K2 + 1);
    const int blocks = (int)std::min<long>((total + 255) / 256, 8L * sm_count());
    return launch_cl(k_box_from_spec<R>, dim3(blocks), 256, 0, s, 1, spec, state, mean, n1, n2, K1, K2, status);
}

// The standalone 2-D FFT passes take the compile-time line length where the
// step kernels do (FP32, 2^8 .. 2^12), the runtime-length engine otherwise.
template <class R>
cudaError_t Ops<R>::rows_r2c(const R *in, C *out, int n1, int logm, const C *tw, cudaStream_t s, int *status) {
    Geom g = geom_rows(logm, n1 / 2, 0);
    cudaError_t err = cudaSuccess;
    with_log<R>(logm, [&](auto lc) {
        err = launch_cl(k_rows_r2c<R, decltype(lc)::value>, dim3(g.blocks), g.threads, g.smem, s, 1, in, out, n1, logm,
                        tw, status);
    });
    return err;
}

template <class R>
cudaError_t Ops<R>::rows_c2r(const C *in, R *out, int n1, int logm, const C *tw, cudaStream_t s, int *status) {
    Geom g = geom_rows(logm, n1 / 2, 0);
    cudaError_t err = cudaSuccess;
    with_log<R>(logm, [&](auto lc) {
        err = launch_cl(k_rows_c2r<R, decltype(lc)::value>, dim3(g.blocks), g.threads, g.smem, s, 1, in, out, n1, logm,
                        tw, status);
    });
    return err;
}

template <class R>
cudaError_t Ops<R>::cols(const C *in, C *out, int logn, int ncols, int ld, int dir, const C *tw, cudaStream_t s,
                         int *status) {
    Geom g = geom_cols(logn, (ncols + 1) / 2, 0);
    cudaError_t err = cudaSuccess;
    with_log<R>(logn, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        // FP32 columns of 2^10 .. 2^12 points: 512-thread CTAs of 512/T line
        // groups (one CTA per SM), where the grid still has two CTAs per SM
        if constexpr (sizeof(R) == 4 && L >= 10 && L <= 12) {
            constexpr int G = 512 / ((1 << L) >> 4);
            const int npairs = (ncols + 1) / 2;
            if (npairs >= 2 * G * sm_count()) {
                const dim3 grid((npairs + G - 1) / G);
                const size_t smem = G * group_smem<R>(L);
                if (dir < 0) err = launch_cl(k_cols<R, -1, L, 512>, grid, 512, smem, s, 1, in, out, logn, ncols, ld, tw, status);
                else err = launch_cl(k_cols<R, 1, L, 512>, grid, 512, smem, s, 1, in, out, logn, ncols, ld, tw, status);
                return;
            }
        }
        if (dir < 0)
            err = launch_cl(k_cols<R, -1, L>, dim3(g.blocks), g.threads, g.smem, s, 1, in, out, logn, ncols, ld, tw,
                            status);
        else
            err = launch_cl(k_cols<R, 1, L>, dim3(g.blocks), g.threads, g.smem, s, 1, in, out, logn, ncols, ld, tw,
                            status);
    });
    return err;
}

// pass A with 8 points per thread (compile-time length 2^L): fixed shape
template <class R, int L> static Geom geom_passA8(int ncols) {
    Geom g;
    if constexpr (L > 0) {
        g.threads = ShapeE<L, 8>::THREADS;
        g.blocks = (ncols + ShapeE<L, 8>::G - 1) / ShapeE<L, 8>::G;
        g.smem = (size_t)ShapeE<L, 8>::G * 2 * plane_len_e<8>(1 << L) * sizeof(typename VecOf<R>::type);
    } else {
        g.threads = g.blocks = 0;
        g.smem = 0;
    }
    return g;
}

// FP64 lines of 2^4 .. 2^7 points: 8 points per thread, one line pair per
// CTA (the runtime kernels give such lines 2^LOG/16 threads, a quarter warp
// at 128 points, and are bound by the latency of their FP64 chains)
template <class R> static bool small_fp64(int logn) { return sizeof(R) == 8 && logn >= 4 && logn <= 7; }
// Points per thread of the FP64 short-line kernels: 4 (a warp per 128-point
// line pair), or 8 with FLAME_FP64_POINTS=8 (read at every launch, so tests
// can run both).  Measured on the 128 x 256 FP64 trajectory: 46.1 us per
// step with 4, 78.4 us with 8: the lines' FP64 chains are latency-bound,
// and a full warp per line pair halves each thread's chain.
static int fp64_points() {
    const char *v = getenv("FLAME_FP64_POINTS");
    return (v && strcmp(v, "8") == 0) ? 8 : 4;
}
template <class R, int E> static Geom geom_small_fp64(int logn, int nlines, size_t extra) {
    Geom g;
    g.threads = (1 << logn) / E;
    g.blocks = nlines;
    g.smem = 2 * (size_t)plane_len_e<E>(1 << logn) * sizeof(typename VecOf<R>::type) + extra;
    return g;
}
// CTA of the one-line kernels (k_passA1/B1/C1): `groups` line
// groups of 2^logn / E threads, each with its own exchange planes, and
// `extra` bytes more (pass B's parked g of two rows); one CTA per unit
template <class R, int E> static Geom geom_short1(int logn, int units, int groups, size_t extra) {
    Geom g;
    g.threads = groups * ((1 << logn) / E);
    g.blocks = units;
    g.smem = (size_t)groups * 2 * plane_len_e<E>(1 << logn) * sizeof(R) + extra;
    return g;
}
// FP32 lines with one-line kernels (E = 16): 2^8 .. 2^11 points
template <class R> static bool one_line_fp32(int logn) { return sizeof(R) == 4 && logn >= 8 && logn <= 11; }
// calls f(integral_constant<E>) with the chosen points per thread
template <class F> static void with_fp64_points(F &&f) {
    if (fp64_points() == 4) f(std::integral_constant<int, 4>{});
    else f(std::integral_constant<int, 8>{});
}

template <class R>
cudaError_t Ops<R>::passA(const FlameDesc &d, cudaStream_t s, int variant, const CUtensorMap *uv_map) {
    if constexpr (sizeof(R) == 8) if (small_fp64<R>(d.a.logn1)) {
        cudaError_t err = cudaErrorInvalidValue;
        with_fp64_points([&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const Geom g = geom_short1<R, E>(d.a.logn1, d.a.K2 + 1, 2, 0);
            static_for<4, 8>([&](auto lc) {
                constexpr int L = decltype(lc)::value;
                if (d.a.logn1 == L)
                    err = launch_s(d.l2_state, k_passA1<R, L, E>, dim3(d.tiles ? d.tiles : g.blocks), g.threads, g.smem, s, 1, d, 0);
            });
        });
        return err;
    }
    if (variant == kVariantOneLine && one_line_fp32<R>(d.a.logn1)) {
        cudaError_t err = cudaErrorInvalidValue;
        const Geom g = geom_short1<R, 16>(d.a.logn1, d.a.K2 + 1, 2, 0);
        static_for<8, 12>([&](auto lc) {
            constexpr int L = decltype(lc)::value;
            if (d.a.logn1 == L)
                err = launch_s(d.l2_state, k_passA1<R, L, 16>, dim3(d.tiles ? d.tiles : g.blocks), g.threads, g.smem, s,
                               1, d, 0);
        });
        return err;
    }
    Geom g = geom_cols(d.a.logn1, d.a.K2 + 1, 0);
    cudaError_t err = cudaSuccess;
    with_log<R>(d.a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        constexpr int cl = cluster_of<R, L>();
        if (sizeof(R) == 4 && L > 0 && variant == kVariantTma && uv_map) {  // tensor-store write-out
            const int pf = resident_ctas((const void *)k_passAt<R, L>, g);
            err = launch_s(d.l2_state, k_passAt<R, L>, dim3(d.tiles ? d.tiles : g.blocks), g.threads, g.smem, s, 1, d, pf, *uv_map);
        } else if (cl > 1 && (variant == kVariantDirect || variant == kVariantTma)) {  // direct stores
            Geom gd = g;
            const int pf = resident_ctas((const void *)k_passAd<R, L>, gd);
            err = launch_s(d.l2_state, k_passAd<R, L>, dim3(d.tiles ? d.tiles : gd.blocks), gd.threads, gd.smem, s, 1, d, pf);
        } else if (sizeof(R) == 4 && L > 0 && variant == kVariantRadix8A) {
            const Geom g8 = geom_passA8<R, L>(d.a.K2 + 1);
            constexpr int cl8 = ShapeE<L, 8>::CL;
            const int pf = resident_ctas((const void *)k_passA8<R, L>, g8);
            err = launch_s(d.l2_state, k_passA8<R, L>, dim3(d.tiles ? d.tiles : round_up(g8.blocks, cl8)), g8.threads, g8.smem, s, cl8, d, pf);
        } else {
            // the compile-time kernels assume Shape<L>::G groups per CTA
            Geom gl = cl > 1 ? geom_cols(d.a.logn1, d.a.K2 + 1, Shape<L>::G) : g;
            const int pf = resident_ctas((const void *)k_passA<R, L>, gl);
            err = launch_s(d.l2_state, k_passA<R, L>, dim3(d.tiles ? d.tiles : round_up(gl.blocks, cl)), gl.threads, gl.smem, s, cl, d, pf);
        }
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}
// pass B parks one row of |z|^2 (N2/2 complex) per group in shared memory
template <class R> static Geom geom_passB(int logm, int nlines, int hint = 0) {
    return make_geom<R>(logm, nlines, hint, (size_t)(1 << logm) * sizeof(typename VecOf<R>::c));
}

// Line groups per CTA of a grouped (ensemble) launch over n flames of
// nlines lines each.  Per flame, make_geom shrinks G until one flame's grid
// spans two CTAs per SM; with FLAME_BATCH_GEOM=1 G is chosen for the class's
// n * nlines lines instead (the flames fill the GPU together).  Returns the
// hint for make_geom (0: per-flame choice).
template <class R> static int batch_groups(int logn, int nlines, int n, size_t extra = 0) {
    const char *v = getenv("FLAME_BATCH_GEOM");
    if (!v || strcmp(v, "1") != 0) return 0;
    const Geom all = make_geom<R>(logn, nlines * n, 0, extra);
    return all.threads / ((1 << logn) >> 4);
}

// pass B with 8 points per thread: 512-thread CTAs, padding every 8 slots
template <class R> static Geom geom_passB8(int logm, int nlines) {
    const int T = (1 << logm) >> 3;
    const int G = T >= 512 ? 1 : 512 / T;
    Geom g;
    g.threads = G * T;
    g.blocks = (nlines + G - 1) / G;
    g.smem = (size_t)G * (2 * (size_t)plane_len_e<8>(1 << logm) * sizeof(typename VecOf<R>::type) +
                          (size_t)(1 << logm) * sizeof(typename VecOf<R>::c));
    return g;
}

template <class R>
cudaError_t Ops<R>::passB(const FlameDesc &d, cudaStream_t s, int variant, const CUtensorMap *gk_map) {
    if constexpr (sizeof(R) == 8) if (small_fp64<R>(d.a.logm)) {  // + M entries of the parked |z|^2 per row pair
        cudaError_t err = cudaErrorInvalidValue;
        with_fp64_points([&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const Geom g = geom_short1<R, E>(d.a.logm, d.a.n1 / 2, 4, (size_t)4 * (1 << d.a.logm) * sizeof(R));
            static_for<4, 8>([&](auto lc) {
                constexpr int L = decltype(lc)::value;
                if (d.a.logm == L) err = launch_s(L2Window{nullptr, 0, 0.f}, k_passB1<R, L, E>, dim3(g.blocks), g.threads, g.smem, s, 1, d, 0);
            });
        });
        return err;
    }
    if (variant == kVariantOneLineB && one_line_fp32<R>(d.a.logm)) {
        cudaError_t err = cudaErrorInvalidValue;
        const Geom g = geom_short1<R, 16>(d.a.logm, d.a.n1 / 2, 4, (size_t)4 * (1 << d.a.logm) * sizeof(R));
        static_for<8, 12>([&](auto lc) {
            constexpr int L = decltype(lc)::value;
            if (d.a.logm == L)
                err = launch_s(L2Window{nullptr, 0, 0.f}, k_passB1<R, L, 16>, dim3(g.blocks), g.threads, g.smem, s, 1, d, 0);
        });
        return err;
    }
    Geom g = geom_passB<R>(d.a.logm, d.a.n1 / 2);
    cudaError_t err = cudaSuccess;
    with_log<R>(d.a.logm, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if constexpr (sizeof(R) == 4 && L == 12) if (variant == kVariantWarpB) {
            Geom gb = g;
            gb.smem += kTwSmemBytes;
            if (gk_map) {
                const int pf = resident_ctas((const void *)k_passBw<R>, gb);
                err = launch_s(L2Window{nullptr, 0, 0.f}, k_passBw<R>, dim3(gb.blocks), gb.threads, gb.smem, s, 1, d, pf,
                               *gk_map);
            } else {
                const int pf = resident_ctas((const void *)k_passBwd<R>, gb);
                err = launch_s(L2Window{nullptr, 0, 0.f}, k_passBwd<R>, dim3(gb.blocks), gb.threads, gb.smem, s, 1, d, pf);
            }
            return;
        }
        if (sizeof(R) == 4 && L > 0 && (variant == kVariantTmaB || variant == kVariantWarpB) && gk_map) {  // tensor-store write-out
            Geom gb = g;
            if (kSharedTw<R, L, 16>) gb.smem += kTwSmemBytes;
            const int pf = resident_ctas((const void *)k_passBt<R, L>, gb);
            err = launch_s(L2Window{nullptr, 0, 0.f}, k_passBt<R, L>, dim3(gb.blocks), gb.threads, gb.smem, s, 1, d, pf, *gk_map);
        } else if (sizeof(R) == 4 && L > 0 && variant == kVariantRadix8) {
            const Geom g8 = geom_passB8<R>(L, d.a.n1 / 2);
            const int pf = resident_ctas((const void *)k_passB8<R, L>, g8);
            err = launch_s(L2Window{nullptr, 0, 0.f}, k_passB8<R, L>, dim3(g8.blocks), g8.threads, g8.smem, s, 1, d, pf);
        } else {
            Geom gb = g;
            if (kSharedTw<R, L, 16>) gb.smem += kTwSmemBytes;
            const int pf = resident_ctas((const void *)k_passB<R, L>, gb);
            err = launch_s(L2Window{nullptr, 0, 0.f}, k_passB<R, L>, dim3(gb.blocks), gb.threads, gb.smem, s, 1, d, pf);
        }
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}
template <class R> cudaError_t Ops<R>::passB_area(const FlameDesc &d, cudaStream_t s) {
    using Vt = typename VecOf<R>::type;
    const int M = 1 << d.a.logm;
    cudaError_t err = cudaErrorNotSupported;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return cudaErrorNotSupported;
    }
    const size_t area_extra = 3 * (size_t)M * sizeof(Vt);
    if constexpr (sizeof(R) == 8) if (small_fp64<R>(d.a.logm)) {
        with_fp64_points([&](auto ec) {
            constexpr int E = decltype(ec)::value;
            Geom g = geom_small_fp64<R, E>(d.a.logm, d.a.n1 / 2, (size_t)M * sizeof(typename VecOf<R>::c) + area_extra);
            if (g.smem + 4096 > (size_t)optin) return;
            static_for<4, 8>([&](auto lc) {
                constexpr int L = decltype(lc)::value;
                if (d.a.logm == L)
                    err = launch_cl(k_passB_area<R, L, E, 128>, dim3(g.blocks), g.threads, g.smem, s, 1, d);
            });
        });
        return err;
    }
    // FP32 compile-time rows: 8 points per thread, 512-thread CTAs (one per
    // SM: the area buffers take most of the shared memory, and 16 warps hide
    // more latency than the 8 of 16 points per thread)
    if constexpr (sizeof(R) == 4) if (d.a.logm >= 8 && d.a.logm <= 12) {
        Geom g = geom_passB8<R>(d.a.logm, d.a.n1 / 2);
        const int G = g.threads / (M / 8);
        g.smem += (size_t)G * area_extra;
        if (g.smem + 4096 > (size_t)optin) return cudaErrorNotSupported;
        with_log<R>(d.a.logm, [&](auto lc) {
            constexpr int L = decltype(lc)::value;
            if constexpr (L > 0) err = launch_cl(k_passB_area<R, L, 8, 512>, dim3(g.blocks), g.threads, g.smem, s, 1, d);
        });
        if (err != cudaSuccess) return err;
        return cudaGetLastError();
    }
    Geom g = make_geom<R>(d.a.logm, d.a.n1 / 2, 0, (size_t)M * sizeof(typename VecOf<R>::c) + area_extra);
    with_log<R>(d.a.logm, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        Geom ga = g;
        if (kSharedTw<R, L, 16>) ga.smem += kTwSmemBytes;
        if (ga.smem + 4096 > (size_t)optin) {
            err = cudaErrorNotSupported;
            return;
        }
        err = launch_cl(k_passB_area<R, L, 16, 256>, dim3(ga.blocks), ga.threads, ga.smem, s, 1, d);
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

template <class R> cudaError_t Ops<R>::passC(const FlameDesc &d, cudaStream_t s) {
    if constexpr (sizeof(R) == 8) if (small_fp64<R>(d.a.logn1)) {
        cudaError_t err = cudaErrorInvalidValue;
        with_fp64_points([&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const Geom g = geom_short1<R, E>(d.a.logn1, (d.a.K2 + 2) / 2, 2, 0);
            static_for<4, 8>([&](auto lc) {
                constexpr int L = decltype(lc)::value;
                if (d.a.logn1 == L)
                    err = launch_s(d.l2_state, k_passC1<R, L, E>, dim3(d.tiles ? d.tiles : g.blocks), g.threads, g.smem,
                                   s, 1, d, 0);
            });
        });
        return err;
    }
    if (d.onec && one_line_fp32<R>(d.a.logn1)) {
        cudaError_t err = cudaErrorInvalidValue;
        const Geom g = geom_short1<R, 16>(d.a.logn1, (d.a.K2 + 2) / 2, 2, 0);
        static_for<8, 12>([&](auto lc) {
            constexpr int L = decltype(lc)::value;
            if (d.a.logn1 == L)
                err = launch_s(d.l2_state, k_passC1<R, L, 16>, dim3(d.tiles ? d.tiles : g.blocks), g.threads, g.smem, s,
                               1, d, 0);
        });
        return err;
    }
    Geom g = geom_cols(d.a.logn1, (d.a.K2 + 2) / 2, 0);
    cudaError_t err = cudaSuccess;
    const bool gen = general_epilogue(d);
    with_log<R>(d.a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (gen) {
            const int pf = resident_ctas((const void *)k_passC<R, L, true>, g);
            err = launch_s(d.l2_state, k_passC<R, L, true>, dim3(d.tiles ? d.tiles : g.blocks), g.threads, g.smem, s, 1,
                           d, pf);
        } else {
            const int pf = resident_ctas((const void *)k_passC<R, L, false>, g);
            err = launch_s(d.l2_state, k_passC<R, L, false>, dim3(d.tiles ? d.tiles : g.blocks), g.threads, g.smem, s,
                           1, d, pf);
        }
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}
template <class R>
cudaError_t Ops<R>::passCA(const FlameDesc &d, cudaStream_t s, const CUtensorMap *uv_map) {
    if (sizeof(R) != 4 || !uv_map || d.a.logn1 < 8 || d.a.logn1 > 12) return cudaErrorNotSupported;
    Geom g = geom_cols(d.a.logn1, (d.a.K2 + 2) / 2, 0);
    cudaError_t err = cudaErrorNotSupported;
    with_log<R>(d.a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if constexpr (sizeof(R) == 4 && L > 0) {
            if (general_epilogue(d)) {
                const int pf = resident_ctas((const void *)k_passCA<R, L, true>, g);
                err = launch_s(d.l2_state, k_passCA<R, L, true>, dim3(g.blocks), g.threads, g.smem, s, 1, d, pf,
                               *uv_map);
            } else {
                const int pf = resident_ctas((const void *)k_passCA<R, L, false>, g);
                err = launch_s(d.l2_state, k_passCA<R, L, false>, dim3(g.blocks), g.threads, g.smem, s, 1, d, pf,
                               *uv_map);
            }
        }
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}
template <class R>
cudaError_t Ops<R>::passA_batch(const FlameDesc *ds, int n, const StepArgs &a, cudaStream_t s, int variant,
                                const CUtensorMap *maps) {
    if constexpr (sizeof(R) == 8) if (small_fp64<R>(a.logn1)) {  // the kernels of passA, so that a flame's ensemble step equals its own
        cudaError_t err = cudaErrorInvalidValue;
        with_fp64_points([&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const Geom g = geom_short1<R, E>(a.logn1, a.K2 + 1, 2, 0);
            static_for<4, 8>([&](auto lc) {
                constexpr int L = decltype(lc)::value;
                if (a.logn1 == L) err = launch_cl(k_passA1_n<R, L, E>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
            });
        });
        return err;
    }
    if (variant == kVariantOneLine && one_line_fp32<R>(a.logn1)) {
        cudaError_t err = cudaErrorInvalidValue;
        const Geom g = geom_short1<R, 16>(a.logn1, a.K2 + 1, 2, 0);
        static_for<8, 12>([&](auto lc) {
            constexpr int L = decltype(lc)::value;
            if (a.logn1 == L) err = launch_cl(k_passA1_n<R, L, 16>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
        });
        return err;
    }
    Geom g = geom_cols(a.logn1, a.K2 + 1, batch_groups<R>(a.logn1, a.K2 + 1, n));
    cudaError_t err = cudaSuccess;
    with_log<R>(a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        constexpr int cl = cluster_of<R, L>();
        if (sizeof(R) == 4 && L > 0 && variant == kVariantTma && maps) {
            err = launch_cl(k_passAt_n<R, L>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0, maps);
        } else if (cl > 1 && (variant == kVariantDirect || variant == kVariantTma)) {
            err = launch_cl(k_passAd_n<R, L>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
        } else if (sizeof(R) == 4 && L > 0 && variant == kVariantRadix8A) {
            const Geom g8 = geom_passA8<R, L>(a.K2 + 1);
            constexpr int cl8 = ShapeE<L, 8>::CL;
            err = launch_cl(k_passA8_n<R, L>, dim3(round_up(g8.blocks, cl8), n), g8.threads, g8.smem, s, cl8, ds, 0);
        } else {
            Geom gl = cl > 1 ? geom_cols(a.logn1, a.K2 + 1, Shape<L>::G) : g;
            err = launch_cl(k_passA_n<R, L>, dim3(round_up(gl.blocks, cl), n), gl.threads, gl.smem, s, cl, ds, 0);
        }
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}
template <class R>
cudaError_t Ops<R>::passB_batch(const FlameDesc *ds, int n, const StepArgs &a, cudaStream_t s, int variant,
                                const CUtensorMap *maps) {
    if constexpr (sizeof(R) == 8) if (small_fp64<R>(a.logm)) {
        cudaError_t err = cudaErrorInvalidValue;
        with_fp64_points([&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const Geom g = geom_short1<R, E>(a.logm, a.n1 / 2, 4, (size_t)4 * (1 << a.logm) * sizeof(R));
            static_for<4, 8>([&](auto lc) {
                constexpr int L = decltype(lc)::value;
                if (a.logm == L) err = launch_cl(k_passB1_n<R, L, E>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
            });
        });
        return err;
    }
    if (variant == kVariantOneLineB && one_line_fp32<R>(a.logm)) {
        cudaError_t err = cudaErrorInvalidValue;
        const Geom g = geom_short1<R, 16>(a.logm, a.n1 / 2, 4, (size_t)4 * (1 << a.logm) * sizeof(R));
        static_for<8, 12>([&](auto lc) {
            constexpr int L = decltype(lc)::value;
            if (a.logm == L) err = launch_cl(k_passB1_n<R, L, 16>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
        });
        return err;
    }
    Geom g = geom_passB<R>(a.logm, a.n1 / 2,
                           batch_groups<R>(a.logm, a.n1 / 2, n, (size_t)(1 << a.logm) * sizeof(typename VecOf<R>::c)));
    cudaError_t err = cudaSuccess;
    with_log<R>(a.logm, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if constexpr (sizeof(R) == 4 && L == 12) if (variant == kVariantWarpB) {
            if (maps) err = launch_cl(k_passBw_n<R>, dim3(g.blocks, n), g.threads, g.smem + kTwSmemBytes, s, 1, ds, 0, maps);
            else err = launch_cl(k_passBwd_n<R>, dim3(g.blocks, n), g.threads, g.smem + kTwSmemBytes, s, 1, ds, 0);
            return;
        }
        if (sizeof(R) == 4 && L > 0 && (variant == kVariantTmaB || variant == kVariantWarpB) && maps) {
            const size_t sm = g.smem + (kSharedTw<R, L, 16> ? kTwSmemBytes : 0);
            err = launch_cl(k_passBt_n<R, L>, dim3(g.blocks, n), g.threads, sm, s, 1, ds, 0, maps);
        } else if (sizeof(R) == 4 && L > 0 && variant == kVariantRadix8) {
            const Geom g8 = geom_passB8<R>(L, a.n1 / 2);
            err = launch_cl(k_passB8_n<R, L>, dim3(g8.blocks, n), g8.threads, g8.smem, s, 1, ds, 0);
        } else {
            const size_t sm = g.smem + (kSharedTw<R, L, 16> ? kTwSmemBytes : 0);
            err = launch_cl(k_passB_n<R, L>, dim3(g.blocks, n), g.threads, sm, s, 1, ds, 0);
        }
    });
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}
template <class R>
cudaError_t Ops<R>::passC_batch(const FlameDesc *ds, int n, const StepArgs &a, cudaStream_t s, bool one_line) {
    if (one_line && one_line_fp32<R>(a.logn1)) {
        cudaError_t err = cudaErrorInvalidValue;
        const Geom g = geom_short1<R, 16>(a.logn1, (a.K2 + 2) / 2, 2, 0);
        static_for<8, 12>([&](auto lc) {
            constexpr int L = decltype(lc)::value;
            if (a.logn1 == L) err = launch_cl(k_passC1_n<R, L, 16>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
        });
        return err;
    }
    if constexpr (sizeof(R) == 8) if (small_fp64<R>(a.logn1)) {
        cudaError_t err = cudaErrorInvalidValue;
        with_fp64_points([&](auto ec) {
            constexpr int E = decltype(ec)::value;
            const Geom g = geom_short1<R, E>(a.logn1, (a.K2 + 2) / 2, 2, 0);
            static_for<4, 8>([&](auto lc) {
                constexpr int L = decltype(lc)::value;
                if (a.logn1 == L) err = launch_cl(k_passC1_n<R, L, E>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
            });
        });
        return err;
    }
    Geom g = geom_cols(a.logn1, (a.K2 + 2) / 2, batch_groups<R>(a.logn1, (a.K2 + 2) / 2, n));
    cudaError_t e = cudaSuccess;
    with_log<R>(a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        e = launch_cl(k_passC_n<R, L>, dim3(g.blocks, n), g.threads, g.smem, s, 1, ds, 0);
    });
    return e;
}

// one row per CTA (N2/32 threads): exchange buffer + one parked row
template <class R> static Geom geom_row1(int logm, int nrows) {
    Geom g;
    g.threads = (1 << logm) >> 4;
    g.blocks = nrows;
    g.smem = group_smem<R>(logm) + (size_t)(1 << logm) * sizeof(typename VecOf<R>::c);
    return g;
}

// The area and adjoint kernels take the column length (log2 N1) or the
// half row length (log2 N2/2) as their compile-time LOG (0: any length).
template <class R> cudaError_t Ops<R>::area(const AdjDesc &d, cudaStream_t s) {
    const StepArgs &a = d.a;
    Geom ga = geom_cols(a.logn1, a.K2 + 1, 0);
    Geom gb = geom_row1<R>(a.logm, a.n1);
    cudaError_t e = cudaSuccess;
    with_log<R>(a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        e = launch_cl(k_areaA<R, L>, dim3(ga.blocks), ga.threads, ga.smem, s, 1, d);
    });
    with_log<R>(a.logm, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (e == cudaSuccess) e = launch_cl(k_areaB<R, L>, dim3(gb.blocks), gb.threads, gb.smem, s, 1, d);
    });
    with_log<R>(a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (e == cudaSuccess) e = launch_cl(k_areaC<R, L>, dim3(ga.blocks), ga.threads, ga.smem, s, 1, d);
    });
    return e;
}

template <class R> cudaError_t Ops<R>::adj_step(const AdjDesc &d, cudaStream_t s) {
    const StepArgs &a = d.a;
    FlameDesc f;
    memset(&f, 0, sizeof f);
    f.a = a;
    f.state = const_cast<void *>(d.state);
    f.uv = d.uv;
    f.tw1 = d.tw1;
    cudaError_t e = passA(f, s, kVariantDirect);  // compile-time kernel with direct stores where there is one
    if (e != cudaSuccess) return e;
    Geom gl = geom_cols(a.logn1, (a.K2 + 2) / 2, 0);
    Geom gb = geom_row1<R>(a.logm, a.n1);
    Geom ga = geom_cols(a.logn1, a.K2 + 1, 0);
    with_log<R>(a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        e = launch_cl(k_adjL<R, L>, dim3(gl.blocks), gl.threads, gl.smem, s, 1, d);
    });
    with_log<R>(a.logm, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (e == cudaSuccess) e = launch_cl(k_adjB<R, L>, dim3(gb.blocks), gb.threads, gb.smem, s, 1, d);
    });
    with_log<R>(a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        if (e == cudaSuccess) e = launch_cl(k_adjC<R, L>, dim3(ga.blocks), ga.threads, ga.smem, s, 1, d);
    });
    return e;
}

// Columns per tile of pass A (tiles = CTAs; clustered variants launch whole
// clusters) and column pairs per tile of pass C, with the tile granularity a
// partial launch must respect (flame_step_host).
template <class R> void Ops<R>::tiles(const StepArgs &a, int variant, int *colsA, int *quantA, int *pairsC) {
    *quantA = 1;
    if (small_fp64<R>(a.logn1) || (variant == kVariantOneLine && one_line_fp32<R>(a.logn1))) {
        *colsA = 1;
        *pairsC = 1;
        return;
    }
    Geom g = make_geom<R>(a.logn1, a.K2 + 1, 0);
    *colsA = g.threads >> (a.logn1 - 4);
    with_log<R>(a.logn1, [&](auto lc) {
        constexpr int L = decltype(lc)::value;
        constexpr int cl = cluster_of<R, L>();
        if constexpr (sizeof(R) == 4 && L > 0) {
            if (variant == kVariantRadix8A) {
                *colsA = ShapeE<L, 8>::G;
                *quantA = ShapeE<L, 8>::CL;
            } else if (cl > 1 && variant == kVariantDefault) {
                *colsA = Shape<L>::G;
                *quantA = cl;
            }
        }
    });
    Geom gc = make_geom<R>(a.logn1, (a.K2 + 2) / 2, 0);
    *pairsC = gc.threads >> (a.logn1 - 4);
}

}  // namespace flame
