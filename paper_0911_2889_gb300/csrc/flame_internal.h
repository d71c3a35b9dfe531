// flame_internal.h -- declarations shared by the host runtime and the
// per-precision kernel translation units.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <type_traits>

namespace flame {

constexpr unsigned kLinearOnly = 1u;
constexpr unsigned kNonlinearOnly = 2u;
constexpr int kStatusNonfinite = 0;
constexpr int kStatusTimeout = 1;
constexpr int kStatusBounds = 2;
// The status word is followed by three words that the index-checking build
// (FLAME_DEBUG_BOUNDS) fills on its first failed check: the check's site,
// the index and the extent it was checked against.
constexpr int kStatusWords = 4;

// Sites of the index checks of the FLAME_DEBUG_BOUNDS build (reported by
// flame_sync_status with the failing index).
enum BoundsSite : int {
    kSiteAState = 1,    // pass A: state column entry
    kSiteAUv = 2,       // pass A: (U, V) store (direct and cluster write-outs)
    kSiteATma = 3,      // pass A: tensor-store coordinates (column, row pair)
    kSiteBUv = 4,       // pass B: row-pair (U, V) load
    kSiteBGk = 5,       // pass B: G store (direct write-out)
    kSiteBTma = 6,      // pass B: tensor-store coordinates (row pair, column pair)
    kSiteBArow = 7,     // pass B (area variant): row-pair area sum; state column 0
    kSiteCGk = 8,       // pass C: column-pair load
    kSiteCState = 9,    // pass C: state load and store (incl. the k2 = 0 mirror)
    kSiteCForcing = 10, // pass C: forcing entry
    kSiteCSave = 11,    // pass C: stage buffer entry
    kSiteCRec = 12,     // pass C: record entry, area row sums
    kSiteCAUv = 13,     // fused pass C + A: (U, V) store and tensor-store coordinates
    kSiteFftIn = 14,    // standalone 2-D FFT passes: input entry
    kSiteFftOut = 15,   // standalone 2-D FFT passes: output entry
    kSiteBoxSpec = 16,  // state from a field: spectrum entry and state entry
    kSiteProbe = 17,    // flame_debug_bounds_probe (a check with no access)
};
// One index check of (i, n) with no memory access, recorded in status
// (index-checking build); returns cudaErrorNotSupported in the normal build.
cudaError_t bounds_probe(int *status, int i, int n, cudaStream_t s);

// Time-stepping stage of a pass C launch (the update its epilogue applies,
// with F = omega Phi + N, N = c ghat + f the non-stiff part, E the exact
// propagator of the linear part over the step):
//   Euler:  Phi <- Phi + dt F(Phi)
//   Heun1:  save <- Phi;  Phi <- Phi + dt F(Phi)                 (predictor)
//   Heun2:  Phi <- (save + Phi + dt F(Phi)) / 2                  (corrector)
//   IF1:    save <- E (Phi + dt/2 N);  Phi <- E (Phi + dt N)     (Lawson-Heun)
//   IF2:    Phi <- save + dt/2 N(Phi)
// The mean mode follows with omega_0 = 0, E_0 = 1.  Stages 1 advance t to
// t_{n+1}; stages 2 evaluate at t_{n+1} and leave t there.
constexpr int kStageEuler = 0;
constexpr int kStageHeun1 = 1;
constexpr int kStageHeun2 = 2;
constexpr int kStageIF1 = 3;
constexpr int kStageIF2 = 4;

// Kernel variants chosen by the autotuner (0 = default shape).
constexpr int kVariantDefault = 0;
constexpr int kVariantDirect = 1;   // pass A: direct stores (no cluster write-out)
constexpr int kVariantRadix8 = 1;   // pass B: 8 points per thread, 512-thread CTAs
constexpr int kVariantRadix8A = 2;  // pass A: 8 points per thread, cluster write-out
constexpr int kVariantTma = 3;      // pass A: column written by tensor stores (FP32)
constexpr int kVariantTmaB = 2;     // pass B: row pair written by tensor stores (FP32)
constexpr int kVariantOneLine = 4;  // pass A (and with it pass C): one line per thread group (FP32, 2^8..2^11)
constexpr int kVariantOneLineB = 3; // pass B: one line per thread group (FP32, 2^8..2^11)
constexpr int kVariantWarpB = 4;    // pass B: 4096-point rows with warp-local exchanges, tensor-store write-out (FP32)

// Plain-old-data arguments of the step kernels.
struct StepArgs {
    int n1, n2;        // grid
    int logn1, logm;   // log2 N1, log2 (N2/2)
    int K1, K2;        // retained harmonics
    int ldk;           // row length of the compact box and workspaces (K2+1)
    double s1, s2;     // kappa = (s1 k1, s2 k2)
    float s1f, s2f;    // s1, s2 rounded once on the host (FP32 kernels)
    double gamma, t0, dt;
    unsigned flags;
};

// Everything one flame's step passes need: parameters, the caller's state
// buffers and the handle's tables and workspace.  Passed by value for a
// single flame, or as a device array indexed by blockIdx.y for an ensemble.
struct L2Window {
    const void *base;
    size_t bytes;
    float hit;  // fraction of the window's accesses that persist
};

struct FlameDesc {
    StepArgs a;
    void *state;            // compact box (in place)
    void *uv;               // N1 x ldk x (U, V) workspace
    void *gk;               // N1 x ldk workspace
    const void *tw1;        // twiddles of length N1
    const void *twm;        // twiddles of length N2/2 (+ real table)
    const double *t_in;     // caller's t (read by pass B)
    // the step's coefficients, derived from t once by pass B (block 0) and
    // read by pass C: [0] t_n, [1] c = 1/(2 r0^2), then from byte 16 the
    // kernel-precision CoefR (1/r0^2, gamma/(2 r0), c/(N1 N2), dt); 48 bytes,
    // 16-byte aligned (handle scratch)
    double *coef;
    double *mean;           // caller's mean mode
    double *t_out;          // caller's t (written by pass C)
    int *status;            // handle's device status word
    // two-stage schemes: the stage of this pass C launch (kStage*) and the
    // box-layout buffer and FP64 scalar that carry a term from stage 1 to
    // stage 2 (unused by the Euler stage)
    int stage;
    void *save;
    double *save_mean;
    // forcing term f_k of eq. (SivCurv1c): a caller-owned box (same layout
    // and precision as the state, k = 0 entry ignored) or null for f = 0,
    // and the mean-mode forcing f_0
    const void *forcing;
    double forcing0;
    // per-step record of the averaged diagnostics (Sec. 2), or null: entry
    // n mod rec_cap (4 doubles) of the step t_n -> t_{n+1} gets t_n, Phi_0(t_n)
    // and <Phi_t>(t_n) = c(t_n) mean |grad Phi_n|^2 + f_0 (the mean mode's
    // right-hand side), and a NaN area slot; written by the first stage
    double *rec;
    int rec_cap;
    // area in the record: 0 = none (NaN), 1 = summed by pass C from the
    // per-row-pair sums arow[N1/2] that the area variant of pass B writes,
    // 2 = the scalar *aval computed by the separate area kernels
    int rec_area;
    double *arow;
    const double *aval;
    // a launch over part of the tiles (pass A and C of one flame): tiles
    // [tile0, tile0 + tiles) of the full grid; tiles = 0: all
    int tile0, tiles;
    // pass C with one line per thread group (set with pass A's one-line
    // variant; FP32 column lengths 2^8 .. 2^11)
    int onec;
    // L2 persisting window over the state for the launches of passes A and
    // C (a launch attribute, not read by the kernels); bytes = 0: none
    L2Window l2_state;
};

// Workspace pointers of the area / adjoint kernels.
struct AdjDesc {
    StepArgs a;
    const void *state;   // forward state Phi (column-major box)
    const void *lam;     // adjoint lambda (column-major box), lambda_0 in *lam0
    void *lam_out;       // updated lambda (may equal lam)
    void *grad;          // dA/dPhi output (column-major box)
    const double *lam0;  // lambda_0 (mean-mode component of lambda)
    const double *mean;  // mean mode Phi_0
    const double *t;     // time (r0 = t for the area; t_n for the adjoint)
    void *uv;            // N1 x ldk pairs, row-major
    void *gk;            // N1 x ldk, row-major (lambda columns) or column-major
    void *aw;            // N1 x ldk pairs, column-major
    double *rowsum;      // N1 per-row partial area sums
    double *area;        // area output
    double *dmean;       // dA/dPhi_0 output
    double *dgamma;      // dL/dgamma accumulator (atomic)
    const void *tw1, *twm;
};

// Launch geometry of a line-FFT kernel.
struct Geom {
    int threads;       // blockDim.x
    int blocks;        // gridDim.x
    size_t smem;       // dynamic shared memory bytes
};

// Sets the thread-local message returned by flame_last_error().
void set_last_error(const char *msg);

// Per-precision launchers (defined in flame_f32.cu / flame_f64.cu).
template <class R> struct Ops {
    using C = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    static cudaError_t init_twiddles(C *tab, int logN, cudaStream_t s);
    // (status: the handle's status words, for the index checks of the
    // FLAME_DEBUG_BOUNDS build; unused otherwise)
    static cudaError_t rows_r2c(const R *in, C *out, int n1, int logm, const C *tw, cudaStream_t s,
                                int *status = nullptr);
    static cudaError_t rows_c2r(const C *in, R *out, int n1, int logm, const C *tw, cudaStream_t s,
                                int *status = nullptr);
    static cudaError_t cols(const C *in, C *out, int logn, int ncols, int ld, int dir, const C *tw,
                            cudaStream_t s, int *status = nullptr);
    // retained modes of an r2c spectrum -> compact box + FP64 mean
    static cudaError_t box_from_spec(const C *spec, C *state, double *mean, int n1, int n2, int K1, int K2,
                                     cudaStream_t s, int *status = nullptr);
    // One step pass for one flame (desc by value) or for nflames flames of
    // the same grid (descs: device array of nflames entries, shape from a).
    // variant: kVariantDefault, or a tuned alternative (pass A: kVariantDirect
    // = no cluster write-out, kVariantTma = tensor-store write-out through
    // uv_map, a map of d.uv made by encode_uv_map; pass B: kVariantRadix8 = 8
    // points per thread)
    static cudaError_t passA(const FlameDesc &d, cudaStream_t s, int variant = 0,
                             const CUtensorMap *uv_map = nullptr);
    static cudaError_t passB(const FlameDesc &d, cudaStream_t s, int variant = 0,
                             const CUtensorMap *gk_map = nullptr);
    static cudaError_t passC(const FlameDesc &d, cudaStream_t s);
    // Pass B that also sums the surface area of its rows (area variant,
    // arow[pair]); cudaErrorNotSupported when its shared memory exceeds the
    // device's limit.
    static cudaError_t passB_area(const FlameDesc &d, cudaStream_t s);
    // Pass C of one step fused with pass A of the next (FP32, 256 <= N1 <=
    // 4096, uv written through uv_map); cudaErrorNotSupported otherwise.
    static cudaError_t passCA(const FlameDesc &d, cudaStream_t s, const CUtensorMap *uv_map);
    // maps (nullable): per-flame tensor maps in device memory (uv maps for
    // pass A, gk maps for pass B) for the tensor-store variants
    static cudaError_t passA_batch(const FlameDesc *descs, int nflames, const StepArgs &a, cudaStream_t s,
                                   int variant = 0, const CUtensorMap *maps = nullptr);
    static cudaError_t passB_batch(const FlameDesc *descs, int nflames, const StepArgs &a, cudaStream_t s,
                                   int variant = 0, const CUtensorMap *maps = nullptr);
    static cudaError_t passC_batch(const FlameDesc *descs, int nflames, const StepArgs &a, cudaStream_t s,
                                   bool one_line = false);
    // Tiles (CTAs) of passes A and C: columns per pass-A tile, the tile
    // multiple a partial pass-A launch must use (clusters), column pairs per
    // pass-C tile
    static void tiles(const StepArgs &a, int variant, int *colsA, int *quantA, int *pairsC);
    // geometry used by the step passes (for the autotuner and the tests)
    static Geom geom_cols(int logn, int nlines, int groups_hint);
    static Geom geom_rows(int logm, int nlines, int groups_hint);
    // Area objective (and its gradient when d.grad / d.dmean are set): 3 kernels.
    static cudaError_t area(const AdjDesc &d, cudaStream_t s);
    // One adjoint step at (d.state, d.t): pass A on the forward state, column
    // synthesis of lambda, row pass, column pass with the lambda update.
    static cudaError_t adj_step(const AdjDesc &d, cudaStream_t s);
};

// Row pairs per tensor store of the uv write-out of pass A (<= 256).
__host__ __device__ constexpr int uv_box_pairs(int n1) { return n1 / 2 < 256 ? n1 / 2 : 256; }

// Column pairs per tensor store of the gk write-out of pass B (<= 256).
__host__ __device__ constexpr int gk_box_pairs(int ldk) { return (ldk + 1) / 2 < 256 ? (ldk + 1) / 2 : 256; }

// Tensor map of an FP32 uv workspace (n1 rows, ldk columns) for the
// tensor-store write-out of pass A: dimensions (8 floats of a row pair, k2,
// row pair), box (8, 1, uv_box_pairs(n1)).  False when the CUDA driver has no
// tensor-map encoder or rejects the map (the variant is then not offered).
bool encode_uv_map(CUtensorMap *map, void *uv, int n1, int ldk);
// Tensor map of an FP32 gk workspace (n1 rows, ldk columns, the column count
// rounded up to even) for the tensor-store write-out of pass B: dimensions
// (8 floats of a row pair and column pair, row pair, column pair), box
// (8, 1, gk_box_pairs(ldk)).
bool encode_gk_map(CUtensorMap *map, void *gk, int n1, int ldk);

}  // namespace flame
