// flame_api.cu -- host runtime behind the C ABI of include/flame.h:
// parameter validation, handle and workspace ownership, twiddle tables,
// launch sequencing, CUDA-graph capture of multi-step calls, ensembles,
// error reporting.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include <unistd.h>  // getpid (the tuner cache file's temporary name)

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "flame.h"
#include "flame_internal.h"
#include "fft_engine.cuh"

using flame::FlameDesc;
using flame::Ops;
using flame::StepArgs;

namespace {

thread_local std::string g_err;

flame_status fail(flame_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CUDA_TRY(expr)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) return fail(FLAME_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// Host-side fault injection for the error-path tests:
// FLAME_FAULT_INJECT=alloc|launch|param makes the next matching call fail
// before it touches the device.
bool inject(const char *what) {
    const char *v = getenv("FLAME_FAULT_INJECT");
    return v && strcmp(v, what) == 0;
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }
int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

constexpr int kGraphChunk = 256;  // steps per captured graph
constexpr int kBatchChunk = 8;    // ensemble steps per captured graph
constexpr int kGraphCache = 8;
constexpr int kRetiredMax = 64;

}  // namespace

void flame::set_last_error(const char *msg) { g_err = msg; }

namespace {
// NVTX range over a host-side scope: one per ABI call and one per pass
// enqueued outside a graph, so that a profiler attached to the process
// (ncu --nvtx, nsys) attributes the kernels to the call and pass that
// launched them.  Without a tool attached a push/pop costs a few
// nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace
#define FLAME_RANGE(name) NvtxRange flame_nvtx_range_(name)

namespace {
// the CUDA driver's tensor-map encoder, looked up once (null when unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return encode;
}
}  // namespace

bool flame::encode_gk_map(CUtensorMap *map, void *gk, int n1, int ldk) {
    const auto encode = tensor_map_encoder();
    if (!encode || !map || !gk || n1 < 2 || (n1 & 1) || ldk < 1) return false;
    // gk as floats: (8 floats: rows 2p, 2p+1 x columns 2q, 2q+1) x row pair
    // (32-byte stride) x column pair (n1 x 16-byte stride)
    const cuuint64_t dims[3] = {8, (cuuint64_t)(n1 / 2), (cuuint64_t)((ldk + 1) / 2)};
    const cuuint64_t strides[2] = {32, (cuuint64_t)n1 * 16};
    const cuuint32_t box[3] = {8, 1, (cuuint32_t)flame::gk_box_pairs(ldk)};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, gk, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool flame::encode_uv_map(CUtensorMap *map, void *uv, int n1, int ldk) {
    const auto encode = tensor_map_encoder();
    if (!encode || !map || !uv || n1 < 2 || (n1 & 1) || ldk < 1) return false;
    // uv as floats: (8 floats of a row pair) x k2 (32-byte stride) x row pair
    const cuuint64_t dims[3] = {8, (cuuint64_t)ldk, (cuuint64_t)(n1 / 2)};
    const cuuint64_t strides[2] = {32, (cuuint64_t)ldk * 32};
    const cuuint32_t box[3] = {8, 1, (cuuint32_t)flame::uv_box_pairs(n1)};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, uv, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Time-integration schemes of the multi-step entry points: explicit Euler,
// Heun's method and the integrating-factor RK2 (Lawson-Heun) step, as
// sequences of pass C stages (kStage*).
enum Scheme { kSchemeEuler = 0, kSchemeHeun = 1, kSchemeIF = 2 };

struct GraphEntry {
    const void *state;
    const double *mean, *t;
    int n, scheme;
    const void *forcing;  // the forcing in force when captured
    double forcing0;
    double *rec;          // the record in force when captured
    int rec_cap;
    bool rec_area;
    cudaGraphExec_t exec;
};

struct flame_ctx {
    flame_params p;  // resolved
    StepArgs sa;
    int logn1, logm;
    int device;
    size_t csz;       // bytes of one complex element
    void *tw1, *twm;  // twiddle tables
    void *uv, *gk;    // step workspaces
    void *spec;       // c2r workspace, N1 x (N2/2 + 1)
    void *aw;         // area / adjoint workspace, N1 x ldk pairs
    double *rowsum;   // N1 per-row area sums
    double *dscal;    // [1]: lambda_0, [2]: dgamma, [3]: dA/dPhi_0 scratch, [4]: the mean-mode
                      // term two-stage schemes carry between stages; [8..15]: step coefficients
    int *status;
    cudaStream_t cap;  // capture stream
    std::vector<GraphEntry> graphs;
    // graphs evicted from the caches above, which a stream may still be
    // running: destroyed by flame_destroy after its device synchronisation,
    // or all at once when kRetiredMax of them have piled up, so that an
    // eviction does not wait for the device
    std::vector<cudaGraphExec_t> retired;
    // ensemble state (owned by the first handle of a batch call): the
    // descriptors, then the flames' uv maps and gk maps (FP32)
    void *batch_desc = nullptr;
    size_t batch_cap = 0;
    void *batch_host = nullptr;  // pinned staging of the descriptors' upload
    size_t batch_host_cap = 0;
    cudaEvent_t batch_up = nullptr;  // recorded after the last upload from the staging
    std::vector<FlameDesc> batch_key;
    // graphs of the current binding: (steps per launch, executable)
    std::vector<std::pair<int, cudaGraphExec_t>> batch_graphs;
    // side streams and events of a capture with one branch per size class
    std::vector<cudaStream_t> batch_streams;
    std::vector<cudaEvent_t> batch_events;
    // adjoint arena (grown on demand by flame_adjoint) and the graphs of its
    // calls, keyed by every pointer and size of the call
    void *adj = nullptr;
    size_t adj_cap = 0;
    struct AdjGraph {
        std::vector<const void *> key;
        cudaGraphExec_t exec;
    };
    std::vector<AdjGraph> adj_graphs;
    // kernel variants picked by the autotuner for passes A and B
    int var_a = 0, var_b = 0;
    // the variants the grouped (ensemble) launches of this grid take: the
    // fastest two-line ones (an ensemble fills the GPU without the one-line
    // kernels, which measured slower there)
    int var_a_bat = 0, var_b_bat = 0;
    // tensor map of uv for the tensor-store variant of pass A (FP32)
    CUtensorMap uv_map, gk_map;  // tensor maps of uv and gk for the tensor-store variants (FP32)
    bool has_uv_map = false, has_gk_map = false;
    const CUtensorMap *map() const { return has_uv_map ? &uv_map : nullptr; }
    const CUtensorMap *gmap() const { return has_gk_map ? &gk_map : nullptr; }
    // multi-step runs fuse pass C of each step with pass A of the next
    bool fuse = false;
    // L2 persisting window over the caller's state (passes A and C)
    size_t l2_state_bytes = 0;
    float l2_state_hit = 0.f;
    // forcing term of eq. (SivCurv1c) (flame_set_forcing): caller-owned box
    // or null, and the mean-mode forcing
    const void *forcing = nullptr;
    double forcing0 = 0.0;
    // per-step diagnostics record (flame_set_record): caller-owned device
    // array of 4 rec_cap doubles, or null
    double *rec = nullptr;
    int rec_cap = 0;
    bool rec_area = false;  // the record includes the surface area
    // flame_step_host: device copies of the state, mean mode and time, the
    // copy stream and the chunk events (created on first use)
    void *io = nullptr;
    cudaStream_t cpy = nullptr;
    std::vector<cudaEvent_t> io_ev;
};

namespace {

template <class R> flame_status alloc_tables(flame_ctx *h) {
    using C = typename Ops<R>::C;
    CUDA_TRY(Ops<R>::init_twiddles(static_cast<C *>(h->tw1), h->logn1, h->cap));
    CUDA_TRY(Ops<R>::init_twiddles(static_cast<C *>(h->twm), h->logm, h->cap));
    return FLAME_OK;
}

void free_ctx(flame_ctx *h) {
    if (!h) return;
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    for (auto &g : h->adj_graphs) cudaGraphExecDestroy(g.exec);
    for (cudaGraphExec_t g : h->retired) cudaGraphExecDestroy(g);
    for (auto &g : h->batch_graphs) cudaGraphExecDestroy(g.second);
    cudaFree(h->batch_desc);
    cudaFreeHost(h->batch_host);
    if (h->batch_up) cudaEventDestroy(h->batch_up);
    for (cudaStream_t q : h->batch_streams) cudaStreamDestroy(q);
    for (cudaEvent_t ev : h->batch_events) cudaEventDestroy(ev);
    cudaFree(h->tw1);
    cudaFree(h->twm);
    cudaFree(h->uv);
    cudaFree(h->gk);
    cudaFree(h->spec);
    cudaFree(h->aw);
    cudaFree(h->rowsum);
    cudaFree(h->adj);
    cudaFree(h->dscal);
    cudaFree(h->status);
    cudaFree(h->io);
    for (auto e : h->io_ev) cudaEventDestroy(e);
    if (h->cpy) cudaStreamDestroy(h->cpy);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

FlameDesc make_desc(flame_ctx *h, void *state, double *mean, double *t) {
    FlameDesc d;
    memset(&d, 0, sizeof d);  // descriptors are compared bytewise
    d.a = h->sa;
    d.state = state;
    d.uv = h->uv;
    d.gk = h->gk;
    d.tw1 = h->tw1;
    d.twm = h->twm;
    d.t_in = t;
    d.coef = h->dscal + 8;
    d.mean = mean;
    d.t_out = t;
    d.status = h->status;
    if (h->l2_state_bytes) d.l2_state = flame::L2Window{state, h->l2_state_bytes, h->l2_state_hit};
    d.stage = flame::kStageEuler;
    // the two-stage schemes carry one box between their stages in the area
    // workspace (N1 (K2+1) pairs, larger than the box) and one FP64 scalar
    d.save = h->aw;
    d.save_mean = h->dscal + 4;
    d.forcing = h->forcing;
    d.forcing0 = h->forcing0;
    d.rec = h->rec;
    d.rec_cap = h->rec_cap;
    d.onec = h->var_a == flame::kVariantOneLine;
    return d;
}

bool first_stage(int stage) {
    return stage == flame::kStageEuler || stage == flame::kStageHeun1 || stage == flame::kStageIF1;
}

// A recorded step with the surface area: pass B's area variant sums the
// area of the rows it transforms (rec_area = 1); where that variant does not
// fit in shared memory (FP64 rows of 8192 points) the separate area kernels
// compute it first, into handle scratch (rec_area = 2).
cudaError_t enqueue_step_area(flame_ctx *h, FlameDesc d, cudaStream_t s) {
    cudaError_t e;
    d.rec_area = 1;
    d.arow = h->rowsum;
    const bool f64 = h->p.prec == FLAME_FP64;
    if ((e = f64 ? Ops<double>::passA(d, s, h->var_a) : Ops<float>::passA(d, s, h->var_a, h->map())) != cudaSuccess)
        return e;
    e = f64 ? Ops<double>::passB_area(d, s) : Ops<float>::passB_area(d, s);
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        flame::AdjDesc ad;
        memset(&ad, 0, sizeof ad);
        ad.a = h->sa;
        ad.state = d.state;
        ad.mean = d.mean;
        ad.t = d.t_in;
        ad.uv = h->uv;
        ad.gk = h->gk;
        ad.aw = h->aw;
        ad.rowsum = h->rowsum;
        ad.area = h->dscal + 6;
        ad.dmean = h->dscal + 3;
        ad.tw1 = h->tw1;
        ad.twm = h->twm;
        // the area kernels use the step's workspaces: run them, then the
        // step's passes from the start
        if ((e = f64 ? Ops<double>::area(ad, s) : Ops<float>::area(ad, s)) != cudaSuccess) return e;
        d.rec_area = 2;
        d.aval = h->dscal + 6;
        if ((e = f64 ? Ops<double>::passA(d, s, h->var_a) : Ops<float>::passA(d, s, h->var_a, h->map())) !=
            cudaSuccess)
            return e;
        e = f64 ? Ops<double>::passB(d, s, h->var_b) : Ops<float>::passB(d, s, h->var_b, h->gmap());
    }
    if (e != cudaSuccess) return e;
    return f64 ? Ops<double>::passC(d, s) : Ops<float>::passC(d, s);
}

cudaError_t enqueue_step(flame_ctx *h, const FlameDesc &d, cudaStream_t s) {
    cudaError_t e;
    if (d.rec && h->rec_area && first_stage(d.stage)) return enqueue_step_area(h, d, s);
    if (h->p.prec == FLAME_FP64) {
        {
            FLAME_RANGE("flame pass A");
            if ((e = Ops<double>::passA(d, s, h->var_a)) != cudaSuccess) return e;
        }
        {
            FLAME_RANGE("flame pass B");
            if ((e = Ops<double>::passB(d, s, h->var_b)) != cudaSuccess) return e;
        }
        FLAME_RANGE("flame pass C");
        return Ops<double>::passC(d, s);
    }
    {
        FLAME_RANGE("flame pass A");
        if ((e = Ops<float>::passA(d, s, h->var_a, h->map())) != cudaSuccess) return e;
    }
    {
        FLAME_RANGE("flame pass B");
        if ((e = Ops<float>::passB(d, s, h->var_b, h->gmap())) != cudaSuccess) return e;
    }
    FLAME_RANGE("flame pass C");
    return Ops<float>::passC(d, s);
}

// The pass C stages of one step of a scheme.
int scheme_stages(int scheme, int *stages) {
    if (scheme == kSchemeHeun) {
        stages[0] = flame::kStageHeun1;
        stages[1] = flame::kStageHeun2;
        return 2;
    }
    if (scheme == kSchemeIF) {
        stages[0] = flame::kStageIF1;
        stages[1] = flame::kStageIF2;
        return 2;
    }
    stages[0] = flame::kStageEuler;
    return 1;
}

// n steps of a scheme: every stage is one evaluation of the right-hand side
// (passes A and B) and a pass C that applies the stage's update.  With
// fusion, pass C of each stage runs fused with pass A of the next:
// A, (B, CA) x (stages - 1), B, C.  Same arithmetic as separate passes.
cudaError_t enqueue_scheme(flame_ctx *h, FlameDesc d, int scheme, int n, cudaStream_t s) {
    int st[2];
    const int ns = scheme_stages(scheme, st);
    const int total = ns * n;
    cudaError_t e = cudaSuccess;
    if (h->fuse && total > 1) {
        e = Ops<float>::passA(d, s, h->var_a, h->map());
        for (int i = 0; i < total && e == cudaSuccess; ++i) {
            d.stage = st[i % ns];
            FlameDesc dc = d;
            if (d.rec && h->rec_area && first_stage(d.stage)) {
                dc.rec_area = 1;
                dc.arow = h->rowsum;
                e = Ops<float>::passB_area(dc, s);
            } else {
                e = Ops<float>::passB(d, s, h->var_b, h->gmap());
            }
            if (e == cudaSuccess) e = i + 1 < total ? Ops<float>::passCA(dc, s, h->map()) : Ops<float>::passC(dc, s);
        }
        return e;
    }
    for (int i = 0; i < total && e == cudaSuccess; ++i) {
        d.stage = st[i % ns];
        e = enqueue_step(h, d, s);
    }
    return e;
}

// The state is written by pass C and read by the next step's pass A (and by
// the following pass C).  A persisting L2 window over it (a per-launch
// attribute of passes A and C) keeps it resident while uv and gk stream
// through the rest of the L2; as it is rewritten in place every step, its
// lines need not go back to HBM in between.  (A second window over gk, for
// pass B's writes, measured slower: it leaves too little L2 to pass A's uv
// stores.)  The set-aside is a limit of this process's context, raised to
// the state's size when the device allows it and never lowered.
// FLAME_L2_PERSIST=0 turns the window off.
void setup_l2_window(flame_ctx *h, size_t state_bytes) {
    const char *env = getenv("FLAME_L2_PERSIST");
    if (env && strcmp(env, "0") == 0) return;
    int max_persist = 0, max_window = 0;
    if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, h->device) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (max_persist <= 0 || max_window <= 0) return;
    size_t cur = 0;
    const size_t want = std::min((size_t)max_persist, state_bytes);
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess ||
        (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) ||
        cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cur == 0) return;
    h->l2_state_bytes = std::min(state_bytes, (size_t)max_window);
    h->l2_state_hit = (float)std::min(1.0, (double)cur / (double)h->l2_state_bytes);
}

// ---------------------------------------------------------------- autotuner
// For FP32 grids with compile-time kernels (N1, N2/2 in 256..4096) the
// alternative shapes of passes A and B are timed once per (grid, K,
// precision, device) on scratch buffers, and the fastest is kept for the
// process.  FLAME_AUTOTUNE=0 keeps the default shapes.
using TuneKey = std::tuple<int, int, int, int, int, int>;
// the autotuner's choice for one grid
struct TuneChoice {
    int a, b, fuse, a_bat, b_bat;
};
std::map<TuneKey, TuneChoice> g_tune;
std::mutex g_tune_mu;

// two-line stand-ins of the one-line variants (for the grouped launches when
// only the single-flame choice is known)
int two_line_a(int v) { return v == flame::kVariantOneLine ? flame::kVariantDirect : v; }
int two_line_b(int v) { return v == flame::kVariantOneLineB ? flame::kVariantDefault : v; }

// Autotuner cache file (FLAME_TUNE_CACHE=path): a flat JSON object mapping
// "<GPU name>|<N1>x<N2>|<K1>,<K2>|<precision>" to [pass A variant, pass B
// variant, fused column passes (0/1), pass A and pass B variants of the
// grouped launches] (an entry of the first three alone is read too).  A
// handle created with a key that the
// file holds takes its choice without timing anything; a new choice is added
// to the file (rewritten through a temporary file and a rename, so that a
// reader never sees half a file).  Entries of other keys are kept.
std::string tune_file_key(const flame_ctx *h) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) {
        cudaGetLastError();
        return std::string();
    }
    char buf[512];
    snprintf(buf, sizeof buf, "%s|%dx%d|%d,%d|%s", prop.name, h->p.n_theta, h->p.n_phi, h->p.K1, h->p.K2,
             h->p.prec == FLAME_FP64 ? "fp64" : "fp32");
    for (char *c = buf; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';  // keep the key a plain JSON string
    return buf;
}

// Parses the cache file into key -> choice; a malformed file reads as empty
// (it is then rewritten with the entries this process adds).
std::map<std::string, TuneChoice> read_tune_file(const char *path) {
    std::map<std::string, TuneChoice> out;
    FILE *f = fopen(path, "rb");
    if (!f) return out;
    std::string s;
    char chunk[4096];
    size_t n;
    while ((n = fread(chunk, 1, sizeof chunk, f)) > 0) s.append(chunk, n);
    fclose(f);
    size_t i = 0;
    auto skip = [&]() {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i;
    };
    skip();
    if (i >= s.size() || s[i] != '{') return {};
    ++i;
    while (true) {
        skip();
        if (i < s.size() && s[i] == '}') break;
        if (i >= s.size() || s[i] != '"') return {};
        const size_t e = s.find('"', i + 1);
        if (e == std::string::npos) return {};
        const std::string key = s.substr(i + 1, e - i - 1);
        i = e + 1;
        skip();
        if (i >= s.size() || s[i] != ':') return {};
        ++i;
        skip();
        int a = 0, b = 0, fu = 0, ab = 0, bb = 0, used = 0;
        if (sscanf(s.c_str() + i, "[ %d , %d , %d , %d , %d ]%n", &a, &b, &fu, &ab, &bb, &used) == 5 && used > 0) {
            out[key] = TuneChoice{a, b, fu, ab, bb};
        } else {
            used = 0;
            if (sscanf(s.c_str() + i, "[ %d , %d , %d ]%n", &a, &b, &fu, &used) != 3 || used == 0) return {};
            out[key] = TuneChoice{a, b, fu, two_line_a(a), two_line_b(b)};
        }
        i += (size_t)used;
        skip();
        if (i < s.size() && s[i] == ',') {
            ++i;
            continue;
        }
        skip();
        if (i < s.size() && s[i] == '}') break;
        return {};
    }
    return out;
}

void write_tune_file(const char *path, const std::map<std::string, TuneChoice> &m) {
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return;  // the cache is optional
    fputs("{\n", f);
    size_t k = 0;
    for (const auto &kv : m)
        fprintf(f, "  \"%s\": [%d, %d, %d, %d, %d]%s\n", kv.first.c_str(), kv.second.a, kv.second.b, kv.second.fuse,
                kv.second.a_bat, kv.second.b_bat, ++k < m.size() ? "," : "");
    fputs("}\n", f);
    const bool ok = fclose(f) == 0;
    if (!ok || rename(tmp.c_str(), path) != 0) remove(tmp.c_str());
}

// Fusion of pass C with the next pass A needs the FP32 compile-time column
// kernels and the uv tensor map; FLAME_FUSE=0 disables it.
bool fuse_allowed(const flame_ctx *h) {
    const char *env = getenv("FLAME_FUSE");
    if (env && strcmp(env, "0") == 0) return false;
    // (not with the one-line column passes: the fused pass is a two-line
    // kernel, and fused and separate steps must give the same bits)
    return h->p.prec == FLAME_FP32_MIXED && h->has_uv_map && h->logn1 >= 8 && h->logn1 <= 12 &&
           h->var_a != flame::kVariantOneLine;
}

flame_status autotune(flame_ctx *h) {
    // FLAME_FORCE_VARIANTS=a,b fixes the variants (tests exercise each one)
    const char *force = getenv("FLAME_FORCE_VARIANTS");
    if (force) {
        int va = 0, vb = 0;
        if (sscanf(force, "%d,%d", &va, &vb) == 2) {
            h->var_a = va == 4   ? flame::kVariantOneLine
                       : va == 3 ? flame::kVariantTma
                       : va == 2 ? flame::kVariantRadix8A
                       : va      ? flame::kVariantDirect
                                 : flame::kVariantDefault;
            h->var_b = vb == 4   ? flame::kVariantWarpB
                       : vb == 3 ? flame::kVariantOneLineB
                       : vb == 2 ? flame::kVariantTmaB
                       : vb      ? flame::kVariantRadix8
                                 : flame::kVariantDefault;
            h->var_a_bat = h->var_a;  // forced: the grouped launches take them too
            h->var_b_bat = h->var_b;
            h->fuse = fuse_allowed(h);
            return FLAME_OK;
        }
    }
    const char *env = getenv("FLAME_AUTOTUNE");
    if (env && strcmp(env, "0") == 0) {
        h->fuse = fuse_allowed(h);
        return FLAME_OK;
    }
    if (h->p.prec != FLAME_FP32_MIXED || h->logn1 < 8 || h->logn1 > 12 || h->logm < 8 || h->logm > 12)
        return FLAME_OK;
    const TuneKey key{h->p.n_theta, h->p.n_phi, h->p.K1, h->p.K2, (int)h->p.prec, h->device};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            h->var_a = it->second.a;
            h->var_b = it->second.b;
            h->var_a_bat = it->second.a_bat;
            h->var_b_bat = it->second.b_bat;
            h->fuse = it->second.fuse && fuse_allowed(h);
            return FLAME_OK;
        }
    }
    const char *cache_path = getenv("FLAME_TUNE_CACHE");
    const std::string fkey = cache_path && *cache_path ? tune_file_key(h) : std::string();
    if (!fkey.empty()) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        const auto m = read_tune_file(cache_path);
        auto it = m.find(fkey);
        if (it != m.end()) {
            h->var_a = it->second.a;
            h->var_b = it->second.b;
            h->var_a_bat = it->second.a_bat;
            h->var_b_bat = it->second.b_bat;
            // a variant the handle cannot run (no tensor map) falls back to the default shape
            if (h->var_a == flame::kVariantTma && !h->has_uv_map) h->var_a = flame::kVariantDefault;
            if (h->var_b == flame::kVariantTmaB && !h->has_gk_map) h->var_b = flame::kVariantDefault;
            if (h->var_a_bat == flame::kVariantTma && !h->has_uv_map) h->var_a_bat = flame::kVariantDefault;
            if (h->var_b_bat == flame::kVariantTmaB && !h->has_gk_map) h->var_b_bat = flame::kVariantDefault;
            if (h->var_b == flame::kVariantWarpB && !h->has_gk_map) h->var_b = flame::kVariantDefault;
            if (h->var_b_bat == flame::kVariantWarpB && !h->has_gk_map) h->var_b_bat = flame::kVariantDefault;
            h->fuse = it->second.fuse != 0 && fuse_allowed(h);
            g_tune[key] = TuneChoice{h->var_a, h->var_b, h->fuse ? 1 : 0, h->var_a_bat, h->var_b_bat};
            return FLAME_OK;
        }
    }
    const size_t box = (2 * (size_t)h->p.K1 + 1) * ((size_t)h->p.K2 + 1) * h->csz;
    void *st = nullptr;
    double *sc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(st);
        cudaFree(sc);
    };
    if (cudaMalloc(&st, box) != cudaSuccess || cudaMalloc((void **)&sc, 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return FLAME_OK;  // tuning is optional: keep the defaults
    }
    double init[2] = {0.0, h->p.t0};
    cudaError_t e = cudaMemsetAsync(st, 0, box, h->cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc, init, sizeof init, cudaMemcpyHostToDevice, h->cap);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    FlameDesc d = make_desc(h, st, sc, sc + 1);
    // pass 0: A, 1: B, 2: C then A (variant, with its pass C), 3: C fused with A
    auto time_it = [&](int pass, int variant, float *ms) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        float total = 0.f;
        for (int rep = 0; rep < 4 && r == cudaSuccess; ++rep) {
            r = cudaEventRecord(e0, h->cap);
            if (r == cudaSuccess) {
                if (pass == 0) r = Ops<float>::passA(d, h->cap, variant, h->map());
                else if (pass == 1) r = Ops<float>::passB(d, h->cap, variant, h->gmap());
                else if (pass == 2) {
                    d.onec = variant == flame::kVariantOneLine;
                    r = Ops<float>::passC(d, h->cap);
                    if (r == cudaSuccess) r = Ops<float>::passA(d, h->cap, variant, h->map());
                } else {
                    r = Ops<float>::passCA(d, h->cap, h->map());
                }
            }
            if (r == cudaSuccess) r = cudaEventRecord(e1, h->cap);
            if (r == cudaSuccess) r = cudaEventSynchronize(e1);
            float t = 0.f;
            if (r == cudaSuccess) r = cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) total += t;  // the first run is the warm-up
        }
        *ms = total / 3.f;
        return r;
    };
    // pass A variants are timed with their pass C (the one-line pass A
    // brings the one-line pass C)
    const int avars[5] = {flame::kVariantDefault, flame::kVariantDirect, flame::kVariantRadix8A, flame::kVariantTma,
                          flame::kVariantOneLine};
    const int bvars[5] = {flame::kVariantDefault, flame::kVariantRadix8, flame::kVariantTmaB, flame::kVariantOneLineB,
                          flame::kVariantWarpB};
    float best_a = 1e30f, best_b = 1e30f, best_a2 = 1e30f, best_b2 = 1e30f;
    for (int v : avars) {
        if (v == flame::kVariantTma && !h->has_uv_map) continue;
        if (v == flame::kVariantOneLine && h->logn1 > 11) continue;
        float ms = 0;
        if (e == cudaSuccess) e = time_it(2, v, &ms);
        if (e == cudaSuccess && ms < best_a) {
            best_a = ms;
            h->var_a = v;
        }
        if (e == cudaSuccess && v != flame::kVariantOneLine && ms < best_a2) {
            best_a2 = ms;
            h->var_a_bat = v;
        }
    }
    d.onec = h->var_a == flame::kVariantOneLine;
    for (int v : bvars) {
        if (v == flame::kVariantTmaB && !h->has_gk_map) continue;
        if (v == flame::kVariantOneLineB && h->logm > 11) continue;
        if (v == flame::kVariantWarpB && (h->logm != 12 || !h->has_gk_map)) continue;
        float ms = 0;
        if (e == cudaSuccess) e = time_it(1, v, &ms);
        // the warp-local variant measures level with variant 2 (within the
        // timing noise): it is taken only when clearly faster, so that the
        // choice does not flip from run to run
        if (v == flame::kVariantWarpB) ms *= 1.02f;
        if (e == cudaSuccess && ms < best_b) {
            best_b = ms;
            h->var_b = v;
        }
        if (e == cudaSuccess && v != flame::kVariantOneLineB && ms < best_b2) {
            best_b2 = ms;
            h->var_b_bat = v;
        }
    }
    // Fused or separate column passes: each way, 4 steps captured as one CUDA
    // graph (as flame_step runs them) and replayed; the faster is kept.
    // (Timed launch by launch, with events between the kernels, the fused
    // pass looked faster at 4096 x 8192; as a graph the separate passes are.)
    if (fuse_allowed(h) && e == cudaSuccess) {
        float ms[2] = {0.f, 0.f};
        for (int way = 0; way < 2 && e == cudaSuccess; ++way) {
            h->fuse = way == 1;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t le = enqueue_scheme(h, d, kSchemeEuler, 4, h->cap);
                e = cudaStreamEndCapture(h->cap, &graph);
                if (e == cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(e0, h->cap);
                if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->cap);
                if (e == cudaSuccess) e = cudaEventRecord(e1, h->cap);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms[way] += t;  // the first replay is the warm-up
            }
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        }
        h->fuse = e == cudaSuccess && ms[1] < ms[0];
    }
    cleanup();
    if (e != cudaSuccess) return fail(FLAME_ECUDA, "autotune: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = TuneChoice{h->var_a, h->var_b, h->fuse ? 1 : 0, h->var_a_bat, h->var_b_bat};
    if (!fkey.empty()) {
        auto m = read_tune_file(cache_path);
        m[fkey] = g_tune[key];
        write_tune_file(cache_path, m);
    }
    return FLAME_OK;
}

// Captures n steps of a scheme for one flame on the handle's capture stream.
flame_status capture_steps(flame_ctx *h, const FlameDesc &d, int scheme, int n, cudaGraphExec_t *out) {
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = enqueue_scheme(h, d, scheme, n, h->cap);
    cudaError_t ee = cudaStreamEndCapture(h->cap, &graph);
    if (le != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(FLAME_ECUDA, "graph capture failed: %s",
                    cudaGetErrorString(le != cudaSuccess ? le : ee));
    }
    cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(FLAME_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    return FLAME_OK;
}

// An evicted graph may still be pending on some stream: it joins the
// retired list instead of being destroyed now.
cudaError_t retire_graph(flame_ctx *h, cudaGraphExec_t exec) {
    h->retired.push_back(exec);
    if ((int)h->retired.size() < kRetiredMax) return cudaSuccess;
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    for (cudaGraphExec_t g : h->retired) cudaGraphExecDestroy(g);
    h->retired.clear();
    return cudaSuccess;
}

flame_status step_graph(flame_ctx *h, void *state, double *mean, double *t, int scheme, int n,
                        cudaGraphExec_t *out) {
    for (auto &g : h->graphs)
        if (g.state == state && g.mean == mean && g.t == t && g.n == n && g.scheme == scheme &&
            g.forcing == h->forcing && g.forcing0 == h->forcing0 && g.rec == h->rec && g.rec_cap == h->rec_cap &&
            g.rec_area == h->rec_area) {
            *out = g.exec;
            return FLAME_OK;
        }
    if ((int)h->graphs.size() >= kGraphCache) {
        CUDA_TRY(retire_graph(h, h->graphs.front().exec));
        h->graphs.erase(h->graphs.begin());
    }
    cudaGraphExec_t exec;
    flame_status st = capture_steps(h, make_desc(h, state, mean, t), scheme, n, &exec);
    if (st != FLAME_OK) return st;
    h->graphs.push_back(
        GraphEntry{state, mean, t, n, scheme, h->forcing, h->forcing0, h->rec, h->rec_cap, h->rec_area, exec});
    *out = exec;
    return FLAME_OK;
}

// nsteps steps of a scheme: one step directly, more as CUDA graphs of up to
// kGraphChunk steps (all captured before the first launch, so that a
// capture failure leaves nothing enqueued).
flame_status run_scheme(flame_ctx *h, void *state, double *mean, double *t, int scheme, int nsteps,
                        cudaStream_t s) {
    if (nsteps == 0) return FLAME_OK;
    if (nsteps == 1) {
        CUDA_TRY(enqueue_scheme(h, make_desc(h, state, mean, t), scheme, 1, s));
        return FLAME_OK;
    }
    const int full = nsteps / kGraphChunk, rest = nsteps % kGraphChunk;
    cudaGraphExec_t gfull = nullptr, grest = nullptr;
    if (full) {
        flame_status st = step_graph(h, state, mean, t, scheme, kGraphChunk, &gfull);
        if (st != FLAME_OK) return st;
    }
    if (rest) {
        flame_status st = step_graph(h, state, mean, t, scheme, rest, &grest);
        if (st != FLAME_OK) return st;
    }
    for (int i = 0; i < full; ++i) CUDA_TRY(cudaGraphLaunch(gfull, s));
    if (rest) CUDA_TRY(cudaGraphLaunch(grest, s));
    return FLAME_OK;
}

}  // namespace

extern "C" {

const char *flame_status_str(flame_status s) {
    switch (s) {
    case FLAME_OK: return "ok";
    case FLAME_EINVAL: return "invalid argument";
    case FLAME_ENOMEM: return "out of memory";
    case FLAME_ECUDA: return "CUDA error";
    case FLAME_EUNSUPPORTED: return "unsupported";
    case FLAME_ETIMEOUT: return "device wait timed out";
    case FLAME_ENONFINITE: return "non-finite value";
    case FLAME_EBOUNDS: return "index out of bounds (index-checking build)";
    }
    return "unknown status";
}

const char *flame_last_error(void) { return g_err.c_str(); }

flame_status flame_create(const flame_params *params, flame_t *out) {
    FLAME_RANGE("flame_create");
    if (!params || !out) return fail(FLAME_EINVAL, "flame_create: null pointer");
    if (inject("param")) return fail(FLAME_EINVAL, "flame_create: injected parameter fault");
    flame_params p = *params;
    if (p.prec != FLAME_FP64 && p.prec != FLAME_FP32_MIXED)
        return fail(FLAME_EINVAL, "flame_create: unknown precision %d", (int)p.prec);
    if (!pow2_in(p.n_theta, 16, 4096))
        return fail(FLAME_EUNSUPPORTED, "n_theta=%d: need a power of two in [16, 4096]", p.n_theta);
    if (!pow2_in(p.n_phi, 32, 8192))
        return fail(FLAME_EUNSUPPORTED, "n_phi=%d: need a power of two in [32, 8192]", p.n_phi);
    if (p.K1 < 0 || p.K2 < 0) return fail(FLAME_EINVAL, "negative K");
    if (p.K1 == 0) p.K1 = (p.n_theta - 1) / 4;
    if (p.K2 == 0) p.K2 = (p.n_phi - 1) / 4;
    if (4 * p.K1 + 1 > p.n_theta || 4 * p.K2 + 1 > p.n_phi)
        return fail(FLAME_EINVAL, "need 4K+1 <= N (alias-free padding): K=(%d,%d) N=(%d,%d)", p.K1, p.K2,
                    p.n_theta, p.n_phi);
    if (!(std::isfinite(p.gamma)) || !(p.theta_pi > 0) || !std::isfinite(p.theta_pi))
        return fail(FLAME_EINVAL, "gamma must be finite and theta_pi > 0");
    if (!(p.s1 >= 0) || !(p.s2 >= 0) || !std::isfinite(p.s1) || !std::isfinite(p.s2))
        return fail(FLAME_EINVAL, "s1, s2 must be >= 0");
    if (p.s1 == 0) p.s1 = p.theta_pi;
    if (p.s2 == 0) p.s2 = p.theta_pi;
    if (!(p.t0 > 0) || !(p.dt > 0) || !std::isfinite(p.t0) || !std::isfinite(p.dt))
        return fail(FLAME_EINVAL, "need t0 > 0 and dt > 0");
    if ((p.flags & ~3u) || p.flags == 3u) return fail(FLAME_EINVAL, "bad flags %u", p.flags);
    if (inject("alloc")) return fail(FLAME_ENOMEM, "flame_create: injected allocation fault");

    flame_ctx *h = new flame_ctx();
    h->p = p;
    h->logn1 = ilog2(p.n_theta);
    h->logm = ilog2(p.n_phi / 2);
    h->csz = p.prec == FLAME_FP64 ? sizeof(double2) : sizeof(float2);
    StepArgs &a = h->sa;
    a.n1 = p.n_theta;
    a.n2 = p.n_phi;
    a.logn1 = h->logn1;
    a.logm = h->logm;
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

    auto dev_alloc = [&](void **ptr, size_t bytes) -> bool {
        return cudaMalloc(ptr, bytes) == cudaSuccess;
    };
    cudaError_t ge = cudaGetDevice(&h->device);
    if (ge != cudaSuccess) {
        delete h;
        return fail(FLAME_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ge));
    }
    const size_t n1 = p.n_theta, ldk = a.ldk, m1 = p.n_phi / 2 + 1;
    bool ok = dev_alloc(&h->tw1, flame::tw_alloc_len(h->logn1) * h->csz) &&
              dev_alloc(&h->twm, flame::tw_alloc_len(h->logm) * h->csz) &&
              dev_alloc(&h->uv, n1 * ldk * 2 * h->csz) && dev_alloc(&h->gk, n1 * ((ldk + 1) & ~(size_t)1) * h->csz) &&
              dev_alloc(&h->spec, n1 * m1 * h->csz) && dev_alloc(&h->aw, n1 * ldk * 2 * h->csz) &&
              dev_alloc((void **)&h->rowsum, n1 * sizeof(double)) && dev_alloc((void **)&h->dscal, 16 * sizeof(double)) &&
              dev_alloc((void **)&h->status, flame::kStatusWords * sizeof(int));
    if (!ok) {
        cudaGetLastError();
        free_ctx(h);
        return fail(FLAME_ENOMEM, "flame_create: device allocation failed");
    }
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        h->cap = nullptr;
        free_ctx(h);
        return fail(FLAME_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    flame_status st = p.prec == FLAME_FP64 ? alloc_tables<double>(h) : alloc_tables<float>(h);
    if (st == FLAME_OK) {
        e = cudaMemsetAsync(h->status, 0, flame::kStatusWords * sizeof(int), h->cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->dscal, 0, 16 * sizeof(double), h->cap);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->cap);
        if (e != cudaSuccess) st = fail(FLAME_ECUDA, "flame_create: %s", cudaGetErrorString(e));
    }
    if (st == FLAME_OK)
        setup_l2_window(h, (2 * (size_t)p.K1 + 1) * ldk * h->csz);
    if (st == FLAME_OK && p.prec == FLAME_FP32_MIXED && h->logn1 >= 8 && h->logn1 <= 12)
        h->has_uv_map = flame::encode_uv_map(&h->uv_map, h->uv, (int)n1, (int)ldk);
    if (st == FLAME_OK && p.prec == FLAME_FP32_MIXED && h->logm >= 8 && h->logm <= 12)
        h->has_gk_map = flame::encode_gk_map(&h->gk_map, h->gk, (int)n1, (int)ldk);
    if (st == FLAME_OK) st = autotune(h);
    if (st != FLAME_OK) {
        free_ctx(h);
        return st;
    }
    *out = h;
    return FLAME_OK;
}

flame_status flame_fused_steps(flame_t h, int *enabled) {
    if (!h || !enabled) return fail(FLAME_EINVAL, "flame_fused_steps: null pointer");
    *enabled = h->fuse ? 1 : 0;
    return FLAME_OK;
}

flame_status flame_tuning(flame_t h, int *pass_a_variant, int *pass_b_variant) {
    if (!h || !pass_a_variant || !pass_b_variant) return fail(FLAME_EINVAL, "flame_tuning: null pointer");
    *pass_a_variant = h->var_a;
    *pass_b_variant = h->var_b;
    return FLAME_OK;
}

flame_status flame_destroy(flame_t h) {
    if (!h) return FLAME_OK;
    cudaError_t e = cudaDeviceSynchronize();
    // persisting lines of this handle's windows go back to normal lines
    if (h->l2_state_bytes && e == cudaSuccess) e = cudaCtxResetPersistingL2Cache();
    free_ctx(h);
    if (e != cudaSuccess) return fail(FLAME_ECUDA, "flame_destroy: %s", cudaGetErrorString(e));
    return FLAME_OK;
}

flame_status flame_get_params(flame_t h, flame_params *out) {
    if (!h || !out) return fail(FLAME_EINVAL, "flame_get_params: null pointer");
    *out = h->p;
    return FLAME_OK;
}

size_t flame_state_len(flame_t h) { return h ? (size_t)(2 * h->p.K1 + 1) * (size_t)(h->p.K2 + 1) : 0; }

flame_status flame_fft_r2c(flame_t h, const void *real_in, void *spec_out, void *stream) {
    FLAME_RANGE("flame_fft_r2c");
    if (!h || !real_in || !spec_out) return fail(FLAME_EINVAL, "flame_fft_r2c: null pointer");
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_fft_r2c: injected launch fault");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int M = h->p.n_phi / 2;
    if (h->p.prec == FLAME_FP64) {
        using C = double2;
        CUDA_TRY(Ops<double>::rows_r2c(static_cast<const double *>(real_in), static_cast<C *>(spec_out),
                                       h->p.n_theta, h->logm, static_cast<const C *>(h->twm), s, h->status));
        CUDA_TRY(Ops<double>::cols(static_cast<C *>(spec_out), static_cast<C *>(spec_out), h->logn1, M + 1,
                                   M + 1, -1, static_cast<const C *>(h->tw1), s, h->status));
    } else {
        using C = float2;
        CUDA_TRY(Ops<float>::rows_r2c(static_cast<const float *>(real_in), static_cast<C *>(spec_out),
                                      h->p.n_theta, h->logm, static_cast<const C *>(h->twm), s, h->status));
        CUDA_TRY(Ops<float>::cols(static_cast<C *>(spec_out), static_cast<C *>(spec_out), h->logn1, M + 1,
                                  M + 1, -1, static_cast<const C *>(h->tw1), s, h->status));
    }
    return FLAME_OK;
}

flame_status flame_state_from_field(flame_t h, const void *field, void *state, double *mean_mode, void *stream) {
    FLAME_RANGE("flame_state_from_field");
    if (!h || !field || !state || !mean_mode) return fail(FLAME_EINVAL, "flame_state_from_field: null pointer");
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_state_from_field: injected launch fault");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n1 = h->p.n_theta, n2 = h->p.n_phi, M = n2 / 2;
    if (h->p.prec == FLAME_FP64) {
        using C = double2;
        C *spec = static_cast<C *>(h->spec);
        CUDA_TRY(Ops<double>::rows_r2c(static_cast<const double *>(field), spec, n1, h->logm,
                                       static_cast<const C *>(h->twm), s, h->status));
        CUDA_TRY(Ops<double>::cols(spec, spec, h->logn1, M + 1, M + 1, -1, static_cast<const C *>(h->tw1), s, h->status));
        CUDA_TRY(Ops<double>::box_from_spec(spec, static_cast<C *>(state), mean_mode, n1, n2, h->p.K1, h->p.K2, s, h->status));
    } else {
        using C = float2;
        C *spec = static_cast<C *>(h->spec);
        CUDA_TRY(Ops<float>::rows_r2c(static_cast<const float *>(field), spec, n1, h->logm,
                                      static_cast<const C *>(h->twm), s, h->status));
        CUDA_TRY(Ops<float>::cols(spec, spec, h->logn1, M + 1, M + 1, -1, static_cast<const C *>(h->tw1), s, h->status));
        CUDA_TRY(Ops<float>::box_from_spec(spec, static_cast<C *>(state), mean_mode, n1, n2, h->p.K1, h->p.K2, s, h->status));
    }
    return FLAME_OK;
}

flame_status flame_fft_c2r(flame_t h, const void *spec_in, void *real_out, void *stream) {
    FLAME_RANGE("flame_fft_c2r");
    if (!h || !spec_in || !real_out) return fail(FLAME_EINVAL, "flame_fft_c2r: null pointer");
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_fft_c2r: injected launch fault");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int M = h->p.n_phi / 2;
    if (h->p.prec == FLAME_FP64) {
        using C = double2;
        CUDA_TRY(Ops<double>::cols(static_cast<const C *>(spec_in), static_cast<C *>(h->spec), h->logn1, M + 1,
                                   M + 1, 1, static_cast<const C *>(h->tw1), s, h->status));
        CUDA_TRY(Ops<double>::rows_c2r(static_cast<const C *>(h->spec), static_cast<double *>(real_out),
                                       h->p.n_theta, h->logm, static_cast<const C *>(h->twm), s, h->status));
    } else {
        using C = float2;
        CUDA_TRY(Ops<float>::cols(static_cast<const C *>(spec_in), static_cast<C *>(h->spec), h->logn1, M + 1,
                                  M + 1, 1, static_cast<const C *>(h->tw1), s, h->status));
        CUDA_TRY(Ops<float>::rows_c2r(static_cast<const C *>(h->spec), static_cast<float *>(real_out),
                                      h->p.n_theta, h->logm, static_cast<const C *>(h->twm), s, h->status));
    }
    return FLAME_OK;
}

flame_status flame_step_heun(flame_t h, void *state, double *mean_mode, double *t, int nsteps, void *stream) {
    FLAME_RANGE("flame_step_heun");
    if (!h || !state || !mean_mode || !t) return fail(FLAME_EINVAL, "flame_step_heun: null pointer");
    if (nsteps < 0) return fail(FLAME_EINVAL, "flame_step_heun: nsteps=%d < 0", nsteps);
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_step_heun: injected launch fault");
    return run_scheme(h, state, mean_mode, t, kSchemeHeun, nsteps, static_cast<cudaStream_t>(stream));
}

flame_status flame_step_if(flame_t h, void *state, double *mean_mode, double *t, int nsteps, void *stream) {
    FLAME_RANGE("flame_step_if");
    if (!h || !state || !mean_mode || !t) return fail(FLAME_EINVAL, "flame_step_if: null pointer");
    if (nsteps < 0) return fail(FLAME_EINVAL, "flame_step_if: nsteps=%d < 0", nsteps);
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_step_if: injected launch fault");
    return run_scheme(h, state, mean_mode, t, kSchemeIF, nsteps, static_cast<cudaStream_t>(stream));
}

flame_status flame_step(flame_t h, void *state, double *mean_mode, double *t, int nsteps, void *stream) {
    FLAME_RANGE("flame_step");
    if (!h || !state || !mean_mode || !t) return fail(FLAME_EINVAL, "flame_step: null pointer");
    if (nsteps < 0) return fail(FLAME_EINVAL, "flame_step: nsteps=%d < 0", nsteps);
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_step: injected launch fault");
    return run_scheme(h, state, mean_mode, t, kSchemeEuler, nsteps, static_cast<cudaStream_t>(stream));
}

flame_status flame_step_host(flame_t h, void *host_state, double *host_mean, double *host_t, int nsteps,
                             void *stream) {
    FLAME_RANGE("flame_step_host");
    if (!h || !host_state || !host_mean || !host_t) return fail(FLAME_EINVAL, "flame_step_host: null pointer");
    if (nsteps < 0) return fail(FLAME_EINVAL, "flame_step_host: nsteps=%d < 0", nsteps);
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_step_host: injected launch fault");
    if (nsteps == 0) return FLAME_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t ld1 = 2 * (size_t)h->p.K1 + 1, ncol = (size_t)h->p.K2 + 1, colb = ld1 * h->csz;
    const size_t boxb = (ncol * colb + 255) & ~(size_t)255;
    constexpr int kChunks = 8;
    if (!h->io) {
        if (cudaMalloc(&h->io, boxb + 256) != cudaSuccess) {
            cudaGetLastError();
            return fail(FLAME_ENOMEM, "flame_step_host: device allocation failed");
        }
    }
    if (!h->cpy) CUDA_TRY(cudaStreamCreateWithFlags(&h->cpy, cudaStreamNonBlocking));
    while (h->io_ev.size() < 2 * kChunks + 2) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->io_ev.push_back(e);
    }
    cudaEvent_t *ev_in = h->io_ev.data(), *ev_out = ev_in + kChunks, ev_start = ev_in[2 * kChunks],
                ev_done = ev_in[2 * kChunks + 1];
    char *dstate = static_cast<char *>(h->io);
    double *dm = reinterpret_cast<double *>(dstate + boxb), *dtm = dm + 1;
    char *hstate = static_cast<char *>(host_state);
    const bool f64 = h->p.prec == FLAME_FP64;
    int colsA = 1, quantA = 1, pairsC = 1;
    if (f64) Ops<double>::tiles(h->sa, h->var_a, &colsA, &quantA, &pairsC);
    else Ops<float>::tiles(h->sa, h->var_a, &colsA, &quantA, &pairsC);
    const int tilesA = (int)((ncol + colsA - 1) / colsA), unitsA = (tilesA + quantA - 1) / quantA;
    const int tilesC = (int)((((ncol + 1) / 2) + pairsC - 1) / pairsC);
    const int KA = std::min(kChunks, unitsA), KC = std::min(kChunks, tilesC);
    FlameDesc d = make_desc(h, dstate, dm, dtm);
    auto passA = [&](const FlameDesc &x) {
        return f64 ? Ops<double>::passA(x, s, h->var_a) : Ops<float>::passA(x, s, h->var_a, h->map());
    };
    auto passB = [&](const FlameDesc &x) {
        return f64 ? Ops<double>::passB(x, s, h->var_b) : Ops<float>::passB(x, s, h->var_b, h->gmap());
    };
    auto passC = [&](const FlameDesc &x) { return f64 ? Ops<double>::passC(x, s) : Ops<float>::passC(x, s); };
    // the copy stream starts after the work already on the caller's stream
    CUDA_TRY(cudaEventRecord(ev_start, s));
    CUDA_TRY(cudaStreamWaitEvent(h->cpy, ev_start, 0));
    CUDA_TRY(cudaMemcpyAsync(dm, host_mean, sizeof(double), cudaMemcpyHostToDevice, h->cpy));
    CUDA_TRY(cudaMemcpyAsync(dtm, host_t, sizeof(double), cudaMemcpyHostToDevice, h->cpy));
    // state in by column chunks, pass A of the first step on each as it lands
    for (int i = 0; i < KA; ++i) {
        const int u0 = (int)((long)unitsA * i / KA), u1 = (int)((long)unitsA * (i + 1) / KA);
        const int a0 = u0 * quantA, a1 = std::min(u1 * quantA, tilesA + quantA - 1);
        const size_t c0 = (size_t)a0 * colsA, c1 = std::min((size_t)a1 * colsA, ncol);
        if (c1 > c0)
            CUDA_TRY(cudaMemcpyAsync(dstate + c0 * colb, hstate + c0 * colb, (c1 - c0) * colb, cudaMemcpyHostToDevice,
                                     h->cpy));
        CUDA_TRY(cudaEventRecord(ev_in[i], h->cpy));
        CUDA_TRY(cudaStreamWaitEvent(s, ev_in[i], 0));
        FlameDesc di = d;
        di.tile0 = a0;
        di.tiles = a1 - a0;
        CUDA_TRY(passA(di));
    }
    CUDA_TRY(passB(d));
    if (nsteps > 1) {
        CUDA_TRY(passC(d));
        for (int k = 1; k + 1 < nsteps; ++k) CUDA_TRY(enqueue_step(h, d, s));
        CUDA_TRY(passA(d));
        CUDA_TRY(passB(d));
    }
    // the last pass C by column-pair chunks, each copied out as it is done;
    // tile 0 (first chunk) also finishes the mean mode and t
    for (int j = 0; j < KC; ++j) {
        const int q0 = (int)((long)tilesC * j / KC), q1 = (int)((long)tilesC * (j + 1) / KC);
        FlameDesc dj = d;
        dj.tile0 = q0;
        dj.tiles = q1 - q0;
        CUDA_TRY(passC(dj));
        CUDA_TRY(cudaEventRecord(ev_out[j], s));
        CUDA_TRY(cudaStreamWaitEvent(h->cpy, ev_out[j], 0));
        const size_t c0 = (size_t)q0 * pairsC * 2, c1 = std::min((size_t)q1 * pairsC * 2, ncol);
        if (c1 > c0)
            CUDA_TRY(cudaMemcpyAsync(hstate + c0 * colb, dstate + c0 * colb, (c1 - c0) * colb, cudaMemcpyDeviceToHost,
                                     h->cpy));
        if (j == 0) {
            CUDA_TRY(cudaMemcpyAsync(host_mean, dm, sizeof(double), cudaMemcpyDeviceToHost, h->cpy));
            CUDA_TRY(cudaMemcpyAsync(host_t, dtm, sizeof(double), cudaMemcpyDeviceToHost, h->cpy));
        }
    }
    CUDA_TRY(cudaEventRecord(ev_done, h->cpy));
    CUDA_TRY(cudaStreamWaitEvent(s, ev_done, 0));
    return FLAME_OK;
}

flame_status flame_set_record(flame_t h, double *rec, int capacity, int with_area) {
    if (!h) return fail(FLAME_EINVAL, "flame_set_record: null handle");
    if (rec && capacity < 1) return fail(FLAME_EINVAL, "flame_set_record: capacity=%d < 1", capacity);
    h->rec = rec;
    h->rec_cap = rec ? capacity : 0;
    h->rec_area = rec && with_area;
    return FLAME_OK;
}

flame_status flame_set_forcing(flame_t h, const void *forcing, double forcing0) {
    if (!h) return fail(FLAME_EINVAL, "flame_set_forcing: null handle");
    if (!std::isfinite(forcing0)) return fail(FLAME_EINVAL, "flame_set_forcing: forcing0 is not finite");
    h->forcing = forcing;
    h->forcing0 = forcing0;
    return FLAME_OK;
}

flame_status flame_step_pass(flame_t h, int pass, void *state, double *mean_mode, double *t, void *stream) {
    if (!h || !state || !mean_mode || !t) return fail(FLAME_EINVAL, "flame_step_pass: null pointer");
    if (pass < 0 || pass > 3) return fail(FLAME_EINVAL, "flame_step_pass: pass=%d not in 0..3", pass);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const FlameDesc d = make_desc(h, state, mean_mode, t);
    static const char *const names[4] = {"flame pass A", "flame pass B", "flame pass C", "flame pass CA"};
    FLAME_RANGE(names[pass]);
    if (pass == 3) {
        if (!h->fuse) return fail(FLAME_EUNSUPPORTED, "flame_step_pass: no fused column pass for this handle");
        CUDA_TRY(Ops<float>::passCA(d, s, h->map()));
        return FLAME_OK;
    }
    if (h->p.prec == FLAME_FP64)
        CUDA_TRY(pass == 0 ? Ops<double>::passA(d, s, h->var_a)
                 : pass == 1 ? Ops<double>::passB(d, s, h->var_b) : Ops<double>::passC(d, s));
    else
        CUDA_TRY(pass == 0 ? Ops<float>::passA(d, s, h->var_a, h->map())
                 : pass == 1 ? Ops<float>::passB(d, s, h->var_b, h->gmap()) : Ops<float>::passC(d, s));
    return FLAME_OK;
}

flame_status flame_step_batch(const flame_t *hs, void *const *states, double *const *mean_modes,
                              double *const *ts, int nflames, int nsteps, void *stream) {
    FLAME_RANGE("flame_step_batch");
    if (!hs || !states || !mean_modes || !ts) return fail(FLAME_EINVAL, "flame_step_batch: null pointer");
    if (nflames < 0 || nsteps < 0) return fail(FLAME_EINVAL, "flame_step_batch: negative count");
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_step_batch: injected launch fault");
    if (nflames == 0 || nsteps == 0) return FLAME_OK;
    flame_ctx *h0 = hs[0];
    if (!h0) return fail(FLAME_EINVAL, "flame_step_batch: null handle 0");
    for (int i = 0; i < nflames; ++i) {
        if (!hs[i] || !states[i] || !mean_modes[i] || !ts[i])
            return fail(FLAME_EINVAL, "flame_step_batch: null entry %d", i);
        if (hs[i]->p.prec != h0->p.prec || hs[i]->device != h0->device)
            return fail(FLAME_EINVAL, "flame_step_batch: flame %d differs in precision or device", i);
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(FLAME_EINVAL, "flame_step_batch: handle %d repeated (shared workspace)", i);
    }
    // group by grid: one launch per pass and size class
    std::map<std::vector<int>, std::vector<FlameDesc>> classes;
    std::map<std::vector<int>, const flame_ctx *> first;
    for (int i = 0; i < nflames; ++i) {
        const StepArgs &a = hs[i]->sa;
        std::vector<int> key{a.n1, a.n2, a.K1, a.K2};
        classes[key].push_back(make_desc(hs[i], states[i], mean_modes[i], ts[i]));
        if (!first.count(key)) first[key] = hs[i];
    }
    std::vector<FlameDesc> flat;
    std::vector<std::pair<size_t, size_t>> ranges;  // (offset, count) per class
    std::vector<const flame_ctx *> class_handle;
    for (auto &kv : classes) {
        ranges.emplace_back(flat.size(), kv.second.size());
        class_handle.push_back(first[kv.first]);
        flat.insert(flat.end(), kv.second.begin(), kv.second.end());
    }
    // Per-flame tensor maps for the tensor-store variants, in the order of
    // flat; with FLAME_BATCH_TMA=1 a class uses them when every flame of it
    // has both maps.  Off by default: on the ensemble's grids (256x512 ..
    // 1024x2048) the grouped direct-store kernels measured faster (1.48e11
    // against 1.44e11 grid-point updates/s for 256 uneven flames).
    std::vector<CUtensorMap> maps(2 * flat.size());
    std::vector<bool> class_maps;
    const char *bt = getenv("FLAME_BATCH_TMA");
    const bool batch_tma = bt && strcmp(bt, "1") == 0;
    {
        size_t i = 0;
        for (auto &kv : classes) {
            bool all = true;
            for (size_t j = 0; j < kv.second.size(); ++j, ++i) {
                const flame_ctx *hf = nullptr;
                for (int q = 0; q < nflames && !hf; ++q)
                    if (states[q] == flat[i].state) hf = hs[q];
                all = all && hf && hf->has_uv_map && hf->has_gk_map;
                if (hf && hf->has_uv_map) maps[i] = hf->uv_map;
                if (hf && hf->has_gk_map) maps[flat.size() + i] = hf->gk_map;
            }
            class_maps.push_back(all && batch_tma);
        }
    }
    const size_t dbytes = flat.size() * sizeof(FlameDesc);
    const size_t mofs = (dbytes + 127) & ~(size_t)127;  // maps: 64-byte aligned
    const size_t bytes = mofs + maps.size() * sizeof(CUtensorMap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool same = h0->batch_key.size() == flat.size() && memcmp(h0->batch_key.data(), flat.data(), dbytes) == 0;
    if (!same) {
        // A new binding: its graphs replace the old ones (an executable graph
        // still in flight is freed when it completes) and its descriptors
        // are uploaded on the caller's stream, after the work already
        // enqueued there.  Only growing the buffers waits for that stream.
        for (auto &g : h0->batch_graphs) cudaGraphExecDestroy(g.second);
        h0->batch_graphs.clear();
        h0->batch_key.clear();
        if (h0->batch_cap < bytes || h0->batch_host_cap < bytes) {
            CUDA_TRY(cudaStreamSynchronize(s));
            if (h0->batch_cap < bytes) {
                cudaFree(h0->batch_desc);
                h0->batch_desc = nullptr;
                h0->batch_cap = 0;
                if (cudaMalloc(&h0->batch_desc, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(FLAME_ENOMEM, "flame_step_batch: descriptor allocation failed");
                }
                h0->batch_cap = bytes;
            }
            if (h0->batch_host_cap < bytes) {
                cudaFreeHost(h0->batch_host);
                h0->batch_host = nullptr;
                h0->batch_host_cap = 0;
                if (cudaMallocHost(&h0->batch_host, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(FLAME_ENOMEM, "flame_step_batch: staging allocation failed");
                }
                h0->batch_host_cap = bytes;
            }
        } else if (h0->batch_up) {
            // the staging buffer may still feed the previous upload: wait
            // for that copy only
            CUDA_TRY(cudaEventSynchronize(h0->batch_up));
        }
        if (!h0->batch_up) CUDA_TRY(cudaEventCreateWithFlags(&h0->batch_up, cudaEventDisableTiming));
        char *hb = static_cast<char *>(h0->batch_host);
        memcpy(hb, flat.data(), dbytes);
        memcpy(hb + mofs, maps.data(), maps.size() * sizeof(CUtensorMap));
        CUDA_TRY(cudaMemcpyAsync(h0->batch_desc, hb, bytes, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaEventRecord(h0->batch_up, s));
        h0->batch_key = flat;
    }
    const FlameDesc *dev = static_cast<const FlameDesc *>(h0->batch_desc);
    const CUtensorMap *dmaps = reinterpret_cast<const CUtensorMap *>(static_cast<char *>(h0->batch_desc) + mofs);
    // FLAME_BATCH_VARIANTS=a,b: the grouped launches use these pass A and B
    // variants (in flame_tuning's numbering) instead of the variants the
    // autotuner chose for a single flame of the class's grid
    int force_a = -1, force_b = -1;
    if (const char *bv = getenv("FLAME_BATCH_VARIANTS")) {
        int fa = 0, fb = 0;
        if (sscanf(bv, "%d,%d", &fa, &fb) == 2) {
            force_a = fa;
            force_b = fb;
        }
    }
    // one pass of one size class: a grouped launch over the class's flames
    auto enqueue_pass = [&](size_t ci, int pass, cudaStream_t q) -> cudaError_t {
        const auto &rg = ranges[ci];
        const StepArgs &a = flat[rg.first].a;
        const FlameDesc *d = dev + rg.first;
        const int nf = (int)rg.second;
        const flame_ctx *hc = class_handle[ci];
        const CUtensorMap *um = class_maps[ci] ? dmaps + rg.first : nullptr;
        const CUtensorMap *gm = class_maps[ci] ? dmaps + flat.size() + rg.first : nullptr;
        const int va = force_a >= 0 ? force_a : hc->var_a_bat, vb = force_b >= 0 ? force_b : hc->var_b_bat;
        if (h0->p.prec == FLAME_FP64)
            return pass == 0 ? Ops<double>::passA_batch(d, nf, a, q, va)
                 : pass == 1 ? Ops<double>::passB_batch(d, nf, a, q, vb)
                             : Ops<double>::passC_batch(d, nf, a, q);
        return pass == 0 ? Ops<float>::passA_batch(d, nf, a, q, va, um)
             : pass == 1 ? Ops<float>::passB_batch(d, nf, a, q, vb, gm)
                         : Ops<float>::passC_batch(d, nf, a, q, va == flame::kVariantOneLine);
    };
    // n steps of every flame.  In one stream: per step and pass, one grouped
    // launch per size class.  With FLAME_BATCH_STREAMS=1 the capture forks
    // one branch per size class (its own stream, joined at the end), so that
    // the classes' passes are independent nodes of the graph and a
    // compute-bound pass of one class may run beside a memory-bound pass of
    // another.
    const char *bs = getenv("FLAME_BATCH_STREAMS");
    const bool branches = bs && strcmp(bs, "1") == 0 && ranges.size() > 1;
    auto enqueue_steps = [&](int n, cudaStream_t q) -> cudaError_t {
        cudaError_t le = cudaSuccess;
        if (!branches) {
            for (int st = 0; st < n && le == cudaSuccess; ++st)
                for (int pass = 0; pass < 3 && le == cudaSuccess; ++pass)
                    for (size_t ci = 0; ci < ranges.size() && le == cudaSuccess; ++ci) le = enqueue_pass(ci, pass, q);
            return le;
        }
        const size_t nc = ranges.size();
        while (h0->batch_streams.size() < nc) {
            cudaStream_t ns = nullptr;
            if ((le = cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking)) != cudaSuccess) return le;
            h0->batch_streams.push_back(ns);
        }
        while (h0->batch_events.size() < nc + 1) {
            cudaEvent_t ev = nullptr;
            if ((le = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return le;
            h0->batch_events.push_back(ev);
        }
        if ((le = cudaEventRecord(h0->batch_events[nc], q)) != cudaSuccess) return le;  // fork
        for (size_t ci = 0; ci < nc && le == cudaSuccess; ++ci) {
            cudaStream_t b = h0->batch_streams[ci];
            le = cudaStreamWaitEvent(b, h0->batch_events[nc], 0);
            for (int st = 0; st < n && le == cudaSuccess; ++st)
                for (int pass = 0; pass < 3 && le == cudaSuccess; ++pass) le = enqueue_pass(ci, pass, b);
            if (le == cudaSuccess) le = cudaEventRecord(h0->batch_events[ci], b);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(q, h0->batch_events[ci], 0);  // join
        }
        return le;
    };
    // graphs of kBatchChunk steps (fewer for a short call), replayed
    auto graph_of = [&](int n, cudaGraphExec_t *out) -> flame_status {
        const int key = n | (branches ? 1 << 30 : 0);  // steps and capture form
        for (auto &g : h0->batch_graphs)
            if (g.first == key) {
                *out = g.second;
                return FLAME_OK;
            }
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(h0->cap, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = enqueue_steps(n, h0->cap);
        const cudaError_t ee = cudaStreamEndCapture(h0->cap, &graph);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(FLAME_ECUDA, "flame_step_batch capture: %s", cudaGetErrorString(le != cudaSuccess ? le : ee));
        }
        const cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(FLAME_ECUDA, "flame_step_batch instantiate: %s", cudaGetErrorString(ie));
        h0->batch_graphs.emplace_back(key, *out);
        return FLAME_OK;
    };
    const int chunk = nsteps < kBatchChunk ? nsteps : kBatchChunk;
    const int full = nsteps / chunk, rest = nsteps % chunk;
    cudaGraphExec_t gfull = nullptr, grest = nullptr;
    flame_status st = graph_of(chunk, &gfull);
    if (st == FLAME_OK && rest) st = graph_of(rest, &grest);
    if (st != FLAME_OK) return st;
    for (int i = 0; i < full; ++i) CUDA_TRY(cudaGraphLaunch(gfull, s));
    if (rest) CUDA_TRY(cudaGraphLaunch(grest, s));
    return FLAME_OK;
}

flame_status flame_area(flame_t h, const void *state, const double *mean_mode, const double *t,
                        double *area_out, void *dA_dstate, double *dA_dmean, void *stream) {
    FLAME_RANGE("flame_area");
    if (!h || !state || !mean_mode || !t || !area_out) return fail(FLAME_EINVAL, "flame_area: null pointer");
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_area: injected launch fault");
    flame::AdjDesc d;
    memset(&d, 0, sizeof d);
    d.a = h->sa;
    d.state = state;
    d.mean = mean_mode;
    d.t = t;
    d.uv = h->uv;
    d.gk = h->gk;
    d.aw = h->aw;
    d.rowsum = h->rowsum;
    d.area = area_out;
    d.grad = dA_dstate;
    d.dmean = dA_dmean ? dA_dmean : h->dscal + 3;
    d.tw1 = h->tw1;
    d.twm = h->twm;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->p.prec == FLAME_FP64) CUDA_TRY(Ops<double>::area(d, s));
    else CUDA_TRY(Ops<float>::area(d, s));
    return FLAME_OK;
}

flame_status flame_adjoint(flame_t h, const void *state0, const double *mean0, const double *t_start, int nsteps,
                           int ckpt_every, const void *lambda_T, const double *lambda0_T, void *grad_state0,
                           double *grad_mean0, double *grad_gamma, void *stream) {
    FLAME_RANGE("flame_adjoint");
    if (!h || !state0 || !mean0 || !t_start || !lambda_T || !lambda0_T || !grad_state0 || !grad_mean0 || !grad_gamma)
        return fail(FLAME_EINVAL, "flame_adjoint: null pointer");
    if (nsteps < 0) return fail(FLAME_EINVAL, "flame_adjoint: nsteps=%d < 0", nsteps);
    if (nsteps > 0 && ckpt_every < 1) return fail(FLAME_EINVAL, "flame_adjoint: ckpt_every=%d < 1", ckpt_every);
    if (inject("launch")) return fail(FLAME_ECUDA, "flame_adjoint: injected launch fault");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t ld1 = 2 * (size_t)h->p.K1 + 1, ldk = (size_t)h->p.K2 + 1;
    const size_t box = ld1 * ldk * h->csz;
    const size_t k0 = (size_t)h->p.K1 * h->csz;  // byte offset of the k = 0 entry
    const int K = nsteps > 0 ? (ckpt_every < nsteps ? ckpt_every : nsteps) : 1;
    const int nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    // arena: nseg checkpoints, K trajectory states, lambda; 2 doubles each for
    // the checkpoint and trajectory (mean, t)
    const size_t nbox = (size_t)nseg + K + 1;
    const size_t need = nbox * box + 2 * ((size_t)nseg + K) * sizeof(double) + 256;
    if (h->adj_cap < need) {
        CUDA_TRY(cudaDeviceSynchronize());
        for (auto &g : h->adj_graphs) cudaGraphExecDestroy(g.exec);  // they point into the old arena
        h->adj_graphs.clear();
        cudaFree(h->adj);
        h->adj = nullptr;
        h->adj_cap = 0;
        if (cudaMalloc(&h->adj, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(FLAME_ENOMEM, "flame_adjoint: cannot allocate %zu bytes of checkpoints", need);
        }
        h->adj_cap = need;
    }
    char *base = static_cast<char *>(h->adj);
    auto ckpt = [&](int i) { return base + (size_t)i * box; };
    auto traj = [&](int i) { return base + ((size_t)nseg + i) * box; };
    char *lam = base + ((size_t)nseg + K) * box;
    double *ckm = reinterpret_cast<double *>(base + nbox * box);  // ckm[i], ckt = ckm + nseg
    double *ckt = ckm + nseg;
    double *trm = ckt + nseg;
    double *trt = trm + K;
    double *lam0 = h->dscal + 1, *dgam = h->dscal + 2;
    const bool f64 = h->p.prec == FLAME_FP64;
    auto step1 = [&](void *st, double *m, double *t, cudaStream_t q) -> cudaError_t {
        FlameDesc d = make_desc(h, st, m, t);
        d.rec = nullptr;  // the recomputed steps are not recorded
        d.rec_cap = 0;
        return enqueue_step(h, d, q);
    };
    // The forward sweep, the recomputations and the adjoint steps run on the
    // handle's arena only (the caller's inputs are copied in before, the
    // results out after), captured once per (arena, nsteps, ckpt_every) and
    // replayed as a graph: at small grids the ~10 operations per step would
    // otherwise be bound by the host's launch rate.
#define ADJ_TRY(x)                          \
    do {                                    \
        const cudaError_t e_ = (x);         \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        // forward sweep from ckpt(0): checkpoints every K steps
        for (int g = 1; g < nseg; ++g) {
            ADJ_TRY(cudaMemcpyAsync(ckpt(g), ckpt(g - 1), box, cudaMemcpyDeviceToDevice, q));
            ADJ_TRY(cudaMemcpyAsync(ckm + g, ckm + g - 1, sizeof(double), cudaMemcpyDeviceToDevice, q));
            ADJ_TRY(cudaMemcpyAsync(ckt + g, ckt + g - 1, sizeof(double), cudaMemcpyDeviceToDevice, q));
            for (int i = 0; i < K; ++i) ADJ_TRY(step1(ckpt(g), ckm + g, ckt + g, q));
        }
        // reverse sweep from lam, lam0 (the final adjoint)
        ADJ_TRY(cudaMemsetAsync(lam + k0, 0, h->csz, q));
        ADJ_TRY(cudaMemsetAsync(dgam, 0, sizeof(double), q));
        flame::AdjDesc d;
        memset(&d, 0, sizeof d);
        d.a = h->sa;
        d.lam = lam;
        d.lam_out = lam;
        d.lam0 = lam0;
        d.uv = h->uv;
        d.gk = h->gk;
        d.aw = h->aw;
        d.dgamma = dgam;
        d.tw1 = h->tw1;
        d.twm = h->twm;
        for (int g = nseg - 1; g >= 0; --g) {
            const int len = (g == nseg - 1) ? nsteps - g * K : K;
            ADJ_TRY(cudaMemcpyAsync(traj(0), ckpt(g), box, cudaMemcpyDeviceToDevice, q));
            ADJ_TRY(cudaMemcpyAsync(trm, ckm + g, sizeof(double), cudaMemcpyDeviceToDevice, q));
            ADJ_TRY(cudaMemcpyAsync(trt, ckt + g, sizeof(double), cudaMemcpyDeviceToDevice, q));
            for (int i = 1; i < len; ++i) {
                ADJ_TRY(cudaMemcpyAsync(traj(i), traj(i - 1), box, cudaMemcpyDeviceToDevice, q));
                ADJ_TRY(cudaMemcpyAsync(trm + i, trm + i - 1, sizeof(double), cudaMemcpyDeviceToDevice, q));
                ADJ_TRY(cudaMemcpyAsync(trt + i, trt + i - 1, sizeof(double), cudaMemcpyDeviceToDevice, q));
                ADJ_TRY(step1(traj(i), trm + i, trt + i, q));
            }
            for (int i = len - 1; i >= 0; --i) {
                d.state = traj(i);
                d.t = trt + i;
                if (f64) ADJ_TRY(Ops<double>::adj_step(d, q));
                else ADJ_TRY(Ops<float>::adj_step(d, q));
            }
        }
        return cudaSuccess;
    };
#undef ADJ_TRY
    if (nseg == 0) {  // no step: the gradient is the final adjoint
        CUDA_TRY(cudaMemcpyAsync(grad_state0, lambda_T, box, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(grad_mean0, lambda0_T, sizeof(double), cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemsetAsync(grad_gamma, 0, sizeof(double), s));
        return FLAME_OK;
    }
    // the forward recomputations include the forcing in force (constant
    // forcing leaves the step's Jacobian, hence the adjoint step, unchanged)
    size_t f0bits = 0;
    memcpy(&f0bits, &h->forcing0, sizeof f0bits);
    const std::vector<const void *> key{h->adj, reinterpret_cast<const void *>((size_t)nsteps),
                                        reinterpret_cast<const void *>((size_t)ckpt_every), h->forcing,
                                        reinterpret_cast<const void *>(f0bits)};
    cudaGraphExec_t exec = nullptr;
    for (auto &g : h->adj_graphs)
        if (g.key == key) exec = g.exec;
    if (!exec) {
        if (h->adj_graphs.size() >= 4) {
            CUDA_TRY(retire_graph(h, h->adj_graphs.front().exec));
            h->adj_graphs.erase(h->adj_graphs.begin());
        }
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = enqueue(h->cap);
        const cudaError_t ee = cudaStreamEndCapture(h->cap, &graph);
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(FLAME_ECUDA, "flame_adjoint: graph capture failed: %s",
                        cudaGetErrorString(le != cudaSuccess ? le : ee));
        }
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(FLAME_ECUDA, "flame_adjoint: graph instantiate: %s", cudaGetErrorString(ie));
        h->adj_graphs.push_back(flame_ctx::AdjGraph{key, exec});
    }
    CUDA_TRY(cudaMemcpyAsync(ckpt(0), state0, box, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ckm, mean0, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ckt, t_start, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(lam, lambda_T, box, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(lam0, lambda0_T, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaGraphLaunch(exec, s));
    CUDA_TRY(cudaMemcpyAsync(grad_state0, lam, box, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(grad_mean0, lam0, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(grad_gamma, dgam, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return FLAME_OK;
}

flame_status flame_debug_bounds_probe(flame_t h, int index, int extent, void *stream) {
    if (!h) return fail(FLAME_EINVAL, "flame_debug_bounds_probe: null handle");
    const cudaError_t e = flame::bounds_probe(h->status, index, extent, static_cast<cudaStream_t>(stream));
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        return fail(FLAME_EUNSUPPORTED, "flame_debug_bounds_probe: not an index-checking build");
    }
    CUDA_TRY(e);
    return FLAME_OK;
}

flame_status flame_sync_status(flame_t h) {
    if (!h) return fail(FLAME_EINVAL, "flame_sync_status: null handle");
    CUDA_TRY(cudaDeviceSynchronize());
    int v[flame::kStatusWords] = {0, 0, 0, 0};
    CUDA_TRY(cudaMemcpy(v, h->status, sizeof v, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(h->status, 0, sizeof v));
    if (v[0] & (1 << flame::kStatusBounds))
        return fail(FLAME_EBOUNDS, "index check failed at site %d: index %d not in [0, %d) (the access was skipped)",
                    v[1], v[2], v[3]);
    if (v[0] & (1 << flame::kStatusTimeout)) return fail(FLAME_ETIMEOUT, "a device-side wait timed out");
    if (v[0] & (1 << flame::kStatusNonfinite)) return fail(FLAME_ENONFINITE, "a step produced NaN or Inf");
    return FLAME_OK;
}

}  // extern "C"
