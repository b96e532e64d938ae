// Host runtime behind the C ABI of include/hji.h: grid handles, validation,
// device buffers, the per-solve set-up, the tile list, and the march loop.
//
// The march runs as CUDA graphs of `check_every` steps (every RK stage of
// every grid in the batch is one persistent kernel launch over the shared
// tile list).  Kernels skip the tiles of grids that have stopped, so the host
// keeps one graph in flight ahead of the one it checks; it reads a single
// device counter of still-marching grids per graph and never syncs per step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "hji_common.cuh"

using hji::InstDesc;
using hji::InstState;

namespace hji {

// TMA descriptors of an instance's fields.  The encoder comes from the
// driver through the runtime's entry-point lookup (no link against the
// driver library).  Dimensions are listed fastest first with the true node
// counts, so a box reaching past the grid reads zeros there; row strides use
// the padded pitch.
bool encode_maps(InstDesc& D, bool f32, int scheme, int variant, const char** why) {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    if (!encode) {
        *why = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    const int nd = D.ndim;
    int TY, TX;
    tile_dims(nd, variant, TY, TX);
    const int G = ghost_width(scheme);
    const int GY = nd >= 2 ? G : 0;
    const size_t es = f32 ? 4 : 8;
    cuuint64_t dims[MAXD], strides[MAXD];
    for (int i = 0; i < nd; ++i) dims[i] = (cuuint64_t)D.n[nd - 1 - i];
    for (int i = 1; i < nd; ++i) strides[i - 1] = (cuuint64_t)D.stride[nd - 1 - i] * es;
    const cuuint32_t wbox[MAXD] = {(cuuint32_t)(TX + 8), (cuuint32_t)(TY + 2 * GY), 1, 1};
    const cuuint32_t nbox[MAXD] = {(cuuint32_t)TX, (cuuint32_t)TY, 1, 1};
    const cuuint32_t estr[MAXD] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    auto enc = [&](int slot, const void* ptr, const cuuint32_t* box) {
        if (!ptr) {
            std::memset(&D.tm[slot], 0, sizeof(CUtensorMap));
            return true;
        }
        const CUresult r = encode(&D.tm[slot], dt, (cuuint32_t)nd, const_cast<void*>(ptr), dims, strides,
                                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            *why = "cuTensorMapEncodeTiled rejected a field";
            return false;
        }
        return true;
    };
    bool ok = enc(TM_WIN_V0, D.V[0], wbox) && enc(TM_WIN_V1, D.V[1], wbox) &&
              enc(TM_WIN_W1, D.W1, wbox) && enc(TM_WIN_W2, D.W2, wbox) && enc(TM_NODE_L, D.l, nbox);
    if (f32) {
        ok = ok && enc(TM_WIN_LO0, D.Vlo[0], wbox) && enc(TM_WIN_LO1, D.Vlo[1], wbox);
        std::memset(&D.tm[TM_NODE_V0], 0, 2 * sizeof(CUtensorMap));
    } else {
        ok = ok && enc(TM_NODE_V0, D.V[0], nbox) && enc(TM_NODE_V1, D.V[1], nbox);
        std::memset(&D.tm[TM_WIN_LO0], 0, 2 * sizeof(CUtensorMap));
    }
    return ok;
}

}  // namespace hji

struct hji_grid_s {
    int ndim = 0;
    int64_t n[HJI_MAX_DIM] = {1, 1, 1, 1};
    double lo[HJI_MAX_DIM] = {0, 0, 0, 0};
    double hi[HJI_MAX_DIM] = {0, 0, 0, 0};
    double dx[HJI_MAX_DIM] = {1, 1, 1, 1};
    int periodic[HJI_MAX_DIM] = {0, 0, 0, 0};
    hji_precision prec = HJI_F64;
    size_t esize = 8;
    int64_t ncells = 0;
    int64_t pitch = 0;               // padded length of the fastest axis (elements)
    int64_t nalloc = 0;              // elements of one field: pitch x (rows of the other axes)
    int device = 0;
    bool has_alloc = false;
    hji_allocator alloc{};
    void* V[2] = {nullptr, nullptr};
    void* W1 = nullptr;
    void* W2 = nullptr;
    void* Vlo[2] = {nullptr, nullptr};  // FP32 grids: low words of the compensated value (with V[])
    void* l = nullptr;
    void* snap = nullptr;            // snapshot of V for the interval test (allocated on first use)
    void* table = nullptr;
    size_t table_bytes = 0;
    InstState* state = nullptr;      // device
    InstDesc* d_desc = nullptr;      // descriptors of the solves this grid leads
    int desc_cap = 0;
    int* d_active = nullptr;         // device counter for single-grid solves
    unsigned long long* d_tiles = nullptr;
    size_t tiles_cap = 0;
    int* d_ntiles = nullptr;
    int* h_active = nullptr;         // pinned host mirrors
    InstState* h_state = nullptr;
    bool has_dyn = false;
    hji::Dyn dyn{};
    bool has_value = false;
    int cur = 0;
    std::string err;
    // Graph cache for single-grid solves.
    cudaGraphExec_t graph = nullptr;
    long long graph_key[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    cudaStream_t cap_stream = nullptr;
};

struct hji_engine_s {
    int ndim = 0;
    bool has_alloc = false;
    hji_allocator alloc{};            // device allocations of the engine's own buffers
    hji_precision prec = HJI_F64;
    hji_solve_opts o{};
    int chunk = 32;
    int max_slots = 0;
    size_t budget = 0;
    size_t in_use = 0;
    cudaStream_t s = nullptr;
    cudaStream_t cap = nullptr;
    InstDesc* d_desc = nullptr;       // max_slots descriptors
    int* d_counts = nullptr;          // [0] marching instances, [1] tiles in the list
    unsigned long long* d_tiles = nullptr;
    size_t tiles_cap = 0;
    int* h_counts = nullptr;          // pinned mirror of d_counts
    cudaGraphExec_t graph = nullptr;
    int grid[2] = {0, 0};  // CTAs of the stage launches (non-last, last)
    int variant = 0;
    cudaEvent_t ev = nullptr;
    bool inflight = false;
    int launched_active = 0;          // instances marching when the chunk was launched
    struct Slot {
        bool used = false;
        hji_grid g = nullptr;
        int64_t tag = 0;
        size_t bytes = 0;
        hji_init init = HJI_INIT_STANDARD;
        std::chrono::steady_clock::time_point t0;
    };
    struct Req {
        hji_grid g;
        int64_t tag;
        hji_init init;
        bool has_k;
    };
    struct Done {
        int64_t tag;
        hji_solve_stats st;
        hji_status status;
    };
    std::vector<Slot> slots;
    std::vector<InstDesc> h_desc;
    std::deque<Req> queue;
    std::vector<Done> done;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

hji_status fail(hji_grid g, hji_status s, const std::string& msg) {
    if (g) g->err = msg;
    else g_create_error = msg;
    return s;
}

hji_status cuda_fail(hji_grid g, cudaError_t e, const char* where) {
    return fail(g, HJI_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HJI_CUDA(g, call)                                        \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((g), e_, #call); \
    } while (0)

void* dev_alloc(hji_grid g, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (g->has_alloc) return g->alloc.alloc(bytes, s, g->alloc.ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(hji_grid g, void* p, cudaStream_t s) {
    if (!p) return;
    if (g->has_alloc) g->alloc.free(p, s, g->alloc.ctx);
    else cudaFreeAsync(p, s);
}

// Copies between a dense C-order array (rows of n[ndim-1] elements) and a
// grid field whose rows are padded to the grid's pitch.
cudaError_t copy_rows(hji_grid g, void* dst, size_t dpitch, const void* src, size_t spitch,
                      cudaMemcpyKind kind, cudaStream_t s) {
    const size_t w = (size_t)g->n[g->ndim - 1] * g->esize;
    const size_t rows = (size_t)(g->nalloc / g->pitch);
    if (rows == 1 || (dpitch == w && spitch == w)) return cudaMemcpyAsync(dst, src, w * rows, kind, s);
    if (dpitch < (1ull << 31) && spitch < (1ull << 31))
        return cudaMemcpy2DAsync(dst, dpitch, src, spitch, w, rows, kind, s);
    cudaError_t e = cudaSuccess;  // rows too long for a 2-D copy: few of them
    for (size_t r = 0; r < rows && e == cudaSuccess; ++r)
        e = cudaMemcpyAsync(static_cast<char*>(dst) + r * dpitch,
                            static_cast<const char*>(src) + r * spitch, w, kind, s);
    return e;
}
cudaError_t copy_in(hji_grid g, void* field, const void* dense, cudaMemcpyKind kind, cudaStream_t s) {
    return copy_rows(g, field, (size_t)g->pitch * g->esize, dense,
                     (size_t)g->n[g->ndim - 1] * g->esize, kind, s);
}
cudaError_t copy_out(hji_grid g, void* dense, const void* field, cudaMemcpyKind kind, cudaStream_t s) {
    return copy_rows(g, dense, (size_t)g->n[g->ndim - 1] * g->esize, field,
                     (size_t)g->pitch * g->esize, kind, s);
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
    }
    return sms;
}

bool finite_all(const double* p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

struct StagePlan {
    int in, out;
    double aV, aE;
    bool last;
};

int rk_plan(int rk, StagePlan* p) {
    if (rk == 1) {
        p[0] = {0, 3, 0.0, 1.0, true};
        return 1;
    }
    if (rk == 2) {
        p[0] = {0, 1, 0.0, 1.0, false};
        p[1] = {1, 3, 0.5, 0.5, true};
        return 2;
    }
    p[0] = {0, 1, 0.0, 1.0, false};
    p[1] = {1, 2, 0.75, 0.25, false};
    p[2] = {2, 3, 1.0 / 3.0, 2.0 / 3.0, true};
    return 3;
}

// Kernel flavours beyond the default stage kernel.
constexpr int kFlavorInterval = 1;  // last stage with Sec. V's interval test
constexpr int kFlavorLocalLF = 2;   // local Lax-Friedrichs (interval test included)

int flavor_of(const hji_solve_opts* o) {
    return (o->interval > 0.0 ? kFlavorInterval : 0) | (o->local_lf ? kFlavorLocalLF : 0);
}

hji::StageLauncher launcher(bool f32, int ndim, int scheme, bool last, int variant, int flavor) {
    if (flavor & kFlavorLocalLF)
        return f32 ? hji::stage_launcher_llf_f32(ndim, scheme, last)
                   : hji::stage_launcher_llf_f64(ndim, scheme, last);
    const bool interval = (flavor & kFlavorInterval) != 0;
    return f32 ? hji::stage_launcher_f32(ndim, scheme, last, variant, interval)
               : hji::stage_launcher_f64(ndim, scheme, last, variant, interval);
}

// CTAs of one stage launch: as many as fit on every SM at once (each stage
// kernel has its own occupancy), at most one per tile.
int stage_grid(bool f32, int ndim, int scheme, long long total_tiles, int variant, bool last,
               int flavor) {
    const bool interval = (flavor & kFlavorInterval) != 0;
    const int b = (flavor & kFlavorLocalLF)
                      ? (f32 ? hji::stage_max_blocks_llf_f32(ndim, scheme, last)
                             : hji::stage_max_blocks_llf_f64(ndim, scheme, last))
                      : (f32 ? hji::stage_max_blocks_f32(ndim, scheme, last, variant, interval)
                             : hji::stage_max_blocks_f64(ndim, scheme, last, variant, interval));
    long long g = (long long)num_sms() * b;
    if (g > total_tiles) g = total_tiles;
    return g < 1 ? 1 : (int)g;
}

// AUTO takes the multi-step launch when a stage has at least this many
// tiles per resident CTA.
constexpr long long kMultiStepTilesPerCta = 4;

// ---- tile-shape choices made by hji_autotune, per problem class ----
std::mutex g_tune_mu;
std::map<std::vector<long long>, int> g_tune;
// Set only while hji_autotune times a variant (on the calling thread).
thread_local int g_force_variant = -1;
// Set only while hji_stage_times runs its march (on the calling thread):
// where the per-stage kernel durations go.
struct StageTimer {
    double ms[3];
    int ns;
};
thread_local StageTimer* g_stage_timer = nullptr;

int size_bucket(long long cells) {
    int b = 0;
    while (cells > 1) {
        cells >>= 1;
        ++b;
    }
    return b;
}

std::vector<long long> tune_key(hji_precision prec, int ndim, const hji_solve_opts* o, int bucket) {
    return {(long long)prec, ndim, (long long)o->scheme, o->rk_order, bucket};
}

// The tile shape for a launch: the autotuned choice for this class (the
// nearest tuned size bucket), else variant 0.
int pick_variant(hji_precision prec, int ndim, const hji_solve_opts* o, long long cells) {
    if (ndim != 2) return 0;
    if (g_force_variant >= 0) return g_force_variant;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int b = size_bucket(cells);
    int best = 0, dist = 1 << 30;
    for (const auto& kv : g_tune) {
        const auto& k = kv.first;
        if (k[0] != (long long)prec || k[1] != ndim || k[2] != (long long)o->scheme || k[3] != o->rk_order)
            continue;
        const int d = (int)(k[4] > b ? k[4] - b : b - k[4]);
        if (d < dist) {
            dist = d;
            best = kv.second;
        }
    }
    return best;
}

void tile_grid(int ndim, const int64_t* n, long long& tx, long long& ty, long long& planes,
               int variant) {
    int TY, TX;
    hji::tile_dims(ndim, variant, TY, TX);
    tx = (n[ndim - 1] + TX - 1) / TX;
    ty = ndim >= 2 ? (n[ndim - 2] + TY - 1) / TY : 1;
    planes = 1;
    for (int a = 0; a < ndim - 2; ++a) planes *= n[a];
}

hji_status validate_opts(hji_grid g, const hji_solve_opts* o) {
    if (!o) return fail(g, HJI_E_INVALID, "opts is NULL");
    if (o->scheme != HJI_ENO1 && o->scheme != HJI_ENO2 && o->scheme != HJI_WENO5)
        return fail(g, HJI_E_INVALID, "unknown scheme");
    if (o->rk_order < 1 || o->rk_order > 3) return fail(g, HJI_E_INVALID, "rk_order must be 1, 2 or 3");
    if (!(o->cfl > 0.0 && o->cfl <= 1.0)) return fail(g, HJI_E_INVALID, "cfl must be in (0, 1]");
    if (!(o->tol >= 0.0) || !std::isfinite(o->tol)) return fail(g, HJI_E_INVALID, "tol must be finite and >= 0");
    if (!(o->horizon >= 0.0) || !std::isfinite(o->horizon))
        return fail(g, HJI_E_INVALID, "horizon must be finite and >= 0");
    if (o->init != HJI_INIT_STANDARD && o->init != HJI_INIT_USER_K && o->init != HJI_INIT_RESIDENT)
        return fail(g, HJI_E_INVALID, "unknown init mode");
    if (!(o->tol_rate >= 0.0) || !std::isfinite(o->tol_rate))
        return fail(g, HJI_E_INVALID, "tol_rate must be finite and >= 0");
    if (o->tile_variant < 0 || o->tile_variant > hji::kTileVariants)
        return fail(g, HJI_E_INVALID, "tile_variant must be 0..HJI_TILE_VARIANTS");
    if (o->march < HJI_MARCH_AUTO || o->march > HJI_MARCH_MULTI_STEP)
        return fail(g, HJI_E_INVALID, "unknown march mode");
    if (!(o->interval >= 0.0) || !std::isfinite(o->interval) || !(o->interval_tol >= 0.0) ||
        !std::isfinite(o->interval_tol))
        return fail(g, HJI_E_INVALID, "interval and interval_tol must be finite and >= 0");
    if ((o->brs != 0 && o->brs != 1) || (o->local_lf != 0 && o->local_lf != 1))
        return fail(g, HJI_E_INVALID, "brs and local_lf must be 0 or 1");
    if (!(o->discount >= 0.0 && o->discount <= 1.0))
        return fail(g, HJI_E_INVALID, "discount must be in [0, 1] (0 and 1: off)");
    if (o->brs && o->discount > 0.0 && o->discount < 1.0)
        return fail(g, HJI_E_INVALID, "discount applies to the projected march, not to brs");
    return HJI_OK;
}

// Make sure the stage buffers, the interval test's snapshot and the term
// table exist for this solve.
hji_status ensure_buffers(hji_grid g, int rk, cudaStream_t s, bool snapshot) {
    const size_t bytes = (size_t)g->nalloc * g->esize;
    if (snapshot && !g->snap) {
        g->snap = dev_alloc(g, bytes, s);
        if (!g->snap) return fail(g, HJI_E_NOMEM, "snapshot buffer allocation failed");
    }
    if (rk >= 2 && !g->W1) {
        g->W1 = dev_alloc(g, bytes, s);
        if (!g->W1) return fail(g, HJI_E_NOMEM, "stage buffer allocation failed");
    }
    if (rk >= 3 && !g->W2) {
        g->W2 = dev_alloc(g, bytes, s);
        if (!g->W2) return fail(g, HJI_E_NOMEM, "stage buffer allocation failed");
    }
    long long nmax = 0;
    for (int a = 0; a < g->ndim; ++a) nmax = g->n[a] > nmax ? g->n[a] : nmax;
    const size_t tb = (size_t)HJI_MAX_TERMS * nmax * g->esize;
    if (!g->table) {
        g->table = dev_alloc(g, tb, s);
        if (!g->table) return fail(g, HJI_E_NOMEM, "table allocation failed");
        g->table_bytes = tb;
    }
    return HJI_OK;
}

// Element strides of a grid's fields: C order, the fastest axis padded to
// `pitch`.
void field_strides(int ndim, const int64_t* n, long long pitch, long long* stride) {
    long long s = 1;
    for (int a = ndim - 1; a >= 0; --a) {
        stride[a] = s;
        s *= (a == ndim - 1) ? pitch : n[a];
    }
}

hji_status make_desc(hji_grid g, const hji_solve_opts* o, int* active, int variant, InstDesc& D) {
    std::memset(&D, 0, sizeof(D));
    D.ndim = g->ndim;
    for (int a = HJI_MAX_DIM - 1; a >= 0; --a) {
        D.n[a] = (int)g->n[a];
        D.periodic[a] = g->periodic[a];
        D.lo[a] = g->lo[a];
        D.dx[a] = g->dx[a];
    }
    field_strides(g->ndim, g->n, g->pitch, D.stride);
    D.ncells = g->ncells;
    D.nalloc = g->nalloc;
    D.dyn = g->dyn;
    D.cfl = o->cfl;
    D.tol = o->tol;
    D.tol_rate = o->tol_rate;
    D.interval = o->interval;
    D.interval_tol = o->interval_tol;
    D.snap = o->interval > 0.0 ? g->snap : nullptr;
    D.brs = o->brs;
    D.local_lf = o->local_lf;
    D.discount = o->discount;
    D.horizon = o->horizon;
    D.max_steps = o->max_steps > 0 ? o->max_steps : 1000000;
    D.V[0] = g->V[0];
    D.V[1] = g->V[1];
    D.W1 = g->W1;
    D.W2 = g->W2;
    D.Vlo[0] = g->Vlo[0];
    D.Vlo[1] = g->Vlo[1];
    D.l = g->l;
    D.table = g->table;
    long long nmax = 0;
    for (int a = 0; a < g->ndim; ++a) nmax = g->n[a] > nmax ? g->n[a] : nmax;
    D.table_stride = nmax;
    D.history = nullptr;
    D.history_len = 0;
    long long tx, ty, planes;
    tile_grid(g->ndim, g->n, tx, ty, planes, variant);
    D.tiles_x = tx;
    D.tiles_y = ty;
    D.tiles_per_plane = tx * ty;
    D.ntiles = tx * ty * planes;
    D.state = g->state;
    D.active = active;
    const char* why = nullptr;
    if (!hji::encode_maps(D, g->prec == HJI_F32, o->scheme, variant, &why))
        return fail(g, HJI_E_CUDA, std::string("tensor map: ") + why);
    return HJI_OK;
}

// Capture `steps` steps of the march (all RK stages) into a graph.
hji_status capture_chunk(hji_grid g, cudaStream_t cap, bool f32, int ndim, int scheme, int rk,
                         int steps, const hji::StageArgs& base, const int* grid, int variant,
                         int flavor, cudaGraphExec_t* out) {
    StagePlan plan[3];
    const int ns = rk_plan(rk, plan);
    hji::StageLauncher L[3];
    for (int i = 0; i < ns; ++i) {
        L[i] = launcher(f32, ndim, scheme, plan[i].last, variant, flavor);
        if (!L[i]) return fail(g, HJI_E_INVALID, "no kernel for this ndim/scheme");
    }
    HJI_CUDA(g, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < steps && e == cudaSuccess; ++s) {
        for (int i = 0; i < ns && e == cudaSuccess; ++i) {
            hji::StageArgs a = base;
            a.stage_in = plan[i].in;
            a.stage_out = plan[i].out;
            a.aV = plan[i].aV;
            a.aE = plan[i].aE;
            a.aVf = (float)plan[i].aV;
            a.aEf = (float)plan[i].aE;
            a.reads_v = plan[i].aV != 0.0 ? 1 : 0;
            e = L[i](a, grid[plan[i].last ? 1 : 0], cap);
        }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(g, e, "stage launch during capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(g, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaGraphInstantiate");
    return HJI_OK;
}

// Capture one multi-step march launch (every stage of `steps` steps, with
// grid-wide barriers) into a graph: the barrier counter is zeroed first.
hji_status capture_march(hji_grid g, cudaStream_t cap, bool f32, int ndim, int scheme, int rk,
                         int steps, const hji::StageArgs& base, int grid, int variant,
                         bool interval, const int* active, unsigned* barrier, int* fault,
                         cudaGraphExec_t* out) {
    hji::MarchLauncher L = f32 ? hji::march_launcher_f32(ndim, scheme, variant, interval)
                               : hji::march_launcher_f64(ndim, scheme, variant, interval);
    if (!L) return fail(g, HJI_E_INVALID, "no march kernel for this ndim/scheme");
    StagePlan plan[3];
    const int ns = rk_plan(rk, plan);
    hji::MarchArgs m;
    std::memset(&m, 0, sizeof(m));
    for (int i = 0; i < ns; ++i) {
        hji::StageArgs a = base;
        a.stage_in = plan[i].in;
        a.stage_out = plan[i].out;
        a.aV = plan[i].aV;
        a.aE = plan[i].aE;
        a.aVf = (float)plan[i].aV;
        a.aEf = (float)plan[i].aE;
        a.reads_v = plan[i].aV != 0.0 ? 1 : 0;
        m.st[i] = a;
    }
    m.ns = ns;
    m.steps = steps;
    m.barrier = barrier;
    m.active = active;
    m.fault = fault;
    HJI_CUDA(g, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(barrier, 0, sizeof(unsigned), cap);
    if (e == cudaSuccess) e = L(m, grid, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(g, e, "march launch during capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(g, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(g, e, "cudaGraphInstantiate");
    return HJI_OK;
}

// The march of hji_stage_times: o->max_steps steps, each stage kernel
// launched on its own between two events (no graph, no convergence check),
// every event recorded before one synchronisation; the mean duration of each
// RK stage's kernel goes to T.
cudaError_t timed_march(const hji_solve_opts* o, bool f32, int ndim, const hji::StageArgs& base,
                        const int* grid, int variant, cudaStream_t s, StageTimer* T) {
    StagePlan plan[3];
    const int ns = rk_plan(o->rk_order, plan);
    hji::StageLauncher Lk[3];
    for (int i = 0; i < ns; ++i) {
        Lk[i] = launcher(f32, ndim, o->scheme, plan[i].last, variant, flavor_of(o));
        if (!Lk[i]) return cudaErrorInvalidValue;
    }
    const int steps = o->max_steps;
    std::vector<cudaEvent_t> ev(2 * (size_t)ns * steps, nullptr);
    cudaError_t e = cudaSuccess;
    size_t made = 0;
    for (; made < ev.size() && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e != cudaSuccess) --made;
    for (int st = 0; st < steps && e == cudaSuccess; ++st) {
        for (int i = 0; i < ns && e == cudaSuccess; ++i) {
            hji::StageArgs a = base;
            a.stage_in = plan[i].in;
            a.stage_out = plan[i].out;
            a.aV = plan[i].aV;
            a.aE = plan[i].aE;
            a.aVf = (float)plan[i].aV;
            a.aEf = (float)plan[i].aE;
            a.reads_v = plan[i].aV != 0.0 ? 1 : 0;
            const size_t k = 2 * ((size_t)st * ns + i);
            e = cudaEventRecord(ev[k], s);
            if (e == cudaSuccess) e = Lk[i](a, grid[plan[i].last ? 1 : 0], s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[k + 1], s);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int i = 0; i < 3; ++i) T->ms[i] = 0.0;
    T->ns = ns;
    for (int st = 0; st < steps && e == cudaSuccess; ++st) {
        for (int i = 0; i < ns && e == cudaSuccess; ++i) {
            const size_t k = 2 * ((size_t)st * ns + i);
            float ms = 0.0f;
            e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            T->ms[i] += ms / steps;
        }
    }
    for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    return e;
}

// The march shared by hji_solve (count == 1) and hji_batch_solve.
hji_status run(int count, hji_grid* grids, const void* const* l, const void* const* k,
               int ptr_is_device, const hji_solve_opts* o, cudaStream_t s, hji_solve_stats* stats) {
    const auto t0 = std::chrono::steady_clock::now();
    hji_grid g0 = grids[0];
    hji_status st = validate_opts(g0, o);
    if (st != HJI_OK) return st;
    const bool f32 = g0->prec == HJI_F32;
    const int ndim = g0->ndim;
    const int gw = hji::ghost_width(o->scheme);
    for (int i = 0; i < count; ++i) {
        hji_grid g = grids[i];
        if (!g) return fail(g0, HJI_E_INVALID, "NULL grid in batch");
        if (g->prec != g0->prec || g->ndim != ndim)
            return fail(g0, HJI_E_INVALID, "grids of a batch must share precision and ndim");
        if (!g->has_dyn) return fail(g, HJI_E_STATE, "dynamics not set");
        if (!l || !l[i]) return fail(g, HJI_E_INVALID, "l is NULL");
        for (int a = 0; a < ndim; ++a)
            if (g->n[a] < 2 * gw + 1)
                return fail(g, HJI_E_INVALID, "grid too small for the scheme's stencil");
        if (o->init == HJI_INIT_USER_K && (!k || !k[i]))
            return fail(g, HJI_E_INVALID, "HJI_INIT_USER_K needs k");
        if (o->init == HJI_INIT_RESIDENT && !g->has_value)
            return fail(g, HJI_E_STATE, "HJI_INIT_RESIDENT without a previous value");
        for (int j = 0; j < i; ++j)
            if (grids[j] == g) return fail(g0, HJI_E_INVALID, "grid listed twice in a batch");
        st = ensure_buffers(g, o->rk_order, s, o->interval > 0.0);
        if (st != HJI_OK) return st;
    }
    const cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

    // The tile shape for this launch (autotuned per class, else variant 0).
    long long cells_all = 0;
    for (int i = 0; i < count; ++i) cells_all += grids[i]->ncells;
    int variant = pick_variant(g0->prec, ndim, o, cells_all / count);
    if (o->tile_variant > 0 && g_force_variant < 0)
        variant = (ndim == 2 && o->tile_variant <= hji::kTileVariants) ? o->tile_variant - 1 : 0;
    if (o->local_lf) variant = 0;  // the local-dissipation kernels have the default shape
    // Launch-wide device scratch (descriptors, tile list, counters) lives on
    // the first grid and is reused (grown on demand) by every solve it leads,
    // together with the captured graph of a chunk.
    std::vector<InstDesc> H(count);
    long long total_tiles = 0;
    for (int i = 0; i < count; ++i) {
        long long tx, ty, planes;
        tile_grid(ndim, grids[i]->n, tx, ty, planes, variant);
        total_tiles += tx * ty * planes;
    }
    if (total_tiles >= (1ll << 31)) return fail(g0, HJI_E_INVALID, "too many tiles");
    auto drop_graph = [&]() {
        if (g0->graph) {
            cudaGraphExecDestroy(g0->graph);
            g0->graph = nullptr;
        }
    };
    if (g0->desc_cap < count) {
        dev_free(g0, g0->d_desc, s);
        g0->d_desc = (InstDesc*)dev_alloc(g0, sizeof(InstDesc) * count, s);
        g0->desc_cap = g0->d_desc ? count : 0;
        drop_graph();
        if (!g0->d_desc) return fail(g0, HJI_E_NOMEM, "descriptor allocation failed");
    }
    if (g0->tiles_cap < (size_t)total_tiles) {
        dev_free(g0, g0->d_tiles, s);
        g0->d_tiles = (unsigned long long*)dev_alloc(g0, sizeof(unsigned long long) * total_tiles, s);
        g0->tiles_cap = g0->d_tiles ? (size_t)total_tiles : 0;
        drop_graph();
        if (!g0->d_tiles) return fail(g0, HJI_E_NOMEM, "tile list allocation failed");
    }
    InstDesc* d_desc = g0->d_desc;
    int* d_active = g0->d_active;
    int* d_ntiles = g0->d_ntiles;
    unsigned long long* d_tiles = g0->d_tiles;
    auto cleanup = [&]() {};

    std::vector<const void*> kptr(count, nullptr);
    std::vector<const void*> kptr_lo(count, nullptr);
    std::vector<unsigned long long> tiles;
    tiles.reserve((size_t)total_tiles);
    for (int i = 0; i < count; ++i) {
        hji_grid g = grids[i];
        cudaError_t e = copy_in(g, g->l, l[i], kind, s);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(g, e, "copy of l");
        }
        if (o->init == HJI_INIT_USER_K) {
            e = copy_in(g, g->V[1], k[i], kind, s);
            if (e != cudaSuccess) {
                cleanup();
                return cuda_fail(g, e, "copy of k");
            }
            kptr[i] = g->V[1];
        } else if (o->init == HJI_INIT_RESIDENT) {
            kptr[i] = g->V[g->cur];
            kptr_lo[i] = g->Vlo[g->cur];
        }
        st = make_desc(g, o, d_active, variant, H[i]);
        if (st != HJI_OK) return st;
        H[i].kinit = kptr[i];
        H[i].kinit_lo = kptr_lo[i];
        for (long long t = 0; t < H[i].ntiles; ++t) tiles.push_back(hji::make_tile(i, t));
        e = cudaMemsetAsync(g->state, 0, sizeof(InstState), s);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(g, e, "state reset");
        }
    }
    int counts[2] = {count, (int)total_tiles};
    cudaError_t e = cudaMemcpyAsync(d_desc, H.data(), sizeof(InstDesc) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(unsigned long long) * total_tiles,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_active, &counts[0], sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ntiles, &counts[1], sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = hji::launch_setup(d_desc, H.data(), count, f32, s);
    if (e == cudaSuccess) e = hji::launch_init(d_desc, H.data(), count, f32, s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(g0, e, "set-up");
    }
    // One sync after set-up: reject NaN/Inf inputs and dynamics without a finite dt.
    for (int i = 0; i < count; ++i) {
        e = cudaMemcpyAsync(&grids[i]->h_state[0], grids[i]->state, sizeof(InstState),
                            cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(g0, e, "set-up sync");
    }
    for (int i = 0; i < count; ++i) {
        const InstState& S = grids[i]->h_state[0];
        if (S.nonfinite) {
            cleanup();
            return fail(grids[i], HJI_E_INVALID, "l or k contains NaN or Inf");
        }
        if (S.status == 2) {
            cleanup();
            return fail(grids[i], HJI_E_INVALID, "dynamics vanish on the grid: no finite CFL step");
        }
    }

    // The march: graphs of `chunk` steps, one in flight ahead of the check.
    // Each graph is either one launch per RK stage, or one multi-step march
    // launch (every CTA resident: at most march_max_blocks per SM).
    const int chunk = o->check_every > 0 ? o->check_every : 32;
    const bool interval = o->interval > 0.0;
    const int flavor = flavor_of(o);
    bool multi = !g_stage_timer && o->march != HJI_MARCH_PER_STAGE && ndim <= 2 && !o->local_lf;
    int mgrid = 0;
    if (multi) {
        const int b = f32 ? hji::march_max_blocks_f32(ndim, o->scheme, variant, interval)
                          : hji::march_max_blocks_f64(ndim, o->scheme, variant, interval);
        long long gm = (long long)num_sms() * b;
        // AUTO: the multi-step launch pays a grid-wide barrier per stage in
        // place of a kernel boundary; that wins when every CTA has several
        // tiles per stage, and loses on short stages of a tile or two per
        // CTA (measured: 8192^2 and a batch of 256 grids faster, 1001^2
        // slower).
        if (o->march == HJI_MARCH_AUTO && total_tiles < kMultiStepTilesPerCta * gm) gm = 0;
        if (gm > total_tiles) gm = total_tiles;
        mgrid = (int)gm;
        multi = mgrid >= 1;
    }
    const int grid[2] = {
        multi ? mgrid : stage_grid(f32, ndim, o->scheme, total_tiles, variant, false, flavor),
        multi ? 0 : stage_grid(f32, ndim, o->scheme, total_tiles, variant, true, flavor)};
    hji::StageArgs base{d_desc, d_tiles, d_ntiles, 0, 0, 0.0, 0.0, 0.0f, 0.0f, 0};
    // the tile count and, for one grid, the list itself are known here
    base.ntiles_imm = (int)total_tiles;
    base.direct = count == 1 ? 1 : 0;
    unsigned* d_barrier = reinterpret_cast<unsigned*>(d_active + 2);
    int* d_fault = d_active + 3;
    cudaGraphExec_t exec = nullptr;
    // The graph's kernels read descriptors and the tile list from the
    // leader's scratch, so it stays valid while those buffers and the launch
    // shape (scheme, RK order, chunk, grid, tile shape, launch mode) are
    // unchanged; its launches also carry the tile count (and, for one grid,
    // take the list as 0 .. n-1), which is therefore part of the key.
    const long long key[9] = {(long long)o->scheme, o->rk_order, chunk, grid[0], grid[1],
                              variant + (multi ? 16 : 0) + 32 * flavor, ndim, f32 ? 1 : 0,
                              2 * total_tiles + base.direct};
    if (g_stage_timer) {
        // the timed march launches its stages one by one
    } else if (g0->graph && std::memcmp(key, g0->graph_key, sizeof(key)) == 0) {
        exec = g0->graph;
    } else {
        drop_graph();
        st = multi ? capture_march(g0, g0->cap_stream, f32, ndim, o->scheme, o->rk_order, chunk, base,
                                   mgrid, variant, interval, d_active, d_barrier, d_fault, &exec)
                   : capture_chunk(g0, g0->cap_stream, f32, ndim, o->scheme, o->rk_order, chunk, base,
                                   grid, variant, flavor, &exec);
        if (st != HJI_OK) return st;
        g0->graph = exec;
        std::memcpy(g0->graph_key, key, sizeof(key));
    }
    if (multi) {
        e = cudaMemsetAsync(d_fault, 0, sizeof(int), s);
        if (e != cudaSuccess) return cuda_fail(g0, e, "march fault flag");
    }
    long long stage_launches = 0;
    if (g_stage_timer) {
        e = timed_march(o, f32, ndim, base, grid, variant, s, g_stage_timer);
        stage_launches = (long long)o->max_steps * o->rk_order;
        if (e != cudaSuccess) return cuda_fail(g0, e, "timed march");
    } else {
        int* h_active = g0->h_active;  // two pinned slots
        cudaEvent_t ev[2];
        cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
        e = cudaSuccess;
        long long graphs = 0;
        for (long long it = 0;; ++it) {
            ++graphs;
            e = cudaGraphLaunch(exec, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h_active[it & 1], d_active, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[it & 1], s);
            if (e != cudaSuccess) break;
            if (it > 0) {
                e = cudaEventSynchronize(ev[(it - 1) & 1]);
                if (e != cudaSuccess) break;
                if (h_active[(it - 1) & 1] <= 0) break;
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        stage_launches = multi ? graphs : graphs * (long long)chunk * o->rk_order;
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(g0, e, "march");
        }
    }
    for (int i = 0; i < count; ++i) {
        e = cudaMemcpyAsync(grids[i]->h_state, grids[i]->state, sizeof(InstState), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) break;
    }
    int h_fault = 0;
    if (e == cudaSuccess && multi)
        e = cudaMemcpyAsync(&g0->h_active[1], d_fault, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && multi) h_fault = g0->h_active[1];
    cleanup();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g0, e, "final state");
    const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    hji_status result = HJI_OK;
    for (int i = 0; i < count; ++i) {
        hji_grid g = grids[i];
        const InstState& S = *g->h_state;
        g->cur = S.cur;
        g->has_value = true;
        hji_status si = HJI_OK;
        if (S.check_count) {
            si = fail(g, HJI_E_CHECK, check_message(S));
        } else if (S.status == 1) {
            si = fail(g, HJI_E_NONFINITE, "the march produced NaN or Inf");
        } else if (S.status == 4) {
            si = fail(g, HJI_E_TIMEOUT, "a bounded device wait gave up (a tile copy never arrived)");
        } else if (h_fault) {
            si = fail(g, HJI_E_TIMEOUT, "a bounded grid-barrier wait of the march kernel gave up");
        } else if (!S.converged) {
            si = fail(g, HJI_E_NOT_CONVERGED, "stopped by the horizon or the step cap");
        }
        if (result == HJI_OK && si != HJI_OK) result = si;
        if (stats) {
            hji_solve_stats& o_ = stats[i];
            o_.steps = S.steps;
            o_.tau = S.tau;
            o_.dt = S.dt;
            o_.final_max_dV = S.last_delta;
            o_.wall_ms = wall;
            for (int a = 0; a < HJI_MAX_DIM; ++a) o_.alpha[a] = a < g->ndim ? S.alpha[a] : 0.0;
            o_.converged = S.converged;
            long long setup = 0;
            for (int j = 0; j < count; ++j) setup += 2 + (grids[j]->dyn.nterms > 0 ? 1 : 0);
            o_.kernel_launches = setup + stage_launches;
        }
    }
    return result;
}

}  // namespace

extern "C" {

const char* hji_status_string(hji_status s) {
    switch (s) {
        case HJI_OK: return "ok";
        case HJI_E_INVALID: return "invalid argument";
        case HJI_E_NOMEM: return "out of device memory";
        case HJI_E_CUDA: return "CUDA error";
        case HJI_E_NOT_CONVERGED: return "not converged";
        case HJI_E_TIMEOUT: return "timeout";
        case HJI_E_STATE: return "call out of order";
        case HJI_E_NONFINITE: return "non-finite value";
        case HJI_E_CHECK: return "index check failed";
    }
    return "unknown status";
}

const char* hji_last_error(hji_grid g) { return g ? g->err.c_str() : g_create_error.c_str(); }

hji_status hji_grid_create(int ndim, const int64_t* n, const double* lo, const double* hi,
                           const int* periodic, hji_precision prec, const hji_allocator* alloc,
                           hji_grid* out) {
    if (!out) return fail(nullptr, HJI_E_INVALID, "out is NULL");
    *out = nullptr;
    if (ndim < 1 || ndim > HJI_MAX_DIM) return fail(nullptr, HJI_E_INVALID, "ndim must be 1..4");
    if (!n || !lo || !hi) return fail(nullptr, HJI_E_INVALID, "n, lo, hi must not be NULL");
    if (prec != HJI_F64 && prec != HJI_F32) return fail(nullptr, HJI_E_INVALID, "unknown precision");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, HJI_E_INVALID, "allocator lacks alloc/free");
    int64_t total = 1;
    for (int a = 0; a < ndim; ++a) {
        if (n[a] < 3) return fail(nullptr, HJI_E_INVALID, "every axis needs at least 3 nodes");
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(hi[a] > lo[a]))
            return fail(nullptr, HJI_E_INVALID, "bounds must be finite with hi > lo");
        total *= n[a];
        if (total > 2147483647ll) return fail(nullptr, HJI_E_INVALID, "grid too large (max 2^31-1 nodes)");
    }
    hji_grid g = new (std::nothrow) hji_grid_s();
    if (!g) return fail(nullptr, HJI_E_NOMEM, "host allocation failed");
    g->ndim = ndim;
    for (int a = 0; a < ndim; ++a) {
        g->n[a] = n[a];
        g->lo[a] = lo[a];
        g->hi[a] = hi[a];
        g->periodic[a] = periodic ? (periodic[a] != 0) : 0;
        g->dx[a] = g->periodic[a] ? (hi[a] - lo[a]) / (double)n[a] : (hi[a] - lo[a]) / (double)(n[a] - 1);
    }
    g->prec = prec;
    g->esize = prec == HJI_F32 ? 4 : 8;
    g->ncells = total;
    g->pitch = hji::pitch_of(n[ndim - 1]);
    g->nalloc = total / n[ndim - 1] * g->pitch;
    cudaGetDevice(&g->device);
    if (alloc) {
        g->has_alloc = true;
        g->alloc = *alloc;
    }
    cudaStream_t s = nullptr;
    const size_t bytes = (size_t)g->nalloc * g->esize;
    g->V[0] = dev_alloc(g, bytes, s);
    g->V[1] = dev_alloc(g, bytes, s);
    g->l = dev_alloc(g, bytes, s);
    if (prec == HJI_F32) {
        g->Vlo[0] = dev_alloc(g, bytes, s);
        g->Vlo[1] = dev_alloc(g, bytes, s);
    }
    g->state = (InstState*)dev_alloc(g, sizeof(InstState), s);
    g->d_desc = (InstDesc*)dev_alloc(g, sizeof(InstDesc), s);
    g->desc_cap = g->d_desc ? 1 : 0;
    // [0] marching instances, [1] tiles in the list, [2] grid-barrier counter
    // and [3] fault flag of the multi-step march kernel
    g->d_active = (int*)dev_alloc(g, sizeof(int) * 4, s);
    bool ok = g->V[0] && g->V[1] && g->l && g->state && g->d_desc && g->d_active &&
              (prec != HJI_F32 || (g->Vlo[0] && g->Vlo[1]));
    g->d_ntiles = ok ? g->d_active + 1 : nullptr;
    if (ok && cudaMallocHost(&g->h_state, sizeof(InstState) * 2) != cudaSuccess) ok = false;
    if (ok && cudaMallocHost(&g->h_active, sizeof(int) * 2) != cudaSuccess) ok = false;
    if (ok && cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) ok = false;
    if (ok && cudaStreamSynchronize(s) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        hji_grid_destroy(g);
        return fail(nullptr, HJI_E_NOMEM, "device allocation failed");
    }
    *out = g;
    return HJI_OK;
}

hji_status hji_grid_destroy(hji_grid g) {
    if (!g) return HJI_OK;
    cudaStream_t s = nullptr;
    cudaStreamSynchronize(s);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    void* bufs[] = {g->V[0], g->V[1], g->W1, g->W2, g->Vlo[0], g->Vlo[1], g->l, g->snap, g->table,
                    g->state, g->d_desc, g->d_active, g->d_tiles};
    for (void* p : bufs) dev_free(g, p, s);
    if (g->h_state) cudaFreeHost(g->h_state);
    if (g->h_active) cudaFreeHost(g->h_active);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    cudaStreamSynchronize(s);
    delete g;
    return HJI_OK;
}

hji_status hji_dynamics_set(hji_grid g, const hji_dynamics* d) {
    if (!g) return fail(nullptr, HJI_E_INVALID, "grid is NULL");
    if (!d) return fail(g, HJI_E_INVALID, "dynamics is NULL");
    const int n = g->ndim;
    if (d->m < 0 || d->m > HJI_MAX_INPUTS || d->q < 0 || d->q > HJI_MAX_INPUTS)
        return fail(g, HJI_E_INVALID, "m and q must be in 0..4");
    if (d->nterms < 0 || d->nterms > HJI_MAX_TERMS) return fail(g, HJI_E_INVALID, "nterms must be in 0..8");
    if (d->m > 0 && (!d->G || !d->ulo || !d->uhi)) return fail(g, HJI_E_INVALID, "m > 0 needs G, ulo, uhi");
    if (d->q > 0 && (!d->E || !d->dlo || !d->dhi)) return fail(g, HJI_E_INVALID, "q > 0 needs E, dlo, dhi");
    if (d->nterms > 0 && (!d->term_row || !d->term_axis || !d->term_fn || !d->term_w))
        return fail(g, HJI_E_INVALID, "nterms > 0 needs the term arrays");
    hji::Dyn D;
    std::memset(&D, 0, sizeof(D));
    D.m = d->m;
    D.q = d->q;
    D.nterms = d->nterms;
    for (int i = 0; i < n; ++i) {
        D.c[i] = d->c ? d->c[i] : 0.0;
        for (int j = 0; j < n; ++j) D.A[i * HJI_MAX_DIM + j] = d->A ? d->A[i * n + j] : 0.0;
        for (int j = 0; j < d->m; ++j) D.G[i * HJI_MAX_INPUTS + j] = d->G[i * d->m + j];
        for (int j = 0; j < d->q; ++j) D.E[i * HJI_MAX_INPUTS + j] = d->E[i * d->q + j];
    }
    for (int j = 0; j < d->m; ++j) {
        D.ulo[j] = d->ulo[j];
        D.uhi[j] = d->uhi[j];
        if (!(D.ulo[j] <= D.uhi[j])) return fail(g, HJI_E_INVALID, "ulo > uhi");
    }
    for (int j = 0; j < d->q; ++j) {
        D.dlo[j] = d->dlo[j];
        D.dhi[j] = d->dhi[j];
        if (!(D.dlo[j] <= D.dhi[j])) return fail(g, HJI_E_INVALID, "dlo > dhi");
    }
    for (int t = 0; t < d->nterms; ++t) {
        if (d->term_row[t] < 0 || d->term_row[t] >= n || d->term_axis[t] < 0 || d->term_axis[t] >= n)
            return fail(g, HJI_E_INVALID, "term row/axis out of range");
        if (d->term_fn[t] < HJI_FN_TAN || d->term_fn[t] > HJI_FN_COS)
            return fail(g, HJI_E_INVALID, "unknown term function");
        D.term_row[t] = d->term_row[t];
        D.term_axis[t] = d->term_axis[t];
        D.term_fn[t] = d->term_fn[t];
        D.term_w[t] = d->term_w[t];
    }
    const double* arrs[] = {D.c, D.A, D.G, D.E, D.ulo, D.uhi, D.dlo, D.dhi, D.term_w};
    const int lens[] = {HJI_MAX_DIM, HJI_MAX_DIM * HJI_MAX_DIM, HJI_MAX_DIM * HJI_MAX_INPUTS,
                        HJI_MAX_DIM * HJI_MAX_INPUTS, HJI_MAX_INPUTS, HJI_MAX_INPUTS, HJI_MAX_INPUTS,
                        HJI_MAX_INPUTS, HJI_MAX_TERMS};
    for (int i = 0; i < 9; ++i)
        if (!finite_all(arrs[i], lens[i])) return fail(g, HJI_E_INVALID, "dynamics contain NaN or Inf");
    g->dyn = D;
    g->has_dyn = true;
    return HJI_OK;
}

hji_status hji_solve(hji_grid g, const void* l, const void* k, int ptr_is_device,
                     const hji_solve_opts* o, void* cuda_stream, hji_solve_stats* stats) {
    if (!g) return fail(nullptr, HJI_E_INVALID, "grid is NULL");
    const void* la[1] = {l};
    const void* ka[1] = {k};
    return run(1, &g, la, ka, ptr_is_device, o, (cudaStream_t)cuda_stream, stats);
}

hji_status hji_batch_solve(int count, hji_grid* grids, const void* const* l, const void* const* k,
                           int ptr_is_device, const hji_solve_opts* o, void* cuda_stream,
                           hji_solve_stats* stats) {
    if (count < 1 || count > 65535 || !grids) return fail(nullptr, HJI_E_INVALID, "count must be 1..65535");
    if (!grids[0]) return fail(nullptr, HJI_E_INVALID, "NULL grid in batch");
    return run(count, grids, l, k, ptr_is_device, o, (cudaStream_t)cuda_stream, stats);
}

hji_status hji_value_get(hji_grid g, void* out, int ptr_is_device, void* cuda_stream) {
    if (!g) return fail(nullptr, HJI_E_INVALID, "grid is NULL");
    if (!out) return fail(g, HJI_E_INVALID, "out is NULL");
    if (!g->has_value) return fail(g, HJI_E_STATE, "no value yet: call hji_solve first");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    HJI_CUDA(g, copy_out(g, out, g->V[g->cur],
                         ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    HJI_CUDA(g, cudaStreamSynchronize(s));
    return HJI_OK;
}

hji_status hji_value_transfer(hji_grid dst, hji_grid src, void* cuda_stream) {
    if (!dst || !src) return fail(dst ? dst : src, HJI_E_INVALID, "grid is NULL");
    if (dst == src) return fail(dst, HJI_E_INVALID, "source and destination are the same grid");
    if (dst->ndim != src->ndim) return fail(dst, HJI_E_INVALID, "grids differ in ndim");
    for (int a = 0; a < dst->ndim; ++a)
        if (dst->n[a] != src->n[a]) return fail(dst, HJI_E_INVALID, "grids differ in node counts");
    if (!src->has_value) return fail(dst, HJI_E_STATE, "source grid has no value yet");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool sf = src->prec == HJI_F32, df = dst->prec == HJI_F32;
    HJI_CUDA(dst, hji::launch_convert(src->nalloc, src->V[src->cur], sf ? src->Vlo[src->cur] : nullptr,
                                      sf, dst->V[0], df ? dst->Vlo[0] : nullptr, df, s));
    HJI_CUDA(dst, cudaStreamSynchronize(s));
    dst->cur = 0;
    dst->has_value = true;
    return HJI_OK;
}

// The engine's device buffers come from its allocator (if one was given,
// e.g. a framework's caching allocator), else from cudaMallocAsync, on the
// engine's stream.
static void* engine_alloc(hji_engine e, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (e->has_alloc) return e->alloc.alloc(bytes, e->s, e->alloc.ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, e->s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void engine_free(hji_engine e, void* p) {
    if (!p) return;
    if (e->has_alloc) e->alloc.free(p, e->s, e->alloc.ctx);
    else cudaFreeAsync(p, e->s);
}

static hji_status efail(hji_engine e, hji_status st, const std::string& msg) {
    if (e) e->err = msg;
    else g_create_error = msg;
    return st;
}

static size_t grid_bytes(hji_grid g, int rk) {
    const size_t field = (size_t)g->nalloc * g->esize;
    size_t n = 3 + (rk >= 2 ? 1 : 0) + (rk >= 3 ? 1 : 0) + (g->prec == HJI_F32 ? 2 : 0);
    return n * field + g->table_bytes;
}

const char* hji_engine_last_error(hji_engine e) { return e ? e->err.c_str() : g_create_error.c_str(); }

hji_status hji_engine_create(int ndim, hji_precision prec, const hji_solve_opts* o, int max_slots,
                             size_t budget_bytes, void* cuda_stream, const hji_allocator* alloc,
                             hji_engine* out) {
    if (!out) return efail(nullptr, HJI_E_INVALID, "out is NULL");
    *out = nullptr;
    if (ndim < 1 || ndim > HJI_MAX_DIM) return efail(nullptr, HJI_E_INVALID, "ndim must be 1..4");
    if (prec != HJI_F64 && prec != HJI_F32) return efail(nullptr, HJI_E_INVALID, "unknown precision");
    if (max_slots < 1 || max_slots > 65535) return efail(nullptr, HJI_E_INVALID, "max_slots must be 1..65535");
    hji_status st = validate_opts(nullptr, o);
    if (st != HJI_OK) return st;
    hji_engine e = new (std::nothrow) hji_engine_s();
    if (!e) return efail(nullptr, HJI_E_NOMEM, "host allocation failed");
    e->ndim = ndim;
    e->prec = prec;
    e->o = *o;
    e->chunk = o->check_every > 0 ? o->check_every : 32;
    e->max_slots = max_slots;
    e->budget = budget_bytes;
    e->s = (cudaStream_t)cuda_stream;
    e->slots.resize(max_slots);
    e->h_desc.resize(max_slots);
    if (alloc) {
        e->alloc = *alloc;
        e->has_alloc = true;
    }
    e->d_desc = (InstDesc*)engine_alloc(e, sizeof(InstDesc) * max_slots);
    e->d_counts = (int*)engine_alloc(e, sizeof(int) * 2);
    bool ok = e->d_desc && e->d_counts &&
              cudaMallocHost(&e->h_counts, sizeof(int) * 2) == cudaSuccess &&
              cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMemset(e->d_counts, 0, sizeof(int) * 2) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        hji_engine_destroy(e);
        return efail(nullptr, HJI_E_NOMEM, "engine allocation failed");
    }
    e->variant = o->local_lf ? 0 : pick_variant(prec, ndim, o, 1ll << 20);
    for (int last = 0; last < 2; ++last)
        e->grid[last] = stage_grid(prec == HJI_F32, ndim, o->scheme, 1ll << 40, e->variant, last != 0,
                                   flavor_of(o));
    *out = e;
    return HJI_OK;
}

hji_status hji_engine_destroy(hji_engine e) {
    if (!e) return HJI_OK;
    cudaStreamSynchronize(e->s);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    engine_free(e, e->d_desc);
    engine_free(e, e->d_counts);
    engine_free(e, e->d_tiles);
    cudaStreamSynchronize(e->s);
    if (e->h_counts) cudaFreeHost(e->h_counts);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->ev) cudaEventDestroy(e->ev);
    delete e;
    return HJI_OK;
}

hji_status hji_engine_submit(hji_engine e, hji_grid g, const void* l, const void* k,
                             int ptr_is_device, hji_init init, int64_t tag) {
    if (!e) return efail(nullptr, HJI_E_INVALID, "engine is NULL");
    if (!g || !l) return efail(e, HJI_E_INVALID, "grid and l must not be NULL");
    if (g->ndim != e->ndim || g->prec != e->prec)
        return efail(e, HJI_E_INVALID, "grid ndim/precision differ from the engine's");
    if (!g->has_dyn) return efail(e, HJI_E_STATE, "dynamics not set");
    if (init == HJI_INIT_USER_K && !k) return efail(e, HJI_E_INVALID, "HJI_INIT_USER_K needs k");
    if (init == HJI_INIT_RESIDENT && !g->has_value)
        return efail(e, HJI_E_STATE, "HJI_INIT_RESIDENT without a previous value");
    if (init != HJI_INIT_STANDARD && init != HJI_INIT_USER_K && init != HJI_INIT_RESIDENT)
        return efail(e, HJI_E_INVALID, "unknown init mode");
    const int gw = hji::ghost_width(e->o.scheme);
    for (int a = 0; a < g->ndim; ++a)
        if (g->n[a] < 2 * gw + 1) return efail(e, HJI_E_INVALID, "grid too small for the stencil");
    for (const auto& r : e->queue)
        if (r.g == g) return efail(e, HJI_E_STATE, "grid already has a queued request");
    for (const auto& sl : e->slots)
        if (sl.used && sl.g == g) return efail(e, HJI_E_STATE, "grid already has a marching request");
    hji_status st = ensure_buffers(g, e->o.rk_order, e->s, e->o.interval > 0.0);
    if (st != HJI_OK) return efail(e, st, g->err);
    if (e->budget && grid_bytes(g, e->o.rk_order) > e->budget)
        return efail(e, HJI_E_INVALID, "grid larger than the engine's whole budget");
    const cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t ce = copy_in(g, g->l, l, kind, e->s);
    if (ce == cudaSuccess && init == HJI_INIT_USER_K) ce = copy_in(g, g->V[1], k, kind, e->s);
    if (ce == cudaSuccess && !ptr_is_device) ce = cudaStreamSynchronize(e->s);
    if (ce != cudaSuccess) return efail(e, HJI_E_CUDA, std::string("copy of l/k: ") + cudaGetErrorString(ce));
    e->queue.push_back({g, tag, init, init == HJI_INIT_USER_K});
    return HJI_OK;
}

static hji_status engine_retire(hji_engine e) {
    int marching = 0;
    for (const auto& sl : e->slots) marching += sl.used ? 1 : 0;
    if (marching == 0 || e->h_counts[0] >= e->launched_active) return HJI_OK;
    // Something stopped during the last chunk: find it from the states.
    for (int i = 0; i < e->max_slots; ++i) {
        auto& sl = e->slots[i];
        if (!sl.used) continue;
        cudaError_t ce = cudaMemcpyAsync(sl.g->h_state, sl.g->state, sizeof(InstState), cudaMemcpyDeviceToHost, e->s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->s);
        if (ce != cudaSuccess) return efail(e, HJI_E_CUDA, std::string("state read: ") + cudaGetErrorString(ce));
        const InstState& S = *sl.g->h_state;
        if (!S.stop) continue;
        hji_engine_s::Done d;
        d.tag = sl.tag;
        std::memset(&d.st, 0, sizeof(d.st));
        d.st.steps = S.steps;
        d.st.tau = S.tau;
        d.st.dt = S.dt;
        d.st.final_max_dV = S.last_delta;
        d.st.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - sl.t0).count();
        for (int a = 0; a < HJI_MAX_DIM; ++a) d.st.alpha[a] = a < sl.g->ndim ? S.alpha[a] : 0.0;
        d.st.converged = S.converged;
        if (S.check_count) d.status = HJI_E_CHECK;
        else if (S.nonfinite) d.status = HJI_E_INVALID;
        else if (S.status == 2) d.status = HJI_E_INVALID;
        else if (S.status == 1) d.status = HJI_E_NONFINITE;
        else if (S.status == 4) d.status = HJI_E_TIMEOUT;
        else d.status = S.converged ? HJI_OK : HJI_E_NOT_CONVERGED;
        sl.g->cur = S.cur;
        sl.g->has_value = S.steps > 0 || sl.g->has_value;
        e->done.push_back(d);
        e->in_use -= sl.bytes;
        sl = hji_engine_s::Slot();
    }
    return HJI_OK;
}

hji_status hji_engine_step(hji_engine e, int* active, int* queued) {
    if (!e) return efail(nullptr, HJI_E_INVALID, "engine is NULL");
    cudaError_t ce = cudaSuccess;
    if (e->inflight) {
        ce = cudaEventSynchronize(e->ev);
        e->inflight = false;
        if (ce != cudaSuccess) return efail(e, HJI_E_CUDA, std::string("chunk: ") + cudaGetErrorString(ce));
        hji_status st = engine_retire(e);
        if (st != HJI_OK) return st;
    }
    // Admit what fits (slots and budget), then publish the tile list and the
    // marching count, and only then launch the admitted requests' set-up, so
    // a set-up that stops an instance (no finite dt) decrements the published
    // count.
    const bool f32 = e->prec == HJI_F32;
    std::vector<int> admitted;
    while (!e->queue.empty()) {
        const auto req = e->queue.front();
        const size_t need = grid_bytes(req.g, e->o.rk_order);
        if (e->budget && e->in_use + need > e->budget) break;
        int slot = -1;
        for (int i = 0; i < e->max_slots; ++i)
            if (!e->slots[i].used) {
                slot = i;
                break;
            }
        if (slot < 0) break;
        if (make_desc(req.g, &e->o, e->d_counts, e->variant, e->h_desc[slot]) != HJI_OK)
            return efail(e, HJI_E_CUDA, req.g->err);
        e->queue.pop_front();
        auto& sl = e->slots[slot];
        sl.used = true;
        sl.g = req.g;
        sl.tag = req.tag;
        sl.bytes = need;
        sl.init = req.init;
        sl.t0 = std::chrono::steady_clock::now();
        e->in_use += need;
        admitted.push_back(slot);
    }
    int marching = 0;
    for (const auto& sl : e->slots) marching += sl.used ? 1 : 0;
    if (!admitted.empty() || marching != e->launched_active) {
        // Rebuild the tile list of the admitted slots (slot index = instance).
        std::vector<unsigned long long> tiles;
        for (int i = 0; i < e->max_slots; ++i)
            if (e->slots[i].used)
                for (long long t = 0; t < e->h_desc[i].ntiles; ++t) tiles.push_back(hji::make_tile(i, t));
        if (tiles.size() > e->tiles_cap) {
            engine_free(e, e->d_tiles);
            size_t cap = tiles.size() * 2;
            e->d_tiles = (unsigned long long*)engine_alloc(e, cap * sizeof(unsigned long long));
            if (!e->d_tiles) {
                e->tiles_cap = 0;
                return efail(e, HJI_E_NOMEM, "tile list allocation failed");
            }
            e->tiles_cap = cap;
            if (e->graph) {
                cudaGraphExecDestroy(e->graph);
                e->graph = nullptr;
            }
        }
        int counts[2] = {marching, (int)tiles.size()};
        if (!tiles.empty())
            ce = cudaMemcpyAsync(e->d_tiles, tiles.data(), tiles.size() * sizeof(unsigned long long),
                                 cudaMemcpyHostToDevice, e->s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(e->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, e->s);
        if (ce != cudaSuccess) return efail(e, HJI_E_CUDA, std::string("tile list: ") + cudaGetErrorString(ce));
    }
    for (int slot : admitted) {
        hji_grid g = e->slots[slot].g;
        const hji_init init = e->slots[slot].init;
        InstDesc& D = e->h_desc[slot];
        D.kinit = init == HJI_INIT_USER_K ? g->V[1] : (init == HJI_INIT_RESIDENT ? g->V[g->cur] : nullptr);
        D.kinit_lo = init == HJI_INIT_RESIDENT ? g->Vlo[g->cur] : nullptr;
        ce = cudaMemsetAsync(g->state, 0, sizeof(InstState), e->s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(e->d_desc + slot, &D, sizeof(InstDesc), cudaMemcpyHostToDevice, e->s);
        if (ce == cudaSuccess) ce = hji::launch_setup(e->d_desc + slot, &D, 1, f32, e->s);
        if (ce == cudaSuccess) ce = hji::launch_init(e->d_desc + slot, &D, 1, f32, e->s);
        if (ce != cudaSuccess) return efail(e, HJI_E_CUDA, std::string("admission: ") + cudaGetErrorString(ce));
    }
    e->launched_active = marching;
    if (marching > 0) {
        if (!e->graph) {
            hji::StageArgs base{e->d_desc, e->d_tiles, e->d_counts + 1, 0, 0, 0.0, 0.0, 0.0f, 0.0f, 0};
            hji_status st = capture_chunk(nullptr, e->cap, f32, e->ndim, e->o.scheme, e->o.rk_order,
                                          e->chunk, base, e->grid, e->variant,
                                          flavor_of(&e->o), &e->graph);
            if (st != HJI_OK) return efail(e, st, g_create_error);
        }
        ce = cudaGraphLaunch(e->graph, e->s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(e->h_counts, e->d_counts, sizeof(int) * 2, cudaMemcpyDeviceToHost, e->s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e->ev, e->s);
        if (ce != cudaSuccess) return efail(e, HJI_E_CUDA, std::string("launch: ") + cudaGetErrorString(ce));
        e->inflight = true;
    }
    if (active) *active = marching;
    if (queued) *queued = (int)e->queue.size();
    return HJI_OK;
}

hji_status hji_engine_poll(hji_engine e, int64_t* tags, hji_solve_stats* stats, hji_status* status,
                           int cap, int* count) {
    if (!e || !count) return efail(e, HJI_E_INVALID, "engine and count must not be NULL");
    int n = 0;
    while (n < cap && !e->done.empty()) {
        const auto& d = e->done.front();
        if (tags) tags[n] = d.tag;
        if (stats) stats[n] = d.st;
        if (status) status[n] = d.status;
        e->done.erase(e->done.begin());
        ++n;
    }
    *count = n;
    return HJI_OK;
}

hji_status hji_autotune(hji_grid g, const void* l, int ptr_is_device, const hji_solve_opts* o,
                        int steps, void* cuda_stream, int* chosen, double* ms_per_step) {
    if (!g) return fail(nullptr, HJI_E_INVALID, "grid is NULL");
    hji_status st = validate_opts(g, o);
    if (st != HJI_OK) return st;
    if (steps < 1) return fail(g, HJI_E_INVALID, "steps must be >= 1");
    hji_solve_opts t = *o;
    t.tol = 0.0;
    t.horizon = 0.0;
    t.max_steps = steps;
    t.check_every = steps;
    t.init = HJI_INIT_STANDARD;
    const int nvar = g->ndim == 2 ? hji::kTileVariants : 1;
    double best_ms = 1e300;
    int best = 0;
    for (int v = 0; v < hji::kTileVariants; ++v) {
        if (ms_per_step) ms_per_step[v] = -1.0;
        if (v >= nvar) continue;
        g_force_variant = v;
        // One warm-up solve, then the median of three timed solves (a single
        // host-timed solve of a small grid is too noisy to rank shapes).
        hji_solve_stats s1;
        hji_status r = hji_solve(g, l, nullptr, ptr_is_device, &t, cuda_stream, &s1);  // warm-up
        double rep[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3 && (r == HJI_OK || r == HJI_E_NOT_CONVERGED); ++k) {
            hji_solve_stats s2;
            r = hji_solve(g, l, nullptr, ptr_is_device, &t, cuda_stream, &s2);
            rep[k] = s2.wall_ms / (double)(s2.steps > 0 ? s2.steps : 1);
        }
        g_force_variant = -1;
        if (r != HJI_OK && r != HJI_E_NOT_CONVERGED) return r;
        std::sort(rep, rep + 3);
        const double ms = rep[1];
        if (ms_per_step) ms_per_step[v] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(g->prec, g->ndim, o, size_bucket(g->ncells))] = best;
    }
    if (chosen) *chosen = best;
    return HJI_OK;
}

hji_status hji_stage_times(hji_grid g, const void* l, int ptr_is_device, const hji_solve_opts* o,
                           int steps, void* cuda_stream, double* ms_per_stage) {
    if (!g) return fail(nullptr, HJI_E_INVALID, "grid is NULL");
    hji_status st = validate_opts(g, o);
    if (st != HJI_OK) return st;
    if (steps < 1 || steps > 4096) return fail(g, HJI_E_INVALID, "steps must be 1..4096");
    if (!ms_per_stage) return fail(g, HJI_E_INVALID, "ms_per_stage is NULL");
    hji_solve_opts t = *o;
    t.tol = 0.0;
    t.horizon = 0.0;
    t.max_steps = steps;
    t.check_every = steps;
    t.init = HJI_INIT_STANDARD;
    StageTimer T{};
    g_stage_timer = &T;
    const void* la[1] = {l};
    const void* ka[1] = {nullptr};
    hji_status r = run(1, &g, la, ka, ptr_is_device, &t, (cudaStream_t)cuda_stream, nullptr);
    g_stage_timer = nullptr;
    if (r != HJI_OK && r != HJI_E_NOT_CONVERGED) return r;
    for (int i = 0; i < T.ns; ++i) ms_per_stage[i] = T.ms[i];
    return HJI_OK;
}

hji_status hji_selftest_bounded_wait(int64_t limit_ns, void* cuda_stream) {
    if (limit_ns < 1000000 || limit_ns > 4000000000ll)
        return fail(nullptr, HJI_E_INVALID, "limit_ns must be 1e6..4e9");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int* d = nullptr;
    if (cudaMallocAsync(&d, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, HJI_E_NOMEM, "device allocation failed");
    }
    int h = -1;
    cudaError_t e = cudaMemsetAsync(d, 0xFF, sizeof(int), s);
    if (e == cudaSuccess) e = hji::launch_wait_selftest((unsigned long long)limit_ns, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, HJI_E_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    if (h == 4) return fail(nullptr, HJI_E_TIMEOUT, "the bounded wait gave up, as it should");
    if (h == 0) return fail(nullptr, HJI_E_STATE, "a barrier that nothing completes completed");
    return fail(nullptr, HJI_E_CUDA, "self-test kernel wrote no result");
}

hji_status hji_selftest_index_check(void* cuda_stream, int* checked, int* count, int* site,
                                    int64_t* index, int64_t* extent) {
#ifdef HJI_CHECKED
    const int is_checked = 1;
#else
    const int is_checked = 0;
#endif
    if (checked) *checked = is_checked;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void* d = nullptr;
    const size_t bytes = sizeof(InstState) + 4 * sizeof(long long);
    if (cudaMallocAsync(&d, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, HJI_E_NOMEM, "device allocation failed");
    }
    InstState* d_st = static_cast<InstState*>(d);
    long long* d_out = reinterpret_cast<long long*>(static_cast<char*>(d) + sizeof(InstState));
    InstState h;
    long long out[4] = {-1, -1, -1, -1};
    cudaError_t e = cudaMemsetAsync(d, 0, bytes, s);
    if (e == cudaSuccess) e = hji::launch_check_selftest(d_st, d_out, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_st, sizeof(InstState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(out), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, HJI_E_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    if (count) *count = h.check_count;
    if (site) *site = h.check_site;
    if (index) *index = h.check_index;
    if (extent) *extent = h.check_limit;
    const bool want = is_checked ? (out[0] == 7 && out[1] == 0 && out[2] == 0 && out[3] == 0)
                                 : (out[0] == 0 && out[1] == 0 && out[2] == 0 && out[3] == 0);
    if (!want) return fail(nullptr, HJI_E_STATE, "the index-check recorder returned wrong indices");
    return HJI_OK;
}

hji_status hji_optimal_control(hji_grid g, hji_scheme scheme, void* u_out, void* d_out,
                               int ptr_is_device, void* cuda_stream) {
    if (!g) return fail(nullptr, HJI_E_INVALID, "grid is NULL");
    if (scheme != HJI_ENO1 && scheme != HJI_ENO2 && scheme != HJI_WENO5)
        return fail(g, HJI_E_INVALID, "unknown scheme");
    if (!g->has_dyn) return fail(g, HJI_E_STATE, "dynamics not set");
    if (!g->has_value) return fail(g, HJI_E_STATE, "no value yet");
    const int m = g->dyn.m, q = g->dyn.q;
    if (m > 0 && !u_out) return fail(g, HJI_E_INVALID, "u_out is NULL");
    const int gw = hji::ghost_width(scheme);
    for (int a = 0; a < g->ndim; ++a)
        if (g->n[a] < 2 * gw + 1) return fail(g, HJI_E_INVALID, "grid too small for the scheme's stencil");
    if (m == 0 && (q == 0 || !d_out)) return HJI_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    hji::ControlArgs A;
    std::memset(&A, 0, sizeof(A));
    for (int a = 0; a < HJI_MAX_DIM; ++a) {
        A.n[a] = a < g->ndim ? (int)g->n[a] : 1;
        A.periodic[a] = a < g->ndim ? g->periodic[a] : 0;
        A.inv_dx[a] = a < g->ndim ? 1.0 / g->dx[a] : 1.0;
    }
    field_strides(g->ndim, g->n, g->pitch, A.stride);
    A.v_hi = g->V[g->cur];
    A.v_lo = g->prec == HJI_F32 ? g->Vlo[g->cur] : nullptr;
    std::memcpy(A.G, g->dyn.G, sizeof(A.G));
    std::memcpy(A.E, g->dyn.E, sizeof(A.E));
    std::memcpy(A.ulo, g->dyn.ulo, sizeof(A.ulo));
    std::memcpy(A.uhi, g->dyn.uhi, sizeof(A.uhi));
    std::memcpy(A.dlo, g->dyn.dlo, sizeof(A.dlo));
    std::memcpy(A.dhi, g->dyn.dhi, sizeof(A.dhi));
    A.m = m;
    A.q = d_out ? q : 0;
    A.ncells = g->ncells;
    const size_t ubytes = (size_t)m * g->ncells * g->esize;
    const size_t dbytes = (size_t)A.q * g->ncells * g->esize;
    void* tmp = nullptr;
    if (ptr_is_device) {
        A.u_out = u_out;
        A.d_out = A.q ? d_out : nullptr;
    } else {
        tmp = dev_alloc(g, ubytes + dbytes, s);
        if (!tmp) return fail(g, HJI_E_NOMEM, "control output allocation failed");
        A.u_out = tmp;
        A.d_out = A.q ? static_cast<unsigned char*>(tmp) + ubytes : nullptr;
    }
    cudaError_t e = hji::launch_control(A, g->prec == HJI_F32, g->ndim, scheme, s);
    if (e == cudaSuccess && !ptr_is_device) {
        if (ubytes) e = cudaMemcpyAsync(u_out, A.u_out, ubytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && dbytes) e = cudaMemcpyAsync(d_out, A.d_out, dbytes, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tmp) {
        dev_free(g, tmp, s);
        cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return cuda_fail(g, e, "optimal control");
    return HJI_OK;
}

hji_status hji_grid_info(hji_grid g, int* ndim, int64_t* n, int64_t* num_nodes) {
    if (!g) return fail(nullptr, HJI_E_INVALID, "grid is NULL");
    if (ndim) *ndim = g->ndim;
    if (n)
        for (int a = 0; a < g->ndim; ++a) n[a] = g->n[a];
    if (num_nodes) *num_nodes = g->ncells;
    return HJI_OK;
}

}  // extern "C"
