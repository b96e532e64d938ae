// hji_solve_noalloc: a one-shot solve for callers that must not allocate
// device memory (for example code running inside a framework that owns all
// device memory, a real-time loop that forbids allocator calls, or a
// process whose allocator is already exhausted).  The caller passes l, k and
// the output buffer; every scratch buffer the march needs (the second value
// buffer, the Runge-Kutta stage buffers, the FP32 low words, the term table,
// the tile list, the instance description and march state) lives in one
// file-scope device array of fixed size, HJI_NOALLOC_SCRATCH_BYTES.
//
// The array's host-side name is not a device address: the first call on a
// device, with that device current, takes its address with
// cudaGetSymbolAddress and caches it per device together with the identity of
// the CUDA context it belongs to; a later call in another context of that
// device (after cudaDeviceReset, or a primary context released and made
// again, where the module is loaded anew and the array may move) looks the
// address up again.  Make the first call on a device before any stream
// capture.  Every call shares the array and leaves its
// contents behind; the march state is cleared at the start of each call.
// Calls whose GPU work overlaps (different streams or threads) race on it.
// Nothing here calls cudaMalloc, cudaFree, cudaMallocHost, graph
// instantiation or any other allocating routine.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "hji_common.cuh"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char hji_noalloc_scratch[HJI_NOALLOC_SCRATCH_BYTES];

// Per device: the scratch array's device address and the id of the context
// it was taken in (0: none yet).  Guarded by g_scratch_mu.
struct ScratchSlot {
    unsigned long long ctx_id;
    void* ptr;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch[kMaxDevices] = {};
thread_local char g_err[256] = "";

// The id of the calling thread's current CUDA context (0 if none), from the
// driver through the runtime's entry-point lookup (no link against the
// driver library).  Returns false if the driver does not offer the lookup.
bool current_ctx_id(unsigned long long* id) {
    static std::once_flag once;
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
        else
            cudaGetLastError();
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
        else
            cudaGetLastError();
    });
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    *id = 0;
    if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return true;
    unsigned long long v = 0;
    if (get_id(c, &v) != CUDA_SUCCESS) return false;
    *id = v;
    return true;
}

// The scratch array's device address in the current context of device dev
// (set-up once per device and context; see the top of this file).
hji_status scratch_address(int dev, cudaStream_t s, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    unsigned long long id = 0;
    if (!current_ctx_id(&id)) {
        std::snprintf(g_err, sizeof(g_err), "the driver offers no context identity lookup");
        return HJI_E_CUDA;
    }
    if (id != 0 && g_scratch[dev].ctx_id == id && g_scratch[dev].ptr != nullptr) {
        *out = static_cast<unsigned char*>(g_scratch[dev].ptr);
        return HJI_OK;
    }
    // A look-up is due: refuse it inside a stream capture.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) {
        std::snprintf(g_err, sizeof(g_err), "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
        return HJI_E_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) {
        std::snprintf(g_err, sizeof(g_err),
                      "the first call in this device context came during a stream capture; "
                      "make one call before capturing");
        return HJI_E_STATE;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, hji_noalloc_scratch);
    if (e != cudaSuccess) {
        std::snprintf(g_err, sizeof(g_err), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return HJI_E_CUDA;
    }
    if (id == 0 && (!current_ctx_id(&id) || id == 0)) {  // the look-up made the context
        std::snprintf(g_err, sizeof(g_err), "no current CUDA context after the symbol look-up");
        return HJI_E_CUDA;
    }
    g_scratch[dev].ctx_id = id;
    g_scratch[dev].ptr = p;
    *out = static_cast<unsigned char*>(p);
    return HJI_OK;
}

hji_status nfail(hji_status s, const char* msg) {
    std::snprintf(g_err, sizeof(g_err), "%s", msg);
    return s;
}

hji_status ncuda(cudaError_t e, const char* where) {
    std::snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
    return HJI_E_CUDA;
}

__global__ void fill_tiles(unsigned long long* tiles, long long ntiles) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntiles;
         t += (long long)gridDim.x * blockDim.x)
        tiles[t] = hji::make_tile(0, t);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool all_finite(const double* p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

extern "C" const char* hji_noalloc_last_error(void) { return g_err; }

extern "C" hji_status hji_solve_noalloc(int ndim, const int64_t* n, const double* lo,
                                        const double* hi, const int* periodic,
                                        hji_precision prec, const hji_dynamics* dyn,
                                        const void* l, const void* k, void* v_out,
                                        const hji_solve_opts* o, void* cuda_stream,
                                        hji_solve_stats* stats) {
    using hji::InstDesc;
    using hji::InstState;
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (ndim < 1 || ndim > HJI_MAX_DIM || !n || !lo || !hi) return nfail(HJI_E_INVALID, "bad grid");
    if (prec != HJI_F64 && prec != HJI_F32) return nfail(HJI_E_INVALID, "unknown precision");
    if (!dyn || !l || !v_out || !o) return nfail(HJI_E_INVALID, "NULL argument");
    if (o->scheme != HJI_ENO1 && o->scheme != HJI_ENO2 && o->scheme != HJI_WENO5)
        return nfail(HJI_E_INVALID, "unknown scheme");
    if (o->rk_order < 1 || o->rk_order > 3) return nfail(HJI_E_INVALID, "rk_order must be 1..3");
    if (!(o->cfl > 0.0 && o->cfl <= 1.0)) return nfail(HJI_E_INVALID, "cfl must be in (0, 1]");
    if (!(o->tol >= 0.0) || !std::isfinite(o->tol) || !(o->horizon >= 0.0) ||
        !std::isfinite(o->horizon))
        return nfail(HJI_E_INVALID, "tol and horizon must be finite and >= 0");
    if (!(o->tol_rate >= 0.0) || !std::isfinite(o->tol_rate))
        return nfail(HJI_E_INVALID, "tol_rate must be finite and >= 0");
    if (o->tile_variant < 0 || o->tile_variant > hji::kTileVariants)
        return nfail(HJI_E_INVALID, "tile_variant must be 0..HJI_TILE_VARIANTS");
    if (o->interval != 0.0)
        return nfail(HJI_E_INVALID, "the interval test is not available without allocation");
    if (o->local_lf != 0)
        return nfail(HJI_E_INVALID, "local Lax-Friedrichs is not available without allocation");
    if (o->brs != 0 && o->brs != 1) return nfail(HJI_E_INVALID, "brs must be 0 or 1");
    if (!(o->discount >= 0.0 && o->discount <= 1.0))
        return nfail(HJI_E_INVALID, "discount must be in [0, 1] (0 and 1: off)");
    if (o->brs && o->discount > 0.0 && o->discount < 1.0)
        return nfail(HJI_E_INVALID, "discount applies to the projected march, not to brs");
    if (o->init == HJI_INIT_USER_K && !k) return nfail(HJI_E_INVALID, "HJI_INIT_USER_K needs k");
    if (o->init != HJI_INIT_STANDARD && o->init != HJI_INIT_USER_K && o->init != HJI_INIT_RESIDENT)
        return nfail(HJI_E_INVALID, "unknown init mode");
    const int gw = hji::ghost_width(o->scheme);
    long long cells = 1, nmax = 0;
    for (int a = 0; a < ndim; ++a) {
        if (n[a] < 2 * gw + 1) return nfail(HJI_E_INVALID, "grid too small for the stencil");
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(hi[a] > lo[a]))
            return nfail(HJI_E_INVALID, "bounds must be finite with hi > lo");
        cells *= n[a];
        if (cells > 2147483647ll) return nfail(HJI_E_INVALID, "grid too large");
        nmax = n[a] > nmax ? n[a] : nmax;
    }
    // Dynamics, packed like hji_dynamics_set does.
    if (dyn->m < 0 || dyn->m > HJI_MAX_INPUTS || dyn->q < 0 || dyn->q > HJI_MAX_INPUTS ||
        dyn->nterms < 0 || dyn->nterms > HJI_MAX_TERMS)
        return nfail(HJI_E_INVALID, "m, q must be 0..4 and nterms 0..8");
    if ((dyn->m > 0 && (!dyn->G || !dyn->ulo || !dyn->uhi)) ||
        (dyn->q > 0 && (!dyn->E || !dyn->dlo || !dyn->dhi)) ||
        (dyn->nterms > 0 && (!dyn->term_row || !dyn->term_axis || !dyn->term_fn || !dyn->term_w)))
        return nfail(HJI_E_INVALID, "dynamics arrays missing");
    InstDesc D;
    std::memset(&D, 0, sizeof(D));
    hji::Dyn& f = D.dyn;
    f.m = dyn->m;
    f.q = dyn->q;
    f.nterms = dyn->nterms;
    for (int i = 0; i < ndim; ++i) {
        f.c[i] = dyn->c ? dyn->c[i] : 0.0;
        for (int j = 0; j < ndim; ++j) f.A[i * HJI_MAX_DIM + j] = dyn->A ? dyn->A[i * ndim + j] : 0.0;
        for (int j = 0; j < dyn->m; ++j) f.G[i * HJI_MAX_INPUTS + j] = dyn->G[i * dyn->m + j];
        for (int j = 0; j < dyn->q; ++j) f.E[i * HJI_MAX_INPUTS + j] = dyn->E[i * dyn->q + j];
    }
    for (int j = 0; j < dyn->m; ++j) {
        f.ulo[j] = dyn->ulo[j];
        f.uhi[j] = dyn->uhi[j];
        if (!(f.ulo[j] <= f.uhi[j])) return nfail(HJI_E_INVALID, "ulo > uhi");
    }
    for (int j = 0; j < dyn->q; ++j) {
        f.dlo[j] = dyn->dlo[j];
        f.dhi[j] = dyn->dhi[j];
        if (!(f.dlo[j] <= f.dhi[j])) return nfail(HJI_E_INVALID, "dlo > dhi");
    }
    for (int t = 0; t < dyn->nterms; ++t) {
        if (dyn->term_row[t] < 0 || dyn->term_row[t] >= ndim || dyn->term_axis[t] < 0 ||
            dyn->term_axis[t] >= ndim || dyn->term_fn[t] < HJI_FN_TAN || dyn->term_fn[t] > HJI_FN_COS)
            return nfail(HJI_E_INVALID, "bad term");
        f.term_row[t] = dyn->term_row[t];
        f.term_axis[t] = dyn->term_axis[t];
        f.term_fn[t] = dyn->term_fn[t];
        f.term_w[t] = dyn->term_w[t];
    }
    if (!all_finite(f.c, HJI_MAX_DIM) || !all_finite(f.A, HJI_MAX_DIM * HJI_MAX_DIM) ||
        !all_finite(f.G, HJI_MAX_DIM * HJI_MAX_INPUTS) || !all_finite(f.E, HJI_MAX_DIM * HJI_MAX_INPUTS) ||
        !all_finite(f.ulo, HJI_MAX_INPUTS) || !all_finite(f.uhi, HJI_MAX_INPUTS) ||
        !all_finite(f.dlo, HJI_MAX_INPUTS) || !all_finite(f.dhi, HJI_MAX_INPUTS) ||
        !all_finite(f.term_w, HJI_MAX_TERMS))
        return nfail(HJI_E_INVALID, "dynamics contain NaN or Inf");

    // Scratch layout and the size check.
    const bool f32 = prec == HJI_F32;
    const size_t es = f32 ? 4 : 8;
    // Tile shape: a forced 2-D variant (tile_variant 1..3) or variant 0
    // (no autotuned choice is consulted here).
    const int variant = (ndim == 2 && o->tile_variant > 0) ? o->tile_variant - 1 : 0;
    long long tx, ty, planes = 1;
    int TX, TY;
    hji::tile_dims(ndim, variant, TY, TX);
    tx = (n[ndim - 1] + TX - 1) / TX;
    ty = ndim >= 2 ? (n[ndim - 2] + TY - 1) / TY : 1;
    for (int a = 0; a < ndim - 2; ++a) planes *= n[a];
    const long long ntiles = tx * ty * planes;
    const long long pitch = hji::pitch_of(n[ndim - 1]);
    const long long rows = cells / n[ndim - 1];
    const long long nalloc = pitch * rows;
    const size_t field = align256((size_t)nalloc * es);
    size_t off = 0;
    const size_t o_state = off; off += align256(sizeof(InstState));
    const size_t o_desc = off;  off += align256(sizeof(InstDesc));
    const size_t o_ints = off;  off += 256;
    const size_t o_tiles = off; off += align256((size_t)ntiles * sizeof(unsigned long long));
    const size_t o_table = off; off += align256((size_t)HJI_MAX_TERMS * nmax * es);
    const size_t o_v0 = off;    off += field;
    const size_t o_v1 = off;    off += field;
    const size_t o_l = off;     off += field;
    const size_t o_w1 = off;    off += o->rk_order >= 2 ? field : 0;
    const size_t o_w2 = off;    off += o->rk_order >= 3 ? field : 0;
    const size_t o_lo = off;    off += f32 ? field : 0;
    const size_t o_lo1 = off;   off += f32 ? field : 0;
    if (off > (size_t)HJI_NOALLOC_SCRATCH_BYTES) {
        std::snprintf(g_err, sizeof(g_err),
                      "grid needs %zu bytes of scratch; hji_solve_noalloc holds %u", off,
                      (unsigned)HJI_NOALLOC_SCRATCH_BYTES);
        return HJI_E_INVALID;
    }

    // Once per device and context: the device address of the scratch array.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ncuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return nfail(HJI_E_INVALID, "device index out of range");
    unsigned char* base = nullptr;
    {
        const hji_status as = scratch_address(dev, s, &base);
        if (as != HJI_OK) return as;
    }
    InstState* d_state = reinterpret_cast<InstState*>(base + o_state);
    InstDesc* d_desc = reinterpret_cast<InstDesc*>(base + o_desc);
    int* d_ints = reinterpret_cast<int*>(base + o_ints);  // [0] active, [1] ntiles
    unsigned long long* d_tiles = reinterpret_cast<unsigned long long*>(base + o_tiles);

    D.ndim = ndim;
    for (int a = HJI_MAX_DIM - 1; a >= 0; --a) {
        D.n[a] = a < ndim ? (int)n[a] : 1;
        D.periodic[a] = (a < ndim && periodic) ? (periodic[a] != 0) : 0;
        D.lo[a] = a < ndim ? lo[a] : 0.0;
        D.dx[a] = a < ndim ? (D.periodic[a] ? (hi[a] - lo[a]) / (double)n[a]
                                            : (hi[a] - lo[a]) / (double)(n[a] - 1))
                           : 1.0;
    }
    {
        long long stride = 1;  // C order, fastest axis padded to the pitch
        for (int a = ndim - 1; a >= 0; --a) {
            D.stride[a] = stride;
            stride *= (a == ndim - 1) ? pitch : n[a];
        }
    }
    D.ncells = cells;
    D.nalloc = nalloc;
    D.cfl = o->cfl;
    D.tol = o->tol;
    D.tol_rate = o->tol_rate;
    D.brs = o->brs;
    D.discount = o->discount;
    D.horizon = o->horizon;
    D.max_steps = o->max_steps > 0 ? o->max_steps : 1000000;
    D.V[0] = base + o_v0;
    D.V[1] = base + o_v1;
    D.W1 = o->rk_order >= 2 ? base + o_w1 : nullptr;
    D.W2 = o->rk_order >= 3 ? base + o_w2 : nullptr;
    D.Vlo[0] = f32 ? base + o_lo : nullptr;
    D.Vlo[1] = f32 ? base + o_lo1 : nullptr;
    D.l = base + o_l;
    D.table = base + o_table;
    D.table_stride = nmax;
    D.tiles_x = tx;
    D.tiles_y = ty;
    D.tiles_per_plane = tx * ty;
    D.ntiles = ntiles;
    D.state = d_state;
    D.active = d_ints;
    D.kinit = o->init == HJI_INIT_STANDARD ? nullptr : D.V[1];
    D.kinit_lo = nullptr;
    {
        const char* why = nullptr;
        if (!hji::encode_maps(D, f32, o->scheme, variant, &why)) return nfail(HJI_E_CUDA, why);
    }
    // l (and k, or the caller's previous value for HJI_INIT_RESIDENT) into
    // the padded scratch fields.
    const size_t wrow = (size_t)n[ndim - 1] * es, prow = (size_t)pitch * es;
    if (rows > 1 && prow >= (1ull << 31)) return nfail(HJI_E_INVALID, "rows too long for hji_solve_noalloc");
    auto rows_copy = [&](void* dst, size_t dp, const void* src, size_t sp) {
        if (rows == 1 || dp == sp)
            return cudaMemcpyAsync(dst, src, wrow * (size_t)rows, cudaMemcpyDeviceToDevice, s);
        return cudaMemcpy2DAsync(dst, dp, src, sp, wrow, (size_t)rows, cudaMemcpyDeviceToDevice, s);
    };

    const int counts[2] = {1, (int)ntiles};
    e = rows_copy(D.l, prow, l, wrow);
    if (e == cudaSuccess && o->init != HJI_INIT_STANDARD)
        e = rows_copy(D.V[1], prow, o->init == HJI_INIT_USER_K ? k : v_out, wrow);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_state, 0, sizeof(InstState), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_desc, &D, sizeof(InstDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ints, counts, sizeof(counts), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        long long b = (ntiles + 255) / 256;
        fill_tiles<<<(int)(b < 1024 ? (b < 1 ? 1 : b) : 1024), 256, 0, s>>>(d_tiles, ntiles);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = hji::launch_setup(d_desc, &D, 1, f32, s);
    if (e == cudaSuccess) e = hji::launch_init(d_desc, &D, 1, f32, s);
    InstState hs;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, d_state, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ncuda(e, "set-up");
    if (hs.nonfinite) return nfail(HJI_E_INVALID, "l or k contains NaN or Inf");
    if (hs.status == 2) return nfail(HJI_E_INVALID, "dynamics vanish on the grid: no finite CFL step");

    // The march: chunks of check_every steps launched directly (no graph).
    hji::StageLauncher L[3];
    int ins[3], outs[3];
    double aV[3], aE[3];
    int ns;
    if (o->rk_order == 1) {
        ns = 1;
        ins[0] = 0; outs[0] = 3; aV[0] = 0.0; aE[0] = 1.0;
    } else if (o->rk_order == 2) {
        ns = 2;
        ins[0] = 0; outs[0] = 1; aV[0] = 0.0; aE[0] = 1.0;
        ins[1] = 1; outs[1] = 3; aV[1] = 0.5; aE[1] = 0.5;
    } else {
        ns = 3;
        ins[0] = 0; outs[0] = 1; aV[0] = 0.0; aE[0] = 1.0;
        ins[1] = 1; outs[1] = 2; aV[1] = 0.75; aE[1] = 0.25;
        ins[2] = 2; outs[2] = 3; aV[2] = 1.0 / 3.0; aE[2] = 2.0 / 3.0;
    }
    int sms = 1;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return ncuda(e, "cudaDeviceGetAttribute");
    long long grid[3];  // per stage: as many CTAs as fit on every SM, at most one per tile
    for (int i = 0; i < ns; ++i) {
        const bool last = i == ns - 1;
        L[i] = f32 ? hji::stage_launcher_f32(ndim, o->scheme, last, variant)
                   : hji::stage_launcher_f64(ndim, o->scheme, last, variant);
        if (!L[i]) return nfail(HJI_E_INVALID, "no kernel for this ndim/scheme");
        const int b = f32 ? hji::stage_max_blocks_f32(ndim, o->scheme, last, variant)
                          : hji::stage_max_blocks_f64(ndim, o->scheme, last, variant);
        grid[i] = (long long)sms * b;
        if (grid[i] > ntiles) grid[i] = ntiles;
        if (grid[i] < 1) grid[i] = 1;
    }
    const int chunk = o->check_every > 0 ? o->check_every : 32;
    long long launches = 2 + (dyn->nterms > 0 ? 1 : 0) + 1;
    for (;;) {
        for (int st = 0; st < chunk && e == cudaSuccess; ++st) {
            for (int i = 0; i < ns && e == cudaSuccess; ++i) {
                hji::StageArgs a{d_desc, d_tiles, d_ints + 1, ins[i], outs[i], aV[i], aE[i],
                                 (float)aV[i], (float)aE[i], aV[i] != 0.0 ? 1 : 0};
                e = L[i](a, (int)grid[i], s);
                ++launches;
            }
        }
        int active = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&active, d_ints, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ncuda(e, "march");
        if (active <= 0) break;
    }
    e = cudaMemcpyAsync(&hs, d_state, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = rows_copy(v_out, wrow, hs.cur == 1 ? D.V[1] : D.V[0], prow);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ncuda(e, "final state");
    if (stats) {
        stats->steps = hs.steps;
        stats->tau = hs.tau;
        stats->dt = hs.dt;
        stats->final_max_dV = hs.last_delta;
        stats->wall_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        for (int a = 0; a < HJI_MAX_DIM; ++a) stats->alpha[a] = a < ndim ? hs.alpha[a] : 0.0;
        stats->converged = hs.converged;
        stats->kernel_launches = launches;
    }
    if (hs.check_count) return nfail(HJI_E_CHECK, hji::check_message(hs).c_str());
    if (hs.status == 1) return nfail(HJI_E_NONFINITE, "the march produced NaN or Inf");
    if (hs.status == 4) return nfail(HJI_E_TIMEOUT, "a bounded device wait gave up");
    if (!hs.converged) return nfail(HJI_E_NOT_CONVERGED, "stopped by the horizon or the step cap");
    g_err[0] = '\0';
    return HJI_OK;
}
