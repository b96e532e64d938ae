// Internal device-side data structures of the HJI reachability solver.
//
// One "instance" is one grid with its dynamics, value buffers and march state.
// Every kernel works on a batch of instances through a flat tile list, so a
// single grid is a batch of one and uneven grids share one launch.
#pragma once

#include <cstdint>
#include <string>
#include <cuda.h>
#include <cuda_runtime.h>

#include "hji.h"

namespace hji {

constexpr int MAXD = HJI_MAX_DIM;
constexpr int MAXU = HJI_MAX_INPUTS;
constexpr int MAXT = HJI_MAX_TERMS;
constexpr int kThreads = 256;  // every stencil kernel uses 256-thread CTAs

// Dynamics f(x,u,d) = c + A x + sum_t w_t phi_t(x[axis_t]) e_{row_t} + G u + E d
// (Sec. II-A, Eq. (1), control-affine form), stored dense at the maximum
// sizes so the kernels index with compile-time strides.
struct Dyn {
    int m, q, nterms, pad_;
    double c[MAXD];
    double A[MAXD * MAXD];  // A[i*MAXD + j]
    double G[MAXD * MAXU];  // G[i*MAXU + j]
    double E[MAXD * MAXU];  // E[i*MAXU + k]
    double ulo[MAXU], uhi[MAXU], dlo[MAXU], dhi[MAXU];
    double term_w[MAXT];
    int term_row[MAXT], term_axis[MAXT], term_fn[MAXT];
};

// Mutable march state of one instance (device memory, written by kernels).
// Per-instance constants of the stage kernels in one precision, formed once
// per solve by the set-up pass (FP64 arithmetic, then rounded), so that each
// stage kernel's per-CTA context load is plain copies: FP64 arithmetic runs
// at a small fraction of the FP32 rate on this GPU, and a few dozen dependent
// FP64 operations per CTA at the start of every launch were on its critical
// path.
//
// The stage kernels carry p- + p+ = 2 pbar per axis instead of pbar, so the
// Hamiltonian's constants (cmid, A, G, E, and the term table) are stored
// halved: every term of H is linear in pbar, and halving is exact.
template <typename T>
struct CtxConst {
    T lo[MAXD], dx[MAXD], inv_dx[MAXD], half_alpha[MAXD];
    T cmid[MAXD];  // c + G umid + E dmid: the box centres' share of the drift
    T A[MAXD * MAXD], G[MAXD * MAXU], E[MAXD * MAXU];
    T urad[MAXU], drad[MAXU];  // half-widths of the control and disturbance boxes
    T arad[MAXD];              // sum_j urad_j |G_aj| + sum_k drad_k |E_ak| per row a
    T dt;
};

struct InstState {
    unsigned long long delta_bits;  // max|dV| of the step in flight (bits of a double >= 0)
    unsigned int tiles_done;        // tiles of the step's last stage finished so far
    int cur;                        // index (0/1) of the buffer holding V^n
    int stop;                       // 1 once converged, capped or failed
    int converged;                  // 1 if max|dV| < tol ended the march
    int status;                     // 0 ok, 1 non-finite value, 2 no finite dt, 3 bad input
    int pad_;
    long long steps;                // full steps taken
    double tau;                     // steps * dt, accumulated in FP64
    double last_delta;              // max|dV| of the last finished step
    // set-up reductions (alpha, CFL rate) for this solve
    unsigned long long alpha_bits[MAXD];
    unsigned long long rate_bits;
    unsigned int setup_done;
    unsigned int nonfinite;         // set by the init pass if l or k has NaN/Inf
    double dt;
    double alpha[MAXD];
    CtxConst<double> kd;  // the stage kernels' constants (set-up pass)
    CtxConst<float> kf;
    double stop_delta;    // tol + tol_rate dt: a step whose max|dV| is below it converges
    // Interval test (Sec. V): every K-th step compares V with the snapshot
    // taken K steps earlier; K = 0 when the test is off.
    long long interval_K;
    unsigned long long interval_bits;  // max|V - snapshot| of the step in flight (bits of a double)
    double last_interval_change;       // of the last finished interval
    // Bounds-checked debug build only (HJI_CHECKED): index checks that
    // failed, and the first one's site (CheckSite), index and extent.
    int check_count;
    int check_site;
    long long check_index;
    long long check_limit;
};

// Sites of the debug build's index checks (the message of a failed check
// names them).
enum CheckSite {
    CK_TILE = 1,     // tile index within the instance's tile count
    CK_TILE_GEO,     // tile origin and slow-axis indices inside the grid
    CK_TMA_X,        // tensor-copy x coordinate on a 16-byte boundary
    CK_TMA_DST,      // tensor-copy destination on a 128-byte boundary
    CK_GHOST_WRITE,  // ghost node slot inside the staged window
    CK_GHOST_READ,   // edge nodes an extrapolated ghost reads, inside the window
    CK_GHOST_LINE,   // periodic ghost line inside the field
    CK_DIFF_READ,    // window rows the y-differences read
    CK_DIFF_WRITE,   // slot of a y-difference
    CK_YSET_READ,    // y-differences a WENO5 set reads
    CK_YSET_WRITE,   // slot of a set's y-derivatives
    CK_PLANE,        // slow-axis stencil plane inside the field
    CK_XWINDOW,      // window row segment of a run's x-stencil
    CK_DIFF_Y,       // y-differences an ENO y-stencil reads
    CK_TABLE,        // per-term table entry
    CK_NODE_SMEM,    // staged l / V^n at the run's nodes
    CK_NODE_GLOBAL,  // the run's nodes in the fields it reads and writes
    CK_NUM_SITES
};

// The text of a failed check (host side).
std::string check_message(const InstState& S);

#ifdef HJI_CHECKED
// Record a failed index check: the first one's site, index and extent, and
// how many failed.
static __device__ __noinline__ void check_miss(InstState* st, int site, long long i, long long n) {
    if (atomicAdd(&st->check_count, 1) == 0) {
        st->check_site = site;
        st->check_index = i;
        st->check_limit = n;
    }
}
// [i, i + w) inside [0, n): i, else 0 after recording the miss.
__device__ __forceinline__ long long checked_index(InstState* st, int site, long long i, long long w,
                                                   long long n) {
    if (i < 0 || i + w > n) {
        check_miss(st, site, i, n);
        return 0;
    }
    return i;
}
// A condition that must hold; false after recording the miss.
__device__ __forceinline__ bool checked_cond(InstState* st, int site, bool ok, long long v,
                                             long long n) {
    if (!ok) check_miss(st, site, v, n);
    return ok;
}
#endif

// Tensor maps of one instance (TMA descriptors, encoded on the host):
// "window" maps copy a tile with its ghost halo (TX + 8 columns starting 4
// left of the tile, TY + 2G rows), "node" maps copy the tile's own nodes.
enum TensorMapSlot {
    TM_WIN_V0, TM_WIN_V1,    // V[0], V[1]: FP64 stage input / FP32 high word
    TM_WIN_LO0, TM_WIN_LO1,  // FP32 low words Vlo[0], Vlo[1]
    TM_WIN_W1, TM_WIN_W2,    // stage buffers (FP64 states, FP32 increments)
    TM_NODE_L,               // l
    TM_NODE_V0, TM_NODE_V1,  // FP64 V^n for the last stage's combination
    kNumMaps
};

// Read-only description of one instance for one solve.
//
// Fields are stored in C order with the fastest axis padded to a pitch that
// is a multiple of 8 elements (stride[ndim-2] = pitch), so that every row
// starts on a 32-byte boundary: the alignment TMA needs for its row strides
// and for 16-byte vector accesses of four FP32 (or two FP64) nodes.
struct InstDesc {
    CUtensorMap tm[kNumMaps];  // 128-byte aligned (the type says so)
    int ndim;
    int periodic[MAXD];
    int n[MAXD];
    long long stride[MAXD];   // element strides, C order, fastest axis padded
    long long ncells;         // nodes
    long long nalloc;         // elements of one field (pitch x rows)
    double lo[MAXD], dx[MAXD];
    Dyn dyn;
    double cfl, tol, horizon, tol_rate;
    double interval, interval_tol;  // Sec. V's interval test (interval 0: off)
    int brs;                  // 1: no projection onto V <= l (Eq. (5) alone)
    int local_lf;             // 1: node-wise Lax-Friedrichs coefficients
    double discount;          // gamma of discounted reachability (Sec. II-C); 0 or 1: off
    void* snap;               // its snapshot of V (the high word for FP32), or null
    long long max_steps;
    void* V[2];               // ping-pong value buffers: V[cur] = V^n
    void* W1;                 // stage buffers of the Runge-Kutta step: stage
    void* W2;                 // states (FP64) or stage increments (FP32)
    void* Vlo[2];             // FP32 only: low words, ping-pong with V: V^n = V[cur] + Vlo[cur]
    void* l;                  // target function l(x)
    void* table;              // per-term tables: table[t*n_max + i] = w_t phi_t(x_axis(i)) / 2
                              // (halved like the stage kernels' other drift constants)
    long long table_stride;
    double* history;          // optional max|dV| per step (FP64), may be null
    long long history_len;
    long long tiles_x, tiles_y, tiles_per_plane, ntiles;  // tile grid of this instance
    InstState* state;
    int* active;              // batch-wide count of instances still marching (may be null)
    const void* kinit;        // warm start read by the init pass (null: V0 = l)
    const void* kinit_lo;     // FP32: low word of kinit when it is a resident value (else null)
};

// Tile list entry: instance index in the high 16 bits, tile index within the
// instance in the low 48 bits.
__host__ __device__ inline unsigned long long make_tile(int inst, long long local) {
    return (static_cast<unsigned long long>(inst) << 48) |
           (static_cast<unsigned long long>(local) & 0xFFFFFFFFFFFFull);
}

// Tile shapes.  A thread updates one run of four consecutive nodes of the
// fastest axis.  1-D tiles are 248 nodes (the staged window of 256 is the
// largest TMA box; threads past the 62nd idle).  N-D tiles cover the two
// fastest axes at a fixed index of the slower axes (which are read from
// global memory / L2 directly): TY rows x TX columns with (TY + 1) x TX / 4
// = 256, so that the TY + 1 sets of five y-differences a WENO5 tile column
// needs are one per thread (the TY x TX / 4 runs of the tile use all but
// one row of threads).  Variant 0 is 31 x 32 nodes (the least halo per
// node), and 2-D grids also have variant 1 (15 x 64) and variant 2
// (63 x 16), which fit narrow or short grids with less padding; the
// autotuner picks per problem class.  Every shape runs the same per-node
// arithmetic, so results do not depend on it.
constexpr int kTileVariants = 3;
constexpr int kPitchAlign = 8;  // elements
template <int NDIM, int V = 0>
struct TileShape {
    static constexpr int TY = (NDIM == 1) ? 1 : (V == 1 ? 15 : (V == 2 ? 63 : 31));
    static constexpr int TX = (NDIM == 1) ? 248 : (V == 1 ? 64 : (V == 2 ? 16 : 32));
    static constexpr int GROUPS = TX / 4;  // 4-node runs per row
    static_assert(NDIM == 1 || (TY + 1) * GROUPS == kThreads, "one y-set per thread");
};
inline void tile_dims(int ndim, int variant, int& ty, int& tx) {
    if (ndim == 1) {
        ty = 1;
        tx = 248;
        return;
    }
    const int v = ndim == 2 ? variant : 0;
    ty = v == 1 ? 15 : (v == 2 ? 63 : 31);
    tx = v == 1 ? 64 : (v == 2 ? 16 : 32);
}
inline long long pitch_of(long long nx) { return (nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign; }

inline int ghost_width(int scheme) { return scheme == HJI_ENO1 ? 1 : (scheme == HJI_ENO2 ? 2 : 3); }

// Arguments of one Runge-Kutta stage launch.
//
// FP64 grids store stage states: the stencil input is W = V^n, W1 or W2 and
// the stage writes aV V^n + aE (W + dt L(W)).
// FP32 grids store stage increments D = W - V^n (small numbers keep full
// relative precision) and V^n as an unevaluated sum hi + lo of two floats:
// the stencil input is W = hi + D_in, a stage writes
// D_out = aE (D_in + dt L(W)), and the last stage adds its increment to
// (hi, lo) with an error-free two-sum.  Both are the same Runge-Kutta step:
// aV + aE = 1 gives aV V + aE (W + dt L) = V + aE (D_in + dt L).
struct StageArgs {
    const InstDesc* insts;
    const unsigned long long* tiles;
    const int* ntiles;     // device scalar: tiles in the list
    int stage_in;          // 0: V[cur], 1: W1/D1, 2: W2/D2 (stencil input)
    int stage_out;         // 1: W1/D1, 2: W2/D2, 3: V[cur^1]
    double aV, aE;
    float aVf, aEf;        // the same coefficients for FP32 kernels
    int reads_v;           // aV != 0
    // Known at launch for a single solve (0: read them from device memory,
    // as engines do, whose tile lists change between launches):
    int ntiles_imm;        // > 0: the number of tiles in the list
    int direct;            // 1: the list is one instance's tiles 0 .. n-1 in order
};

using StageLauncher = cudaError_t (*)(const StageArgs&, int grid, cudaStream_t);

// Arguments of the multi-step march kernel: one cooperative launch runs
// every RK stage (st[0..ns-1]) of up to `steps` steps, with a grid-wide
// barrier after each stage, and ends early once no instance is marching.
struct MarchArgs {
    StageArgs st[3];
    int ns;            // RK stages per step
    int steps;         // steps this launch may run
    unsigned* barrier; // grid-barrier counter, zero at launch
    const int* active; // instances of the batch still marching
    int* fault;        // set to 1 when a bounded wait gave up
};
using MarchLauncher = cudaError_t (*)(const MarchArgs&, int grid, cudaStream_t);
// Multi-step march kernels exist for 1-D and 2-D grids (null / 0 otherwise).
MarchLauncher march_launcher_f64(int ndim, int scheme, int variant = 0, bool interval = false);
MarchLauncher march_launcher_f32(int ndim, int scheme, int variant = 0, bool interval = false);
int march_max_blocks_f64(int ndim, int scheme, int variant = 0, bool interval = false);
int march_max_blocks_f32(int ndim, int scheme, int variant = 0, bool interval = false);

// Kernel dispatch tables (one per precision); `variant` selects the tile
// shape (only 2-D grids have more than variant 0); `interval` picks the last
// stage with Sec. V's interval test compiled in.
StageLauncher stage_launcher_f64(int ndim, int scheme, bool last, int variant = 0,
                                 bool interval = false);
// Local Lax-Friedrichs variants (default tile shape; the last stage has the
// interval test compiled in).
StageLauncher stage_launcher_llf_f64(int ndim, int scheme, bool last);
StageLauncher stage_launcher_llf_f32(int ndim, int scheme, bool last);
int stage_max_blocks_llf_f64(int ndim, int scheme, bool last);
int stage_max_blocks_llf_f32(int ndim, int scheme, bool last);
StageLauncher stage_launcher_f32(int ndim, int scheme, bool last, int variant = 0,
                                 bool interval = false);
int stage_max_blocks_f64(int ndim, int scheme, bool last, int variant = 0, bool interval = false);
int stage_max_blocks_f32(int ndim, int scheme, bool last, int variant = 0, bool interval = false);

// Arguments of the optimal-control pass (hji_control.cu): a grid's current
// value (padded C-order fields; FP32 grids add the low word) and the input
// matrices and bounds, in FP64 (converted to the kernel's precision).
struct ControlArgs {
    int n[MAXD];
    int periodic[MAXD];
    long long stride[MAXD];
    double inv_dx[MAXD];
    const void* v_hi;
    const void* v_lo;   // FP32: low word of the value (null for FP64)
    double G[MAXD * MAXU], E[MAXD * MAXU];
    double ulo[MAXU], uhi[MAXU], dlo[MAXU], dhi[MAXU];
    int m, q;
    long long ncells;
    void* u_out;        // m dense grid-shaped arrays, one after another
    void* d_out;        // q of them, or null
};
cudaError_t launch_control(const ControlArgs& a, bool f32, int ndim, int scheme, cudaStream_t s);

// Set-up kernels (hji_setup.cu).
cudaError_t launch_setup(const InstDesc* d_insts, const InstDesc* h_insts, int count, bool f32,
                         cudaStream_t s);
// One launch per pass covers all `count` instances (blockIdx.y picks one);
// the init pass reads each instance's warm start from its kinit / keep_lo.
cudaError_t launch_init(const InstDesc* d_insts, const InstDesc* h_insts, int count, bool f32,
                        cudaStream_t s);
// Encode the tensor maps of D for the given precision, scheme and tile
// variant (host; D's field pointers, sizes and strides must be set).
// Returns false (with a message) if the driver rejects a map.
bool encode_maps(InstDesc& D, bool f32, int scheme, int variant, const char** why);
// Bounded-wait self-test (hji_setup.cu): *d_result = 4 when the wait gave up.
cudaError_t launch_wait_selftest(unsigned long long limit_ns, int* d_result, cudaStream_t s);
// The debug build's check recorder on fixed indices (none of them is used to
// address memory): out[0..3] and the record in *st.  A no-op in the product
// build.
cudaError_t launch_check_selftest(InstState* st, long long* out, cudaStream_t s);
cudaError_t launch_convert(long long n, const void* src_hi, const void* src_lo, bool src_f32,
                           void* dst_hi, void* dst_lo, bool dst_f32, cudaStream_t s);

}  // namespace hji
