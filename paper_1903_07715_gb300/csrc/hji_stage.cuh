// The fused Runge-Kutta stage kernel: one launch advances one stage of every
// live instance in the batch.  Per tile of nodes it
//   1. stages the stencil input W (tile + ghost halo of the two fastest axes)
//      in shared memory, building ghost nodes beyond the grid edge by linear
//      extrapolation (or periodic wrap) while loading;
//   2. forms the one-sided derivatives p-, p+ along every axis (ENO1, ENO2 or
//      HJ-WENO5; slower axes read their stencil lines from L2 directly);
//   3. evaluates the closed-form control-affine Hamiltonian of Eq. (6) at the
//      averaged gradient plus the Lax-Friedrichs dissipation;
//   4. combines the Euler stage W + dt L(W) with V^n (TVD Runge-Kutta);
//   5. on the last stage applies min(., l) (Eq. (7)-(8)), reduces
//      max|V^{n+1} - V^n| (warp shuffle -> CTA -> one 64-bit atomic), and the
//      CTA finishing an instance's last tile advances that instance's step
//      counter, tau, stop flag and buffer index.
// Tiles of instances that have stopped are skipped, so launches queued after
// convergence do no work and no step past the stop point ever runs.
#pragma once

#include <cfloat>

#include "hji_common.cuh"

namespace hji {

template <typename T>
struct Num;
template <>
struct Num<double> {
    static __device__ __forceinline__ double weno_tiny() { return 1e-60; }
};

template <int SCHEME>
struct Ghost {
    static constexpr int G = SCHEME == HJI_ENO1 ? 1 : (SCHEME == HJI_ENO2 ? 2 : 3);
};

// Of two second differences the one of smaller magnitude; a tie keeps the
// lower-index one.  The comparison is made on undivided differences, which
// selects exactly as comparing Q = S / (2 dx) would.
template <typename T>
__device__ __forceinline__ T smaller_mag(T a, T b) {
    return fabs(a) <= fabs(b) ? a : b;
}

// HJ-WENO5 (Jiang and Peng) on undivided one-sided differences v1..v5, with
// eps = 1e-6 max(v^2) + tiny as in the textbook form (the relative part is
// scale free, so undivided differences give the divided-difference weights).
// FP64 forms the normalised weights d_k / (S_k + eps)^2 as
// d_k q_k / sum_j d_j q_j with q_1 = (b2 b3)^2, q_2 = (b1 b3)^2,
// q_3 = (b1 b2)^2, b_k = S_k + eps: one division.  FP32 uses the fast
// reciprocals r_k = 1/b_k, a_k = d_k r_k^2 and 1/sum a_k; tiny = 1e-18 keeps
// sum a_k below 2^126 (the range of the fast division) while exceeding
// 1e-6 max(v^2) only where every |v| < 1e-6 (flat data, where the weights do
// not matter).
template <typename T>
__device__ __forceinline__ T weno5(T v1, T v2, T v3, T v4, T v5) {
    const T phi1 = v1 * T(1.0 / 3.0) - v2 * T(7.0 / 6.0) + v3 * T(11.0 / 6.0);
    const T phi2 = -v2 * T(1.0 / 6.0) + v3 * T(5.0 / 6.0) + v4 * T(1.0 / 3.0);
    const T phi3 = v3 * T(1.0 / 3.0) + v4 * T(5.0 / 6.0) - v5 * T(1.0 / 6.0);
    const T a = v1 - T(2) * v2 + v3, b = v1 - T(4) * v2 + T(3) * v3;
    const T c = v2 - T(2) * v3 + v4, d = v2 - v4;
    const T e = v3 - T(2) * v4 + v5, f = T(3) * v3 - T(4) * v4 + v5;
    const T s1 = T(13.0 / 12.0) * a * a + T(0.25) * b * b;
    const T s2 = T(13.0 / 12.0) * c * c + T(0.25) * d * d;
    const T s3 = T(13.0 / 12.0) * e * e + T(0.25) * f * f;
    const T vm = fmax(fmax(fmax(v1 * v1, v2 * v2), fmax(v3 * v3, v4 * v4)), v5 * v5);
    if constexpr (sizeof(T) == 4) {
        const float eps = 1e-6f * vm + 1e-18f;
        const float r1 = __fdividef(1.0f, s1 + eps);
        const float r2 = __fdividef(1.0f, s2 + eps);
        const float r3 = __fdividef(1.0f, s3 + eps);
        const float a1 = 0.1f * (r1 * r1), a2 = 0.6f * (r2 * r2), a3 = 0.3f * (r3 * r3);
        const float num = a1 * phi1 + a2 * phi2 + a3 * phi3;
        return __fdividef(num, a1 + a2 + a3);
    } else {
        const T eps = T(1e-6) * vm + Num<T>::weno_tiny();
        const T b1 = s1 + eps, b2 = s2 + eps, b3 = s3 + eps;
        const T b12 = b1 * b2, b13 = b1 * b3, b23 = b2 * b3;
        const T w1 = T(0.1) * (b23 * b23);
        const T w2 = T(0.6) * (b13 * b13);
        const T w3 = T(0.3) * (b12 * b12);
        const T num = w1 * phi1 + w2 * phi2 + w3 * phi3;
        return num / (w1 + w2 + w3);
    }
}

// (p-, p+) at node c from the 2G undivided differences D[k] = W[k+1] - W[k]
// of its stencil line W[0..2G] (node c = W[G]; D[G-1] is the backward and
// D[G] the forward difference).
template <typename T, int SCHEME>
__device__ __forceinline__ void one_sided_diffs(const T* D, T inv_dx, T& pm, T& pp) {
    if constexpr (SCHEME == HJI_ENO1) {
        pm = D[0] * inv_dx;
        pp = D[1] * inv_dx;
    } else if constexpr (SCHEME == HJI_ENO2) {
        const T Sm = D[1] - D[0], S0 = D[2] - D[1], Sp = D[3] - D[2];
        pm = (D[1] + T(0.5) * smaller_mag(Sm, S0)) * inv_dx;
        pp = (D[2] - T(0.5) * smaller_mag(S0, Sp)) * inv_dx;
    } else {
        pm = weno5<T>(D[0], D[1], D[2], D[3], D[4]) * inv_dx;
        pp = weno5<T>(D[5], D[4], D[3], D[2], D[1]) * inv_dx;
    }
}

// A value on the grid as an unevaluated sum h + l.  FP64 grids use l = 0.
// FP32 grids use h = the high word of V^n and l = its low word plus the
// stage increment: differences of neighbours, (h1 - h0) + (l1 - l0), then
// keep the precision of the difference itself instead of the precision of
// the value (the high-word subtraction of close neighbours is exact).
template <typename T>
struct Pair {
    T h, l;
};

template <typename T>
__device__ __forceinline__ Pair<T> load_pair(const T* __restrict__ h, const T* __restrict__ lo,
                                            const T* __restrict__ d, long long i) {
    Pair<T> p;
    p.h = __ldg(h + i);
    p.l = T(0);
    if (lo != nullptr) p.l = __ldg(lo + i);
    if (d != nullptr) p.l += __ldg(d + i);
    return p;
}

// The ghost node e + k (e - i1) (linear extrapolation by k nodes beyond the
// edge node e, i1 its inner neighbour).  With l = 0 (FP64) this is exactly
// the textbook expression; with pairs the rounding errors of k*(e.h - i1.h)
// and of the high-word sum are carried into the low word.
template <typename T>
__device__ __forceinline__ Pair<T> extrapolate(Pair<T> e, Pair<T> i1, int k) {
    Pair<T> g;
    const T kk = T(k);
    if constexpr (sizeof(T) == 8) {
        g.h = e.h + kk * (e.h - i1.h);
        g.l = T(0);
    } else {
        const T dh = e.h - i1.h;
        const T t = kk * dh;
        const T te = fmaf(kk, dh, -t);      // exact error of the product
        const T sh = e.h + t;               // two-sum of e.h + t
        const T bp = sh - e.h;
        const T se = (e.h - (sh - bp)) + (t - bp);
        g.h = sh;
        g.l = e.l + kk * (e.l - i1.l) + (te + se);
    }
    return g;
}

// Node j (possibly outside [0, n)) of a line with element stride s whose
// node 0 is at element offset 0 of h/lo/d: periodic wrap, or extrapolation.
template <typename T>
__device__ __forceinline__ Pair<T> line_pair(const T* __restrict__ h, const T* __restrict__ lo,
                                            const T* __restrict__ d, int j, int n, long long s,
                                            int periodic) {
    if (j >= 0 && j < n) return load_pair(h, lo, d, (long long)j * s);
    if (periodic) {
        int w = j % n;
        if (w < 0) w += n;
        return load_pair(h, lo, d, (long long)w * s);
    }
    const bool low = j < 0;
    const int k = low ? -j : j - (n - 1);
    const Pair<T> e = load_pair(h, lo, d, (long long)(low ? 0 : n - 1) * s);
    const Pair<T> i1 = load_pair(h, lo, d, (long long)(low ? 1 : n - 2) * s);
    return extrapolate(e, i1, k);
}

// Undivided difference of two neighbouring pairs.
template <typename T>
__device__ __forceinline__ T pair_diff(const Pair<T>& b, const Pair<T>& a) {
    if constexpr (sizeof(T) == 8) {
        return b.h - a.h;
    } else {
        return (b.h - a.h) + (b.l - a.l);
    }
}

// Shared-memory copy of what a tile needs from its instance, in precision T.
template <typename T>
struct TileCtx {
    int inst;
    int stop;
    int cur;
    int m, q, nterms;
    int n[MAXD];
    int periodic[MAXD];
    long long stride[MAXD];
    long long tiles_x, tiles_per_plane, ntiles;
    T lo[MAXD], dx[MAXD], inv_dx[MAXD], half_alpha[MAXD];
    T c[MAXD], A[MAXD * MAXD], G[MAXD * MAXU], E[MAXD * MAXU];
    T ulo[MAXU], uhi[MAXU], dlo[MAXU], dhi[MAXU];
    int term_row[MAXT], term_axis[MAXT];
    T dt;
    const T* win;   // stencil input (FP64: the stage state; FP32: V^n hi word)
    const T* din;   // FP32: stage increment added to win (null for stage 1)
    const T* vcur;
    T* wout;
    T* vlo;         // FP32: low word of V^n, updated in place by the last stage
    const T* l;
    const T* table;
    long long table_stride;
};

// Fill the tile context; called by every thread of the CTA (each copies a
// slice), followed by __syncthreads() at the call site.
static_assert(MAXD == 4 && MAXU == 4 && MAXT == 8 && kThreads > 96,
              "load_ctx hands out slices for these sizes");
template <typename T>
__device__ void load_ctx(TileCtx<T>& C, const InstDesc* __restrict__ insts, int inst,
                         const StageArgs& a) {
    const InstDesc& D = insts[inst];
    const int t = threadIdx.x;
    if (t < MAXD * MAXD) C.A[t] = T(D.dyn.A[t]);
    else if (t < 32) C.G[t - 16] = T(D.dyn.G[t - 16]);
    else if (t < 48) C.E[t - 32] = T(D.dyn.E[t - 32]);
    else if (t < 52) C.ulo[t - 48] = T(D.dyn.ulo[t - 48]);
    else if (t < 56) C.uhi[t - 52] = T(D.dyn.uhi[t - 52]);
    else if (t < 60) C.dlo[t - 56] = T(D.dyn.dlo[t - 56]);
    else if (t < 64) C.dhi[t - 60] = T(D.dyn.dhi[t - 60]);
    else if (t < 72) {
        C.term_row[t - 64] = D.dyn.term_row[t - 64];
        C.term_axis[t - 64] = D.dyn.term_axis[t - 64];
    } else if (t < 76) {
        const int i = t - 72;
        InstState* st = D.state;
        C.n[i] = D.n[i];
        C.periodic[i] = D.periodic[i];
        C.stride[i] = D.stride[i];
        C.lo[i] = T(D.lo[i]);
        C.dx[i] = T(D.dx[i]);
        C.inv_dx[i] = T(1.0 / D.dx[i]);
        C.half_alpha[i] = T(0.5 * st->alpha[i]);
        C.c[i] = T(D.dyn.c[i]);
    } else if (t == 96) {
        InstState* st = D.state;
        const int cur = *((volatile int*)&st->cur);
        C.inst = inst;
        C.stop = *((volatile int*)&st->stop);
        C.cur = cur;
        C.m = D.dyn.m;
        C.q = D.dyn.q;
        C.nterms = D.dyn.nterms;
        C.dt = T(*((volatile double*)&st->dt));
        C.tiles_x = D.tiles_x;
        C.tiles_per_plane = D.tiles_per_plane;
        C.ntiles = D.ntiles;
        const T* vc = static_cast<const T*>(D.V[cur]);
        const T* stage =
            a.stage_in == 0 ? nullptr : static_cast<const T*>(a.stage_in == 1 ? D.W1 : D.W2);
        C.vcur = vc;
        if constexpr (sizeof(T) == 4) {
            C.win = vc;
            C.din = stage;
        } else {
            C.win = stage ? stage : vc;
            C.din = nullptr;
        }
        C.vlo = static_cast<T*>(D.Vlo);
        C.wout = a.stage_out == 3 ? static_cast<T*>(D.V[cur ^ 1])
                                  : static_cast<T*>(a.stage_out == 1 ? D.W1 : D.W2);
        C.l = static_cast<const T*>(D.l);
        C.table = static_cast<const T*>(D.table);
        C.table_stride = D.table_stride;
    }
}

// Finish one step of an instance: called by the single thread whose tile was
// the instance's last one in this (last) stage.
__device__ inline void finish_step(const InstDesc& D) {
    InstState* st = D.state;
    __threadfence();
    const double d = __longlong_as_double((long long)atomicAdd(&st->delta_bits, 0ull));
    const long long steps = st->steps + 1;
    const double tau = st->tau + st->dt;
    st->last_delta = d;
    st->steps = steps;
    st->tau = tau;
    st->cur ^= 1;
    if (D.history != nullptr && steps - 1 < D.history_len) D.history[steps - 1] = d;
    st->delta_bits = 0ull;
    st->tiles_done = 0u;
    if (!(d <= DBL_MAX)) {  // NaN or Inf
        st->status = 1;
        st->stop = 1;
    } else if (d < D.tol + D.tol_rate * st->dt) {
        st->converged = 1;
        st->stop = 1;
    } else if (D.horizon > 0.0 && tau >= D.horizon) {
        st->stop = 1;
    } else if (steps >= D.max_steps) {
        st->stop = 1;
    }
    if (st->stop && D.active != nullptr) atomicSub(D.active, 1);
    __threadfence();
}

// ---- asynchronous global -> shared copies (cp.async, 4 or 8 bytes) ----
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Dynamic shared-memory layout of one stage kernel (units of T): two
// buffers of the staged tile (high words; FP32 also low words and stage
// increments), two buffers of l (and, FP64, of V^n) for the tile nodes, and
// the per-tile neighbour differences.
template <typename T, int NDIM, int SCHEME, bool LAST, int V>
struct StageSmem {
    static constexpr int G = Ghost<SCHEME>::G;
    static constexpr int TY = TileShape<NDIM, V>::TY;
    static constexpr int TX = TileShape<NDIM, V>::TX;
    static constexpr int GY = (NDIM >= 2) ? G : 0;
    static constexpr int SW = TX + 2 * G;
    static constexpr int SH = TY + 2 * GY;
    static constexpr int NR = SH * SW;
    static constexpr int NI = TY * TX;
    static constexpr int DXW = SW - 1;
    static constexpr int DYH = SH - 1;
    static constexpr bool INCR = sizeof(T) == 4;
    static constexpr int RH = 0;
    static constexpr int RL = RH + 2 * NR;
    static constexpr int RD = RL + (INCR ? 2 * NR : 0);
    static constexpr int LT = RD + (INCR ? 2 * NR : 0);
    static constexpr int VN = LT + (LAST ? 2 * NI : 0);
    static constexpr int DX = VN + ((LAST && !INCR) ? 2 * NI : 0);
    static constexpr int DY = DX + TY * DXW;
    static constexpr int NT = DY + (NDIM >= 2 ? DYH * TX : 0);
    static constexpr size_t BYTES = NT * sizeof(T);
};

// Where tile `local` of an instance sits.  N-D tiles are enumerated with the
// last slow axis fastest, so consecutive tiles of a CTA's run are neighbours
// along that axis and share most of their slow-axis stencil lines in L1.
struct TileGeo {
    long long base;
    int sidx[MAXD];
    int y0, x0;
};

template <typename T, int NDIM, int TY, int TX>
__device__ __forceinline__ TileGeo tile_geo(const TileCtx<T>& C, long long local) {
    TileGeo g;
    long long tip = local;
    g.base = 0;
    if constexpr (NDIM >= 3) {
        long long r = local;
        const int ls = NDIM - 3;  // last slow axis
        g.sidx[ls] = static_cast<int>(r % C.n[ls]);
        r /= C.n[ls];
        tip = r % C.tiles_per_plane;
        r /= C.tiles_per_plane;
        for (int ax = ls - 1; ax >= 0; --ax) {
            g.sidx[ax] = static_cast<int>(r % C.n[ax]);
            r /= C.n[ax];
        }
        for (int ax = 0; ax <= ls; ++ax) g.base += (long long)g.sidx[ax] * C.stride[ax];
    }
    const int by = static_cast<int>(tip / C.tiles_x);
    const int bx = static_cast<int>(tip - (long long)by * C.tiles_x);
    g.y0 = by * TY;
    g.x0 = bx * TX;
    return g;
}

// The CTA's walk over the tile list: runs of R consecutive tiles, run r
// going to CTA r mod gridDim (R = 1, plain cyclic, for short lists; up to 8
// for long ones, where consecutive tiles share an instance context).
struct TileWalk {
    int R, nruns, ntiles, ti, run, rr;
    __device__ TileWalk(int n) : ntiles(n) {
        R = max(1, min(8, n / (static_cast<int>(gridDim.x) * 4)));
        nruns = (n + R - 1) / R;
        run = blockIdx.x;
        ti = run * R;
        rr = 0;
    }
    __device__ int next() {
        if (run >= nruns) return -1;
        const int t = ti;
        if (++rr == R || ti + 1 >= ntiles) {
            run += gridDim.x;
            ti = run * R;
            rr = 0;
        } else {
            ++ti;
        }
        return t;
    }
};

template <typename T, int NDIM, int SCHEME, bool LAST, int V>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? (NDIM <= 2 ? 5 : 3) : 3)
    stage_kernel(const StageArgs a) {
    using L = StageSmem<T, NDIM, SCHEME, LAST, V>;
    constexpr int G = L::G, TY = L::TY, TX = L::TX, GY = L::GY, SW = L::SW, SH = L::SH;
    constexpr int NR = L::NR, NI = L::NI, DXW = L::DXW, DYH = L::DYH;
    constexpr int ROWS_PER_PASS = kThreads / TX;
    constexpr int CELLS = (TY + ROWS_PER_PASS - 1) / ROWS_PER_PASS;
    constexpr int AX = NDIM - 1;  // fastest axis
    constexpr int AY = NDIM >= 2 ? NDIM - 2 : 0;  // second fastest axis (used if NDIM >= 2)
    constexpr bool INCR = L::INCR;  // FP32: increments + compensated V

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* dxs = sm + L::DX;  // dxs[r][c] = W(r, c+1) - W(r, c), tile rows
    T* dys = sm + L::DY;  // dys[r][c] = W(r+1, c) - W(r, c)
    __shared__ TileCtx<T> C;
    __shared__ T red[kThreads / 32];

    const int ntiles = *a.ntiles;
    // Stage coefficients in the kernel's precision (no conversion in FP32).
    T cV, cE;
    if constexpr (INCR) {
        cV = a.aVf;
        cE = a.aEf;
    } else {
        cV = a.aV;
        cE = a.aE;
    }
    const bool reads_v = a.reads_v != 0;
    const bool has_d = INCR && a.stage_in != 0;
    const int tx = threadIdx.x % TX;
    const int ty = threadIdx.x / TX;
    int loaded = -1;

    // Staged-window walk of this thread: element s = threadIdx.x + k kThreads
    // sits at row r, column c; stepping by kThreads adds SR rows and SC
    // columns (no divisions in the loops).
    constexpr int SR = kThreads / SW, SC = kThreads % SW;
    const int r_first = threadIdx.x / SW, c_first = threadIdx.x % SW;

    // Issue the asynchronous copies of a tile's stencil input (and l, V^n)
    // into buffer b.  Nodes outside the grid are filled in afterwards.
    auto issue = [&](const TileGeo& tg, int b) {
        const int nx = C.n[AX];
        const int ny = NDIM >= 2 ? C.n[AY] : 1;
        const int sy = NDIM >= 2 ? static_cast<int>(C.stride[AY]) : 0;
        const T* hp = C.win + tg.base;
        const T* lp = INCR ? C.vlo + tg.base : nullptr;
        const T* dp = C.din ? C.din + tg.base : nullptr;
        const bool inside = tg.x0 - G >= 0 && tg.x0 + TX + G <= nx &&
                            (NDIM < 2 || (tg.y0 - GY >= 0 && tg.y0 + TY + GY <= ny));
        T* dh = sm + L::RH + b * NR;
        T* dl = sm + L::RL + b * NR;
        T* dd = sm + L::RD + b * NR;
        int r = r_first, c = c_first;
        int goff = (tg.y0 - GY + r) * sy + (tg.x0 - G + c);
        for (int s = threadIdx.x; s < NR; s += kThreads) {
            bool ok = inside;
            if (!inside) {
                const int gy = tg.y0 - GY + r, gx = tg.x0 - G + c;
                ok = ((NDIM < 2) || (gy >= 0 && gy < ny)) && gx >= 0 && gx < nx;
            }
            if (ok) {
                cp_async<sizeof(T)>(dh + s, hp + goff);
                if constexpr (INCR) {
                    cp_async<sizeof(T)>(dl + s, lp + goff);
                    if (dp) cp_async<sizeof(T)>(dd + s, dp + goff);
                }
            }
            c += SC;
            r += SR;
            goff += SR * sy + SC;
            if (c >= SW) {
                c -= SW;
                ++r;
                goff += sy - SW;
            }
        }
        if constexpr (LAST) {
            // Tile nodes: thread (ty, tx) takes rows ty, ty + ROWS_PER_PASS, ...
            const T* lg = C.l + tg.base;
            const T* vg = C.vcur + tg.base;
            const int gx = tg.x0 + tx;
#pragma unroll
            for (int k = 0; k < CELLS; ++k) {
                const int ry = ty + k * ROWS_PER_PASS;
                const int gy = tg.y0 + ry;
                if (ry < TY && gy < ny && gx < nx) {
                    const int si = ry * TX + tx;
                    const int gi = gy * sy + gx;
                    cp_async<sizeof(T)>(sm + L::LT + b * NI + si, lg + gi);
                    if constexpr (!INCR) cp_async<sizeof(T)>(sm + L::VN + b * NI + si, vg + gi);
                }
            }
        }
        cp_async_commit();
    };

    TileWalk walk(ntiles);
    int t = walk.next();
    int buf = 0;
    bool issued = false;
    while (t >= 0) {
        const unsigned long long entry = a.tiles[t];
        const int inst = static_cast<int>(entry >> 48);
        const long long local = static_cast<long long>(entry & 0xFFFFFFFFFFFFull);
        if (inst != loaded) {
            __syncthreads();  // everyone is done with the previous context
            load_ctx<T>(C, a.insts, inst, a);
            __syncthreads();
            loaded = inst;
        }
        if (C.stop) {  // uniform across the CTA; nothing was issued for it
            t = walk.next();
            issued = false;
            continue;
        }
        const TileGeo tg = tile_geo<T, NDIM, TY, TX>(C, local);
        if (!issued) issue(tg, buf);
        // Prefetch the next tile of the walk while this one is computed.
        const int tn = walk.next();
        bool pref = false;
        if (tn >= 0) {
            const unsigned long long en = a.tiles[tn];
            if (static_cast<int>(en >> 48) == inst) {
                issue(tile_geo<T, NDIM, TY, TX>(C, static_cast<long long>(en & 0xFFFFFFFFFFFFull)),
                      buf ^ 1);
                pref = true;
            }
        }
        if (pref) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();

        const int nx = C.n[AX];
        const int ny = NDIM >= 2 ? C.n[AY] : 1;
        const long long sy = NDIM >= 2 ? C.stride[AY] : 0;
        const int y0 = tg.y0, x0 = tg.x0;
        const T* __restrict__ hp = C.win + tg.base;
        const T* __restrict__ lp = INCR ? C.vlo + tg.base : nullptr;
        const T* __restrict__ dp = C.din ? C.din + tg.base : nullptr;
        T* rh = sm + L::RH + buf * NR;
        T* rl = sm + L::RL + buf * NR;
        T* rd = sm + L::RD + buf * NR;
        // FP32 stages 2+: fold the increment into the low word once per node.
        if constexpr (INCR) {
            if (has_d) {
                for (int s = threadIdx.x; s < NR; s += kThreads) rl[s] += rd[s];
                __syncthreads();
            }
        }
        auto pair_at = [&](int s) {
            Pair<T> p;
            p.h = rh[s];
            p.l = T(0);
            if constexpr (INCR) p.l = rl[s];
            return p;
        };

        // 1. Ghost nodes of tiles that reach beyond the grid edge: linear
        //    extrapolation from the two edge nodes (both inside the staged
        //    window), or, on a periodic axis, the wrapped node.
        const bool edge = x0 - G < 0 || x0 + TX + G > nx ||
                          (NDIM >= 2 && (y0 - GY < 0 || y0 + TY + GY > ny));
        if (edge) {
            for (int s = threadIdx.x; s < NR; s += kThreads) {
                const int r = s / SW, c = s - r * SW;
                const int gy = y0 - GY + r, gx = x0 - G + c;
                const bool iny = (NDIM < 2) || (gy >= 0 && gy < ny);
                const bool inx = gx >= 0 && gx < nx;
                if (iny && inx) continue;
                Pair<T> v;
                if (iny) {
                    if (C.periodic[AX]) {
                        const long long r0 = (long long)gy * sy;
                        v = line_pair<T>(hp + r0, lp ? lp + r0 : nullptr, dp ? dp + r0 : nullptr,
                                         gx, nx, 1, 1);
                    } else {
                        const bool low = gx < 0;
                        const int ce = (low ? 0 : nx - 1) - (x0 - G);
                        const int ci = (low ? 1 : nx - 2) - (x0 - G);
                        v = extrapolate(pair_at(r * SW + ce), pair_at(r * SW + ci),
                                        low ? -gx : gx - (nx - 1));
                    }
                } else if (inx) {
                    if (C.periodic[AY]) {
                        v = line_pair<T>(hp + gx, lp ? lp + gx : nullptr, dp ? dp + gx : nullptr,
                                         gy, ny, sy, 1);
                    } else {
                        const bool low = gy < 0;
                        const int re = (low ? 0 : ny - 1) - (y0 - GY);
                        const int ri = (low ? 1 : ny - 2) - (y0 - GY);
                        v = extrapolate(pair_at(re * SW + c), pair_at(ri * SW + c),
                                        low ? -gy : gy - (ny - 1));
                    }
                } else {
                    v.h = T(0);  // corner of the halo: never used by an axis-aligned stencil
                    v.l = T(0);
                }
                // Written after every read of this pass: ghost nodes only
                // read in-grid nodes, and no thread writes an in-grid node.
                rh[s] = v.h;
                if constexpr (INCR) rl[s] = v.l;
            }
            __syncthreads();
        }
        // 2. Each neighbour difference once per tile (FP32: on the pairs).
        {
            constexpr int XR = kThreads / DXW, XC = kThreads % DXW;
            int r = threadIdx.x / DXW, c = threadIdx.x % DXW;
            for (int i = threadIdx.x; i < TY * DXW; i += kThreads) {
                const int s0 = (r + GY) * SW + c;
                dxs[i] = pair_diff(pair_at(s0 + 1), pair_at(s0));
                c += XC;
                r += XR;
                if (c >= DXW) {
                    c -= DXW;
                    ++r;
                }
            }
        }
        if constexpr (NDIM >= 2) {
            for (int i = threadIdx.x; i < DYH * TX; i += kThreads) {
                const int r = i / TX, c = i - r * TX;
                const int s0 = r * SW + c + G;
                dys[i] = pair_diff(pair_at(s0 + SW), pair_at(s0));
            }
        }
        __syncthreads();

        // 3-5. Each thread updates CELLS nodes of the tile.
        T dmax = T(0);
#pragma unroll
        for (int k = 0; k < CELLS; ++k) {
            const int ry = ty + k * ROWS_PER_PASS;
            const int gy = y0 + ry, gx = x0 + tx;
            if (ry >= TY || gy >= ny || gx >= nx) continue;
            T pm[NDIM], pp[NDIM];
            T D[2 * G];
            const int c0 = (ry + GY) * SW + (tx + G);  // this node in the staged tile
            const int ci = ry * TX + tx;               // this node among the tile nodes
#pragma unroll
            for (int o = 0; o < 2 * G; ++o) D[o] = dxs[ry * DXW + tx + o];
            one_sided_diffs<T, SCHEME>(D, C.inv_dx[AX], pm[AX], pp[AX]);
            if constexpr (NDIM >= 2) {
#pragma unroll
                for (int o = 0; o < 2 * G; ++o) D[o] = dys[(ry + o) * TX + tx];
                one_sided_diffs<T, SCHEME>(D, C.inv_dx[AY], pm[AY], pp[AY]);
            }
            const long long off = (long long)gy * sy + gx;  // within the plane
#pragma unroll
            for (int ax = 0; ax < NDIM - 2; ++ax) {
                // Slower axes: the stencil line straight from global memory
                // (L1/L2).  The slow index is the same for the whole tile, so
                // a tile away from that axis' edges takes the strided path.
                const long long st = C.stride[ax];
                Pair<T> line[2 * G + 1];
                if (tg.sidx[ax] >= G && tg.sidx[ax] < C.n[ax] - G) {
#pragma unroll
                    for (int o = -G; o <= G; ++o)
                        line[o + G] = load_pair<T>(hp, lp, dp, off + o * st);
                } else {
                    const long long l0 = off - (long long)tg.sidx[ax] * st;
#pragma unroll
                    for (int o = -G; o <= G; ++o)
                        line[o + G] = line_pair<T>(hp + l0, lp ? lp + l0 : nullptr,
                                                   dp ? dp + l0 : nullptr, tg.sidx[ax] + o,
                                                   C.n[ax], st, C.periodic[ax]);
                }
#pragma unroll
                for (int o = 0; o < 2 * G; ++o) D[o] = pair_diff(line[o + 1], line[o]);
                one_sided_diffs<T, SCHEME>(D, C.inv_dx[ax], pm[ax], pp[ax]);
            }
            // Node coordinates and the drift f0(x) = c + A x + terms.
            int idx[NDIM];
#pragma unroll
            for (int ax = 0; ax < NDIM - 2; ++ax) idx[ax] = tg.sidx[ax];
            if constexpr (NDIM >= 2) idx[AY] = gy;
            idx[AX] = gx;
            T x[NDIM], pbar[NDIM];
#pragma unroll
            for (int ax = 0; ax < NDIM; ++ax) {
                x[ax] = C.lo[ax] + T(idx[ax]) * C.dx[ax];
                pbar[ax] = T(0.5) * (pp[ax] + pm[ax]);
            }
            T h = T(0);
#pragma unroll
            for (int i = 0; i < NDIM; ++i) {
                T fi = C.c[i];
#pragma unroll
                for (int j = 0; j < NDIM; ++j) fi += C.A[i * MAXD + j] * x[j];
                h += pbar[i] * fi;
            }
            for (int tt = 0; tt < C.nterms; ++tt) {
                const int ax = C.term_axis[tt];
                h += pbar[C.term_row[tt]] * __ldg(C.table + tt * C.table_stride + idx[ax]);
            }
            // max_u <G^T p, u> and min_d <E^T p, d> over the boxes (Eq. (6)).
            for (int j = 0; j < C.m; ++j) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < NDIM; ++i) s += C.G[i * MAXU + j] * pbar[i];
                h += fmax(s * C.ulo[j], s * C.uhi[j]);
            }
            for (int j = 0; j < C.q; ++j) {
                T r = T(0);
#pragma unroll
                for (int i = 0; i < NDIM; ++i) r += C.E[i * MAXU + j] * pbar[i];
                h += fmin(r * C.dlo[j], r * C.dhi[j]);
            }
            // Lax-Friedrichs: L = H(pbar) + sum alpha_a (p+ - p-) / 2.
            T Lv = h;
#pragma unroll
            for (int ax = 0; ax < NDIM; ++ax) Lv += C.half_alpha[ax] * (pp[ax] - pm[ax]);
            // Runge-Kutta stage combination.
            const long long gidx = tg.base + off;
            if constexpr (INCR) {
                const T dc = has_d ? rd[c0] : T(0);
                const T inc = cE * (dc + C.dt * Lv);
                if constexpr (!LAST) {
                    C.wout[gidx] = inc;
                } else {
                    // V^n + inc as an unevaluated float pair (error-free
                    // two-sum), then min(., l) of Eq. (7)-(8).
                    const T hi = rh[c0];
                    const T lo = has_d ? C.vlo[gidx] : rl[c0];
                    const T sl = lo + inc;
                    T nh = hi + sl;
                    const T bb = nh - hi;
                    T nl = (hi - (nh - bb)) + (sl - bb);
                    const T lv = sm[L::LT + buf * NI + ci];
                    if (nh > lv || (nh == lv && nl > T(0))) {
                        nh = lv;
                        nl = T(0);
                    }
                    const T ch = fabs((nh - hi) + (nl - lo));
                    dmax = (ch > dmax || ch != ch) ? ch : dmax;
                    C.wout[gidx] = nh;
                    C.vlo[gidx] = nl;
                }
            } else {
                const T wc = rh[c0];
                const T eul = wc + C.dt * Lv;
                T out;
                T vn = wc;
                if (reads_v) {
                    if constexpr (LAST) vn = sm[L::VN + buf * NI + ci];
                    else vn = __ldg(C.vcur + gidx);
                    out = cV * vn + cE * eul;
                } else {
                    out = eul;
                }
                if constexpr (LAST) {
                    const T lv = sm[L::LT + buf * NI + ci];
                    out = fmin(out, lv);
                    const T ch = fabs(out - vn);
                    dmax = (ch > dmax || ch != ch) ? ch : dmax;
                }
                C.wout[gidx] = out;
            }
        }

        if constexpr (LAST) {
            // CTA max of |dV| (NaN wins), then the instance-wide reduction.
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T other = __shfl_xor_sync(0xffffffffu, dmax, o);
                dmax = (other > dmax || other != other) ? other : dmax;
            }
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dmax;
            __syncthreads();
            if (threadIdx.x == 0) {
                T mt = red[0];
                for (int w = 1; w < kThreads / 32; ++w) mt = (red[w] > mt || red[w] != red[w]) ? red[w] : mt;
                const double m = static_cast<double>(mt);
                const InstDesc& D = a.insts[inst];
                InstState* st = D.state;
                atomicMax(&st->delta_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
                __threadfence();
                const unsigned int prev = atomicAdd(&st->tiles_done, 1u);
                if (prev + 1 == static_cast<unsigned int>(C.ntiles)) finish_step(D);
            }
        }
        __syncthreads();  // buffer `buf` is refilled by the prefetch after next
        buf ^= 1;
        t = tn;
        issued = pref;
    }
    cp_async_wait<0>();
}

template <typename T, int NDIM, int SCHEME, bool LAST, int V>
cudaError_t launch_stage(const StageArgs& a, int grid, cudaStream_t s) {
    using L = StageSmem<T, NDIM, SCHEME, LAST, V>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(stage_kernel<T, NDIM, SCHEME, LAST, V>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(L::BYTES));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    stage_kernel<T, NDIM, SCHEME, LAST, V><<<grid, kThreads, L::BYTES, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int NDIM, int SCHEME, bool LAST, int V>
int max_blocks_stage() {
    using L = StageSmem<T, NDIM, SCHEME, LAST, V>;
    cudaFuncSetAttribute(stage_kernel<T, NDIM, SCHEME, LAST, V>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L::BYTES));
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stage_kernel<T, NDIM, SCHEME, LAST, V>,
                                                      kThreads, L::BYTES) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

}  // namespace hji
