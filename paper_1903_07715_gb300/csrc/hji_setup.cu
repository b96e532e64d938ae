// Per-solve set-up passes, run once before the march:
//   * term tables: w_t phi_t(x_axis) / 2 per node of the term's axis, so the
//     stage kernel evaluates tan/sin/cos terms by a table read;
//   * dissipation coefficients and CFL step: alpha_a = max over nodes of
//     max_{u,d} |f_a(x,u,d)| and dt = cfl / max over nodes of
//     sum_a max_{u,d}|f_a| / dx_a, reduced in FP64 (warp shuffle -> CTA ->
//     64-bit atomics; the last CTA turns the maxima into dt);
//   * initial value: V = l (Sec. II-B) or V = min(k, l) (Sec. III, proof of
//     Thm. 1), flagging NaN/Inf in l or k.
#include <cfloat>

#include "hji_common.cuh"
#include "hji_stage.cuh"

namespace hji {

__device__ __forceinline__ double apply_fn(int fn, double x) {
    if (fn == HJI_FN_TAN) return tan(x);
    if (fn == HJI_FN_SIN) return sin(x);
    return cos(x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) table_kernel(const InstDesc* __restrict__ insts) {
    const InstDesc& D = insts[blockIdx.z];
    T* table = static_cast<T*>(D.table);
    for (int t = blockIdx.y; t < D.dyn.nterms; t += gridDim.y) {
        const int ax = D.dyn.term_axis[t];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D.n[ax];
             i += gridDim.x * blockDim.x) {
            const double x = D.lo[ax] + (double)i * D.dx[ax];
            // halved, like the other drift constants of the stage kernels
            table[t * D.table_stride + i] = T(0.5 * D.dyn.term_w[t] * apply_fn(D.dyn.term_fn[t], x));
        }
    }
}

constexpr int kAlphaTab = 2048;  // term values cached per CTA (FP64)
constexpr int kAlphaChunk = 16;  // consecutive nodes per alpha thread

// The stage kernels' per-instance constants in both precisions, from the
// descriptor and this solve's alpha and dt (thread 0 of the set-up pass's
// last CTA).
__device__ void fill_ctx_const(const InstDesc& D, InstState* st) {
    CtxConst<double>& kd = st->kd;
    CtxConst<float>& kf = st->kf;
    // cmid, A, G, E halved: the stage kernels multiply them by 2 pbar.
    for (int i = 0; i < MAXD * MAXD; ++i) {
        kd.A[i] = 0.5 * D.dyn.A[i];
        kf.A[i] = static_cast<float>(kd.A[i]);
    }
    for (int i = 0; i < MAXD * MAXU; ++i) {
        kd.G[i] = 0.5 * D.dyn.G[i];
        kf.G[i] = static_cast<float>(kd.G[i]);
        kd.E[i] = 0.5 * D.dyn.E[i];
        kf.E[i] = static_cast<float>(kd.E[i]);
    }
    for (int j = 0; j < MAXU; ++j) {
        kd.urad[j] = 0.5 * (D.dyn.uhi[j] - D.dyn.ulo[j]);
        kf.urad[j] = static_cast<float>(kd.urad[j]);
        kd.drad[j] = 0.5 * (D.dyn.dhi[j] - D.dyn.dlo[j]);
        kf.drad[j] = static_cast<float>(kd.drad[j]);
    }
    for (int i = 0; i < MAXD; ++i) {
        kd.lo[i] = D.lo[i];
        kd.dx[i] = D.dx[i];
        kd.inv_dx[i] = 1.0 / D.dx[i];
        kd.half_alpha[i] = 0.5 * st->alpha[i];
        double cm = D.dyn.c[i];
        for (int j = 0; j < MAXU; ++j) {
            cm += D.dyn.G[i * MAXU + j] * (0.5 * (D.dyn.ulo[j] + D.dyn.uhi[j]));
            cm += D.dyn.E[i * MAXU + j] * (0.5 * (D.dyn.dlo[j] + D.dyn.dhi[j]));
        }
        kd.cmid[i] = 0.5 * cm;
        double ar = 0.0;
        for (int j = 0; j < MAXU; ++j) {
            ar += fabs(D.dyn.G[i * MAXU + j]) * kd.urad[j];
            ar += fabs(D.dyn.E[i * MAXU + j]) * kd.drad[j];
        }
        kd.arad[i] = ar;
        kf.arad[i] = static_cast<float>(ar);
        kf.lo[i] = static_cast<float>(kd.lo[i]);
        kf.dx[i] = static_cast<float>(kd.dx[i]);
        kf.inv_dx[i] = static_cast<float>(kd.inv_dx[i]);
        kf.half_alpha[i] = static_cast<float>(kd.half_alpha[i]);
        kf.cmid[i] = static_cast<float>(kd.cmid[i]);
    }
    kd.dt = st->dt;
    kf.dt = static_cast<float>(st->dt);
    st->stop_delta = D.tol + D.tol_rate * st->dt;
    long long K = 0;
    if (D.interval > 0.0 && D.snap != nullptr) {
        K = llround(D.interval / st->dt);
        if (K < 1) K = 1;
    }
    st->interval_K = K;
    st->interval_bits = 0ull;
}

__global__ void __launch_bounds__(kThreads) alpha_kernel(const InstDesc* __restrict__ insts) {
    const InstDesc& D = insts[blockIdx.y];
    const int nd = D.ndim;
    const int fa = nd - 1;  // fastest axis
    const int nx = D.n[fa];
    const Dyn& f = D.dyn;
    // w_t phi_t(x) depends on one coordinate: tabulate it once per CTA when
    // the term axes are short enough, instead of once per node.
    __shared__ double tab[kAlphaTab];
    __shared__ int tab_off[MAXT];
    int total = 0;
    for (int t = 0; t < f.nterms; ++t) total += D.n[f.term_axis[t]];
    const bool use_tab = total <= kAlphaTab;
    if (use_tab) {
        int o = 0;
        for (int t = 0; t < f.nterms; ++t) {
            if (threadIdx.x == 0) tab_off[t] = o;
            const int ax = f.term_axis[t];
            for (int i = threadIdx.x; i < D.n[ax]; i += blockDim.x)
                tab[o + i] = f.term_w[t] * apply_fn(f.term_fn[t], D.lo[ax] + (double)i * D.dx[ax]);
            o += D.n[ax];
        }
    }
    __syncthreads();
    auto term = [&](int t, int i) {
        const int ax = f.term_axis[t];
        return use_tab ? tab[tab_off[t] + i]
                       : f.term_w[t] * apply_fn(f.term_fn[t], D.lo[ax] + (double)i * D.dx[ax]);
    };
    // f_a is affine in (u, d): its range over the boxes is centre +- radius,
    // so max |f_a| = |centre| + radius, with the radius the same at every
    // node and the centre c_a + G umid + E dmid + sum_b A_ab x_b + terms.
    // (Loops over axes run to MAXD with a guard, so the per-axis arrays stay
    // in registers.)
    double radius[MAXD], cconst[MAXD], inv_dx[MAXD];
#pragma unroll
    for (int a = 0; a < MAXD; ++a) {
        if (a >= nd) {
            radius[a] = cconst[a] = inv_dx[a] = 0.0;
            continue;
        }
        double c = f.c[a], r = 0.0;
        for (int j = 0; j < f.m; ++j) {
            c += f.G[a * MAXU + j] * (0.5 * (f.ulo[j] + f.uhi[j]));
            r += fabs(f.G[a * MAXU + j]) * (0.5 * (f.uhi[j] - f.ulo[j]));
        }
        for (int k = 0; k < f.q; ++k) {
            c += f.E[a * MAXU + k] * (0.5 * (f.dlo[k] + f.dhi[k]));
            r += fabs(f.E[a * MAXU + k]) * (0.5 * (f.dhi[k] - f.dlo[k]));
        }
        cconst[a] = c;
        radius[a] = r;
        inv_dx[a] = 1.0 / D.dx[a];
    }
    // Each thread takes chunks of consecutive nodes; along a row of the
    // fastest axis only x_fa changes, so the rest of each centre (rowc) is
    // formed once per row the chunk touches.
    constexpr int kChunk = kAlphaChunk;
    const int ncells = static_cast<int>(D.ncells);
    double amax[MAXD] = {0.0, 0.0, 0.0, 0.0};
    double rmax = 0.0;
    double rowc[MAXD];
    const long long nchunks = (static_cast<long long>(ncells) + kChunk - 1) / kChunk;
    for (long long ch = blockIdx.x * (long long)blockDim.x + threadIdx.x; ch < nchunks;
         ch += (long long)gridDim.x * blockDim.x) {
        int c = static_cast<int>(ch * kChunk);
        const int cend = min(c + kChunk, ncells);
        int row = c / nx;
        int i = c - row * nx;
        bool fresh = true;
        for (; c < cend; ++c, ++i) {
            if (i == nx) {
                i = 0;
                ++row;
                fresh = true;
            }
            if (fresh) {  // the row's constant part of every centre
                fresh = false;
                double xs[MAXD];  // coordinates of the slower axes
                int idx[MAXD];
                int r = row;
#pragma unroll
                for (int a = MAXD - 1; a >= 0; --a) {
                    idx[a] = 0;
                    xs[a] = 0.0;
                    if (a < nd - 1) {
                        idx[a] = r % D.n[a];
                        r /= D.n[a];
                        xs[a] = D.lo[a] + (double)idx[a] * D.dx[a];
                    }
                }
#pragma unroll
                for (int a = 0; a < MAXD; ++a) {
                    double cc = cconst[a];
#pragma unroll
                    for (int b = 0; b < MAXD; ++b)
                        if (b < nd - 1) cc += f.A[a * MAXD + b] * xs[b];
                    for (int t = 0; t < f.nterms; ++t) {
                        const int ax = f.term_axis[t];
                        if (f.term_row[t] == a && ax != fa) {
                            int ia = idx[0];
#pragma unroll
                            for (int b = 1; b < MAXD; ++b) ia = ax == b ? idx[b] : ia;
                            cc += term(t, ia);
                        }
                    }
                    rowc[a] = cc;
                }
            }
            const double xf = D.lo[fa] + (double)i * D.dx[fa];
            double rate = 0.0;
#pragma unroll
            for (int a = 0; a < MAXD; ++a) {
                if (a >= nd) break;
                double centre = rowc[a] + f.A[a * MAXD + fa] * xf;
                for (int t = 0; t < f.nterms; ++t)
                    if (f.term_row[t] == a && f.term_axis[t] == fa) centre += term(t, i);
                const double al = fabs(centre) + radius[a];
                amax[a] = fmax(amax[a], al);
                rate += al * inv_dx[a];
            }
            rmax = fmax(rmax, rate);
        }
    }
    __shared__ double red[kThreads / 32][MAXD + 1];
#pragma unroll
    for (int a = 0; a <= MAXD; ++a) {
        double v = a < MAXD ? amax[a] : rmax;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][a] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        InstState* st = D.state;
        for (int a = 0; a <= MAXD; ++a) {
            double v = red[0][a];
            for (int w = 1; w < kThreads / 32; ++w) v = fmax(v, red[w][a]);
            unsigned long long* dst = a < MAXD ? &st->alpha_bits[a] : &st->rate_bits;
            atomicMax(dst, static_cast<unsigned long long>(__double_as_longlong(v)));
        }
        __threadfence();
        if (atomicAdd(&st->setup_done, 1u) + 1 == gridDim.x) {
            __threadfence();
            for (int a = 0; a < MAXD; ++a)
                st->alpha[a] = __longlong_as_double((long long)atomicAdd(&st->alpha_bits[a], 0ull));
            const double rate = __longlong_as_double((long long)atomicAdd(&st->rate_bits, 0ull));
            if (rate > 0.0 && rate <= DBL_MAX) {
                st->dt = D.cfl / rate;
            } else {
                st->dt = 0.0;
                st->status = 2;
                if (atomicExch(&st->stop, 1) == 0 && D.active != nullptr) atomicSub(D.active, 1);
            }
            fill_ctx_const(D, st);
            __threadfence();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) init_kernel(const InstDesc* __restrict__ insts) {
    const InstDesc& D = insts[blockIdx.y];
    const T* __restrict__ k = static_cast<const T*>(D.kinit);
    const T* __restrict__ klo_p = static_cast<const T*>(D.kinit_lo);
    const T* l = static_cast<const T*>(D.l);
    T* V = static_cast<T*>(D.V[0]);
    // FP32 grids: the low word of V starts at zero, or, when k is the grid's
    // own resident value, keeps that value's low word.
    T* Vlo = static_cast<T*>(D.Vlo[0]);
    T* snap = static_cast<T*>(D.snap);
    // Fields are rows of the fastest axis padded to the pitch; pad elements
    // are left alone.
    const int nx = D.n[D.ndim - 1];
    const long long pitch = D.ndim >= 2 ? D.stride[D.ndim - 2] : D.nalloc;
    unsigned int bad = 0u;
    const bool small = D.nalloc < (1ll << 32);  // 32-bit column arithmetic suffices
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < D.nalloc;
         c += (long long)gridDim.x * blockDim.x) {
        const long long col = small ? static_cast<long long>(static_cast<unsigned>(c) %
                                                             static_cast<unsigned>(pitch))
                                    : c % pitch;
        if (col >= nx) continue;
        const T lv = l[c];
        T v = lv, vlo = T(0);
        if (!isfinite(lv)) bad = 1u;
        if (k != nullptr) {
            const T kv = k[c];
            const T klo = (klo_p != nullptr && Vlo != nullptr) ? klo_p[c] : T(0);
            if (!isfinite(kv)) bad = 1u;
            // With the projection off (Eq. (5) alone) the start is k as given.
            if (D.brs || kv < lv || (kv == lv && klo < T(0))) {
                v = kv;
                vlo = klo;
            }
        }
        V[c] = v;
        if (Vlo != nullptr) Vlo[c] = vlo;
        if (snap != nullptr) snap[c] = v;  // the interval test's first reference
    }
    bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
    if (bad && (threadIdx.x & 31) == 0) atomicOr(&D.state->nonfinite, 1u);
}

// Resident-value transfer between grids of different precision.
__global__ void __launch_bounds__(kThreads)
    convert_kernel(long long n, const void* src_hi, const void* src_lo, int src_f32, void* dst_hi,
                   void* dst_lo, int dst_f32) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        double v;
        if (src_f32) {
            v = (double)static_cast<const float*>(src_hi)[c];
            if (src_lo) v += (double)static_cast<const float*>(src_lo)[c];
        } else {
            v = static_cast<const double*>(src_hi)[c];
        }
        if (dst_f32) {
            const float h = (float)v;
            static_cast<float*>(dst_hi)[c] = h;
            if (dst_lo) static_cast<float*>(dst_lo)[c] = (float)(v - (double)h);
        } else {
            static_cast<double*>(dst_hi)[c] = v;
        }
    }
}

// Self-test of the bounded TMA wait: one CTA arms an mbarrier for 16 bytes
// that no copy delivers, so its phase never completes, and waits on it with
// the stage kernel's bounded routine.  result = 4 (the status a stage kernel
// records) when the wait gave up, 0 if the phase completed.  Nothing is in
// flight on the barrier when the CTA leaves.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int* result) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(b, 16u);
    __syncthreads();
    const bool ok = mbar_wait_bounded(b, 0u, limit_ns);
    const int gave_up = __syncthreads_or(!ok);
    if (threadIdx.x == 0) *result = gave_up ? 4 : 0;
}

cudaError_t launch_wait_selftest(unsigned long long limit_ns, int* d_result, cudaStream_t s) {
    wait_selftest_kernel<<<1, 64, 0, s>>>(limit_ns, d_result);
    return cudaGetLastError();
}

// The debug build's recorder on a 10-element extent: one index inside, a
// 4-wide range past the end, one index before the start, and a failed
// condition.  The indices are only compared, never used as addresses.
__global__ void check_selftest_kernel(InstState* st, long long* out) {
#ifdef HJI_CHECKED
    out[0] = checked_index(st, CK_TILE, 7, 1, 10);
    out[1] = checked_index(st, CK_PLANE, 8, 4, 10);
    out[2] = checked_index(st, CK_XWINDOW, -1, 1, 10);
    out[3] = checked_cond(st, CK_TMA_X, false, 3, 4) ? 1 : 0;
#else
    (void)st;
    (void)out;
#endif
}

cudaError_t launch_check_selftest(InstState* st, long long* out, cudaStream_t s) {
    check_selftest_kernel<<<1, 1, 0, s>>>(st, out);
    return cudaGetLastError();
}

static const char* const kCheckSiteNames[CK_NUM_SITES] = {
    "",
    "tile index",
    "tile origin",
    "tensor-copy x coordinate (16-byte boundary)",
    "tensor-copy destination (128-byte boundary)",
    "ghost node slot",
    "extrapolation source in the window",
    "periodic ghost line",
    "y-difference source rows",
    "y-difference slot",
    "WENO5 set source",
    "WENO5 set result slot",
    "slow-axis stencil plane",
    "x-stencil window segment",
    "ENO y-stencil differences",
    "term table entry",
    "staged node values",
    "node fields",
};

std::string check_message(const InstState& S) {
    const int site = S.check_site;
    const char* name = site > 0 && site < CK_NUM_SITES ? kCheckSiteNames[site] : "unknown site";
    return "index check failed " + std::to_string(S.check_count) + " time(s); first: " + name +
           " (site " + std::to_string(site) + "), index " + std::to_string(S.check_index) +
           " against extent " + std::to_string(S.check_limit);
}

static int grid_for(long long work, int cap);

cudaError_t launch_convert(long long n, const void* src_hi, const void* src_lo, bool src_f32,
                           void* dst_hi, void* dst_lo, bool dst_f32, cudaStream_t s) {
    convert_kernel<<<grid_for(n, 4096), kThreads, 0, s>>>(n, src_hi, src_lo, src_f32 ? 1 : 0, dst_hi,
                                                          dst_lo, dst_f32 ? 1 : 0);
    return cudaGetLastError();
}

static int grid_for(long long work, int cap) {
    long long b = (work + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return static_cast<int>(b);
}

cudaError_t launch_setup(const InstDesc* d_insts, const InstDesc* h_insts, int count, bool f32,
                         cudaStream_t s) {
    long long cmax = 0, nmax = 0;
    int tmax = 0;
    for (int i = 0; i < count; ++i) {
        const InstDesc& H = h_insts[i];
        cmax = H.ncells > cmax ? H.ncells : cmax;
        tmax = H.dyn.nterms > tmax ? H.dyn.nterms : tmax;
        for (int a = 0; a < H.ndim; ++a) nmax = H.n[a] > nmax ? H.n[a] : nmax;
    }
    if (tmax > 0) {
        dim3 grid(grid_for(nmax, 64), tmax, count);
        if (f32)
            table_kernel<float><<<grid, kThreads, 0, s>>>(d_insts);
        else
            table_kernel<double><<<grid, kThreads, 0, s>>>(d_insts);
    }
    // Each alpha thread takes chunks of kAlphaChunk nodes.
    alpha_kernel<<<dim3(grid_for((cmax + kAlphaChunk - 1) / kAlphaChunk, 1024), count), kThreads, 0,
                   s>>>(d_insts);
    return cudaGetLastError();
}

cudaError_t launch_init(const InstDesc* d_insts, const InstDesc* h_insts, int count, bool f32,
                        cudaStream_t s) {
    long long cmax = 0;
    for (int i = 0; i < count; ++i) cmax = h_insts[i].ncells > cmax ? h_insts[i].ncells : cmax;
    const dim3 grid(grid_for(cmax, 4096), count);
    if (f32)
        init_kernel<float><<<grid, kThreads, 0, s>>>(d_insts);
    else
        init_kernel<double><<<grid, kThreads, 0, s>>>(d_insts);
    return cudaGetLastError();
}

}  // namespace hji
