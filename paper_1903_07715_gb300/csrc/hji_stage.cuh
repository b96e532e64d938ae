// The fused Runge-Kutta stage kernel: one launch advances one stage of every
// live instance in the batch.  Per tile of nodes it
//   1. copies the stencil input W (tile + ghost halo of the two fastest axes)
//      into shared memory with TMA (one thread issues the tensor copies of
//      the next tile while the CTA computes the current one), then builds the
//      ghost nodes beyond the grid edge by linear extrapolation (or periodic
//      wrap);
//   2. forms the one-sided derivatives p-, p+ along every axis (ENO1, ENO2 or
//      HJ-WENO5): each thread takes runs of four consecutive nodes of the
//      fastest axis, whose WENO5 stencils share smoothness indicators, and
//      slower axes read their stencil lines from L2 directly;
//   3. evaluates the closed-form control-affine Hamiltonian of Eq. (6) at the
//      averaged gradient plus the Lax-Friedrichs dissipation;
//   4. combines the Euler stage W + dt L(W) with V^n (TVD Runge-Kutta);
//   5. on the last stage applies min(., l) (Eq. (7)-(8)), reduces
//      max|V^{n+1} - V^n| (warp shuffle -> CTA -> one 64-bit atomic), and the
//      CTA finishing an instance's last tile advances that instance's step
//      counter, tau, stop flag and buffer index.
// Tiles of instances that have stopped are skipped, so launches queued after
// convergence do no work and no step past the stop point ever runs.
//
// Every wait on a TMA copy is bounded (kWaitNs); a CTA whose copy does not
// arrive records the failure (HJI_E_TIMEOUT) in the instance's state, stops
// the instance and returns.
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
//
// The textbook evaluation is rewritten on differences of the v's, which
// neighbouring stencils share.  With e_k = v_k - v_{k+1} (k = 1..4):
//   smoothness indicators S_A = 13/12 (e1 - e2)^2 + 1/4 (e1 - 3 e2)^2,
//                         S_B = 13/12 (e2 - e3)^2 + 1/4 (e2 + e3)^2,
//                         S_C = 13/12 (e3 - e4)^2 + 1/4 (3 e3 - e4)^2
//   (the usual (v1 - 2v2 + v3), (v1 - 4v2 + 3v3), ... written in e's);
//   candidate polynomials: phi_1 - phi_2 = t1 / 3 and phi_3 - phi_2 = t3 / 6
//   with the third differences t1 = e1 - 2e2 + e3, t3 = e2 - 2e3 + e4, so
//   sum_k w_k phi_k = phi_2 + (alpha_1 t1 / 3 + alpha_3 t3 / 6) / sum alpha
//   (alpha_k = d_k / (S_k + eps)^2, d = (0.1, 0.6, 0.3)); and
//   max v^2 = (max |v|)^2.
// The derivative on the reversed differences (v5..v1) has the same three
// indicators in reverse order (the indicator formula is symmetric under
// reversing its triple) and third differences (-t3, -t1), so one set of
// five differences serves p+ of one node and p- of its neighbour.
//
// Two exact rescalings shape the arithmetic into fused multiply-adds:
//   * the normalised weights do not change when every S_k and eps are
//     multiplied by one factor, so the indicators are formed as
//     S'_k = S_k / (13/12) = p_k^2 + (3/13) q_k^2 with eps' = (12/13) eps;
//   * numerator and denominator of the weighted correction are multiplied
//     by 30:  forward  (z1 t1 + 1.5 z3 t3) / (3 z1 + 18 z2 + 9 z3),
//             reversed (z3 t3 + 1.5 z1 t1) / (9 z1 + 18 z2 + 3 z3),
//     so a set's products A = z1 t1, B = z3 t3 and u = 18 z2 serve both of
//     its derivatives.
//
// WenoSet holds z1, z3, A, B, u of a set, where (z1, z2, z3) are the
// weights d_k / b_k^2 up to a common factor (b = S' + eps'):
//   FP64: z = ((b_B b_C)^2, (b_A b_C)^2, (b_A b_B)^2), the common factor
//         (b_A b_B b_C)^2, one division (tiny = 1e-60 keeps the fourth
//         powers above the FP64 range floor);
//   FP32: z = (r_A^2, r_B^2, r_C^2), r = 1/b by the hardware's approximate
//         reciprocal; tiny = 1e-18 keeps r^2 and the weighted sums below
//         2^126, inside the normal range, while exceeding 1e-6 max(v^2)
//         only where every |v| < 1e-6 (flat data, where the weights do not
//         matter).
template <typename T>
struct WenoSet {
    T z1, z3, A, B, u;
};

// The hardware's approximate reciprocal (PTX rcp.approx.ftz.f32, one
// special-function instruction).  The WENO5 weights' denominators lie far
// inside the normal range (at least 1e-18 and below 2^126), where it is
// what a fast division by them computes, without that division's checks
// for the range ends.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// A set from its first differences e1..e4, m = max |v_k| and its third
// differences t1, t3.
template <typename T>
__device__ __forceinline__ WenoSet<T> weno_set(T e1, T e2, T e3, T e4, T m, T t1, T t3) {
    constexpr T kq = T(3.0 / 13.0);           // (1/4) / (13/12)
    constexpr T keps = T(1e-6 * 12.0 / 13.0);  // eps' = eps / (13/12)
    const T pA = e1 - e2, qA = e1 - T(3) * e2;
    const T pB = e2 - e3, qB = e2 + e3;
    const T pC = e3 - e4, qC = T(3) * e3 - e4;
    const T sA = fma(pA, pA, (kq * qA) * qA);
    const T sB = fma(pB, pB, (kq * qB) * qB);
    const T sC = fma(pC, pC, (kq * qC) * qC);
    T z1, z2, z3;
    if constexpr (sizeof(T) == 4) {
        const float eps = fmaf(keps * m, m, 1e-18f * (12.0f / 13.0f));
        const float rA = rcp_approx(sA + eps);
        const float rB = rcp_approx(sB + eps);
        const float rC = rcp_approx(sC + eps);
        z1 = rA * rA;
        z2 = rB * rB;
        z3 = rC * rC;
    } else {
        const T eps = fma(keps * m, m, Num<T>::weno_tiny() * T(12.0 / 13.0));
        const T bA = sA + eps, bB = sB + eps, bC = sC + eps;
        const T pBC = bB * bC, pAC = bA * bC, pAB = bA * bB;
        z1 = pBC * pBC;
        z2 = pAC * pAC;
        z3 = pAB * pAB;
    }
    WenoSet<T> w;
    w.z1 = z1;
    w.z3 = z3;
    w.A = z1 * t1;
    w.B = z3 * t3;
    w.u = T(18) * z2;
    return w;
}

template <typename T>
__device__ __forceinline__ T ratio(T num, T den) {
    if constexpr (sizeof(T) == 4) return num * rcp_approx(den);
    else return num / den;
}

// p- on the forward set v1..v5 (phi_2 = -v2/6 + 5 v3/6 + v4/3).
template <typename T>
__device__ __forceinline__ T weno_fwd(T v2, T v3, T v4, const WenoSet<T>& w) {
    const T phi2 = v3 * T(5.0 / 6.0) - v2 * T(1.0 / 6.0) + v4 * T(1.0 / 3.0);
    const T num = fma(T(1.5), w.B, w.A);
    const T den = fma(T(3), w.z1, fma(T(9), w.z3, w.u));
    return phi2 + ratio(num, den);
}
// p+ on the same set read in reverse (v5..v1).
template <typename T>
__device__ __forceinline__ T weno_rev(T v2, T v3, T v4, const WenoSet<T>& w) {
    const T phi2 = v3 * T(5.0 / 6.0) - v4 * T(1.0 / 6.0) + v2 * T(1.0 / 3.0);
    const T num = fma(T(1.5), w.A, w.B);
    const T den = fma(T(9), w.z1, fma(T(3), w.z3, w.u));
    return phi2 - ratio(num, den);
}

// ---- Two FP32 lanes per instruction ----
// Blackwell's packed FP32 instructions (add / mul / fma on .f32x2) do two
// lanes in one issue slot, each lane rounded as the scalar instruction
// would be.  The WENO5 y-set pass evaluates four independent tile columns
// per thread, which pair up as (0, 1) and (2, 3).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp2(float2 a) {  // the scalar path's reciprocal, per lane
    return make_float2(rcp_approx(a.x), rcp_approx(a.y));
}

// weno_set on two lanes (FP32): the same arithmetic; 3 e3 - e4 enters only
// squared, so its negation e4 - 3 e3 (one fused operation) is used.
__device__ __forceinline__ WenoSet<float2> weno_set2(float2 e1, float2 e2, float2 e3, float2 e4, float2 m,
                                                    float2 t1, float2 t3) {
    const float2 kq = f2(3.0f / 13.0f);
    const float2 pA = sub2(e1, e2), qA = fma2(e2, f2(-3.0f), e1);
    const float2 pB = sub2(e2, e3), qB = add2(e2, e3);
    const float2 pC = sub2(e3, e4), qCn = fma2(e3, f2(-3.0f), e4);
    const float2 sA = fma2(pA, pA, mul2(mul2(kq, qA), qA));
    const float2 sB = fma2(pB, pB, mul2(mul2(kq, qB), qB));
    const float2 sC = fma2(pC, pC, mul2(mul2(kq, qCn), qCn));
    const float2 eps = fma2(mul2(f2(float(1e-6 * 12.0 / 13.0)), m), m, f2(1e-18f * (12.0f / 13.0f)));
    const float2 rA = rcp2(add2(sA, eps)), rB = rcp2(add2(sB, eps)), rC = rcp2(add2(sC, eps));
    WenoSet<float2> w;
    w.z1 = mul2(rA, rA);
    w.z3 = mul2(rC, rC);
    w.A = mul2(w.z1, t1);
    w.B = mul2(w.z3, t3);
    w.u = mul2(f2(18.0f), mul2(rB, rB));
    return w;
}
__device__ __forceinline__ float2 ratio2(float2 num, float2 den) { return mul2(num, rcp2(den)); }
__device__ __forceinline__ float2 weno_fwd2(float2 v2, float2 v3, float2 v4, const WenoSet<float2>& w) {
    const float2 phi2 = fma2(v4, f2(1.0f / 3.0f), fma2(v2, f2(-1.0f / 6.0f), mul2(v3, f2(5.0f / 6.0f))));
    const float2 num = fma2(f2(1.5f), w.B, w.A);
    const float2 den = fma2(f2(3.0f), w.z1, fma2(f2(9.0f), w.z3, w.u));
    return add2(phi2, ratio2(num, den));
}
__device__ __forceinline__ float2 weno_rev2(float2 v2, float2 v3, float2 v4, const WenoSet<float2>& w) {
    const float2 phi2 = fma2(v2, f2(1.0f / 3.0f), fma2(v4, f2(-1.0f / 6.0f), mul2(v3, f2(5.0f / 6.0f))));
    const float2 num = fma2(f2(1.5f), w.A, w.B);
    const float2 den = fma2(f2(9.0f), w.z1, fma2(f2(3.0f), w.z3, w.u));
    return sub2(phi2, ratio2(num, den));
}

// WENO5 (p-, p+) from the six differences D[0..5] of one node.
template <typename T>
__device__ __forceinline__ void weno5_pair(const T* D, T inv_dx, T& pm, T& pp) {
    T E[5], Tt[3];
#pragma unroll
    for (int k = 0; k < 5; ++k) E[k] = D[k] - D[k + 1];
#pragma unroll
    for (int k = 0; k < 3; ++k) Tt[k] = E[k] - T(2) * E[k + 1] + E[k + 2];
    const T m14 = fmax(fmax(fabs(D[1]), fabs(D[2])), fmax(fabs(D[3]), fabs(D[4])));
    const WenoSet<T> wa = weno_set(E[0], E[1], E[2], E[3], fmax(m14, fabs(D[0])), Tt[0], Tt[1]);
    const WenoSet<T> wb = weno_set(E[1], E[2], E[3], E[4], fmax(m14, fabs(D[5])), Tt[1], Tt[2]);
    pm = weno_fwd(D[1], D[2], D[3], wa) * inv_dx;
    pp = weno_rev(D[2], D[3], D[4], wb) * inv_dx;
}

// The same on two lanes (FP32; two nodes' stencil lines, lane by lane the
// scalar arithmetic): WENO5 from six differences per lane, and the
// smaller-magnitude choice of ENO2 per lane (no packed compare).
__device__ __forceinline__ void weno5_pair2(const float2* D, float2 inv_dx, float2& pm, float2& pp) {
    float2 E[5], Tt[3];
#pragma unroll
    for (int k = 0; k < 5; ++k) E[k] = sub2(D[k], D[k + 1]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Tt[k] = add2(fma2(E[k + 1], f2(-2.0f), E[k]), E[k + 2]);
    const float m14x = fmaxf(fmaxf(fabsf(D[1].x), fabsf(D[2].x)), fmaxf(fabsf(D[3].x), fabsf(D[4].x)));
    const float m14y = fmaxf(fmaxf(fabsf(D[1].y), fabsf(D[2].y)), fmaxf(fabsf(D[3].y), fabsf(D[4].y)));
    const WenoSet<float2> wa =
        weno_set2(E[0], E[1], E[2], E[3],
                  make_float2(fmaxf(m14x, fabsf(D[0].x)), fmaxf(m14y, fabsf(D[0].y))), Tt[0], Tt[1]);
    const WenoSet<float2> wb =
        weno_set2(E[1], E[2], E[3], E[4],
                  make_float2(fmaxf(m14x, fabsf(D[5].x)), fmaxf(m14y, fabsf(D[5].y))), Tt[1], Tt[2]);
    pm = mul2(weno_fwd2(D[1], D[2], D[3], wa), inv_dx);
    pp = mul2(weno_rev2(D[2], D[3], D[4], wb), inv_dx);
}
__device__ __forceinline__ float2 smaller_mag2(float2 a, float2 b) {
    return make_float2(fabsf(a.x) <= fabsf(b.x) ? a.x : b.x, fabsf(a.y) <= fabsf(b.y) ? a.y : b.y);
}
template <int SCHEME>
__device__ __forceinline__ void one_sided_diffs2(const float2* D, float2 inv_dx, float2& pm, float2& pp) {
    if constexpr (SCHEME == HJI_ENO1) {
        pm = mul2(D[0], inv_dx);
        pp = mul2(D[1], inv_dx);
    } else if constexpr (SCHEME == HJI_ENO2) {
        const float2 Sm = sub2(D[1], D[0]), S0 = sub2(D[2], D[1]), Sp = sub2(D[3], D[2]);
        pm = mul2(fma2(f2(0.5f), smaller_mag2(Sm, S0), D[1]), inv_dx);
        pp = mul2(fma2(f2(-0.5f), smaller_mag2(S0, Sp), D[2]), inv_dx);
    } else {
        weno5_pair2(D, inv_dx, pm, pp);
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
        weno5_pair(D, inv_dx, pm, pp);
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

// Loads of fields a kernel never writes go through the read-only data path
// (__ldg).  COH = true marks a caller (the multi-step march kernel) in which
// the field may have been written earlier in the same launch by another CTA:
// those loads are made at L2 (__ldcg), which is coherent, instead.
template <bool COH, typename T>
__device__ __forceinline__ T ld_field(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

template <typename T, bool COH = false>
__device__ __forceinline__ Pair<T> load_pair(const T* __restrict__ h, const T* __restrict__ lo,
                                            const T* __restrict__ d, long long i) {
    Pair<T> p;
    p.h = ld_field<COH>(h + i);
    p.l = T(0);
    if (lo != nullptr) p.l = ld_field<COH>(lo + i);
    if (d != nullptr) p.l += ld_field<COH>(d + i);
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
template <typename T, bool COH = false>
__device__ __forceinline__ Pair<T> line_pair(const T* __restrict__ h, const T* __restrict__ lo,
                                            const T* __restrict__ d, int j, int n, long long s,
                                            int periodic) {
    if (j >= 0 && j < n) return load_pair<T, COH>(h, lo, d, (long long)j * s);
    if (periodic) {
        int w = j % n;
        if (w < 0) w += n;
        return load_pair<T, COH>(h, lo, d, (long long)w * s);
    }
    const bool low = j < 0;
    const int k = low ? -j : j - (n - 1);
    const Pair<T> e = load_pair<T, COH>(h, lo, d, (long long)(low ? 0 : n - 1) * s);
    const Pair<T> i1 = load_pair<T, COH>(h, lo, d, (long long)(low ? 1 : n - 2) * s);
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

// ---- four consecutive values (16 bytes FP32, 32 bytes FP64) ----
template <typename T>
struct Q4 {
    T v[4];
};
template <typename T>
__device__ __forceinline__ Q4<T> ld4(const T* p) {  // shared or global, 16-byte aligned
    Q4<T> q;
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        q.v[0] = a.x; q.v[1] = a.y; q.v[2] = a.z; q.v[3] = a.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        q.v[0] = a.x; q.v[1] = a.y; q.v[2] = b.x; q.v[3] = b.y;
    }
    return q;
}
template <typename T, bool COH = false>
__device__ __forceinline__ Q4<T> ldg4(const T* p) {  // global, 16-byte aligned (see ld_field)
    Q4<T> q;
    if constexpr (sizeof(T) == 4) {
        const float4 a = ld_field<COH>(reinterpret_cast<const float4*>(p));
        q.v[0] = a.x; q.v[1] = a.y; q.v[2] = a.z; q.v[3] = a.w;
    } else {
        const double2 a = ld_field<COH>(reinterpret_cast<const double2*>(p));
        const double2 b = ld_field<COH>(reinterpret_cast<const double2*>(p) + 1);
        q.v[0] = a.x; q.v[1] = a.y; q.v[2] = b.x; q.v[3] = b.y;
    }
    return q;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T* v) {  // 16-byte aligned
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
}

// The interval test's per-node work on a step that ends an interval: the
// largest |V^{n+1} - snapshot| over a run's valid nodes goes into imax and
// V^{n+1} (the high word for FP32) replaces the snapshot.  Each node's
// snapshot is read and written by the thread that owns the node.
template <typename T, bool COH>
__device__ __forceinline__ void interval_check(T* snap, const T* v, int nvalid, T& imax) {
    if (nvalid == 4) {
        const Q4<T> s = ldg4<T, COH>(snap);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const T ch = fabs(v[i] - s.v[i]);
            imax = (ch > imax || ch != ch) ? ch : imax;
        }
        st4(snap, v);
    } else {
        for (int i = 0; i < nvalid; ++i) {
            const T ch = fabs(v[i] - ld_field<COH>(snap + i));
            imax = (ch > imax || ch != ch) ? ch : imax;
            snap[i] = v[i];
        }
    }
}

// ---- The bounds-checked debug build ----
// Compiled with -DHJI_CHECKED (a second library from the same sources),
// every index the tile and halo code forms is tested against the extent of
// the array it addresses before the access.  A miss is recorded in the
// instance's state (the first site, index and extent, and a count; the
// solve then fails with HJI_E_CHECK) and the access goes to element 0
// instead, so the march never touches memory outside its arrays.  In the
// product build the checks compile to nothing.
#ifdef HJI_CHECKED
#define HJI_CHK(site, i, w, n) \
    static_cast<decltype(i)>(::hji::checked_index(C.state, (site), (i), (w), (n)))
#define HJI_CHK_COND(site, ok, v, n) ::hji::checked_cond(C.state, (site), (ok), (v), (n))
// An offset `off` from element `base` of a field: the offset, or -base (the
// field's element 0) after a miss.
#define HJI_CHK_REL(site, base, off, w, n) \
    static_cast<decltype(off)>(::hji::checked_index(C.state, (site), (base) + (off), (w), (n)) - (base))
#else
#define HJI_CHK(site, i, w, n) (i)
#define HJI_CHK_COND(site, ok, v, n) true
#define HJI_CHK_REL(site, base, off, w, n) (off)
#endif

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
    int tiles_x, tiles_per_plane, ntiles;
    T lo[MAXD], dx[MAXD], inv_dx[MAXD], half_alpha[MAXD];
    T cmid[MAXD], A[MAXD * MAXD], G[MAXD * MAXU], E[MAXD * MAXU];
    T urad[MAXU], drad[MAXU];  // half-widths of the control and disturbance boxes
    T arad[MAXD];              // per row: sum_j urad_j |G_aj| + sum_k drad_k |E_ak|
    int term_row[MAXT], term_axis[MAXT];
    int project;               // 1: V <- min(V, l) after the step (Eq. (7)); 0: Eq. (5) alone
    // Discounted reachability (Sec. II-C): the step's result is scaled by
    // gamma before the projection.  FP64 keeps gamma; the FP32 compensated
    // form keeps 1 - gamma and subtracts (1 - gamma) V~ from the increment.
    int discounted;
    T disc;
    T dt;
    const T* win;   // stencil input (FP64: the stage state; FP32: V^n hi word)
    const T* din;   // FP32: stage increment added to win (null for stage 1)
    const T* vcur;
    T* wout;
    const T* vlo;   // FP32: low word of V^n
    T* vlo_out;     // FP32: low word of V^{n+1}, written by the last stage
    const T* l;
    const T* table;
    long long table_stride;
    // The last stage's step bookkeeping (finish_step), read at context load:
    // none of it changes during a launch before the instance's last tile.
    InstState* state;
    int* active;
    double* history;
    long long history_len, steps0, max_steps;
    double tau0, dt_d, stop_delta, horizon;
    // Interval test (Sec. V): on a step that ends an interval the last stage
    // compares V^{n+1} with the snapshot and replaces it.
    T* snap;
    int boundary;
    double interval_tol;
    // Extents the debug build's index checks test against: elements of one
    // field, and of the term table.
    long long nalloc, table_elems;
    // TMA descriptors of the fields this stage copies.
    const CUtensorMap* tm_win;   // stencil input (high word)
    const CUtensorMap* tm_lo;    // FP32 low word of V^n
    const CUtensorMap* tm_d;     // FP32 stage increment
    const CUtensorMap* tm_l;     // l at the tile nodes
    const CUtensorMap* tm_vn;    // FP64 V^n at the tile nodes
};

// Half of row a of the drift at a node, f0_a(x)/2 with f0_a(x) = c_a +
// G_a umid + E_a dmid + A_a x + the nonlinear terms of row a (the context's
// drift constants and the term table are stored halved): with arad_a it
// gives half the node's own dissipation coefficient,
// max_{u,d} |f_a(x,u,d)| / 2 = |f0_a(x)/2| + arad_a / 2 (local
// Lax-Friedrichs).  idx are the node's indices; the fastest index may lie
// past the grid's edge for the tail of a run (its table reads are clamped,
// its result unused).
template <typename T, int NDIM>
__device__ __forceinline__ T row_drift(const TileCtx<T>& C, const int* idx, int a) {
    T f = C.cmid[a];
#pragma unroll
    for (int j = 0; j < NDIM; ++j) f += C.A[a * MAXD + j] * (C.lo[j] + T(idx[j]) * C.dx[j]);
    for (int tt = 0; tt < C.nterms; ++tt) {
        if (C.term_row[tt] != a) continue;
        const int ax = C.term_axis[tt];
        int ia = idx[0];
#pragma unroll
        for (int r = 1; r < NDIM; ++r) ia = ax == r ? idx[r] : ia;
        f += __ldg(C.table + tt * C.table_stride +
                   HJI_CHK_REL(CK_TABLE, (long long)tt * C.table_stride, min(ia, C.n[ax] - 1), 1,
                               C.table_elems));
    }
    return f;
}

// The set-up pass's constants of an instance in precision T.
template <typename T>
__device__ __forceinline__ const CtxConst<T>& ctx_const(const InstState* st) {
    if constexpr (sizeof(T) == 4) return st->kf;
    else return st->kd;
}

// Fill the tile context; called by every thread of the CTA (each copies a
// slice), followed by __syncthreads() at the call site.  Not inlined: the
// stage kernels keep fewer registers live across their tile loop (the FP32
// 1-D/2-D and 4-D ENO2 ones spill none) with the context load as a call.
static_assert(MAXD == 4 && MAXU == 4 && MAXT == 8 && kThreads > 96,
              "load_ctx hands out slices for these sizes");
template <typename T, bool COH>
__device__ __noinline__ void load_ctx(TileCtx<T>& C, const InstDesc* __restrict__ insts, int inst,
                                      const StageArgs& a) {
    const InstDesc& D = insts[inst];
    const CtxConst<T>& K = ctx_const<T>(D.state);
    const int t = threadIdx.x;
    if (t < MAXD * MAXD) C.A[t] = K.A[t];
    else if (t < 32) C.G[t - 16] = K.G[t - 16];
    else if (t < 48) C.E[t - 32] = K.E[t - 32];
    else if (t < 52) C.urad[t - 48] = K.urad[t - 48];
    else if (t < 56) C.drad[t - 52] = K.drad[t - 52];
    else if (t < 64) {
        // threads 56..63 have no slice
    } else if (t < 72) {
        C.term_row[t - 64] = D.dyn.term_row[t - 64];
        C.term_axis[t - 64] = D.dyn.term_axis[t - 64];
    } else if (t < 76) {
        const int i = t - 72;
        C.n[i] = D.n[i];
        C.periodic[i] = D.periodic[i];
        C.stride[i] = D.stride[i];
        C.lo[i] = K.lo[i];
        C.dx[i] = K.dx[i];
        C.inv_dx[i] = K.inv_dx[i];
        C.half_alpha[i] = K.half_alpha[i];
        C.cmid[i] = K.cmid[i];
        C.arad[i] = K.arad[i];
    } else if (t == 96) {
        // Both buffers' pointers are read beside the state pointer, so that
        // only the choice between them waits for the buffer index (two
        // dependent loads before the first tile copy, not three).
        void* const v0 = D.V[0];
        void* const v1 = D.V[1];
        void* const lo0 = D.Vlo[0];
        void* const lo1 = D.Vlo[1];
        InstState* st = D.state;
        const int cur = *((volatile int*)&st->cur);
        C.inst = inst;
        C.stop = *((volatile int*)&st->stop);
        C.cur = cur;
        C.m = D.dyn.m;
        C.q = D.dyn.q;
        C.project = D.brs ? 0 : 1;
        C.discounted = (D.discount > 0.0 && D.discount < 1.0) ? 1 : 0;
        C.disc = sizeof(T) == 4 ? T(1.0 - D.discount) : T(D.discount);
        C.nterms = D.dyn.nterms;
        C.dt = K.dt;
        C.tiles_x = static_cast<int>(D.tiles_x);
        C.tiles_per_plane = static_cast<int>(D.tiles_per_plane);
        C.ntiles = static_cast<int>(D.ntiles);
        const T* vc = static_cast<const T*>(cur ? v1 : v0);
        const T* stage =
            a.stage_in == 0 ? nullptr : static_cast<const T*>(a.stage_in == 1 ? D.W1 : D.W2);
        const int tm_v = cur ? TM_WIN_V1 : TM_WIN_V0;
        const int tm_s = a.stage_in == 1 ? TM_WIN_W1 : TM_WIN_W2;
        C.vcur = vc;
        if constexpr (sizeof(T) == 4) {
            C.win = vc;
            C.din = stage;
            C.tm_win = &D.tm[tm_v];
            C.tm_d = stage ? &D.tm[tm_s] : nullptr;
        } else {
            C.win = stage ? stage : vc;
            C.din = nullptr;
            C.tm_win = &D.tm[stage ? tm_s : tm_v];
            C.tm_d = nullptr;
        }
        C.tm_lo = &D.tm[cur ? TM_WIN_LO1 : TM_WIN_LO0];
        C.tm_l = &D.tm[TM_NODE_L];
        C.tm_vn = &D.tm[cur ? TM_NODE_V1 : TM_NODE_V0];
        C.vlo = static_cast<const T*>(cur ? lo1 : lo0);
        C.vlo_out = static_cast<T*>(cur ? lo0 : lo1);
        C.wout = a.stage_out == 3 ? static_cast<T*>(cur ? v0 : v1)
                                  : static_cast<T*>(a.stage_out == 1 ? D.W1 : D.W2);
        C.l = static_cast<const T*>(D.l);
        C.table = static_cast<const T*>(D.table);
        C.table_stride = D.table_stride;
        C.nalloc = D.nalloc;
        C.table_elems = (long long)D.dyn.nterms * D.table_stride;
        C.state = st;
        C.active = D.active;
        C.history = D.history;
        C.history_len = D.history_len;
        // steps and tau change at the end of every step (finish_step); the
        // multi-step march kernel (COH) reads them after a step of the same
        // launch, so at L2.
        if constexpr (COH) {
            C.steps0 = __ldcg(&st->steps);
            C.tau0 = __ldcg(&st->tau);
        } else {
            C.steps0 = st->steps;
            C.tau0 = st->tau;
        }
        C.max_steps = D.max_steps;
        C.dt_d = st->dt;
        C.stop_delta = st->stop_delta;
        C.horizon = D.horizon;
        const long long K = st->interval_K;
        C.snap = static_cast<T*>(D.snap);
        C.boundary = (K > 0 && D.snap != nullptr && (C.steps0 + 1) % K == 0) ? 1 : 0;
        C.interval_tol = D.interval_tol;
    }
}

// Stop an instance once: the thread that flips the flag lowers the
// batch-wide count of marching instances.
__device__ inline void stop_instance(const InstDesc& D) {
    if (atomicExch(&D.state->stop, 1) == 0 && D.active != nullptr) atomicSub(D.active, 1);
}

// Add v to the instance's count of finished tiles with acquire-release order
// (PTX memory model, GPU scope): the caller's earlier max|dV| reduction is
// visible before its count, and the thread whose addition completes the
// count sees every CTA's reduction.
__device__ __forceinline__ unsigned add_tiles_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Finish one step of an instance: called by the single thread whose tile
// count completed the instance's last stage (after add_tiles_acq_rel), with
// the context it loaded for that instance.  The state it writes is read by
// later launches and by the host, both after this kernel has ended.
template <typename T>
__device__ inline void finish_step(const TileCtx<T>& C) {
    InstState* st = C.state;
    const double d = __longlong_as_double((long long)atomicAdd(&st->delta_bits, 0ull));
    const long long steps = C.steps0 + 1;
    const double tau = C.tau0 + C.dt_d;
    st->last_delta = d;
    st->steps = steps;
    st->tau = tau;
    st->cur = C.cur ^ 1;
    if (C.history != nullptr && steps - 1 < C.history_len) C.history[steps - 1] = d;
    st->delta_bits = 0ull;
    st->tiles_done = 0u;
    double di = DBL_MAX;  // the interval's largest change, on a step that ends one
    if (C.boundary) {
        di = __longlong_as_double((long long)atomicAdd(&st->interval_bits, 0ull));
        st->interval_bits = 0ull;
        st->last_interval_change = di;
    }
    bool stop = false;
    if (!(d <= DBL_MAX)) {  // NaN or Inf
        st->status = 1;
        stop = true;
    } else if (d < C.stop_delta || di < C.interval_tol) {
        st->converged = 1;
        stop = true;
    } else if (C.horizon > 0.0 && tau >= C.horizon) {
        stop = true;
    } else if (steps >= C.max_steps) {
        stop = true;
    }
    if (stop && atomicExch(&st->stop, 1) == 0 && C.active != nullptr) atomicSub(C.active, 1);
}

// ---- TMA tensor copies and their mbarriers ----
constexpr unsigned long long kWaitNs = 4000000000ull;  // a bounded wait gives up after 4 s

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Wait for the phase with the given parity; false if it has not completed
// within limit_ns (or 2^26 polls).
static __device__ __noinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity,
                                                      unsigned long long limit_ns = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}
// Tiled tensor copy global -> shared, completing on `bar`; c[] are the
// element coordinates of the box origin, fastest dimension first.
template <int R>
__device__ __forceinline__ void tma_load(unsigned dst, const CUtensorMap* m, const int* c,
                                         unsigned bar) {
    const unsigned long long mp = reinterpret_cast<unsigned long long>(m);
    if constexpr (R == 1) {
        asm volatile(
            "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2}], [%3];" ::"r"(dst), "l"(mp), "r"(c[0]), "r"(bar)
            : "memory");
    } else if constexpr (R == 2) {
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst), "l"(mp), "r"(c[0]), "r"(c[1]), "r"(bar)
            : "memory");
    } else if constexpr (R == 3) {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst), "l"(mp), "r"(c[0]), "r"(c[1]),
            "r"(c[2]), "r"(bar)
            : "memory");
    } else {
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst), "l"(mp), "r"(c[0]), "r"(c[1]),
            "r"(c[2]), "r"(c[3]), "r"(bar)
            : "memory");
    }
}

// Dynamic shared-memory layout of one stage kernel: two buffers, each with
// the staged window (high words; FP32 also low words and stage increments)
// and, for the last stage, l (and, FP64, V^n) at the tile nodes; then the
// y-differences of the current tile and, for WENO5, its y-derivatives.  Window row r, column c holds the node
// (y0 - GY + r, x0 - 4 + c): columns start 4 left of the tile so that every
// copy starts on a 16-byte boundary.
constexpr int round128(int b) { return (b + 127) / 128 * 128; }

template <typename T, int NDIM, int SCHEME, bool LAST, int V>
struct StageSmem {
    using S = TileShape<NDIM, V>;
    static constexpr int G = Ghost<SCHEME>::G;
    static constexpr int TY = S::TY, TX = S::TX, GROUPS = S::GROUPS;
    static constexpr int GY = (NDIM >= 2) ? G : 0;
    static constexpr int SWX = TX + 8;
    static constexpr int SH = TY + 2 * GY;
    static constexpr int WIN = SWX * SH;   // elements of one window field
    static constexpr int NODES = TY * TX;
    static constexpr bool INCR = sizeof(T) == 4;
    static constexpr int WINB = round128(WIN * (int)sizeof(T));
    static constexpr int NODEB = round128(NODES * (int)sizeof(T));
    static constexpr int NF = INCR ? 3 : 1;
    static constexpr int DYSB = NDIM >= 2 ? round128((SH - 1) * TX * (int)sizeof(T)) : 0;
    // WENO5 y-derivatives p-, p+ of the tile nodes, from the set pass.
    static constexpr bool YSETS = NDIM >= 2 && SCHEME == HJI_WENO5;
    static constexpr int PYB = YSETS ? round128(NODES * (int)sizeof(T)) : 0;
    // The last stage stages l (and, FP64, V^n) at the tile nodes with the
    // window, unless (FP32 WENO5) the two l buffers would cost the fourth CTA
    // per SM (233472 B of shared memory, about 2.4 KB of it static and
    // reserved per CTA); it then reads l from L2 where it uses it.
    static constexpr int BASEB = 2 * NF * WINB + DYSB + 2 * PYB + 128;
    static constexpr bool STAGE_L = LAST && (!INCR || 4 * (BASEB + 2 * NODEB + 2400) <= 233472);
    static constexpr int NN = STAGE_L ? (INCR ? 1 : 2) : 0;
    static constexpr int BUFB = NF * WINB + NN * NODEB;
    static constexpr int DYS = 2 * BUFB;
    static constexpr int PMY = DYS + DYSB;
    static constexpr int PPY = PMY + PYB;
    static constexpr int BYTES = PPY + PYB + 128;  // + alignment slack (smem_layout_base)
    static_assert(WINB % 128 == 0 && NODEB % 128 == 0 && DYSB % 128 == 0 && PYB % 128 == 0,
                  "tensor-copy destinations sit on 128-byte boundaries");
    static __host__ __device__ constexpr int H(int b) { return b * BUFB; }
    static __host__ __device__ constexpr int LO(int b) { return b * BUFB + WINB; }
    static __host__ __device__ constexpr int DD(int b) { return b * BUFB + 2 * WINB; }
    static __host__ __device__ constexpr int LT(int b) { return b * BUFB + NF * WINB; }
    static __host__ __device__ constexpr int VN(int b) { return b * BUFB + NF * WINB + NODEB; }
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
__device__ __forceinline__ TileGeo tile_geo(const TileCtx<T>& C, int local) {
    TileGeo g;
    int tip = local;
    g.base = 0;
#pragma unroll
    for (int ax = 0; ax < MAXD; ++ax) g.sidx[ax] = 0;
    if constexpr (NDIM >= 3) {
        int r = local;
        const int ls = NDIM - 3;  // last slow axis
        g.sidx[ls] = r % C.n[ls];
        r /= C.n[ls];
        tip = r % C.tiles_per_plane;
        r /= C.tiles_per_plane;
        for (int ax = ls - 1; ax >= 0; --ax) {
            g.sidx[ax] = r % C.n[ax];
            r /= C.n[ax];
        }
        for (int ax = 0; ax <= ls; ++ax) g.base += (long long)g.sidx[ax] * C.stride[ax];
    }
    const int by = tip / C.tiles_x;
    const int bx = tip - by * C.tiles_x;
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

// Resident CTAs per SM the register budget is cut for: FP32 1-D/2-D stages
// four (64 registers), FP32 3-D/4-D and FP64 two.  (Five for the 2-D ENO2
// stages before the last fits 48 registers without spills, but the tighter
// budget costs more instructions than the fifth CTA hides.)
template <typename T, int NDIM, int SCHEME, bool LAST>
constexpr int kMinBlocks = sizeof(T) != 4 ? 2 : NDIM > 2 ? 2 : 4;

// The kernels' dynamic shared memory (the tile windows and per-tile
// arrays; StageSmem gives the layout, whose blocks sit at multiples of 128
// bytes from its base).  A tiled tensor copy needs a 128-byte-aligned
// shared destination, and the base of dynamic shared memory is only
// guaranteed 16-byte alignment, so the layout starts at the first 128-byte
// boundary (BYTES includes the 128 bytes of slack).  The offset is taken in
// the shared window itself, so the compiler still addresses the layout as
// shared memory.
extern __shared__ __align__(16) unsigned char hji_smem[];

__device__ __forceinline__ unsigned char* smem_layout_base() {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(hji_smem));
    return hji_smem + ((128u - (a & 127u)) & 127u);
}

// One Runge-Kutta stage of every live instance, as run by one CTA over its
// share of the tile list (the body of a stage launch).  The caller owns the
// two mbarriers at shared address bar0 (initialised, count 1) and their
// phase bits; the tile context, reduction slots and tile placements are
// this function's own shared variables.  COH selects coherent loads for
// fields that another CTA may have written earlier in the same launch.
// INTERVAL (last stage only) compiles in Sec. V's interval test; LLF the
// node-wise (local) Lax-Friedrichs coefficients.  Returns
// false when a bounded wait gave up (the failure is recorded in the
// instance's state; the CTA must leave).
template <typename T, int NDIM, int SCHEME, bool LAST, int V, bool COH, bool INTERVAL,
          bool LLF = false>
__device__ __forceinline__ bool stage_pass(const StageArgs& a, unsigned bar0, unsigned& phase) {
    using L = StageSmem<T, NDIM, SCHEME, LAST, V>;
    __shared__ TileCtx<T> C;
    __shared__ T red[2 * (kThreads / 32)];
    __shared__ TileGeo geo_s[2];  // where the tile in each buffer sits (written by thread 0)
    unsigned char* sb = smem_layout_base();
    constexpr int G = L::G, TY = L::TY, TX = L::TX, GROUPS = L::GROUPS;
    constexpr int GY = L::GY, SWX = L::SWX, SH = L::SH, WIN = L::WIN;
    constexpr int AX = NDIM - 1;                  // fastest axis
    constexpr int AY = NDIM >= 2 ? NDIM - 2 : 0;  // second fastest axis (used if NDIM >= 2)
    constexpr bool INCR = L::INCR;                // FP32: increments + compensated V

    T* dys = reinterpret_cast<T*>(sb + L::DYS);  // dys[r][c] = W(r+1, c) - W(r, c), tile columns

    const int ntiles = a.ntiles_imm > 0 ? a.ntiles_imm : *a.ntiles;
    // tile-list entry t (a single instance's list is t itself)
    auto tile_entry = [&](int t) {
        return a.direct ? static_cast<unsigned long long>(t) : a.tiles[t];
    };
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
    // Thread -> (tile row, run of four nodes); for NDIM >= 2 the last row of
    // threads has no run (it takes a y-set in the WENO5 set pass).
    const int grp = threadIdx.x % GROUPS;
    const int ry = threadIdx.x / GROUPS;
    const bool thread_works = NDIM >= 2 ? ry < TY : threadIdx.x < GROUPS;

    // Bytes one tile's copies deliver to its buffer's barrier.
    const unsigned tile_bytes =
        static_cast<unsigned>(WIN * sizeof(T)) * (INCR ? (has_d ? 3u : 2u) : 1u) +
        (L::STAGE_L ? static_cast<unsigned>(TY * TX * sizeof(T)) * ((!INCR && reads_v) ? 2u : 1u) : 0u);

    // Thread 0: start the tensor copies of a tile into buffer b.
    auto issue = [&](const TileGeo& tg, int b) {
        const unsigned bar = bar0 + 8u * b;
        const unsigned base = smem_addr(sb);
        // (A destination off its 128-byte boundary issues no copy: the
        // bounded wait then gives up and the CTA leaves.)
        if (!HJI_CHK_COND(CK_TMA_DST, (base & 127u) == 0u, base, 128)) return;
        mbar_expect_tx(bar, tile_bytes);
        int cw[4] = {tg.x0 - 4, tg.y0 - GY, 0, 0};
        int cn[4] = {tg.x0, tg.y0, 0, 0};
        if constexpr (NDIM >= 3) {
            cw[2] = cn[2] = tg.sidx[NDIM - 3];
            if constexpr (NDIM == 4) cw[3] = cn[3] = tg.sidx[0];
        }
#ifdef HJI_CHECKED
        {
            constexpr int k = 16 / (int)sizeof(T);  // elements per 16 bytes
            bool in = tg.x0 >= 0 && tg.x0 < C.n[AX] && (NDIM < 2 || (tg.y0 >= 0 && tg.y0 < C.n[AY]));
            for (int ax = 0; ax < NDIM - 2; ++ax) in = in && tg.sidx[ax] >= 0 && tg.sidx[ax] < C.n[ax];
            HJI_CHK_COND(CK_TILE_GEO, in, tg.x0, C.n[AX]);
            // an unaligned x would be an illegal copy: round it down
            if (!HJI_CHK_COND(CK_TMA_X, cw[0] % k == 0, cw[0], k)) cw[0] -= ((cw[0] % k) + k) % k;
            if (!HJI_CHK_COND(CK_TMA_X, cn[0] % k == 0, cn[0], k)) cn[0] -= ((cn[0] % k) + k) % k;
        }
#endif
        tma_load<NDIM>(base + L::H(b), C.tm_win, cw, bar);
        if constexpr (INCR) {
            tma_load<NDIM>(base + L::LO(b), C.tm_lo, cw, bar);
            if (has_d) tma_load<NDIM>(base + L::DD(b), C.tm_d, cw, bar);
        }
        if constexpr (L::STAGE_L) {
            tma_load<NDIM>(base + L::LT(b), C.tm_l, cn, bar);
            if constexpr (!INCR) {
                if (reads_v) tma_load<NDIM>(base + L::VN(b), C.tm_vn, cn, bar);
            }
        }
    };

    int loaded = -1;
    TileWalk walk(ntiles);
    int t = walk.next();
    int buf = 0;
    bool issued = false;
    // Last stage: each thread's running max|dV| over the CTA's tiles of the
    // current instance, published (with the tile count) when the CTA moves
    // on to another instance or runs out of tiles.
    T dmax = T(0);
    T imax = T(0);  // the same for the interval test's change, on a step that ends an interval
    (void)imax;
    int run_tiles = 0;
    while (t >= 0) {
        const unsigned long long entry = tile_entry(t);
        const int inst = static_cast<int>(entry >> 48);
        const int local = static_cast<int>(entry & 0xFFFFFFFFFFFFull);
        if (inst != loaded) {
            __syncthreads();  // everyone is done with the previous context
            load_ctx<T, COH>(C, a.insts, inst, a);
            __syncthreads();
            if (threadIdx.x == 0 && !C.stop) {
                tensormap_acquire(C.tm_win);
                if (INCR) tensormap_acquire(C.tm_lo);
                if (has_d) tensormap_acquire(C.tm_d);
                if (L::STAGE_L) tensormap_acquire(C.tm_l);
                if (LAST && !INCR && reads_v) tensormap_acquire(C.tm_vn);
            }
            loaded = inst;
        }
        if (C.stop) {  // uniform across the CTA; nothing was issued for it
            t = walk.next();
            issued = false;
            continue;
        }
        const int tn = walk.next();
        const bool pref = tn >= 0 && static_cast<int>(tile_entry(tn) >> 48) == inst;
        // Buffer `buf` was last read two tiles ago, which every thread
        // finished before the barrier below of the previous tile.  Thread 0
        // places the tiles (one integer division each) for everyone.
        if (threadIdx.x == 0 && !issued) {
            geo_s[buf] = tile_geo<T, NDIM, TY, TX>(C, HJI_CHK(CK_TILE, local, 1, C.ntiles));
            issue(geo_s[buf], buf);
        }
        const bool ok = mbar_wait_bounded(bar0 + 8u * buf, (phase >> buf) & 1u);
        phase ^= 1u << buf;
        // After this barrier every thread is done with the previous tile, so
        // its buffer (buf ^ 1) and the y-differences may be overwritten.
        if (__syncthreads_or(!ok)) {
            // A copy never arrived: record it, stop the instance and leave.
            if (threadIdx.x == 0) {
                const InstDesc& D = a.insts[inst];
                atomicExch(&D.state->status, 4);
                stop_instance(D);
            }
            return false;
        }
        const TileGeo& tg = geo_s[buf];  // read from shared memory where used
        // Prefetch the next tile of the walk while this one is computed.
        if (threadIdx.x == 0 && pref) {
            geo_s[buf ^ 1] = tile_geo<T, NDIM, TY, TX>(
                C, HJI_CHK(CK_TILE, static_cast<int>(tile_entry(tn) & 0xFFFFFFFFFFFFull), 1, C.ntiles));
            issue(geo_s[buf ^ 1], buf ^ 1);
        }

        const int nx = C.n[AX];
        const int ny = NDIM >= 2 ? C.n[AY] : 1;
        const long long sy = NDIM >= 2 ? C.stride[AY] : 0;
        const int y0 = tg.y0, x0 = tg.x0;
        const T* __restrict__ hp = C.win + tg.base;
        const T* __restrict__ lp = INCR ? C.vlo + tg.base : nullptr;
        const T* __restrict__ dp = C.din ? C.din + tg.base : nullptr;
        T* wh = reinterpret_cast<T*>(sb + L::H(buf));
        T* wl = reinterpret_cast<T*>(sb + L::LO(buf));
        const T* wd = reinterpret_cast<const T*>(sb + L::DD(buf));
        // FP32 stages 2+: the stencil input is hi + (lo + d); every reader
        // adds the stage increment to the low word itself.  Ghost slots lie
        // outside the tensor, so their increments read as zero.
        auto pair_at = [&](int r, int c) {
            const int i = HJI_CHK(CK_GHOST_READ, r * SWX + c, 1, WIN);
            Pair<T> p;
            p.h = wh[i];
            p.l = T(0);
            if constexpr (INCR) {
                p.l = wl[i];
                if (has_d) p.l += wd[i];
            }
            return p;
        };

        // 1. Ghost nodes of tiles that reach beyond the grid edge: linear
        //    extrapolation from the two edge nodes (both inside the staged
        //    window), or, on a periodic axis, the wrapped node.  Only the
        //    ghosts an axis-aligned stencil of a tile node reaches are built:
        //    along x for the tile rows, along y for the tile columns.
        const bool edge = x0 - G < 0 || x0 + TX + G > nx ||
                          (NDIM >= 2 && (y0 - GY < 0 || y0 + TY + GY > ny));
        if (edge) {
            constexpr int NXG = 2 * G * TY;
            constexpr int NYG = NDIM >= 2 ? 2 * G * TX : 0;
            for (int s = threadIdx.x; s < NXG + NYG; s += kThreads) {
                Pair<T> v;
                int r, c;
                if (s < NXG) {
                    const int ry = s / (2 * G), j = s - ry * (2 * G);
                    r = GY + ry;
                    const int gy = y0 + ry;
                    const int gx = j < G ? j - G : nx + (j - G);
                    c = gx - x0 + 4;
                    if ((NDIM >= 2 && gy >= ny) || c < 4 - G || c >= 4 + TX + G) continue;
                    if (C.periodic[AX]) {
                        const long long r0 =
                            HJI_CHK_REL(CK_GHOST_LINE, tg.base, (long long)gy * sy, nx, C.nalloc);
                        v = line_pair<T, COH>(hp + r0, lp ? lp + r0 : nullptr, dp ? dp + r0 : nullptr,
                                         gx, nx, 1, 1);
                    } else {
                        const bool low = gx < 0;
                        const int ce = (low ? 0 : nx - 1) - x0 + 4;
                        const int ci = (low ? 1 : nx - 2) - x0 + 4;
                        v = extrapolate(pair_at(r, ce), pair_at(r, ci), low ? -gx : gx - (nx - 1));
                    }
                } else {
                    const int s2 = s - NXG;
                    const int j = s2 / TX, cx = s2 - j * TX;
                    c = 4 + cx;
                    const int gx = x0 + cx;
                    const int gy = j < G ? j - G : ny + (j - G);
                    r = gy - y0 + GY;
                    if (gx >= nx || r < 0 || r >= SH) continue;
                    if (C.periodic[AY]) {
                        const long long c0 = HJI_CHK_REL(CK_GHOST_LINE, tg.base, (long long)gx,
                                                         (long long)(ny - 1) * sy + 1, C.nalloc);
                        v = line_pair<T, COH>(hp + c0, lp ? lp + c0 : nullptr, dp ? dp + c0 : nullptr,
                                         gy, ny, sy, 1);
                    } else {
                        const bool low = gy < 0;
                        const int re = (low ? 0 : ny - 1) - y0 + GY;
                        const int ri = (low ? 1 : ny - 2) - y0 + GY;
                        v = extrapolate(pair_at(re, c), pair_at(ri, c), low ? -gy : gy - (ny - 1));
                    }
                }
                // Written after every read of this pass: ghost nodes only
                // read in-grid nodes, and no thread writes an in-grid node.
                const int gs = HJI_CHK(CK_GHOST_WRITE, r * SWX + c, 1, WIN);
                wh[gs] = v.h;
                if constexpr (INCR) wl[gs] = v.l;
            }
            __syncthreads();
        }
        // 2. y-differences of the tile columns, once per tile (FP32: on the pairs).
        //    Items are dealt from the last thread down, so the items beyond
        //    one per thread fall to the last warp rather than to warp 0,
        //    which also issues the tile copies.
        if constexpr (NDIM >= 2) {
            for (int i = kThreads - 1 - threadIdx.x; i < (SH - 1) * GROUPS; i += kThreads) {
                const int r = i / GROUPS, g4 = i - r * GROUPS;
                const int s0 = HJI_CHK(CK_DIFF_READ, r * SWX + 4 + 4 * g4, SWX + 4, WIN);
                const Q4<T> h0 = ld4(wh + s0), h1 = ld4(wh + s0 + SWX);
                T dv[4];
                if constexpr (INCR) {
                    Q4<T> l0 = ld4(wl + s0), l1 = ld4(wl + s0 + SWX);
                    if (has_d) {
                        const Q4<T> d0 = ld4(wd + s0), d1 = ld4(wd + s0 + SWX);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            l0.v[q] += d0.v[q];
                            l1.v[q] += d1.v[q];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) dv[q] = (h1.v[q] - h0.v[q]) + (l1.v[q] - l0.v[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) dv[q] = h1.v[q] - h0.v[q];
                }
                st4(dys + HJI_CHK(CK_DIFF_WRITE, r * TX + 4 * g4, 4, (SH - 1) * TX), dv);
            }
            __syncthreads();
        }
        // 2b. WENO5 along y by sets: set j of a column is its differences
        //     j .. j+4, which give p- of tile row j (forward) and p+ of tile
        //     row j-1 (reversed), so each set is evaluated once.  Thread
        //     (j, g4) takes set j of columns 4 g4 .. 4 g4 + 3.
        if constexpr (L::YSETS) {
            const int j = threadIdx.x / GROUPS, g4 = threadIdx.x - j * GROUPS;
            const int q0 = HJI_CHK(CK_YSET_READ, j * TX + 4 * g4, 4 * TX + 4, (SH - 1) * TX);
            T q[5][4];
#pragma unroll
            for (int o = 0; o < 5; ++o) {
                const Q4<T> v = ld4(dys + q0 + o * TX);
#pragma unroll
                for (int c = 0; c < 4; ++c) q[o][c] = v.v[c];
            }
            const T iy = C.inv_dx[AY];
            T pmv[4], ppv[4];
            T mc[4];  // the sets' scales m (no packed max)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                mc[c] = fmax(fmax(fmax(fabs(q[0][c]), fabs(q[1][c])), fmax(fabs(q[2][c]), fabs(q[3][c]))),
                             fabs(q[4][c]));
            if constexpr (sizeof(T) == 4) {
                // columns (0, 1) and (2, 3) as two lanes
#pragma unroll
                for (int c = 0; c < 4; c += 2) {
                    float2 v[5], e[4];
#pragma unroll
                    for (int o = 0; o < 5; ++o) v[o] = make_float2(q[o][c], q[o][c + 1]);
#pragma unroll
                    for (int o = 0; o < 4; ++o) e[o] = sub2(v[o], v[o + 1]);
                    const float2 t1 = add2(fma2(e[1], f2(-2.0f), e[0]), e[2]);
                    const float2 t3 = add2(fma2(e[2], f2(-2.0f), e[1]), e[3]);
                    const WenoSet<float2> w =
                        weno_set2(e[0], e[1], e[2], e[3], make_float2(mc[c], mc[c + 1]), t1, t3);
                    const float2 pm = mul2(weno_fwd2(v[1], v[2], v[3], w), f2(iy));
                    const float2 pp = mul2(weno_rev2(v[1], v[2], v[3], w), f2(iy));
                    pmv[c] = pm.x;
                    pmv[c + 1] = pm.y;
                    ppv[c] = pp.x;
                    ppv[c + 1] = pp.y;
                }
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    T e[4];
#pragma unroll
                    for (int o = 0; o < 4; ++o) e[o] = q[o][c] - q[o + 1][c];
                    const T t1 = e[0] - T(2) * e[1] + e[2], t3 = e[1] - T(2) * e[2] + e[3];
                    const WenoSet<T> w = weno_set(e[0], e[1], e[2], e[3], mc[c], t1, t3);
                    pmv[c] = weno_fwd(q[1][c], q[2][c], q[3][c], w) * iy;
                    ppv[c] = weno_rev(q[1][c], q[2][c], q[3][c], w) * iy;
                }
            }
            if (j < TY)
                st4(reinterpret_cast<T*>(sb + L::PMY) + HJI_CHK(CK_YSET_WRITE, j * TX + 4 * g4, 4, TY * TX),
                    pmv);
            if (j > 0)
                st4(reinterpret_cast<T*>(sb + L::PPY) +
                        HJI_CHK(CK_YSET_WRITE, (j - 1) * TX + 4 * g4, 4, TY * TX),
                    ppv);
            __syncthreads();
        }

        // 3-5. Each thread updates a run of 4 nodes of the tile.  The
        // derivatives of each axis are folded at once into the
        // Lax-Friedrichs sum Lv = sum_a alpha_a (p+ - p-) / 2 and the
        // averaged gradient pbar, so they never need to be kept for all axes.
        const int gx0 = x0 + 4 * grp;
        const int gy = y0 + ry;
        if (thread_works && gx0 < nx && (NDIM < 2 || gy < ny)) {
            T Lv[4] = {T(0), T(0), T(0), T(0)};
            T pb[4][NDIM];
            auto fold = [&](int ax, int i, T pm_, T pp_) {
                T ha;
                if constexpr (LLF) {
                    int nid[NDIM];
#pragma unroll
                    for (int b = 0; b < NDIM - 2; ++b) nid[b] = tg.sidx[b];
                    if constexpr (NDIM >= 2) nid[AY] = gy;
                    nid[AX] = gx0 + i;
                    ha = fabs(row_drift<T, NDIM>(C, nid, ax)) + T(0.5) * C.arad[ax];
                } else {
                    ha = C.half_alpha[ax];
                }
                Lv[i] += ha * (pp_ - pm_);
                pb[i][ax] = pp_ + pm_;  // 2 pbar: the Hamiltonian's constants are halved
            };
            const long long gidx =
                HJI_CHK(CK_NODE_GLOBAL, tg.base + (long long)gy * sy + gx0, 4, C.nalloc);
            // FP32 last stage without staged l: its load from L2 is issued
            // here, so that its latency overlaps the derivatives.
            Q4<T> lt_early;
            if constexpr (LAST && INCR && !L::STAGE_L) lt_early = ldg4(C.l + gidx);
            // Slower axes first (their stencil lines are the largest live
            // set): the lines straight from global memory
            // (L1/L2), four nodes per load, differenced plane by plane.  The
            // slow index is the same for the whole tile, so a tile away from
            // that axis' edges takes the direct path.
#pragma unroll
            for (int ax = 0; ax < NDIM - 2; ++ax) {
                const long long st = C.stride[ax];
                const int si = tg.sidx[ax], ns = C.n[ax];
                const long long l0 = gidx - (long long)si * st;  // node 0 of these lines
                auto plane = [&](int j, Pair<T>* out) {
                    const long long o = HJI_CHK(CK_PLANE, l0 + (long long)j * st, 4, C.nalloc);
                    const Q4<T> h = ldg4<T, COH>(C.win + o);
                    Q4<T> lo, dd;
                    if constexpr (INCR) {
                        lo = ldg4<T, COH>(C.vlo + o);
                        if (C.din) dd = ldg4<T, COH>(C.din + o);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        out[i].h = h.v[i];
                        out[i].l = T(0);
                        if constexpr (INCR) {
                            out[i].l = lo.v[i];
                            if (C.din) out[i].l += dd.v[i];
                        }
                    }
                };
                auto plane_any = [&](int j, Pair<T>* out) {
                    if (j >= 0 && j < ns) {
                        plane(j, out);
                    } else if (C.periodic[ax]) {
                        j %= ns;
                        if (j < 0) j += ns;
                        plane(j, out);
                    } else {
                        const bool low = j < 0;
                        Pair<T> e[4], i1[4];
                        plane(low ? 0 : ns - 1, e);
                        plane(low ? 1 : ns - 2, i1);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            out[i] = extrapolate(e[i], i1[i], low ? -j : j - (ns - 1));
                    }
                };
                const bool inner = si >= G && si < ns - G;
                const T is = C.inv_dx[ax];
                if constexpr (INCR) {
                    // FP32: nodes (0, 1) and (2, 3) of the run as two lanes of
                    // packed instructions (the plane loads give them as
                    // aligned pairs); the same arithmetic lane by lane.
                    struct P2 {
                        float2 h[2], l[2];
                    };
                    auto plane2 = [&](int j) {
                        P2 r;
                        if (inner || (j >= 0 && j < ns)) {
                            const long long o = HJI_CHK(CK_PLANE, l0 + (long long)j * st, 4, C.nalloc);
                            const Q4<T> h = ldg4<T, COH>(C.win + o);
                            const Q4<T> lo = ldg4<T, COH>(C.vlo + o);
                            r.h[0] = make_float2(h.v[0], h.v[1]);
                            r.h[1] = make_float2(h.v[2], h.v[3]);
                            r.l[0] = make_float2(lo.v[0], lo.v[1]);
                            r.l[1] = make_float2(lo.v[2], lo.v[3]);
                            if (C.din) {
                                const Q4<T> dd = ldg4<T, COH>(C.din + o);
                                r.l[0] = add2(r.l[0], make_float2(dd.v[0], dd.v[1]));
                                r.l[1] = add2(r.l[1], make_float2(dd.v[2], dd.v[3]));
                            }
                        } else {  // a ghost plane (periodic wrap or extrapolation)
                            Pair<T> out[4];
                            plane_any(j, out);
#pragma unroll
                            for (int k = 0; k < 2; ++k) {
                                r.h[k] = make_float2(out[2 * k].h, out[2 * k + 1].h);
                                r.l[k] = make_float2(out[2 * k].l, out[2 * k + 1].l);
                            }
                        }
                        return r;
                    };
                    // every plane of the line first (their loads in flight
                    // together), then the differences
                    P2 pl[2 * G + 1];
#pragma unroll
                    for (int o = 0; o <= 2 * G; ++o) pl[o] = plane2(si - G + o);
                    float2 D2[2][2 * G];
#pragma unroll
                    for (int o = 0; o < 2 * G; ++o) {
#pragma unroll
                        for (int k = 0; k < 2; ++k)
                            D2[k][o] = add2(sub2(pl[o + 1].h[k], pl[o].h[k]), sub2(pl[o + 1].l[k], pl[o].l[k]));
                    }
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        float2 pm2, pp2;
                        one_sided_diffs2<SCHEME>(D2[k], f2(is), pm2, pp2);
                        fold(ax, 2 * k, pm2.x, pp2.x);
                        fold(ax, 2 * k + 1, pm2.y, pp2.y);
                    }
                } else {
                    T D[2 * G][4];
                    Pair<T> prev[4], cur[4];
                    if (inner) plane(si - G, prev);
                    else plane_any(si - G, prev);
#pragma unroll
                    for (int o = 1 - G; o <= G; ++o) {
                        if (inner) plane(si + o, cur);
                        else plane_any(si + o, cur);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            D[o + G - 1][i] = pair_diff(cur[i], prev[i]);
                            prev[i] = cur[i];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        T Di[2 * G];
#pragma unroll
                        for (int o = 0; o < 2 * G; ++o) Di[o] = D[o][i];
                        T pm_, pp_;
                        one_sided_diffs<T, SCHEME>(Di, is, pm_, pp_);
                        fold(ax, i, pm_, pp_);
                    }
                }
            }
            // x: the window row of this run, columns 4 grp .. 4 grp + 11.
            const int s0 = HJI_CHK(CK_XWINDOW, (ry + GY) * SWX + 4 * grp, 12, WIN);
            {
                T d[11];
                const Q4<T> h0 = ld4(wh + s0), h1 = ld4(wh + s0 + 4), h2 = ld4(wh + s0 + 8);
                const T hv[12] = {h0.v[0], h0.v[1], h0.v[2], h0.v[3], h1.v[0], h1.v[1],
                                  h1.v[2], h1.v[3], h2.v[0], h2.v[1], h2.v[2], h2.v[3]};
                if constexpr (INCR) {
                    const Q4<T> l0 = ld4(wl + s0), l1 = ld4(wl + s0 + 4), l2 = ld4(wl + s0 + 8);
                    T lv[12] = {l0.v[0], l0.v[1], l0.v[2], l0.v[3], l1.v[0], l1.v[1],
                                l1.v[2], l1.v[3], l2.v[0], l2.v[1], l2.v[2], l2.v[3]};
                    if (has_d) {
                        const Q4<T> d0 = ld4(wd + s0), d1 = ld4(wd + s0 + 4), d2 = ld4(wd + s0 + 8);
                        const T dd[12] = {d0.v[0], d0.v[1], d0.v[2], d0.v[3], d1.v[0], d1.v[1],
                                          d1.v[2], d1.v[3], d2.v[0], d2.v[1], d2.v[2], d2.v[3]};
#pragma unroll
                        for (int j = 0; j < 12; ++j) lv[j] += dd[j];
                    }
#pragma unroll
                    for (int j = 4 - G; j < 7 + G; ++j)
                        d[j] = (hv[j + 1] - hv[j]) + (lv[j + 1] - lv[j]);
                } else {
#pragma unroll
                    for (int j = 4 - G; j < 7 + G; ++j) d[j] = hv[j + 1] - hv[j];
                }
                const T ix = C.inv_dx[AX];
                if constexpr (SCHEME == HJI_WENO5) {
                    // Node i: p- on the set d[i+1..i+5], p+ on d[i+2..i+6]
                    // reversed; the set d[j..j+4] serves p+ of node j-2 and
                    // p- of node j-1, with first differences E[j..j+3] and
                    // third differences Tt[j], Tt[j+1] for both.
                    T E[9], Tt[8], a[10];
#pragma unroll
                    for (int j = 1; j <= 8; ++j) E[j] = d[j] - d[j + 1];
#pragma unroll
                    for (int j = 1; j <= 7; ++j) Tt[j] = E[j] - T(2) * E[j + 1] + E[j + 2];
#pragma unroll
                    for (int j = 1; j <= 9; ++j) a[j] = fabs(d[j]);
                    auto set_w = [&](int j) {
                        const T m = fmax(fmax(fmax(a[j], a[j + 1]), fmax(a[j + 2], a[j + 3])), a[j + 4]);
                        return weno_set(E[j], E[j + 1], E[j + 2], E[j + 3], m, Tt[j], Tt[j + 1]);
                    };
                    WenoSet<T> wl = set_w(1);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const WenoSet<T> wr = set_w(i + 2);
                        fold(AX, i, weno_fwd(d[i + 2], d[i + 3], d[i + 4], wl) * ix,
                             weno_rev(d[i + 3], d[i + 4], d[i + 5], wr) * ix);
                        wl = wr;
                    }
                } else if constexpr (SCHEME == HJI_ENO2) {
                    // Node i: second differences S[i+2..i+4]; the choice
                    // between S[j] and S[j+1] serves p+ of node j-3 and p- of
                    // node j-2, so it is made once.
                    T S[8], M[7];
#pragma unroll
                    for (int j = 2; j <= 7; ++j) S[j] = d[j + 1] - d[j];
#pragma unroll
                    for (int j = 2; j <= 6; ++j) M[j] = smaller_mag(S[j], S[j + 1]);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        fold(AX, i, (d[i + 3] + T(0.5) * M[i + 2]) * ix,
                             (d[i + 4] - T(0.5) * M[i + 3]) * ix);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        T pm_, pp_;
                        one_sided_diffs<T, SCHEME>(d + 4 + i - G, ix, pm_, pp_);
                        fold(AX, i, pm_, pp_);
                    }
                }
            }
            // y: WENO5 from the set pass; ENO from rows ry .. ry + 2G - 1 of
            // the difference array.
            if constexpr (L::YSETS) {
                const int ni = HJI_CHK(CK_NODE_SMEM, ry * TX + 4 * grp, 4, TY * TX);
                const Q4<T> m4 = ld4(reinterpret_cast<const T*>(sb + L::PMY) + ni);
                const Q4<T> p4 = ld4(reinterpret_cast<const T*>(sb + L::PPY) + ni);
#pragma unroll
                for (int i = 0; i < 4; ++i) fold(AY, i, m4.v[i], p4.v[i]);
            } else if constexpr (NDIM >= 2) {
                T dy[2 * G][4];
                const int y0i = HJI_CHK(CK_DIFF_Y, ry * TX + 4 * grp, (2 * G - 1) * TX + 4, (SH - 1) * TX);
#pragma unroll
                for (int o = 0; o < 2 * G; ++o) {
                    const Q4<T> q = ld4(dys + y0i + o * TX);
#pragma unroll
                    for (int i = 0; i < 4; ++i) dy[o][i] = q.v[i];
                }
                const T iy = C.inv_dx[AY];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    T D[2 * G];
#pragma unroll
                    for (int o = 0; o < 2 * G; ++o) D[o] = dy[o][i];
                    T pm_, pp_;
                    one_sided_diffs<T, SCHEME>(D, iy, pm_, pp_);
                    fold(AY, i, pm_, pp_);
                }
            }
            // Hamiltonian (Eq. (6)) at pbar.  With the boxes written as
            // mid +- rad, max_u <G^T p, u> = <G^T p, umid> + sum_j urad_j |(G^T p)_j|
            // and min_d <E^T p, d> = <E^T p, dmid> - sum_k drad_k |(E^T p)_k|;
            // the mid parts are folded into the constant drift (cmid), so
            // H = <p, cmid + A x + terms> + sum_j urad_j |.| - sum_k drad_k |.|.
            // Along the run only x[AX] changes, by dx per node.
            {
                int idx[NDIM];
#pragma unroll
                for (int ax = 0; ax < NDIM - 2; ++ax) idx[ax] = tg.sidx[ax];
                if constexpr (NDIM >= 2) idx[AY] = gy;
                idx[AX] = gx0;
                T x[NDIM];
#pragma unroll
                for (int ax = 0; ax < NDIM; ++ax) x[ax] = C.lo[ax] + T(idx[ax]) * C.dx[ax];
#pragma unroll
                for (int r = 0; r < NDIM; ++r) {
                    T f0 = C.cmid[r];
#pragma unroll
                    for (int j = 0; j < NDIM; ++j) f0 += C.A[r * MAXD + j] * x[j];
                    const T step = C.A[r * MAXD + AX] * C.dx[AX];
#pragma unroll
                    for (int i = 0; i < 4; ++i) Lv[i] += pb[i][r] * (f0 + T(i) * step);
                }
                for (int tt = 0; tt < C.nterms; ++tt) {
                    const int ax = C.term_axis[tt], row = C.term_row[tt];
                    const T* tab = C.table + tt * C.table_stride;
                    // pb[i][row] by selects: a runtime index would put pb in local memory.
                    T pr[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        pr[i] = pb[i][0];
#pragma unroll
                        for (int r = 1; r < NDIM; ++r) pr[i] = row == r ? pb[i][r] : pr[i];
                    }
                    int ia = idx[0];
#pragma unroll
                    for (int r = 1; r < NDIM; ++r) ia = ax == r ? idx[r] : ia;
                    if (ax == AX) {
                        const int xa = HJI_CHK_REL(CK_TABLE, (long long)tt * C.table_stride, gx0,
                                                   min(4, nx - gx0), C.table_elems);
#pragma unroll
                        for (int i = 0; i < 4; ++i)  // runs may reach past the edge
                            Lv[i] += pr[i] * __ldg(tab + min(xa + i, nx - 1));
                    } else {
                        const T w = __ldg(
                            tab + HJI_CHK_REL(CK_TABLE, (long long)tt * C.table_stride, ia, 1, C.table_elems));
#pragma unroll
                        for (int i = 0; i < 4; ++i) Lv[i] += pr[i] * w;
                    }
                }
                for (int j = 0; j < C.m; ++j) {
                    T g[NDIM];
#pragma unroll
                    for (int r = 0; r < NDIM; ++r) g[r] = C.G[r * MAXU + j];
                    const T rad = C.urad[j];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        T s = T(0);
#pragma unroll
                        for (int r = 0; r < NDIM; ++r) s += g[r] * pb[i][r];
                        Lv[i] += rad * fabs(s);
                    }
                }
                for (int j = 0; j < C.q; ++j) {
                    T e[NDIM];
#pragma unroll
                    for (int r = 0; r < NDIM; ++r) e[r] = C.E[r * MAXU + j];
                    const T rad = C.drad[j];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        T s = T(0);
#pragma unroll
                        for (int r = 0; r < NDIM; ++r) s += e[r] * pb[i][r];
                        Lv[i] -= rad * fabs(s);
                    }
                }
            }
            // Runge-Kutta stage combination and stores (four nodes at once
            // when the whole run lies inside the grid).
            const int nvalid = min(4, nx - gx0);
            const T dt = C.dt;
            // The run's own stencil input (high word), read again here rather
            // than kept in registers through the derivatives.
            T wc[4];
            {
                const Q4<T> q = ld4(wh + s0 + 4);
#pragma unroll
                for (int i = 0; i < 4; ++i) wc[i] = q.v[i];
            }
            if constexpr (INCR) {
                T dc[4] = {T(0), T(0), T(0), T(0)};
                if (has_d) {
                    const Q4<T> q = ld4(wd + s0 + 4);
#pragma unroll
                    for (int i = 0; i < 4; ++i) dc[i] = q.v[i];
                }
                T inc[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) inc[i] = cE * (dc[i] + dt * Lv[i]);
                if constexpr (!LAST) {
                    if (nvalid == 4) st4(C.wout + gidx, inc);
                    else
                        for (int i = 0; i < nvalid; ++i) C.wout[gidx + i] = inc[i];
                } else {
                    // V^n + inc as an unevaluated float pair (error-free
                    // two-sum), then min(., l) of Eq. (7)-(8).
                    // The low word of V^n, from the window.
                    T lo[4];
                    {
                        const Q4<T> q = ld4(wl + s0 + 4);
#pragma unroll
                        for (int i = 0; i < 4; ++i) lo[i] = q.v[i];
                    }
                    Q4<T> lt;  // l at the run's nodes
                    if constexpr (L::STAGE_L)
                        lt = ld4(reinterpret_cast<const T*>(sb + L::LT(buf)) +
                                 HJI_CHK(CK_NODE_SMEM, ry * TX + 4 * grp, 4, TY * TX));
                    else
                        lt = lt_early;  // (its pad columns are never used)
                    if (C.discounted) {
                        // gamma V~ = V~ - (1 - gamma) V~ with V~ = hi + lo +
                        // inc; the low word's share of (1 - gamma) V~ is below
                        // the pair's rounding and is left out.
#pragma unroll
                        for (int i = 0; i < 4; ++i) inc[i] = fma(-C.disc, wc[i] + inc[i], inc[i]);
                    }
                    T nh[4], nl[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const T hi = wc[i];
                        const T sl = lo[i] + inc[i];
                        T vh = hi + sl;
                        const T bb = vh - hi;
                        T vl = (hi - (vh - bb)) + (sl - bb);
                        const T lv = lt.v[i];
                        if (C.project && (vh > lv || (vh == lv && vl > T(0)))) {
                            vh = lv;
                            vl = T(0);
                        }
                        nh[i] = vh;
                        nl[i] = vl;
                        if (i < nvalid) {
                            const T ch = fabs((vh - hi) + (vl - lo[i]));
                            dmax = (ch > dmax || ch != ch) ? ch : dmax;
                        }
                    }
                    if (nvalid == 4) {
                        st4(C.wout + gidx, nh);
                        st4(C.vlo_out + gidx, nl);
                    } else {
                        for (int i = 0; i < nvalid; ++i) {
                            C.wout[gidx + i] = nh[i];
                            C.vlo_out[gidx + i] = nl[i];
                        }
                    }
                    if constexpr (INTERVAL) {
                        if (C.boundary) interval_check<T, COH>(C.snap + gidx, nh, nvalid, imax);
                    }
                }
            } else {
                T vn[4], out[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) vn[i] = wc[i];
                if (reads_v) {
                    Q4<T> q;
                    if constexpr (LAST)
                        q = ld4(reinterpret_cast<const T*>(sb + L::VN(buf)) +
                                HJI_CHK(CK_NODE_SMEM, ry * TX + 4 * grp, 4, TY * TX));
                    else
                        q = ldg4<T, COH>(C.vcur + gidx);
#pragma unroll
                    for (int i = 0; i < 4; ++i) vn[i] = q.v[i];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const T eul = wc[i] + dt * Lv[i];
                    out[i] = reads_v ? cV * vn[i] + cE * eul : eul;
                }
                if constexpr (LAST) {
                    const Q4<T> lt = ld4(reinterpret_cast<const T*>(sb + L::LT(buf)) +
                                         HJI_CHK(CK_NODE_SMEM, ry * TX + 4 * grp, 4, TY * TX));
                    if (C.discounted) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) out[i] *= C.disc;
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (C.project) out[i] = fmin(out[i], lt.v[i]);
                        if (i < nvalid) {
                            const T ch = fabs(out[i] - vn[i]);
                            dmax = (ch > dmax || ch != ch) ? ch : dmax;
                        }
                    }
                }
                if (nvalid == 4) st4(C.wout + gidx, out);
                else
                    for (int i = 0; i < nvalid; ++i) C.wout[gidx + i] = out[i];
                if constexpr (LAST && INTERVAL) {
                    if (C.boundary) interval_check<T, COH>(C.snap + gidx, out, nvalid, imax);
                }
            }
        }

        if constexpr (LAST) {
            ++run_tiles;
            if (!pref) {  // uniform: the next tile is another instance's, or none
                // CTA max of |dV| (NaN wins), then the instance-wide reduction;
                // the CTA that completes the instance's tile count finishes
                // the step.
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const T other = __shfl_xor_sync(0xffffffffu, dmax, o);
                    dmax = (other > dmax || other != other) ? other : dmax;
                }
                const bool bnd = INTERVAL && C.boundary != 0;  // uniform
                if (bnd) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const T other = __shfl_xor_sync(0xffffffffu, imax, o);
                        imax = (other > imax || other != other) ? other : imax;
                    }
                }
                if ((threadIdx.x & 31) == 0) {
                    red[threadIdx.x >> 5] = dmax;
                    if (bnd) red[kThreads / 32 + (threadIdx.x >> 5)] = imax;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    T mt = red[0];
                    for (int w = 1; w < kThreads / 32; ++w)
                        mt = (red[w] > mt || red[w] != red[w]) ? red[w] : mt;
                    const double m = static_cast<double>(mt);
                    InstState* st = C.state;
                    if (bnd) {
                        T mi = red[kThreads / 32];
                        for (int w = 1; w < kThreads / 32; ++w) {
                            const T r = red[kThreads / 32 + w];
                            mi = (r > mi || r != r) ? r : mi;
                        }
                        atomicMax(&st->interval_bits,
                                  static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(mi))));
                    }
                    atomicMax(&st->delta_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
                    const unsigned int prev = add_tiles_acq_rel(&st->tiles_done, static_cast<unsigned int>(run_tiles));
                    if (prev + static_cast<unsigned int>(run_tiles) == static_cast<unsigned int>(C.ntiles))
                        finish_step(C);
                }
                dmax = T(0);
                if constexpr (INTERVAL) imax = T(0);
                run_tiles = 0;
            }
        }
        buf ^= 1;
        t = tn;
        issued = pref;
    }
    return true;
}

// One launch per Runge-Kutta stage (see stage_pass).
template <typename T, int NDIM, int SCHEME, bool LAST, int V, bool INTERVAL, bool LLF>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T, NDIM, SCHEME, LAST>)
    stage_kernel(const StageArgs a) {
    __shared__ __align__(8) unsigned long long bars[2];
    const unsigned bar0 = smem_addr(&bars[0]);
    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_init_fence();
    }
    __syncthreads();
    unsigned phase = 0u;  // bit b: parity of the next completion of buffer b
    stage_pass<T, NDIM, SCHEME, LAST, V, false, INTERVAL, LLF>(a, bar0, phase);
}

// ---- the multi-step march: every stage of `steps` steps in one launch ----

// Grid-wide barrier of a cooperative launch: every CTA adds one to
// *counter (release, GPU scope) and waits until it reaches `target`
// (acquire), so all global writes made before the barrier by any CTA are
// visible after it, to plain loads and (through the proxy fences) to the
// tensor copies.  The wait is bounded: after kWaitNs, or when another CTA
// has already given up (*fault != 0), the CTA records the failure in
// *fault and the caller leaves.
__device__ __forceinline__ bool grid_sync(unsigned* counter, unsigned target, int* fault) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("fence.proxy.async.global;" ::: "memory");
        unsigned prev;
        asm volatile("atom.release.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(prev)
                     : "l"(counter)
                     : "memory");
        unsigned long long t0 = 0ull;
        for (unsigned it = 0; it < (1u << 30); ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
            if (v >= target) break;
            if (it == 0u) {
                t0 = global_ns();
            } else if ((it & 255u) == 0u) {
                if (global_ns() - t0 > kWaitNs || *reinterpret_cast<volatile int*>(fault) != 0) {
                    ok = 0;
                    break;
                }
            }
            if (it > 64u) __nanosleep(32);
            if (it + 1u == (1u << 30)) ok = 0;
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (!ok) atomicExch(fault, 1);
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T, int NDIM, int SCHEME, int V, bool INTERVAL>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T, NDIM, SCHEME, true>)
    march_kernel(const MarchArgs m) {
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ int go;
    const unsigned bar0 = smem_addr(&bars[0]);
    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_init_fence();
    }
    __syncthreads();
    unsigned phase = 0u;
    unsigned barriers = 0u;
    for (int step = 0; step < m.steps; ++step) {
        for (int i = 0; i < m.ns; ++i) {
            const bool ok =
                i + 1 < m.ns
                    ? stage_pass<T, NDIM, SCHEME, false, V, true, false>(m.st[i], bar0, phase)
                    : stage_pass<T, NDIM, SCHEME, true, V, true, INTERVAL>(m.st[i], bar0, phase);
            if (!ok) {
                if (threadIdx.x == 0) atomicExch(m.fault, 1);
                return;
            }
            ++barriers;
            if (!grid_sync(m.barrier, barriers * gridDim.x, m.fault)) return;
        }
        // Every instance's step bookkeeping is done and visible: stop when
        // none is still marching (a uniform decision of all CTAs).
        if (threadIdx.x == 0) go = *reinterpret_cast<const volatile int*>(m.active) > 0;
        __syncthreads();
        if (!go) return;
    }
}

template <typename T, int NDIM, int SCHEME, int V, bool INTERVAL>
cudaError_t launch_march(const MarchArgs& m, int grid, cudaStream_t s) {
    using L0 = StageSmem<T, NDIM, SCHEME, false, V>;
    using L1 = StageSmem<T, NDIM, SCHEME, true, V>;
    constexpr int BYTES = L0::BYTES > L1::BYTES ? L0::BYTES : L1::BYTES;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(march_kernel<T, NDIM, SCHEME, V, INTERVAL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, march_kernel<T, NDIM, SCHEME, V, INTERVAL>, m);
}

template <typename T, int NDIM, int SCHEME, int V, bool INTERVAL>
int max_blocks_march() {
    using L0 = StageSmem<T, NDIM, SCHEME, false, V>;
    using L1 = StageSmem<T, NDIM, SCHEME, true, V>;
    constexpr int BYTES = L0::BYTES > L1::BYTES ? L0::BYTES : L1::BYTES;
    if (cudaFuncSetAttribute(march_kernel<T, NDIM, SCHEME, V, INTERVAL>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES) != cudaSuccess)
        return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, march_kernel<T, NDIM, SCHEME, V, INTERVAL>,
                                                      kThreads, BYTES) != cudaSuccess)
        return 0;
    return b;
}

template <typename T, int NDIM, int SCHEME, bool LAST, int V, bool INTERVAL, bool LLF = false>
cudaError_t launch_stage(const StageArgs& a, int grid, cudaStream_t s) {
    using L = StageSmem<T, NDIM, SCHEME, LAST, V>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(stage_kernel<T, NDIM, SCHEME, LAST, V, INTERVAL, LLF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(L::BYTES));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    stage_kernel<T, NDIM, SCHEME, LAST, V, INTERVAL, LLF><<<grid, kThreads, L::BYTES, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int NDIM, int SCHEME, bool LAST, int V, bool INTERVAL, bool LLF = false>
int max_blocks_stage() {
    using L = StageSmem<T, NDIM, SCHEME, LAST, V>;
    cudaFuncSetAttribute(stage_kernel<T, NDIM, SCHEME, LAST, V, INTERVAL, LLF>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(L::BYTES));
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stage_kernel<T, NDIM, SCHEME, LAST, V, INTERVAL, LLF>,
                                                      kThreads, L::BYTES) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

}  // namespace hji
