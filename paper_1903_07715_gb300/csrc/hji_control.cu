// The instantaneous optimal control of Eq. (9), u*(x) = argmax_u min_d
// <grad V(x), f(x,u,d)>, at every node of a grid's current value, together
// with the disturbance attaining the inner minimum.
//
// grad V is the average (p- + p+)/2 of the scheme's one-sided derivatives,
// the gradient at which the march evaluates the Hamiltonian, with the same
// ghost nodes (linear extrapolation, periodic wrap).  For control-affine
// dynamics <p, f> = <p, f0(x)> + <G^T p, u> + <E^T p, d>, so over boxes the
// choice separates by component: u*_j = uhi_j if (G^T p)_j >= 0 else ulo_j,
// and d*_k = dlo_k if (E^T p)_k >= 0 else dhi_k (a zero component, where any
// value is optimal, takes the upper control bound and the lower disturbance
// bound).  One thread per node; a post-pass over the converged value, run
// once per query.
#include "hji_common.cuh"
#include "hji_stage.cuh"

namespace hji {

template <typename T, int NDIM, int SCHEME>
__global__ void __launch_bounds__(kThreads) control_kernel(const ControlArgs a) {
    constexpr int G = Ghost<SCHEME>::G;
    const T* __restrict__ h = static_cast<const T*>(a.v_hi);
    const T* __restrict__ lo = static_cast<const T*>(a.v_lo);
    T* uo = static_cast<T*>(a.u_out);
    T* dout = static_cast<T*>(a.d_out);
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < a.ncells;
         node += (long long)gridDim.x * blockDim.x) {
        int idx[NDIM];
        long long r = node, base = 0;
#pragma unroll
        for (int ax = NDIM - 1; ax >= 0; --ax) {
            idx[ax] = static_cast<int>(r % a.n[ax]);
            r /= a.n[ax];
            base += (long long)idx[ax] * a.stride[ax];
        }
        T pbar[NDIM];
#pragma unroll
        for (int ax = 0; ax < NDIM; ++ax) {
            const long long l0 = base - (long long)idx[ax] * a.stride[ax];  // node 0 of the line
            Pair<T> line[2 * G + 1];
#pragma unroll
            for (int o = -G; o <= G; ++o)
                line[o + G] = line_pair<T>(h + l0, lo ? lo + l0 : nullptr, nullptr, idx[ax] + o,
                                           a.n[ax], a.stride[ax], a.periodic[ax]);
            T D[2 * G];
#pragma unroll
            for (int k = 0; k < 2 * G; ++k) D[k] = pair_diff(line[k + 1], line[k]);
            T pm, pp;
            one_sided_diffs<T, SCHEME>(D, T(a.inv_dx[ax]), pm, pp);
            pbar[ax] = T(0.5) * (pp + pm);
        }
        for (int j = 0; j < a.m; ++j) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < NDIM; ++i) s += T(a.G[i * MAXU + j]) * pbar[i];
            uo[(long long)j * a.ncells + node] = s >= T(0) ? T(a.uhi[j]) : T(a.ulo[j]);
        }
        if (dout != nullptr) {
            for (int k = 0; k < a.q; ++k) {
                T s = T(0);
#pragma unroll
                for (int i = 0; i < NDIM; ++i) s += T(a.E[i * MAXU + k]) * pbar[i];
                dout[(long long)k * a.ncells + node] = s >= T(0) ? T(a.dlo[k]) : T(a.dhi[k]);
            }
        }
    }
}

template <typename T, int NDIM>
static cudaError_t launch_control_nd(const ControlArgs& a, int scheme, int grid, cudaStream_t s) {
    if (scheme == HJI_ENO1) control_kernel<T, NDIM, HJI_ENO1><<<grid, kThreads, 0, s>>>(a);
    else if (scheme == HJI_ENO2) control_kernel<T, NDIM, HJI_ENO2><<<grid, kThreads, 0, s>>>(a);
    else control_kernel<T, NDIM, HJI_WENO5><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_control_t(const ControlArgs& a, int ndim, int scheme, int grid,
                                    cudaStream_t s) {
    switch (ndim) {
        case 1: return launch_control_nd<T, 1>(a, scheme, grid, s);
        case 2: return launch_control_nd<T, 2>(a, scheme, grid, s);
        case 3: return launch_control_nd<T, 3>(a, scheme, grid, s);
        default: return launch_control_nd<T, 4>(a, scheme, grid, s);
    }
}

cudaError_t launch_control(const ControlArgs& a, bool f32, int ndim, int scheme, cudaStream_t s) {
    long long blocks = (a.ncells + kThreads - 1) / kThreads;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    return f32 ? launch_control_t<float>(a, ndim, scheme, (int)blocks, s)
               : launch_control_t<double>(a, ndim, scheme, (int)blocks, s);
}

}  // namespace hji
