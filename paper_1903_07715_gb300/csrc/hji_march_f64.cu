// Explicit instantiations of the multi-step march kernel in double (1-D and
// 2-D grids: the 3-D/4-D forms would spill registers, and those grids march
// with one launch per stage), and its dispatch table.
#include "hji_stage.cuh"

namespace hji {

#define HJI_MARCH(ND, SC, V)                                                                   \
    if (ndim == ND && scheme == SC && v == V)                                                   \
        return interval ? launch_march<double, ND, SC, V, true> : launch_march<double, ND, SC, V, false>;
#define HJI_MOCC(ND, SC, V)                                                                    \
    if (ndim == ND && scheme == SC && v == V)                                                   \
        return interval ? max_blocks_march<double, ND, SC, V, true>()                           \
                        : max_blocks_march<double, ND, SC, V, false>();
#define HJI_LOW(X) \
    X(1, HJI_ENO1, 0) X(1, HJI_ENO2, 0) X(1, HJI_WENO5, 0) \
    X(2, HJI_ENO1, 0) X(2, HJI_ENO2, 0) X(2, HJI_WENO5, 0) \
    X(2, HJI_ENO1, 1) X(2, HJI_ENO2, 1) X(2, HJI_WENO5, 1) \
    X(2, HJI_ENO1, 2) X(2, HJI_ENO2, 2) X(2, HJI_WENO5, 2)

MarchLauncher march_launcher_f64(int ndim, int scheme, int variant, bool interval) {
    const int v = ndim == 2 ? variant : 0;
    HJI_LOW(HJI_MARCH)
    return nullptr;
}

int march_max_blocks_f64(int ndim, int scheme, int variant, bool interval) {
    const int v = ndim == 2 ? variant : 0;
    HJI_LOW(HJI_MOCC)
    return 0;
}

}  // namespace hji
