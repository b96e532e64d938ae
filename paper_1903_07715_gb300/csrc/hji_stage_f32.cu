// Explicit instantiations of the fused stage kernel in float, and the
// dispatch table the host runtime uses to pick one.
#include "hji_stage.cuh"

namespace hji {

#define HJI_ENTRY(ND, SC, V)                                                                   \
    if (ndim == ND && scheme == SC && v == V) {                                                 \
        if (!last) return launch_stage<float, ND, SC, false, V, false>;                        \
        return interval ? launch_stage<float, ND, SC, true, V, true>                           \
                        : launch_stage<float, ND, SC, true, V, false>;                         \
    }
#define HJI_OCC(ND, SC, V)                                                                     \
    if (ndim == ND && scheme == SC && v == V) {                                                 \
        if (!last) return max_blocks_stage<float, ND, SC, false, V, false>();                  \
        return interval ? max_blocks_stage<float, ND, SC, true, V, true>()                     \
                        : max_blocks_stage<float, ND, SC, true, V, false>();                   \
    }
#define HJI_ALL(X) \
    X(1, HJI_ENO1, 0) X(1, HJI_ENO2, 0) X(1, HJI_WENO5, 0) \
    X(2, HJI_ENO1, 0) X(2, HJI_ENO2, 0) X(2, HJI_WENO5, 0) \
    X(2, HJI_ENO1, 1) X(2, HJI_ENO2, 1) X(2, HJI_WENO5, 1) \
    X(2, HJI_ENO1, 2) X(2, HJI_ENO2, 2) X(2, HJI_WENO5, 2) \
    X(3, HJI_ENO1, 0) X(3, HJI_ENO2, 0) X(3, HJI_WENO5, 0) \
    X(4, HJI_ENO1, 0) X(4, HJI_ENO2, 0) X(4, HJI_WENO5, 0)

StageLauncher stage_launcher_f32(int ndim, int scheme, bool last, int variant, bool interval) {
    const int v = ndim == 2 ? variant : 0;
    HJI_ALL(HJI_ENTRY)
    return nullptr;
}

int stage_max_blocks_f32(int ndim, int scheme, bool last, int variant, bool interval) {
    const int v = ndim == 2 ? variant : 0;
    HJI_ALL(HJI_OCC)
    return 1;
}

}  // namespace hji
