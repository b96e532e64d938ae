// Explicit instantiations of the fused stage kernel in float, and the
// dispatch table the host runtime uses to pick one.
#include "hji_stage.cuh"

namespace hji {

#define HJI_STAGE_ENTRY(ND, SC) \
    if (ndim == ND && scheme == SC) return last ? launch_stage<float, ND, SC, true> : launch_stage<float, ND, SC, false>;
#define HJI_STAGE_OCC(ND, SC) \
    if (ndim == ND && scheme == SC) return last ? max_blocks_stage<float, ND, SC, true>() : max_blocks_stage<float, ND, SC, false>();
#define HJI_ALL(X) \
    X(1, HJI_ENO1) X(1, HJI_ENO2) X(1, HJI_WENO5) \
    X(2, HJI_ENO1) X(2, HJI_ENO2) X(2, HJI_WENO5) \
    X(3, HJI_ENO1) X(3, HJI_ENO2) X(3, HJI_WENO5) \
    X(4, HJI_ENO1) X(4, HJI_ENO2) X(4, HJI_WENO5)

StageLauncher stage_launcher_f32(int ndim, int scheme, bool last) {
    HJI_ALL(HJI_STAGE_ENTRY)
    return nullptr;
}

int stage_max_blocks_f32(int ndim, int scheme, bool last) {
    HJI_ALL(HJI_STAGE_OCC)
    return 1;
}

}  // namespace hji
