// Explicit instantiations of the stage kernel in float with local
// Lax-Friedrichs dissipation (node-wise coefficients; default tile shape;
// the last stage has the interval test compiled in), and their dispatch.
#include "hji_stage.cuh"

namespace hji {

#define HJI_LLF(ND, SC)                                                                       \
    if (ndim == ND && scheme == SC)                                                            \
        return last ? launch_stage<float, ND, SC, true, 0, true, true>                          \
                    : launch_stage<float, ND, SC, false, 0, false, true>;
#define HJI_LLF_OCC(ND, SC)                                                                   \
    if (ndim == ND && scheme == SC)                                                            \
        return last ? max_blocks_stage<float, ND, SC, true, 0, true, true>()                    \
                    : max_blocks_stage<float, ND, SC, false, 0, false, true>();
#define HJI_DIMS(X) \
    X(1, HJI_ENO1) X(1, HJI_ENO2) X(1, HJI_WENO5) X(2, HJI_ENO1) X(2, HJI_ENO2) X(2, HJI_WENO5) \
    X(3, HJI_ENO1) X(3, HJI_ENO2) X(3, HJI_WENO5) X(4, HJI_ENO1) X(4, HJI_ENO2) X(4, HJI_WENO5)

StageLauncher stage_launcher_llf_f32(int ndim, int scheme, bool last) {
    HJI_DIMS(HJI_LLF)
    return nullptr;
}

int stage_max_blocks_llf_f32(int ndim, int scheme, bool last) {
    HJI_DIMS(HJI_LLF_OCC)
    return 1;
}

}  // namespace hji
