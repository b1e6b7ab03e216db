// FP32 step kernels that record boundary face fluxes for reflux (meshes with coarse/fine
// faces), compiled apart so the translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_STEP_VARIANT(float, launch_step_rfx_f32, FLX_LF, true)
