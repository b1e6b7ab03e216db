// FP64 step kernels that record boundary face fluxes for reflux (meshes with coarse/fine
// faces), compiled apart so the translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_STEP_VARIANT(double, launch_step_rfx_f64, FLX_LF, true)
