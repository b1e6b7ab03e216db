// FP64 step kernels with the HLLD flux that record boundary face fluxes for reflux,
// compiled apart so the translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_STEP_VARIANT(double, launch_step_hlld_rfx_f64, FLX_HLLD, true)
