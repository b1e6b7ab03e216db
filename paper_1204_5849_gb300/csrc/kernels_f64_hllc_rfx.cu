// FP64 step kernels with the HLLC flux that record boundary face fluxes for reflux,
// compiled apart so the translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_STEP_VARIANT(double, launch_step_hllc_rfx_f64, FLX_HLLC, true)
