// FP32 step kernels with the HLLC interface flux (LF and WENO), compiled apart from the
// other FP32 kernels so the translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_STEP_VARIANT(float, launch_step_hllc_f32, FLX_HLLC, false)
