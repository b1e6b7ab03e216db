// FP32 step kernels with the HLLD interface flux (LF and WENO), compiled apart from the
// other FP32 kernels so the translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_STEP_VARIANT(float, launch_step_hlld_f32, FLX_HLLD, false)
