// FP64 step kernels with the HLLD interface flux (LF and WENO), compiled apart from the
// other FP64 kernels so the translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_STEP_VARIANT(double, launch_step_hlld_f64, FLX_HLLD, false)
