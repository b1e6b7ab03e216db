// FP32 step kernels with the HLLC interface flux (LF and WENO), compiled apart from the
// other FP32 kernels so the two translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_HLLC_LAUNCHER(float, f32)
