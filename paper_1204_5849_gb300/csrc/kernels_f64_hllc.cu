// FP64 step kernels with the HLLC interface flux (LF and WENO), compiled apart from the
// other FP64 kernels so the two translation units build in parallel.
#include "kernels_impl.cuh"
MAPGB_DEFINE_HLLC_LAUNCHER(double, f64)
