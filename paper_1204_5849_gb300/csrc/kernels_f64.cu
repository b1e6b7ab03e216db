// FP64 instantiation of the kernels: the plain FP64 form.  Compiled without FMA
// contraction (-fmad=false) so each operation rounds separately.
#include "kernels_impl.cuh"
MAPGB_DEFINE_LAUNCHERS(double, f64)
