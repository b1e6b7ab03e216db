// FP32 instantiation of the kernels: FP32 storage and arithmetic, with the pressure
// recovery redone in FP64 in low internal-energy cells (physics.cuh).
#include "kernels_impl.cuh"
MAPGB_DEFINE_LAUNCHERS(float, f32)
