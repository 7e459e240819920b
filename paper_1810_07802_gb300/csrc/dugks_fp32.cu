// FP32 instantiation of the phase-field DUGKS kernels (FP32 arithmetic on
// distributions stored as FP32 deviations from the rest state).
#include "dugks_launch.cuh"

namespace dugks {
DUGKS_INSTANTIATE(float)
}
