// FP64 instantiation of the phase-field DUGKS kernels.
#include "dugks_launch.cuh"

namespace dugks {
DUGKS_INSTANTIATE(double)
}
