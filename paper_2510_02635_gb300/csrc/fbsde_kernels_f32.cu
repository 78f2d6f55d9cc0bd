// FP32-stream instantiation of the kernels (particle state, increments and moment sums
// in float; regression combination, CG vectors and Newton in double).
#include "fbsde_launch.cuh"

namespace fbsde {
template struct Launch<float>;
}
