// FP64 instantiation of the kernels (double throughout).
#include "fbsde_launch.cuh"

namespace fbsde {
template struct Launch<double>;
}
