// FP64 instantiation of the librykov kernels (RK_FP64 contexts).
#include "rykov_launch_impl.cuh"

namespace rk {
template struct Launch<double>;
}
