// FP32 instantiation of the librykov kernels (RK_MIXED contexts: per-velocity work in
// FP32, reductions compensated and combined in FP64, per-cell/per-face work FP64).
#include "rykov_launch_impl.cuh"

namespace rk {
template struct Launch<float>;
}
