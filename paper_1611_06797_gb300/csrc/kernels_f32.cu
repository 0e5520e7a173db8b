// FP32 (precision form) instantiation of the hot-path kernels.
#include "path_impl.cuh"
namespace ltmp2 {
template struct Path<float>;
}
