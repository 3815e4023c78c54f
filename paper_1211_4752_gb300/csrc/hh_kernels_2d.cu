// 2-D (5-point) instantiations of the stencil kernels.
#include "hh_kernels.cuh"
namespace hh {
HH_INSTANTIATE_DIM(2)
}  // namespace hh
