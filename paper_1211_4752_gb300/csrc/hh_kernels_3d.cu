// 3-D (7-point) instantiations of the stencil kernels.
#include "hh_kernels.cuh"
namespace hh {
HH_INSTANTIATE_DIM(3)
}  // namespace hh
