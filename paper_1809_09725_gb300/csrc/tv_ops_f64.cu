// tv_ops_f64.cu -- explicit instantiation of the 4D TV kernels (see tv_impl.cuh).
#include "tv_impl.cuh"

namespace dr {
template struct TvOps<double, double>;
}  // namespace dr
