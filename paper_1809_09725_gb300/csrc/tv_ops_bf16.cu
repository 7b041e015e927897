// tv_ops_bf16.cu -- explicit instantiation of the 4D TV kernels (see tv_impl.cuh).
#include "tv_impl.cuh"

namespace dr {
template struct TvOps<float, bf16>;
}  // namespace dr
