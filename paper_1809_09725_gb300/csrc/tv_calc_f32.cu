// tv_calc_f32.cu -- explicit instantiation of the 4D TV kernels (see tv_impl.cuh).
#include "tv_impl.cuh"

namespace dr {
template struct TvCalc<float>;
}  // namespace dr
