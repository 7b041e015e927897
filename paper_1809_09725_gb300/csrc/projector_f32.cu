// projector_f32.cu -- instantiates the projector pair for float storage, float arithmetic.
#include "projector_impl.cuh"

namespace dr {
template struct ProjOps<float, float>;
}  // namespace dr
