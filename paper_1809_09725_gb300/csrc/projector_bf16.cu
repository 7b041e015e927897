// projector_bf16.cu -- instantiates the projector pair for bf16 storage, float arithmetic.
#include "projector_impl.cuh"

namespace dr {
template struct ProjOps<bf16, float>;
}  // namespace dr
