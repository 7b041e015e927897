// projector_f64.cu -- instantiates the projector pair for double storage, double arithmetic.
#include "projector_impl.cuh"

namespace dr {
template struct ProjOps<double, double>;
}  // namespace dr
