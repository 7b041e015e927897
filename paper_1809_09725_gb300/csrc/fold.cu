// fold.cu -- instantiates the half-turn folded projector pair (fold_impl.cuh)
// for float and bf16 storage with float arithmetic.
#include <algorithm>
#include <cmath>

#include "fold_impl.cuh"

namespace dr {
template struct FoldOps<float, float>;
template struct FoldOps<bf16, float>;
}  // namespace dr
