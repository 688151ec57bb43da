// Mixed-precision kernels instantiated for BF16-deviation storage.
#include "rlbm_mixed_impl.cuh"

namespace rlbm {
const MixedUnit kMixedBF16 = mixed_unit<StoreBF16>();
}  // namespace rlbm
