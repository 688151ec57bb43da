// Mixed-precision kernels instantiated for FP32 storage.
#include "rlbm_mixed_impl.cuh"

namespace rlbm {
const MixedUnit kMixedF32 = mixed_unit<StoreF32>();
}  // namespace rlbm
