// Mixed-precision kernels instantiated for FP32-deviation storage.
#include "rlbm_mixed_impl.cuh"

namespace rlbm {
const MixedUnit kMixedF32Dev = mixed_unit<StoreF32Dev>();
}  // namespace rlbm
