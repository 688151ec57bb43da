// Mixed-precision kernels instantiated for FP16-deviation storage.
#include "rlbm_mixed_impl.cuh"

namespace rlbm {
const MixedUnit kMixedF16 = mixed_unit<StoreF16>();
}  // namespace rlbm
