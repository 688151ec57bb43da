// Mixed-precision path: the reference equilibria of the domains and the
// dispatch to the per-storage translation units (rlbm_mixed_<storage>.cu),
// which hold the step, initialiser, read-out and copy kernels.
#include "rlbm_mixed_impl.cuh"

namespace rlbm {

namespace {
const MixedUnit& unit(int storage) {
  switch (storage) {
    case ST_F32: return kMixedF32;
    case ST_F32DEV: return kMixedF32Dev;
    case ST_BF16DEV: return kMixedBF16;
    default: return kMixedF16;
  }
}
}  // namespace

// Upload the FP32 tables of every unit and opt the kernels into their shared memory.
cudaError_t prepare_mixed() {
  cudaError_t e = upload_mixed_tables();  // this unit's copy, read by k_prepare_refs
  if (e != cudaSuccess) return e;
  for (int st : {ST_F32, ST_F32DEV, ST_BF16DEV, ST_F16DEV})
    if ((e = unit(st).prepare()) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_prepare_refs(int edf, DomDev* doms, int ndom, cudaStream_t s) {
  const int grid = (ndom + 63) / 64;
  switch (edf) {
    case EDF_MJ: k_prepare_refs<EDF_MJ><<<grid, 64, 0, s>>>(doms, ndom); break;
    case EDF_FD: k_prepare_refs<EDF_FD><<<grid, 64, 0, s>>>(doms, ndom); break;
    default: k_prepare_refs<EDF_BE><<<grid, 64, 0, s>>>(doms, ndom); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_step_mixed(int storage, int edf, const StepArgs& a, int grid, cudaStream_t s) {
  return unit(storage).step(edf, a, grid, s);
}

cudaError_t launch_init_mixed(int storage, int edf, const InitArgs& a, int nx, int ny, cudaStream_t s) {
  return unit(storage).init(edf, a, nx, ny, s);
}

cudaError_t launch_fields_mixed(int storage, int edf, const FieldsArgs& a, int nx, int ny, cudaStream_t s) {
  return unit(storage).fields(edf, a, nx, ny, s);
}

cudaError_t launch_copy_mixed(int storage, const CopyArgs& a, cudaStream_t s) {
  return unit(storage).copy(a, s);
}

}  // namespace rlbm
