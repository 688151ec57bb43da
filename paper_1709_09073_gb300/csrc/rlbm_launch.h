// Kernel launchers shared between the C ABI (rlbm_api.cu) and the kernel
// translation units.
#pragma once
#include <cuda_runtime.h>

#include "rlbm_common.h"

namespace rlbm {

// Initialiser and read-out launches cover one domain (tiles == null: a 2D grid
// over domain `dom`, fields [ny][nx]) or every domain at once (a block per
// tile of the work list, fields packed domain after domain, DomDev::foff).
struct InitArgs {
  const DomDev* doms;
  int dom, kind;
  const double *a, *theta, *ux, *uy;  // device, [ny][nx] or packed
  void* f;                            // population copy to initialise
  unsigned* status;
  const Tile* tiles;                  // null: domain `dom` only
  int ntiles;
};

struct FieldsArgs {
  const DomDev* doms;
  int dom, streamed;
  const void* f;
  double *n, *theta, *ux, *uy, *z;    // device outputs, each may be null
  double* diag;                       // null, or [7][ny][nx]: q^0, q^x, q^y, pi^{x..x} orders 2-5
  unsigned* status;
  const Tile* tiles;                  // null: domain `dom` only; else every domain, packed outputs
  int ntiles;
};

struct CopyArgs {
  const DomDev* doms;
  int dom, to_dense;
  int q0, nq;                         // planes q0 .. q0+nq-1
  void* pop;
  double* dense;                      // [nq][ny+2][nx+2]
};

// FP64 storage (plain method)
cudaError_t prepare_f64();
cudaError_t launch_step_f64(int edf, const StepArgs& a, int grid, cudaStream_t s);
cudaError_t launch_init_f64(int edf, const InitArgs& a, int nx, int ny, cudaStream_t s);
cudaError_t launch_fields_f64(int edf, const FieldsArgs& a, int nx, int ny, cudaStream_t s);
cudaError_t launch_copy_f64(const CopyArgs& a, cudaStream_t s);

// FP32 / 16-bit deviation storage (mixed precision)
cudaError_t prepare_mixed();
cudaError_t launch_prepare_refs(int edf, DomDev* doms, int ndom, cudaStream_t s);
cudaError_t launch_step_mixed(int storage, int edf, const StepArgs& a, int grid, cudaStream_t s);
cudaError_t launch_init_mixed(int storage, int edf, const InitArgs& a, int nx, int ny, cudaStream_t s);
cudaError_t launch_fields_mixed(int storage, int edf, const FieldsArgs& a, int nx, int ny, cudaStream_t s);
cudaError_t launch_copy_mixed(int storage, const CopyArgs& a, cudaStream_t s);

}  // namespace rlbm
