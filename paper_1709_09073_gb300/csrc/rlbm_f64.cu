// FP64 storage (the plain method): fused pull-stream + collide step with all
// arithmetic in FP64, plus the FP64 initialiser, read-out and raw copies.
#include <cuda_runtime.h>

#include "rlbm_kernels.cuh"

namespace rlbm {

// One fused step for every cell of every tile: pull-stream from fin (its halo
// was filled by the previous step), moments, Landau state, equilibrium,
// relaxation (Eq. 3), store to fout and fill fout's halo.
template <int EDF>
__global__ void __launch_bounds__(kThreads) k_step_f64(StepArgs a) {
  extern __shared__ double sm[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const Tile tl = a.tiles[t];
    const DomDev& D = a.doms[tl.dom];
    const int x = tl.x0 + threadIdx.x, y = tl.y0 + threadIdx.y;
    if (x >= D.nx || y >= D.ny) continue;
    const double* __restrict__ fin = static_cast<const double*>(a.fin) + D.off;
    double* __restrict__ fout = static_cast<double*>(a.fout) + D.off;
    const long long c = cell_rel(D, x, y);
    double N[3], T[6];
    pull_moments64<EDF, StoreF64>(fin, D, x, y, c, sm, tid, N, T);
    CellState S;
    unsigned st = cell_state<EDF>(N, T, S);
    const bool ok = !(st & ST_NONPHYSICAL);
    if (ok) {
      // constant tau, or the local tau = 4 (eta/s) / theta + 0.2546 of Sec. 3.5;
      // a body force shifts the velocity the collision uses to u + a tau (Sec. 3.4)
      // (a branch, uniform per domain: the divisions only run for a local tau)
      double tau = D.tau, itau = D.inv_tau;
      if (D.eta_s > 0.0) {
        tau = 4.0 * D.eta_s / S.theta + 0.2546;
        itau = 1.0 / tau;
      }
      double ux = S.ux, uy = S.uy, gam = S.gamma;
      if (D.accel_x != 0.0 || D.accel_y != 0.0) {
        ux += D.accel_x * tau;
        uy += D.accel_y * tau;
        gam = 1.0 / sqrt(1.0 - ux * ux - uy * uy);
      }
      const int oi = D.order - 2;
      double om[12];
#pragma unroll
      for (int d = 0; d < 12; ++d) om[d] = gam * (1.0 - (dcos(d) * ux + dsin(d) * uy)) * itau;
      double zr[21], zi[21];
      // a clamped BE state relaxes to its own equilibrium energy 4 pi theta^3 g_3(z_c)
      const double eps_eq = (st & ST_CLAMPED) ? 4.0 * PI * S.theta * S.theta * S.theta * S.g[2] : S.eps;
      eq_moments<EDF>(S.g, S.theta, ux, uy, gam, S.n, eps_eq, zr, zi, oi);
#pragma unroll 1
      for (int s = 0; s < 6; ++s) {
        double fe[12];
        feq_shell<EDF>(s, zr, zi, fe, oi);
#pragma unroll
        for (int d = 0; d < 12; ++d) {
          const int q = 6 * d + s;
          const double v = sm[q * kThreads + tid];
          const double r = fma(om[d], fe[d] - v, v);
          sm[q * kThreads + tid] = r;
          fout[q * kBlkW + c] = r;
        }
      }
      if (touches_vwall(D, x, y)) write_vwall_ghosts<EDF, StoreF64>(D, x, y, fout, sm, tid, &S, &st);
    } else {
      for (int q = 0; q < 72; ++q) fout[q * kBlkW + c] = sm[q * kThreads + tid];
    }
    write_halo64<EDF, StoreF64>(D, x, y, fout, sm, tid, ok, S.n, S.ux, S.uy, S.gamma, st, ok);
    if (st) atomicOr(a.status, st);
  }
}

template <int EDF>
static cudaError_t prepare_t() {
  cudaError_t e = cudaFuncSetAttribute(k_step_f64<EDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64);
  if (e != cudaSuccess) return e;
  return prepare_common_t<StoreF64, EDF>();
}

// Opt the kernels into 72 KB of dynamic shared memory (once per process).
cudaError_t prepare_f64() {
  cudaError_t e;
  if ((e = prepare_t<EDF_MJ>())) return e;
  if ((e = prepare_t<EDF_FD>())) return e;
  return prepare_t<EDF_BE>();
}

cudaError_t launch_step_f64(int edf, const StepArgs& a, int grid, cudaStream_t s) {
  switch (edf) {
    case EDF_MJ: k_step_f64<EDF_MJ><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
    case EDF_FD: k_step_f64<EDF_FD><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
    default: k_step_f64<EDF_BE><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_init_f64(int edf, const InitArgs& a, int nx, int ny, cudaStream_t s) {
  return launch_init_t<StoreF64>(edf, a, nx, ny, s);
}

cudaError_t launch_fields_f64(int edf, const FieldsArgs& a, int nx, int ny, cudaStream_t s) {
  return launch_fields_t<StoreF64>(edf, a, nx, ny, s);
}

cudaError_t launch_copy_f64(const CopyArgs& a, cudaStream_t s) { return launch_copy_t<StoreF64>(a, s); }

}  // namespace rlbm
