// Staged variant of the mixed-precision step (RLBM_KERNEL_STAGED): the same
// update as k_step_mixed with the same arithmetic in the same order
// (bit-identical results), with the memory traffic reorganised so that one
// tile's loads overlap the previous tile's collision:
//  * the whole pull neighbourhood of a 32 x 4 tile -- for each of the 12
//    directions one TMA box of its six shell planes over rows y0-1 .. y0+4 --
//    is copied into shared memory by 12 bulk-tensor loads on one mbarrier;
//  * every thread pulls its 72 populations (Eqs. 17-18) from those boxes into
//    registers (no global loads and no address arithmetic per population, and
//    no shared-memory column: the block holds 170 registers per thread);
//  * as soon as the block has pulled, one thread issues the next tile's boxes
//    into the same buffer, so they land while this tile collides (a tile at a
//    domain edge first borrows the buffer as the column its halo writer reads
//    and issues the next tile after that);
//  * the collided populations leave by coalesced stores from registers.
// Every wait for a copy is bounded (StepArgs::wait_ns); a wait that runs out
// sets ST_TIMEOUT, lets the copy in flight land (bounded) and ends the kernel.
// Included by rlbm_mixed_impl.cuh after the TMA helpers it shares with
// k_step_mixed_tma.
#pragma once

namespace rlbm {

constexpr int kVariantStaged = 4;  // StepArgs::variant of RLBM_KERNEL_STAGED

#ifndef RLBM_STAGED_MIN_BLOCKS
#define RLBM_STAGED_MIN_BLOCKS 3  // resident blocks per SM: 3 x 69 KB of boxes (FP32), 170 registers
#endif

template <class S>
constexpr size_t staged_smem_bytes() {
  return 12 * (size_t)TmaBox<S>::kBytes;
}

// The 12 boxes of tile t into `boxes`, completing on `bar` (one thread).
template <class S>
__device__ __forceinline__ void staged_issue(const StepArgs& a, int t, unsigned char* boxes, uint64_t* bar) {
  const Tile tl = a.tiles[t];
  const void* map = static_cast<const unsigned char*>(a.tmaps) + (size_t)tl.dom * kTensorMapBytes;
  mbar_expect_tx(bar, 12 * TmaBox<S>::kBytes);
#pragma unroll 1
  for (int d = 0; d < 12; ++d) tma_load_3d(boxes + d * TmaBox<S>::kBytes, map, tl.x0, tl.y0, 6 * d, bar);
}

// Pull of direction d (six shells) from its box into v[0..5], with the shell
// sums A = sum_s p_s v_s, B = sum_s p_s^2 v_s; same weights and order of
// operations as pull_one. `cell` points at the cell's own value in shell 0.
template <int d, class S>
__device__ __forceinline__ void pull_dir_regs(const typename S::T* cell, const DomDev& D, const float pc[6],
                                              const float p2c[6], float v[6], float& A, float& B) {
  using TB = TmaBox<S>;
  constexpr double cx = dcos(d), cy = dsin(d);
  constexpr int sx = sgnd(cx), sy = sgnd(cy);
  constexpr double ax = dabs(cx), ay = dabs(cy);
  constexpr float axr = (float)ax, ayr = (float)ay;
  constexpr float w1 = axr * ayr, w2 = (1.0f - axr) * ayr, w3 = axr * (1.0f - ayr),
                  w4 = (1.0f - axr) * (1.0f - ayr);
  constexpr int o1 = -sx - sy * TB::kW, o2 = -sy * TB::kW, o3 = -sx;
  float a_ = 0.0f, b_ = 0.0f;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const typename S::T* pl = cell + s * TB::kPlaneElems;
    float w;
    if (ax == 0.0 || ay == 0.0) {
      w = S::raw(pl[o1]);
    } else {
      const float v1 = S::raw(pl[o1]), v2 = S::raw(pl[o2]), v3 = S::raw(pl[o3]), v4 = S::raw(pl[0]);
      w = fmaf(w1, v1, fmaf(w2, v2, fmaf(w3, v3, w4 * v4)));
    }
    w = S::decf(w, D, s);
    v[s] = w;
    a_ = fmaf(w, pc[s], a_);
    b_ = fmaf(w, p2c[s], b_);
  }
  A = a_;
  B = b_;
}

// Collision of one cell whose pulled FP32 deviations are in registers v[72]
// (the arithmetic of collide_mixed); kKeep: also leave the relaxed values in
// the column col[q * kThreads] for the halo writer (edge tiles).
template <int EDF, class S, bool kKeep>
__device__ __forceinline__ unsigned collide_regs(const DomDev& D, int x, int y, long long c, const float A[12],
                                                 const float B[12], float v[72], float* col,
                                                 typename S::T* __restrict__ fout) {
  const long long P = D.plane;
  const HarmF ha = harmonics_f(A), hb = harmonics_f(B);
  const df N0 = df_add(df_make(D.n0_hl[0], D.n0_hl[1]), ha.h0);
  const df H0 = df_add(df_make(D.t00_hl[0], D.t00_hl[1]), hb.h0);
  df T[6];
  T[0] = H0;
  T[1] = df_make(hb.c1, 0.0f);
  T[2] = df_make(hb.s1, 0.0f);
  T[3] = df_scale(df_add(H0, hb.c2), 0.5f);
  T[4] = df_make(0.5f * hb.s2, 0.0f);
  T[5] = df_scale(df_add(H0, -hb.c2), 0.5f);
  df ux, uy, eps, gam;
  unsigned st = landau_df(T, ux, uy, eps, gam);
  df n = df_make(0.0f, 0.0f);
  if (!(st & ST_NONPHYSICAL)) {
    n = df_mul(gam, df_sub(N0, df_add(df_mul(ux, ha.c1), df_mul(uy, ha.s1))));
    if (!(n.hi > 0.0f) || !isfinite(n.hi)) st |= ST_NONPHYSICAL;
  }
  const bool ok = !(st & ST_NONPHYSICAL);
  const float uxf = df_to_float(ux), uyf = df_to_float(uy), gf = df_to_float(gam), nf = df_to_float(n);
  if (ok) {
    const float ef = df_to_float(eps);
    float theta, z, g[6];
    if (EDF == EDF_MJ) {
      theta = ef / (2.0f * nf);
      z = nf / (2.0f * kPIf * theta * theta);
#pragma unroll
      for (int i = 0; i < 6; ++i) g[i] = z;
    } else {
      const float target = 0.5f * kPIf * ef * ef / (nf * nf * nf);
      const int zs = solve_z_R_f<EDF>(target, z, g);
      st |= zs;
      if (zs & ST_CLAMPED) theta = sqrtf(nf / (2.0f * kPIf * g[1]));
      else theta = 0.5f * g[1] / g[2] * ef / nf;
    }
    const df nG = df_mul(n, gam);
    df eG2 = df_mul(df_mul(eps, gam), gam);
    if (st & ST_CLAMPED) eG2 = df_make(4.0f * kPIf * theta * theta * theta * g[2] * gf * gf, 0.0f);
    float zr[21], zi[21];
    dz_moments<EDF>(D, g, theta, uxf, uyf, gf, nG.hi, eG2.hi, zr, zi);
    const df u2h = df_scale(df_add(df_mul(ux, ux), df_mul(uy, uy)), 0.5f);
    const df dz10 = df_sub(nG, df_make(D.z1_hl[0], D.z1_hl[1]));
    const df dz20 = df_sub(df_add(eG2, df_mul(eG2, u2h)), df_make(D.z2_hl[0], D.z2_hl[1]));
    zr[1] = df_to_float(dz10);
    zr[3] = df_to_float(dz20);
    const df e15 = df_mul(eG2, 1.5f);
    zr[4] = df_to_float(df_mul(e15, ux));
    zi[4] = df_to_float(df_mul(e15, uy));
    float d10 = 0.0f, d20 = 0.0f, d21r = 0.0f, d21i = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      d10 = fmaf(c_Ef[EDF][k], zr[k * (k + 1) / 2], d10);
      d20 = fmaf(c_Ef[EDF][6 + k], zr[k * (k + 1) / 2], d20);
    }
#pragma unroll
    for (int k = 1; k < 6; ++k) {
      d21r = fmaf(c_Ef[EDF][12 + k], zr[k * (k + 1) / 2 + 1], d21r);
      d21i = fmaf(c_Ef[EDF][12 + k], zi[k * (k + 1) / 2 + 1], d21i);
    }
    zr[1] -= d10;
    zr[3] -= d20;
    zr[4] -= d21r;
    zi[4] -= d21i;
    float itau = (float)D.inv_tau;
    if (D.eta_s > 0.0) itau = 1.0f / (4.0f * (float)D.eta_s / theta + 0.2546f);
    float om[12];
#pragma unroll
    for (int d = 0; d < 12; ++d) om[d] = relax_rate(d, gf, uxf, uyf, itau);
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      float fe[12];
      dfeq_shell<EDF>(s, D.rres[s], zr, zi, fe);
#pragma unroll
      for (int d = 0; d < 12; ++d) {
        const int q = 6 * d + s;
        const float r = fmaf(om[d], fe[d] - v[q], v[q]);
        if constexpr (kKeep) col[q * kThreads] = r;
        fout[q * P + c] = S::encf(r, D, s);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 72; ++q) {
      if constexpr (kKeep) col[q * kThreads] = v[q];
      fout[q * P + c] = S::encf(v[q], D, q % 6);
    }
  }
  if (kKeep && (x == 0 || x == D.nx - 1 || y == 0 || y == D.ny - 1))
    halo_lean<EDF, S>(D, x, y, fout, col, ok, nf, uxf, uyf, gf, &st);
  return st;
}

template <int EDF, class S>
__global__ void __launch_bounds__(kThreads, RLBM_STAGED_MIN_BLOCKS) k_step_staged(StepArgs a) {
  using T = typename S::T;
  using TB = TmaBox<S>;
  extern __shared__ __align__(128) unsigned char sms[];
  __shared__ uint64_t bar;
  unsigned char* boxes = sms;
  float* colbase = reinterpret_cast<float*>(sms);  // the boxes, reused as the column of an edge tile
  const int tid = threadIdx.y * kTileW + threadIdx.x;
  if (blockIdx.x >= a.ntiles) return;  // whole block
  const unsigned long long wait_ns = a.wait_ns ? a.wait_ns : kDefaultWaitNs;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) staged_issue<S>(a, blockIdx.x, boxes, &bar);
  const T* cell0 = reinterpret_cast<const T*>(boxes) + (threadIdx.y + 1) * TB::kW + threadIdx.x + TB::kLpad;
  unsigned it = 0;  // tiles of this block so far = completed phases of the barrier
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++it) {
    const Tile tl = a.tiles[t];
    const DomDev& D = a.doms[tl.dom];
    const int tn = t + gridDim.x;
    float pc[6], p2c[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      pc[s] = c_pf[EDF][s];
      p2c[s] = c_p2f[EDF][s];
    }
    const bool ok = mbar_wait(&bar, it & 1, wait_ns);
    if (__syncthreads_or(!ok)) goto timed_out;
    float v[72], A[12], B[12];
#define RLBM_STAGED_PULL(d) \
    pull_dir_regs<d, S>(cell0 + (d) * TB::kStageElems, D, pc, p2c, v + 6 * (d), A[d], B[d]);
    RLBM_STAGED_PULL(0) RLBM_STAGED_PULL(1) RLBM_STAGED_PULL(2) RLBM_STAGED_PULL(3)
    RLBM_STAGED_PULL(4) RLBM_STAGED_PULL(5) RLBM_STAGED_PULL(6) RLBM_STAGED_PULL(7)
    RLBM_STAGED_PULL(8) RLBM_STAGED_PULL(9) RLBM_STAGED_PULL(10) RLBM_STAGED_PULL(11)
#undef RLBM_STAGED_PULL
    __syncthreads();  // every thread holds its populations: the boxes are free
    const bool edge = tl.x0 == 0 || tl.x0 + kTileW >= D.nx || tl.y0 == 0 || tl.y0 + kTileH >= D.ny;
    if (!edge && tid == 0 && tn < a.ntiles) staged_issue<S>(a, tn, boxes, &bar);  // lands during the collision
    {
      const int x = tl.x0 + threadIdx.x, y = tl.y0 + threadIdx.y;
      if (x < D.nx && y < D.ny) {
        T* __restrict__ fout = static_cast<T*>(a.fout) + D.off;
        const long long c = (long long)(y + 1) * D.pitch + D.lpad + x;
        unsigned st;
        if (edge) st = collide_regs<EDF, S, true>(D, x, y, c, A, B, v, colbase + tid, fout);
        else st = collide_regs<EDF, S, false>(D, x, y, c, A, B, v, nullptr, fout);
        if (st) atomicOr(a.status, st);
      }
    }
    if (edge) {
      __syncthreads();  // the halo writers are done with the column
      if (tid == 0 && tn < a.ntiles) staged_issue<S>(a, tn, boxes, &bar);
    }
  }
  return;
timed_out:
  // a copy did not land in time: report it and let the copy in flight land
  // (bounded by the default limit) so that none writes shared memory after exit
  if (tid == 0) {
    atomicOr(a.status, ST_TIMEOUT);
    mbar_wait(&bar, it & 1);
  }
}

template <class S, int EDF>
static cudaError_t prepare_staged_t() {
  return cudaFuncSetAttribute(k_step_staged<EDF, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)staged_smem_bytes<S>());
}

template <class S>
static cudaError_t launch_staged(int edf, const StepArgs& a, int grid, cudaStream_t s) {
  const size_t sm = staged_smem_bytes<S>();
  switch (edf) {
    case EDF_MJ: k_step_staged<EDF_MJ, S><<<grid, dim3(kTileW, kTileH), sm, s>>>(a); break;
    case EDF_FD: k_step_staged<EDF_FD, S><<<grid, dim3(kTileW, kTileH), sm, s>>>(a); break;
    default: k_step_staged<EDF_BE, S><<<grid, dim3(kTileW, kTileH), sm, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace rlbm
