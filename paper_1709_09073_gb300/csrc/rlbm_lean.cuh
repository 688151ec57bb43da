// Lean variant of the mixed-precision step (RLBM_KERNEL_LEAN, _LEAN2): the same
// update as k_step_mixed with the same arithmetic in the same order, so the
// results are bit-identical, but with fewer issued instructions and shorter
// waits per cell:
//  * the block copies its tile's domain descriptor into shared memory once, so
//    the collision reads its per-domain constants there instead of issuing
//    global loads that the streaming pull may have evicted from L1;
//  * with kCells = 2 each thread owns two adjacent cells of a row, and the
//    bilinear pull of both (Eqs. 17-18) reads each plane row with one aligned
//    pair load plus one single load, against four single loads per cell;
//  * the shell loop of the collision is unrolled, so the projection tables are
//    immediate constant-bank operands instead of indexed constant loads;
//  * the relaxed populations go back into the shared-memory column only in
//    tiles that touch a domain edge (where the halo writer reads them), and
//    the halo writer runs only for edge cells.
// Included by rlbm_mixed_impl.cuh after the helpers it shares with k_step_mixed.
#pragma once

namespace rlbm {

// StepArgs::variant values of the lean kernels (RLBM_KERNEL_LEAN, _LEAN2)
constexpr int kVariantLean = 2, kVariantLean2 = 3;

constexpr int kDomWords = (int)(sizeof(DomDev) / sizeof(unsigned));
static_assert(sizeof(DomDev) % sizeof(unsigned) == 0, "descriptor copied by words");

// Raw stored values as FP32: one element, or an aligned pair (x, x+1).
template <class S>
__device__ __forceinline__ float ld1(const typename S::T* p) {
  return S::raw(*p);
}
template <class S>
__device__ __forceinline__ float2 ld2(const typename S::T* p) {
  using T = typename S::T;
  if constexpr (sizeof(T) == 4) {
    return *reinterpret_cast<const float2*>(p);
  } else if constexpr (S::kind == ST_F16DEV) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
  } else {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  }
}

// Bilinear pull of direction d from one plane for the kCells cells starting at
// element c (v[j] for cell x + j); same weights and order of operations as
// pull_one. For two cells, c is even, so the pair (c, c+1) of a row is 8-byte
// (FP32) or 4-byte (16-bit) aligned.
template <int d, class S, int kCells>
__device__ __forceinline__ void pull_cells(const typename S::T* __restrict__ pl, long long c, int W, float v[kCells]) {
  constexpr double cx = dcos(d), cy = dsin(d);
  constexpr int sx = sgnd(cx), sy = sgnd(cy);
  constexpr double ax = dabs(cx), ay = dabs(cy);
  if constexpr (kCells == 1) {
    v[0] = pull_one<d, float, S>(pl, c, W);
  } else if constexpr (ax == 0.0 || ay == 0.0) {
    const long long o1 = c - sx - (long long)sy * W;
    if constexpr (sx == 0) {
      const float2 p = ld2<S>(pl + o1);
      v[0] = p.x;
      v[1] = p.y;
    } else {
      v[0] = ld1<S>(pl + o1);
      v[1] = ld1<S>(pl + o1 + 1);
    }
  } else {
    constexpr float axr = (float)ax, ayr = (float)ay;
    constexpr float w1 = axr * ayr, w2 = (1.0f - axr) * ayr, w3 = axr * (1.0f - ayr),
                    w4 = (1.0f - axr) * (1.0f - ayr);
    const long long ra = c - (long long)sy * W;  // row y - sy
    // per row: the aligned pair (x, x+1) and the single value x - 1 (sx > 0) or x + 2
    const float2 pa = ld2<S>(pl + ra), pb = ld2<S>(pl + c);
    const float ea = ld1<S>(pl + ra + (sx > 0 ? -1 : 2)), eb = ld1<S>(pl + c + (sx > 0 ? -1 : 2));
    // v1 = f(x - sx, y - sy), v2 = f(x, y - sy), v3 = f(x - sx, y), v4 = f(x, y)
    if constexpr (sx > 0) {
      v[0] = fmaf(w1, ea, fmaf(w2, pa.x, fmaf(w3, eb, w4 * pb.x)));
      v[1] = fmaf(w1, pa.x, fmaf(w2, pa.y, fmaf(w3, pb.x, w4 * pb.y)));
    } else {
      v[0] = fmaf(w1, pa.y, fmaf(w2, pa.x, fmaf(w3, pb.y, w4 * pb.x)));
      v[1] = fmaf(w1, ea, fmaf(w2, pa.y, fmaf(w3, eb, w4 * pb.y)));
    }
  }
}

// The halo writer, kept out of line: only edge cells call it.
template <int EDF, class S>
__device__ __noinline__ void halo_lean(const DomDev& D, int x, int y, typename S::T* __restrict__ fout,
                                       const float* col, bool ok, float n, float ux, float uy, float gam,
                                       unsigned* st) {
  unsigned s = 0;
  write_halo_mixed<EDF, S, true>(D, x, y, fout, col, ok, n, ux, uy, gam, s);
  *st |= s;
}

// Collision of one cell from the harmonic sums of its pulled FP32 deviations
// (ha: shell sums weighted by p, hb: by p^2) and its column col[q * kThreads];
// the arithmetic of collide_mixed, shell loop unrolled. kKeep: write the relaxed
// values back into the column (edge tiles).
template <int EDF, class S, bool kKeep, int kUnroll>
__device__ __forceinline__ unsigned collide_lean(const DomDev& D, int x, int y, long long c, const HarmF& ha,
                                                 const HarmF& hb, float* col, typename S::T* __restrict__ fout) {
  const long long P = D.plane;
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
#pragma unroll kUnroll
    for (int s = 0; s < 6; ++s) {
      float fe[12];
      dfeq_shell<EDF>(s, D.rres[s], zr, zi, fe);
#pragma unroll
      for (int d = 0; d < 12; ++d) {
        const int q = 6 * d + s;
        const float v = col[q * kThreads];
        const float r = fmaf(om[d], fe[d] - v, v);
        if constexpr (kKeep) col[q * kThreads] = r;
        fout[q * P + c] = S::encf(r, D, s);
      }
    }
  } else {
    for (int q = 0; q < 72; ++q) fout[q * P + c] = S::encf(col[q * kThreads], D, q % 6);
  }
  if (kKeep && (x == 0 || x == D.nx - 1 || y == 0 || y == D.ny - 1))
    halo_lean<EDF, S>(D, x, y, fout, col, ok, nf, uxf, uyf, gf, &st);
  return st;
}

#ifndef RLBM_LEAN2_MIN_BLOCKS
#define RLBM_LEAN2_MIN_BLOCKS 6  // resident 64-thread blocks per SM (register budget)
#endif
// shells of the collision unrolled per iteration (1: the tables are indexed
// per shell; 6: all entries are immediate operands, at a register cost)
#ifndef RLBM_LEAN_UNROLL
#define RLBM_LEAN_UNROLL 1
#endif
#ifndef RLBM_LEAN2_UNROLL
#define RLBM_LEAN2_UNROLL 6
#endif

template <int kCells>
constexpr int lean_threads() {
  return kThreads / kCells;
}

// kCells cells of a row per thread, 32 x 4 cells per block, one tile of the work
// list at a time (one block per tile, or a persistent grid).
template <int EDF, class S, int kCells>
__global__ void __launch_bounds__(kThreads / kCells, kCells == 1 ? RLBM_MIXED_MIN_BLOCKS : RLBM_LEAN2_MIN_BLOCKS)
    k_step_lean(StepArgs a) {
  using T = typename S::T;
  constexpr int kUnroll = kCells == 1 ? RLBM_LEAN_UNROLL : RLBM_LEAN2_UNROLL;
  extern __shared__ float smf[];
  __shared__ DomDev sD;
  constexpr int kW = kTileW / kCells;  // threads per tile row
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kW + tx;
  const int cell0 = ty * kTileW + kCells * tx;  // column slot of the thread's first cell
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const Tile tl = a.tiles[t];
    if (t != (int)blockIdx.x) __syncthreads();  // the previous tile is done with sD
    {
      const unsigned* src = reinterpret_cast<const unsigned*>(a.doms + tl.dom);
      unsigned* dst = reinterpret_cast<unsigned*>(&sD);
      for (int i = tid; i < kDomWords; i += kW * kTileH) dst[i] = src[i];
    }
    __syncthreads();
    const DomDev& D = sD;
    const int x = tl.x0 + kCells * tx, y = tl.y0 + ty;
    if (x >= D.nx || y >= D.ny) continue;
    const long long P = D.plane;
    const int W = D.pitch;
    const T* __restrict__ fin = static_cast<const T*>(a.fin) + D.off;
    T* __restrict__ fout = static_cast<T*>(a.fout) + D.off;
    const long long c = (long long)(y + 1) * W + D.lpad + x;
    float* col = smf + cell0;
    float pc[6], p2c[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      pc[s] = c_pf[EDF][s];
      p2c[s] = c_p2f[EDF][s];
    }
    float A[kCells][12], B[kCells][12];
#define RLBM_LEAN_DIR(d)                                                          \
  {                                                                               \
    float a_[kCells], b_[kCells];                                                 \
    _Pragma("unroll") for (int j = 0; j < kCells; ++j) a_[j] = b_[j] = 0.0f;      \
    _Pragma("unroll") for (int s = 0; s < 6; ++s) {                               \
      float v[kCells];                                                            \
      pull_cells<d, S, kCells>(fin + (6 * d + s) * P, c, W, v);                   \
      _Pragma("unroll") for (int j = 0; j < kCells; ++j) {                        \
        v[j] = S::decf(v[j], D, s);                                               \
        a_[j] = fmaf(v[j], pc[s], a_[j]);                                         \
        b_[j] = fmaf(v[j], p2c[s], b_[j]);                                        \
      }                                                                           \
      if constexpr (kCells == 2)                                                  \
        *reinterpret_cast<float2*>(col + (6 * d + s) * kThreads) = make_float2(v[0], v[1]); \
      else                                                                        \
        col[(6 * d + s) * kThreads] = v[0];                                       \
    }                                                                             \
    _Pragma("unroll") for (int j = 0; j < kCells; ++j) {                          \
      A[j][d] = a_[j];                                                            \
      B[j][d] = b_[j];                                                            \
    }                                                                             \
  }
    RLBM_LEAN_DIR(0) RLBM_LEAN_DIR(1) RLBM_LEAN_DIR(2) RLBM_LEAN_DIR(3)
    RLBM_LEAN_DIR(4) RLBM_LEAN_DIR(5) RLBM_LEAN_DIR(6) RLBM_LEAN_DIR(7)
    RLBM_LEAN_DIR(8) RLBM_LEAN_DIR(9) RLBM_LEAN_DIR(10) RLBM_LEAN_DIR(11)
#undef RLBM_LEAN_DIR
    HarmF ha[kCells], hb[kCells];
#pragma unroll
    for (int j = 0; j < kCells; ++j) {
      ha[j] = harmonics_f(A[j]);
      hb[j] = harmonics_f(B[j]);
    }
    // edge tiles keep the relaxed values in the column for the halo writer
    const bool keep = tl.x0 == 0 || tl.x0 + kTileW >= D.nx || tl.y0 == 0 || tl.y0 + kTileH >= D.ny;
    unsigned st = 0;
#pragma unroll 1
    for (int j = 0; j < kCells; ++j) {
      if (x + j >= D.nx) break;
      const HarmF hA = j == 0 ? ha[0] : ha[kCells - 1], hB = j == 0 ? hb[0] : hb[kCells - 1];
      if (keep) st |= collide_lean<EDF, S, true, kUnroll>(D, x + j, y, c + j, hA, hB, col + j, fout);
      else st |= collide_lean<EDF, S, false, kUnroll>(D, x + j, y, c + j, hA, hB, col + j, fout);
    }
    if (st) atomicOr(a.status, st);
  }
}

template <class S, int EDF>
static cudaError_t prepare_lean_t() {
  cudaError_t e = cudaFuncSetAttribute(k_step_lean<EDF, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(72 * kThreads * sizeof(float)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_step_lean<EDF, S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(72 * kThreads * sizeof(float)));
}

template <class S>
static cudaError_t launch_lean(int edf, int cells, const StepArgs& a, int grid, cudaStream_t s) {
  const size_t sm = 72 * kThreads * sizeof(float);
  if (cells == 2) {
    const dim3 blk(kTileW / 2, kTileH);
    switch (edf) {
      case EDF_MJ: k_step_lean<EDF_MJ, S, 2><<<grid, blk, sm, s>>>(a); break;
      case EDF_FD: k_step_lean<EDF_FD, S, 2><<<grid, blk, sm, s>>>(a); break;
      default: k_step_lean<EDF_BE, S, 2><<<grid, blk, sm, s>>>(a); break;
    }
  } else {
    const dim3 blk(kTileW, kTileH);
    switch (edf) {
      case EDF_MJ: k_step_lean<EDF_MJ, S, 1><<<grid, blk, sm, s>>>(a); break;
      case EDF_FD: k_step_lean<EDF_FD, S, 1><<<grid, blk, sm, s>>>(a); break;
      default: k_step_lean<EDF_BE, S, 1><<<grid, blk, sm, s>>>(a); break;
    }
  }
  return cudaGetLastError();
}

}  // namespace rlbm
