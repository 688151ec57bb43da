// Kernels shared by the storage formats: storage policies, the bilinear pull
// (Eqs. 17-18), the FP64 initialiser / read-out / raw copies, and the halo
// writer that fuses the boundary conditions into the producing kernel.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rlbm_device.cuh"
#include "rlbm_launch.h"

namespace rlbm {

constexpr int kThreads = kTileW * kTileH;  // one cell per thread; blocks of one tile
static_assert(kThreads == 128 || kThreads == 256, "tiles of 32 x 4 or 32 x 8 cells");

__host__ __device__ constexpr int sgnd(double v) { return (v > 0.0) - (v < 0.0); }
__host__ __device__ constexpr double dcos(int d) {
  return d == 0 ? 1.0 : d == 1 ? SQRT3_2 : d == 2 ? 0.5 : d == 3 ? 0.0 : d == 4 ? -0.5
       : d == 5 ? -SQRT3_2 : d == 6 ? -1.0 : d == 7 ? -SQRT3_2 : d == 8 ? -0.5 : d == 9 ? 0.0
       : d == 10 ? 0.5 : SQRT3_2;
}
__host__ __device__ constexpr double dsin(int d) { return dcos((d + 9) % 12); }
__host__ __device__ constexpr double dabs(double v) { return v < 0.0 ? -v : v; }

// ------------------------------------------------------------ storage policies
// dec/enc convert between a stored value and the population f in FP64;
// decf/encf between a stored (or interpolated) value and the FP32 deviation
// f - fref used by the mixed-precision step.
struct StoreF64 {
  using T = double;
  static constexpr int kind = ST_F64;
  __device__ static double raw(T v) { return v; }
  __device__ static double dec(double r, const DomDev&, int) { return r; }
  __device__ static T enc(double f, const DomDev&, int) { return f; }
};
struct StoreF32 {
  using T = float;
  static constexpr int kind = ST_F32;
  __device__ static float raw(T v) { return v; }
  __device__ static double dec(double r, const DomDev&, int) { return r; }
  __device__ static T enc(double f, const DomDev&, int) { return (float)f; }
  __device__ static float decf(float r, const DomDev& D, int s) { return r - D.fref[s]; }
  __device__ static T encf(float df, const DomDev& D, int s) { return D.fref[s] + df; }
};
struct StoreBF16 {
  using T = __nv_bfloat16;
  static constexpr int kind = ST_BF16DEV;
  __device__ static float raw(T v) { return __bfloat162float(v); }
  __device__ static double dec(double h, const DomDev& D, int s) { return (double)D.fref[s] + (double)D.a_s[s] * h; }
  __device__ static T enc(double f, const DomDev& D, int s) {
    return __float2bfloat16_rn((float)((f - (double)D.fref[s]) * (double)D.b_s[s]));
  }
  __device__ static float decf(float h, const DomDev& D, int s) { return D.a_s[s] * h; }
  __device__ static T encf(float df, const DomDev& D, int s) { return __float2bfloat16_rn(df * D.b_s[s]); }
};
struct StoreF16 {
  using T = __half;
  static constexpr int kind = ST_F16DEV;
  __device__ static float raw(T v) { return __half2float(v); }
  __device__ static double dec(double h, const DomDev& D, int s) { return (double)D.fref[s] + (double)D.a_s[s] * h; }
  __device__ static T enc(double f, const DomDev& D, int s) {
    return __float2half_rn((float)((f - (double)D.fref[s]) * (double)D.b_s[s]));
  }
  __device__ static float decf(float h, const DomDev& D, int s) { return D.a_s[s] * h; }
  __device__ static T encf(float df, const DomDev& D, int s) { return __float2half_rn(df * D.b_s[s]); }
};

// FP32 absolute deviation h = f - fref: FP32's exponent range covers every
// shell, so no per-shell scale is needed and decoding/encoding in the mixed
// step are exact identities.
struct StoreF32Dev {
  using T = float;
  static constexpr int kind = ST_F32DEV;
  __device__ static float raw(T v) { return v; }
  __device__ static double dec(double h, const DomDev& D, int s) { return (double)D.fref[s] + h; }
  __device__ static T enc(double f, const DomDev& D, int s) { return (float)(f - (double)D.fref[s]); }
  __device__ static float decf(float h, const DomDev&, int) { return h; }
  __device__ static T encf(float df, const DomDev&, int) { return df; }
};

// Element offsets, from a cell's own element, of its neighbours x - 1 and
// x + 1 in the same row (in the next block across a block boundary) and of
// the rows y - 1 and y + 1. Across a periodic side they point at the wrapped
// interior cell (x = nx - 1 for x - 1 of x = 0, row ny - 1 for y - 1 of row 0,
// and so on) rather than at the halo image, which holds the same value when
// it is written: the offsets compose, so a diagonal neighbour wraps in x, in
// y or in both. Every pull therefore reads no periodic halo image.
struct Nbr {
  int xm, xp;
  long long ym, yp;
};
__device__ __forceinline__ Nbr neighbours(const DomDev& D, int x, int y) {
  const int lane = (x + kBlkW) % kBlkW;
  Nbr n;
  n.xm = lane ? -1 : -kBlk + (kBlkW - 1);
  n.xp = lane != kBlkW - 1 ? 1 : kBlk - (kBlkW - 1);
  if (D.bc[0] == BC_PERIODIC) {
    const int span = (int)(cell_rel(D, D.nx - 1, 0) - cell_rel(D, 0, 0));
    if (x == 0) n.xm = span;
    if (x == D.nx - 1) n.xp = -span;
  }
  n.ym = -D.pitch;
  n.yp = D.pitch;
  if (D.bc[2] == BC_PERIODIC) {
    const long long span = (long long)(D.ny - 1) * D.pitch;
    if (y == 0) n.ym = span;
    if (y == D.ny - 1) n.yp = -span;
  }
  return n;
}

// Bilinear interpolated pull of direction d from one plane (Eqs. 17-18): the
// four grid points around x - v_d with weights |v_x||v_y|, (1-|v_x|)|v_y|,
// |v_x|(1-|v_y|), (1-|v_x|)(1-|v_y|); axis directions shift by one cell.
// `pl` points at the cell's own element of the plane. Interpolates the stored
// values (decoding is affine per plane).
template <int d, class R, class S>
__device__ __forceinline__ R pull_one(const typename S::T* __restrict__ pl, const Nbr& nb) {
  constexpr double cx = dcos(d), cy = dsin(d);
  constexpr int sx = sgnd(cx), sy = sgnd(cy);
  constexpr double ax = dabs(cx), ay = dabs(cy);
  const long long ox = sx > 0 ? nb.xm : (sx < 0 ? nb.xp : 0);  // to x - sx
  const long long oy = sy > 0 ? nb.ym : (sy < 0 ? nb.yp : 0);   // to y - sy
  if (ax == 0.0 || ay == 0.0) return (R)S::raw(pl[ox + oy]);
  // weights from the rounded |v_x|, |v_y| (one of them is 1/2): every product and
  // 1 - |v| is exact in R, so the four weights sum to exactly 1 and streaming
  // conserves the global sums of every plane
  constexpr R axr = (R)ax, ayr = (R)ay;
  constexpr R w1 = axr * ayr, w2 = (R(1) - axr) * ayr, w3 = axr * (R(1) - ayr),
              w4 = (R(1) - axr) * (R(1) - ayr);
  const R v1 = (R)S::raw(pl[ox + oy]), v2 = (R)S::raw(pl[oy]), v3 = (R)S::raw(pl[ox]), v4 = (R)S::raw(pl[0]);
  return fma(w1, v1, fma(w2, v2, fma(w3, v3, w4 * v4)));
}

// Pull all 72 populations (FP64) into the thread's shared-memory column and
// return N^mu, T^{mu nu} (Eqs. 20, 22).
template <int EDF, class S>
__device__ __forceinline__ void pull_moments64(const typename S::T* __restrict__ fin, const DomDev& D,
                                               int x, int y, long long c, double* sm, int tid, double N[3],
                                               double T[6]) {
  const Nbr nb = neighbours(D, x, y);
  double A[12], B[12];
#define RLBM_PULL_DIR(d)                                                          \
  {                                                                               \
    double a_ = 0.0, b_ = 0.0;                                                    \
    _Pragma("unroll") for (int s = 0; s < 6; ++s) {                               \
      const double v = S::dec(pull_one<d, double, S>(fin + c + (6 * d + s) * kBlkW, nb), D, s); \
      sm[(6 * d + s) * kThreads + tid] = v;                                       \
      a_ = fma(v, c_p[EDF][s], a_);                                               \
      b_ = fma(v, c_p2[EDF][s], b_);                                              \
    }                                                                             \
    A[d] = a_;                                                                    \
    B[d] = b_;                                                                    \
  }
  RLBM_PULL_DIR(0) RLBM_PULL_DIR(1) RLBM_PULL_DIR(2) RLBM_PULL_DIR(3)
  RLBM_PULL_DIR(4) RLBM_PULL_DIR(5) RLBM_PULL_DIR(6) RLBM_PULL_DIR(7)
  RLBM_PULL_DIR(8) RLBM_PULL_DIR(9) RLBM_PULL_DIR(10) RLBM_PULL_DIR(11)
#undef RLBM_PULL_DIR
  const Harm ha = harmonics(A, false), hb = harmonics(B, true);
  N[0] = ha.h0; N[1] = ha.c1; N[2] = ha.s1;
  T[0] = hb.h0; T[1] = hb.c1; T[2] = hb.s1;
  T[3] = 0.5 * (hb.h0 + hb.c2);
  T[4] = 0.5 * hb.s2;
  T[5] = 0.5 * (hb.h0 - hb.c2);
}

// FP64 equilibrium at (theta, g, u) written through a functor out(q, value).
template <int EDF, class Out>
__device__ __forceinline__ void feq_emit(const double g[6], double theta, double ux, double uy,
                                         double gamma, int oi, Out out) {
  double zr[21], zi[21];
  eq_moments<EDF>(g, theta, ux, uy, gamma, -1.0, -1.0, zr, zi, oi);
#pragma unroll 1
  for (int s = 0; s < 6; ++s) {
    double fe[12];
    feq_shell<EDF>(s, zr, zi, fe, oi);
#pragma unroll
    for (int d = 0; d < 12; ++d) out(6 * d + s, fe[d]);
  }
}

// Halo images of an edge cell (x, y): the halo cells that map to it under the
// boundary conditions. Returns the count; hx/hy/wall receive each target and
// the wall side (-1: copy of the cell, 0..3: fixed-T wall ghost of that side).
// Periodic: wrapped image; zero-gradient: copy; fixed-T wall: f^eq(n_b, u_b,
// theta_wall) from the cell's pre-collision state; an x wall wins at corners.
// images = false leaves out the periodic images (every pull wraps across a
// periodic side instead, see neighbours); only the TMA-staged step, whose
// boxes read the halo as stored, needs them.
__device__ __forceinline__ int halo_targets(const DomDev& D, int x, int y, int hx[8], int hy[8], int wall[8],
                                            bool images = true) {
  const int nx = D.nx, ny = D.ny;
  int xs[3], ys[3], nX = 1, nY = 1;
  xs[0] = x;
  ys[0] = y;
  if (D.bc[0] == BC_PERIODIC) {
    if (images && x == nx - 1) xs[nX++] = -1;
    if (images && x == 0) xs[nX++] = nx;
  } else {
    if (x == 0) xs[nX++] = -1;
    if (x == nx - 1) xs[nX++] = nx;
  }
  if (D.bc[2] == BC_PERIODIC) {
    if (images && y == ny - 1) ys[nY++] = -1;
    if (images && y == 0) ys[nY++] = ny;
  } else {
    // an exchanged side's ghost row is the neighbour's face: nothing to write
    if (y == 0 && D.bc[2] != BC_EXCHANGED) ys[nY++] = -1;
    if (y == ny - 1 && D.bc[3] != BC_EXCHANGED) ys[nY++] = ny;
  }
  int cnt = 0;
  for (int i = 0; i < nX; ++i)
    for (int j = 0; j < nY; ++j) {
      if (i == 0 && j == 0) continue;
      const int tx = xs[i], ty = ys[j];
      int w = -1;
      if (tx == -1 && bc_is_wall(D.bc[0])) w = 0;
      else if (tx == nx && bc_is_wall(D.bc[1])) w = 1;
      else if (ty == -1 && bc_is_wall(D.bc[2])) w = 2;
      else if (ty == ny && bc_is_wall(D.bc[3])) w = 3;
      hx[cnt] = tx;
      hy[cnt] = ty;
      wall[cnt] = w;
      ++cnt;
    }
  return cnt;
}

// Halo writer for kernels that hold the cell's populations in FP64 (smem column).
// Velocity-wall ghosts are skipped when the step has written them already
// (vw_written); otherwise (initial state, or a cell left unrelaxed) they get the
// wall equilibrium f^eq(n_wall, 0, theta_wall).
template <int EDF, class S>
__device__ void write_halo64(const DomDev& D, int x, int y, typename S::T* __restrict__ fout, const double* sm,
                             int tid, bool have_state, double n, double ux, double uy, double gamma,
                             unsigned& st, bool vw_written = false) {
  int hx[8], hy[8], wall[8];
  const int cnt = halo_targets(D, x, y, hx, hy, wall);
  for (int i = 0; i < cnt; ++i) {
    const long long h = cell_rel(D, hx[i], hy[i]);
    if (wall[i] >= 0 && D.bc[wall[i]] == BC_VWALL) {
      if (vw_written) continue;
      const double tw = D.t_wall[wall[i]];
      double z, g[6];
      st |= solve_z_from_n_theta<EDF>(D.n_wall, tw, z, g);
      feq_emit<EDF>(g, tw, 0.0, 0.0, 1.0, D.order - 2,
                    [&](int q, double v) { fout[q * kBlkW + h] = S::enc(v, D, q % 6); });
      continue;
    }
    if (wall[i] < 0 || !have_state) {
      for (int q = 0; q < 72; ++q) fout[q * kBlkW + h] = S::enc(sm[q * kThreads + tid], D, q % 6);
    } else {
      const double tw = D.t_wall[wall[i]];
      double z, g[6];
      st |= solve_z_from_n_theta<EDF>(n, tw, z, g);
      feq_emit<EDF>(g, tw, ux, uy, gamma, D.order - 2,
                    [&](int q, double v) { fout[q * kBlkW + h] = S::enc(v, D, q % 6); });
    }
  }
}

// True when the cell borders a velocity wall (its ghosts need the
// non-equilibrium extrapolation of the step).
__device__ __forceinline__ bool touches_vwall(const DomDev& D, int x, int y) {
  return (x == 0 && D.bc[0] == BC_VWALL) || (x == D.nx - 1 && D.bc[1] == BC_VWALL) ||
         (y == 0 && D.bc[2] == BC_VWALL) || (y == D.ny - 1 && D.bc[3] == BC_VWALL);
}

// Velocity-wall ghosts of a cell (Sec. 3.4): f^eq(n_wall, 0, theta_wall) +
// (f* - f^eq), f* the cell's post-collision populations (smem column) and f^eq
// the equilibrium it relaxes towards -- its state (n, eps, theta, z) at the
// force-shifted velocity u + a tau. At the initial state f* is the initial
// equilibrium. Kept out of line: only edge cells pay for it.
template <int EDF, class S>
__device__ __noinline__ void write_vwall_ghosts(const DomDev& D, int x, int y, typename S::T* __restrict__ fout,
                                                const double* sm, int tid, const CellState* cs, unsigned* st) {
  int hx[8], hy[8], wall[8];
  const int cnt = halo_targets(D, x, y, hx, hy, wall);
  int tw_side = -1;
  for (int i = 0; i < cnt; ++i)
    if (wall[i] >= 0 && D.bc[wall[i]] == BC_VWALL) tw_side = wall[i];
  if (tw_side < 0) return;
  const double tw = D.t_wall[tw_side];  // shared by every velocity wall of the domain
  const int oi = D.order - 2;
  const double tau = D.eta_s > 0.0 ? 4.0 * D.eta_s / cs->theta + 0.2546 : D.tau;
  double ux = cs->ux, uy = cs->uy, gam = cs->gamma;
  if (D.accel_x != 0.0 || D.accel_y != 0.0) {
    ux += D.accel_x * tau;
    uy += D.accel_y * tau;
    gam = 1.0 / sqrt(1.0 - ux * ux - uy * uy);
  }
  double z, g[6], zrw[21], ziw[21], zrc[21], zic[21];
  *st |= solve_z_from_n_theta<EDF>(D.n_wall, tw, z, g);
  eq_moments<EDF>(g, tw, 0.0, 0.0, 1.0, -1.0, -1.0, zrw, ziw, oi);
  eq_moments<EDF>(cs->g, cs->theta, ux, uy, gam, cs->n, cs->eps, zrc, zic, oi);
  for (int s = 0; s < 6; ++s) {
    double few[12], fe[12];
    feq_shell<EDF>(s, zrw, ziw, few, oi);
    feq_shell<EDF>(s, zrc, zic, fe, oi);
    for (int i = 0; i < cnt; ++i) {
      if (wall[i] < 0 || D.bc[wall[i]] != BC_VWALL) continue;
      const long long h = cell_rel(D, hx[i], hy[i]);
      for (int d = 0; d < 12; ++d) {
        const int q = 6 * d + s;
        fout[q * kBlkW + h] = S::enc(few[d] + (sm[q * kThreads + tid] - fe[d]), D, s);
      }
    }
  }
}

// The cell (x, y) of domain `dom` a thread of an initialiser or read-out
// launch covers: a block per tile of the work list, or a 2D grid over one domain.
__device__ __forceinline__ void cell_of_launch(const Tile* tiles, int dom0, int& dom, int& x, int& y) {
  if (tiles) {
    const Tile tl = tiles[blockIdx.x];
    dom = tl.dom;
    x = tl.x0 + threadIdx.x;
    y = tl.y0 + threadIdx.y;
  } else {
    dom = dom0;
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
  }
}

// f = f^eq of the given fields (time zero, FP64 arithmetic), halo included.
template <int EDF, class S>
__global__ void __launch_bounds__(kThreads) k_init(InitArgs a) {
  extern __shared__ double sm[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  int dom, x, y;
  cell_of_launch(a.tiles, a.dom, dom, x, y);
  const DomDev& D = a.doms[dom];
  if (x >= D.nx || y >= D.ny) return;
  const long long i = (a.tiles ? D.foff : 0) + (long long)y * D.nx + x;
  const double theta = a.theta[i], ux = a.ux[i], uy = a.uy[i];
  unsigned st = 0;
  double z, n, g[6];
  if (a.kind == 1) {
    z = a.a[i];
    g_all<EDF>(z, g);
    n = 2.0 * PI * theta * theta * g[1];
  } else {
    n = a.a[i];
    st |= solve_z_from_n_theta<EDF>(n, theta, z, g);
  }
  const double u2 = ux * ux + uy * uy;
  const bool ok = (u2 < 1.0) && (theta > 0.0) && (n > 0.0) && isfinite(z);
  if (!ok) st |= ST_NONPHYSICAL;
  const double gamma = ok ? 1.0 / sqrt(1.0 - u2) : 1.0;
  typename S::T* __restrict__ f = static_cast<typename S::T*>(a.f) + D.off;
  const long long c = cell_rel(D, x, y);
  if (ok) {
    feq_emit<EDF>(g, theta, ux, uy, gamma, D.order - 2, [&](int q, double v) {
      sm[q * kThreads + tid] = v;
      f[q * kBlkW + c] = S::enc(v, D, q % 6);
    });
  } else {
    for (int q = 0; q < 72; ++q) {
      sm[q * kThreads + tid] = nan("");
      f[q * kBlkW + c] = S::enc(nan(""), D, q % 6);
    }
  }
  bool vw = false;
  if (ok && touches_vwall(D, x, y)) {
    CellState cs;
    cs.n = n; cs.theta = theta; cs.ux = ux; cs.uy = uy; cs.z = z; cs.gamma = gamma;
    for (int k = 0; k < 6; ++k) cs.g[k] = g[k];
    cs.eps = 4.0 * PI * theta * theta * theta * g[2];  // Eq. (25)
    write_vwall_ghosts<EDF, S>(D, x, y, f, sm, tid, &cs, &st);
    vw = true;
  }
  write_halo64<EDF, S>(D, x, y, f, sm, tid, ok, n, ux, uy, gamma, st, vw);
  if (st) atomicOr(a.status, st);
}

// Macroscopic fields (FP64) of the streamed (or stored) populations.
template <int EDF, class S>
__global__ void __launch_bounds__(kThreads) k_fields(FieldsArgs a) {
  extern __shared__ double sm[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  int dom, x, y;
  cell_of_launch(a.tiles, a.dom, dom, x, y);
  const DomDev& D = a.doms[dom];
  if (x >= D.nx || y >= D.ny) return;
  const typename S::T* __restrict__ f = static_cast<const typename S::T*>(a.f) + D.off;
  const long long c = cell_rel(D, x, y);
  double N[3], T[6];
  if (a.streamed) {
    pull_moments64<EDF, S>(f, D, x, y, c, sm, tid, N, T);
  } else {
    double A[12], B[12];
    for (int d = 0; d < 12; ++d) {
      double a_ = 0.0, b_ = 0.0;
      for (int s = 0; s < 6; ++s) {
        const double v = S::dec((double)S::raw(f[(6 * d + s) * kBlkW + c]), D, s);
        a_ = fma(v, c_p[EDF][s], a_);
        b_ = fma(v, c_p2[EDF][s], b_);
      }
      A[d] = a_;
      B[d] = b_;
    }
    const Harm ha = harmonics(A, false), hb = harmonics(B, true);
    N[0] = ha.h0; N[1] = ha.c1; N[2] = ha.s1;
    T[0] = hb.h0; T[1] = hb.c1; T[2] = hb.s1;
    T[3] = 0.5 * (hb.h0 + hb.c2);
    T[4] = 0.5 * hb.s2;
    T[5] = 0.5 * (hb.h0 - hb.c2);
  }
  CellState S_;
  unsigned st = cell_state<EDF>(N, T, S_);
  const long long i = (a.tiles ? D.foff : 0) + (long long)y * D.nx + x;
  if (st & ST_NONPHYSICAL) S_.n = S_.theta = S_.ux = S_.uy = S_.z = nan("");
  if (a.n) a.n[i] = S_.n;
  if (a.theta) a.theta[i] = S_.theta;
  if (a.ux) a.ux[i] = S_.ux;
  if (a.uy) a.uy[i] = S_.uy;
  if (a.z) a.z[i] = S_.z;
  if (a.diag) {
    // heat flux q^a = (3 theta g_3 / g_2)(n U^a - N^a), Sec. 3.3, and the
    // diagonal non-equilibrium tensors pi^{x..x} = sum_i (f_i - f^eq_i) (p_i^x)^k,
    // k = 2..5 (Sec. 3.1), with f^eq the fifth-order equilibrium of the cell's
    // Landau state -- the one its next collision relaxes towards
    const long long np = (long long)D.nx * D.ny;
    double out[7];
    if (st & ST_NONPHYSICAL) {
      for (int k = 0; k < 7; ++k) out[k] = nan("");
    } else {
      const double hq = 3.0 * S_.theta * S_.g[2] / S_.g[1];
      out[0] = hq * (S_.n * S_.gamma - N[0]);
      out[1] = hq * (S_.n * S_.gamma * S_.ux - N[1]);
      out[2] = hq * (S_.n * S_.gamma * S_.uy - N[2]);
      const double eps_eq = (st & ST_CLAMPED) ? 4.0 * PI * S_.theta * S_.theta * S_.theta * S_.g[2] : S_.eps;
      double zr[21], zi[21];
      eq_moments<EDF>(S_.g, S_.theta, S_.ux, S_.uy, S_.gamma, S_.n, eps_eq, zr, zi, D.order - 2);
      double p2 = 0.0, p3 = 0.0, p4 = 0.0, p5 = 0.0;
      for (int s = 0; s < 6; ++s) {
        double fe[12];
        feq_shell<EDF>(s, zr, zi, fe, D.order - 2);
#pragma unroll
        for (int d = 0; d < 12; ++d) {
          const int q = 6 * d + s;
          const double v = a.streamed ? sm[q * kThreads + tid] : S::dec((double)S::raw(f[q * kBlkW + c]), D, s);
          const double px = c_p[EDF][s] * dcos(d), w = (v - fe[d]) * px * px;
          p2 += w;
          p3 += w * px;
          p4 += w * px * px;
          p5 += w * px * px * px;
        }
      }
      out[3] = p2;
      out[4] = p3;
      out[5] = p4;
      out[6] = p5;
    }
    for (int k = 0; k < 7; ++k) a.diag[k * np + i] = out[k];
  }
  if (st) atomicOr(a.status, st);
}

// Raw populations (halo included) <-> FP64 [72][ny+2][nx+2].
template <class S>
__global__ void k_copy(CopyArgs a) {
  const DomDev& D = a.doms[a.dom];
  const long long w = D.nx + 2, h = D.ny + 2, tot = (long long)a.nq * w * h;
  typename S::T* pop = static_cast<typename S::T*>(a.pop);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long q = a.q0 + e / (w * h), r = e % (w * h), yy = r / w, xx = r % w;
    const long long src = cell_pos(D, (int)xx - 1, (int)yy - 1) + q * kBlkW;
    if (a.to_dense) a.dense[e] = S::dec((double)S::raw(pop[src]), D, (int)(q % 6));
    else pop[src] = S::enc(a.dense[e], D, (int)(q % 6));
  }
}

constexpr size_t kSmem64 = 72 * kThreads * sizeof(double);

template <class S, int EDF>
cudaError_t prepare_common_t() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_init<EDF, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64)))
    return e;
  return cudaFuncSetAttribute(k_fields<EDF, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64);
}

// Grid of an initialiser or read-out launch: a block per tile, or a 2D grid
// over one nx x ny domain.
inline dim3 launch_grid(const Tile* tiles, int ntiles, int nx, int ny) {
  return tiles ? dim3(ntiles) : dim3((nx + kTileW - 1) / kTileW, (ny + kTileH - 1) / kTileH);
}

template <class S>
cudaError_t launch_init_t(int edf, const InitArgs& a, int nx, int ny, cudaStream_t s) {
  const dim3 grid = launch_grid(a.tiles, a.ntiles, nx, ny);
  switch (edf) {
    case EDF_MJ: k_init<EDF_MJ, S><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
    case EDF_FD: k_init<EDF_FD, S><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
    default: k_init<EDF_BE, S><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
  }
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_fields_t(int edf, const FieldsArgs& a, int nx, int ny, cudaStream_t s) {
  const dim3 grid = launch_grid(a.tiles, a.ntiles, nx, ny);
  switch (edf) {
    case EDF_MJ: k_fields<EDF_MJ, S><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
    case EDF_FD: k_fields<EDF_FD, S><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
    default: k_fields<EDF_BE, S><<<grid, dim3(kTileW, kTileH), kSmem64, s>>>(a); break;
  }
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_copy_t(const CopyArgs& a, cudaStream_t s) {
  k_copy<S><<<1024, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rlbm
