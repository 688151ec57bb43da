// Device arithmetic of the fused stream-collide update (FP64 form).
//
// Per cell: moments N^mu, T^{mu nu} (Eqs. 20, 22) -> Landau frame (Eq. 21) ->
// n, theta, z (Eqs. 23-25) -> the 36 equilibrium moments in harmonic form
// (Appendix) -> the fifth-order discrete equilibrium as a block-diagonal
// projection (Eqs. 10-11) -> Anderson-Witting relaxation (Eq. 3).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rlbm_common.h"
#include "rlbm_tables.h"

namespace rlbm {

// ---------------------------------------------------------------- tables
// Each translation unit that includes this header gets its own copy.
static __constant__ double c_p[3][6] = {RLBM_P_MJ_INIT, RLBM_P_FD_INIT, RLBM_P_BE_INIT};
static __constant__ double c_w[3][6] = {RLBM_W_MJ_INIT, RLBM_W_FD_INIT, RLBM_W_BE_INIT};
static __constant__ double c_p2[3][6] = {RLBM_P2_MJ_INIT, RLBM_P2_FD_INIT, RLBM_P2_BE_INIT};
// projection tables per expansion order N = 2..5 (index N - 2; entries of degree
// above N are zero) and EDF
static __constant__ double c_Q[4][3][126] = {
    {RLBM_QO2_MJ_INIT, RLBM_QO2_FD_INIT, RLBM_QO2_BE_INIT},
    {RLBM_QO3_MJ_INIT, RLBM_QO3_FD_INIT, RLBM_QO3_BE_INIT},
    {RLBM_QO4_MJ_INIT, RLBM_QO4_FD_INIT, RLBM_QO4_BE_INIT},
    {RLBM_Q_MJ_INIT, RLBM_Q_FD_INIT, RLBM_Q_BE_INIT}};
// exact defects of the rounded Q tables in the conserved moments: e1 (N^0, block
// k = 0), e2 (T^00, block 0), e3 (T^0x + i T^0y, block 1), 6 entries each
static __constant__ double c_E[4][3][18] = {
    {RLBM_EO2_MJ_INIT, RLBM_EO2_FD_INIT, RLBM_EO2_BE_INIT},
    {RLBM_EO3_MJ_INIT, RLBM_EO3_FD_INIT, RLBM_EO3_BE_INIT},
    {RLBM_EO4_MJ_INIT, RLBM_EO4_FD_INIT, RLBM_EO4_BE_INIT},
    {RLBM_E_MJ_INIT, RLBM_E_FD_INIT, RLBM_E_BE_INIT}};
constexpr int kOrder5 = 3;  // table index of the fifth order
static __constant__ double c_pnk[63] = RLBM_PNK_INIT;
static __constant__ double c_invpow[6 * RLBM_NSERIES] = RLBM_INVPOW_INIT;
static __constant__ double c_be_exp[6 * RLBM_NEXP] = RLBM_BE_EXP_INIT;
static __constant__ double c_fd_exp[6 * RLBM_NEXP] = RLBM_FD_EXP_INIT;
static __constant__ double c_be_logcoef[6] = RLBM_BE_LOGCOEF_INIT;
static __constant__ double c_be_harm[6] = RLBM_BE_HARM_INIT;
static __constant__ double c_g_zc[6] = RLBM_G_ZC_INIT;

// Offset of harmonic block k in the Q tables: sum_{k'<k} 6 (6 - k').
__host__ __device__ constexpr int qoff(int k) { return 6 * (6 * k - (k * (k - 1)) / 2); }

// ------------------------------------------------------- EDF integrals g_nu
// g[nu-1] = g_nu(z), nu = 1..6 (Eq. 12). MJ: z. BE: Li_nu(z). FD: -Li_nu(-z).
// Power series in z for small z, the expansions in mu = ln z around z = 1
// (zeta values for BE, eta values for FD), and for FD z > 4 the inversion
// formula -Li_nu(-z) = (-1)^nu Li_nu(-1/z) + (ln z)^nu/nu! + 2 sum_j eta(2j) (ln z)^{nu-2j}/(nu-2j)!.
__device__ __forceinline__ void li_series6(double x, double g[6]) {
  // sum_{k>=1} x^k k^{-nu}, |x| <= 1/4
  double xk = 1.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) g[i] = 0.0;
  for (int k = 1; k <= RLBM_NSERIES; ++k) {
    xk *= x;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = fma(xk, c_invpow[i * RLBM_NSERIES + k - 1], g[i]);
    if (fabs(xk) < 1e-18) break;
  }
}

template <int EDF>
__device__ void g_all(double z, double g[6]) {
  if (EDF == EDF_MJ) {
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = z;
    return;
  }
  if (EDF == EDF_BE) {
    if (z <= 0.25) { li_series6(z, g); return; }
    const double mu = log(z);
    double mk = 1.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = 0.0;
    for (int k = 0; k < RLBM_NEXP; ++k) {
#pragma unroll
      for (int i = 0; i < 6; ++i) g[i] = fma(mk, c_be_exp[i * RLBM_NEXP + k], g[i]);
      mk *= mu;
      if (fabs(mk) < 1e-30) break;
    }
    // the k = nu-1 term: mu^{nu-1}/(nu-1)! (H_{nu-1} - ln(-mu))
    const double lnm = log(-mu);
    double mp = 1.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      g[i] = fma(mp * c_be_logcoef[i], c_be_harm[i] / c_be_logcoef[i] - lnm, g[i]);
      mp *= mu;
    }
    return;
  }
  // FD
  if (z <= 0.25) {
    li_series6(-z, g);
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = -g[i];
    return;
  }
  if (z <= 4.0) {
    const double mu = log(z);
    double mk = 1.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = 0.0;
    for (int k = 0; k < RLBM_NEXP; ++k) {
#pragma unroll
      for (int i = 0; i < 6; ++i) g[i] = fma(mk, c_fd_exp[i * RLBM_NEXP + k], g[i]);
      mk *= mu;
      if (fabs(mk) < 1e-30) break;
    }
    return;
  }
  li_series6(-1.0 / z, g);
  const double L = log(z);
  // eta(2) = pi^2/12, eta(4) = 7 pi^4/720, eta(6) = 31 pi^6/30240
  const double eta2 = 0.82246703342411321824, eta4 = 0.94703282949724591758,
               eta6 = 0.98555109129743510410;
  const double L2 = L * L, L3 = L2 * L, L4 = L3 * L, L5 = L4 * L, L6 = L5 * L;
  g[0] = -g[0] + L;
  g[1] = g[1] + L2 / 2.0 + 2.0 * eta2;
  g[2] = -g[2] + L3 / 6.0 + 2.0 * eta2 * L;
  g[3] = g[3] + L4 / 24.0 + 2.0 * eta2 * L2 / 2.0 + 2.0 * eta4;
  g[4] = -g[4] + L5 / 120.0 + 2.0 * eta2 * L3 / 6.0 + 2.0 * eta4 * L;
  g[5] = g[5] + L6 / 720.0 + 2.0 * eta2 * L4 / 24.0 + 2.0 * eta4 * L2 / 2.0 + 2.0 * eta6;
}

// g_1, g_2, g_3 alone (g[0..2] of g_all): what the Newton iterations below need.
// In the series range g_1 has the closed form ln(1 + z) (FD) or -ln(1 - z) (BE),
// and g_2, g_3 take two series instead of six.
template <int EDF>
__device__ __forceinline__ void g123(double z, double g[3]) {
  if (EDF != EDF_MJ && z <= 0.25) {
    const double x = EDF == EDF_BE ? z : -z;
    double xk = 1.0, s2 = 0.0, s3 = 0.0;
    for (int k = 1; k <= RLBM_NSERIES; ++k) {
      xk *= x;
      s2 = fma(xk, c_invpow[RLBM_NSERIES + k - 1], s2);
      s3 = fma(xk, c_invpow[2 * RLBM_NSERIES + k - 1], s3);
      if (fabs(xk) < 1e-18) break;
    }
    g[0] = EDF == EDF_BE ? -log1p(-z) : log1p(z);
    g[1] = EDF == EDF_BE ? s2 : -s2;
    g[2] = EDF == EDF_BE ? s3 : -s3;
    return;
  }
  double g6[6];
  g_all<EDF>(z, g6);
  g[0] = g6[0];
  g[1] = g6[1];
  g[2] = g6[2];
}

// A Newton step d in mu leaves an error of about C d^2, C = |F''/(2F')| of the
// equation solved: at most 0.23 for FD and about 0.12/(1 - z) for BE (computed
// with arbitrary-precision polylogs for both solves below). A Newton step with
// d^2 C_bound < 1e-17 (C_bound = 0.25, or 0.25/(1 - z) for BE) is therefore
// accepted without evaluating the equation again.
template <int EDF>
__device__ __forceinline__ bool newton_done64(double d, double z) {
  const double cb = EDF == EDF_BE ? 0.25 / (1.0 - z) : 0.25;
  return d * d * cb < 1e-17;
}

// Fugacity from (eps, n), FD/BE: g_3^2/g_2^3 = (pi/2) eps^2/n^3 (Eq. 25), solved
// for mu = ln z by safeguarded Newton; BE states below R(z_c) are clamped.
// Start: with w = 1/target = g_2^3/g_3^2 = z + O(z^2), inverting the series gives
// mu = ln w - s w/2 + (119/1728) w^2 - s (85/6912) w^3 + O(w^4) (s = -1 FD, +1 BE),
// 1.4e-6 off in mu at z = 0.17: two Newton steps reach the FP64 floor, a third
// confirms it.
template <int EDF>
__device__ int solve_z_from_R(double target, double& z, double g[6]) {
  if (EDF == EDF_BE && target < RLBM_R_ZC) {
    z = ZC;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = c_g_zc[i];
    return ST_CLAMPED;
  }
  double lo = -60.0, hi = (EDF == EDF_BE) ? log(ZC) : 60.0;
  const double lt = log(target);
  double mu = -lt;
  const double w = 1.0 / target;
  if (w < 0.5) {
    constexpr double kS = EDF == EDF_BE ? 1.0 : -1.0;
    mu = fma(fma(fma(-kS * (85.0 / 6912.0), w, 119.0 / 1728.0), w, -0.5 * kS), w, mu);
  }
  mu = fmin(fmax(mu, lo + 1e-3), hi);
  int st = ST_ZSOLVE;
  double dprev = INFINITY;
  for (int it = 0; it < 80; ++it) {
    double gi[3];
    const double ze = exp(mu);
    g123<EDF>(ze, gi);
    const double F = log(gi[2] * gi[2] / (gi[1] * gi[1] * gi[1])) - lt;
    if (F == 0.0) { st = 0; break; }  // exact root at mu
    const double dF = 2.0 * gi[1] / gi[2] - 3.0 * gi[0] / gi[1];
    if (F > 0.0) lo = mu; else hi = mu;
    double mn = mu - F / dF;
    const bool newton = mn >= lo && mn <= hi;
    if (!newton) mn = 0.5 * (lo + hi);
    const double d = fabs(mn - mu);
    mu = mn;
    // converged: step at the tolerance, a Newton step whose error bound is below
    // it, or no longer shrinking at the noise floor
    if (d <= 1e-15 * fmax(1.0, fabs(mu)) || (newton && newton_done64<EDF>(d, ze)) ||
        (d < 1e-12 && d >= dprev)) {
      st = 0;
      break;
    }
    dprev = d;
  }
  z = exp(mu);
  g_all<EDF>(z, g);
  return st;
}

// Fugacity from (n, theta): n = 2 pi theta^2 g_2(z) (Eq. 25). Start: inverting
// G = g_2(z) gives mu = ln G +- G/4 - (5/288) G^2 +- G^3/288 + O(G^4) (upper
// signs FD, lower BE).
template <int EDF>
__device__ int solve_z_from_n_theta(double n, double theta, double& z, double g[6]) {
  const double G = n / (2.0 * PI * theta * theta);
  if (EDF == EDF_MJ) {
    z = G;
    g_all<EDF>(z, g);
    return 0;
  }
  if (EDF == EDF_BE && G >= c_g_zc[1]) {
    z = ZC;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = c_g_zc[i];
    return ST_CLAMPED;
  }
  double lo = -60.0, hi = (EDF == EDF_BE) ? log(ZC) : 60.0;
  const double lG = log(G);
  double mu = lG;
  if (G < 0.5) {
    constexpr double kS = EDF == EDF_BE ? -1.0 : 1.0;
    mu = fma(fma(fma(kS / 288.0, G, -5.0 / 288.0), G, 0.25 * kS), G, mu);
  }
  mu = fmin(fmax(mu, lo + 1e-3), hi);
  int st = ST_ZSOLVE;
  double dprev = INFINITY;
  for (int it = 0; it < 80; ++it) {
    double gi[3];
    const double ze = exp(mu);
    g123<EDF>(ze, gi);
    const double F = log(gi[1]) - lG;      // increasing in mu
    if (F == 0.0) { st = 0; break; }       // exact root at mu
    const double dF = gi[0] / gi[1];
    if (F < 0.0) lo = mu; else hi = mu;
    double mn = mu - F / dF;
    const bool newton = mn >= lo && mn <= hi;
    if (!newton) mn = 0.5 * (lo + hi);
    const double d = fabs(mn - mu);
    mu = mn;
    // converged: step at the tolerance, a Newton step whose error bound is below
    // it, or no longer shrinking at the noise floor
    if (d <= 1e-15 * fmax(1.0, fabs(mu)) || (newton && newton_done64<EDF>(d, ze)) ||
        (d < 1e-12 && d >= dprev)) {
      st = 0;
      break;
    }
    dprev = d;
  }
  z = exp(mu);
  g_all<EDF>(z, g);
  return st;
}

// ------------------------------------------------------------ Landau frame
// T^a_b U^b = eps U^a (Eq. 21) written for U = gamma (1, u):
//   eps = T00 - m.u,   m_i - Pi_ij u_j = eps u_i,   m = (T01, T02), Pi = T^{ij},
// solved by Newton's method in u from the ideal conformal-fluid estimate
// (eps + P = x with 2 x^2 - 3 T00 x + |m|^2 = 0, u = m / x). The fixed point is
// the eigenvector the paper's power method converges to.
struct Frame {
  double eps, ux, uy, gamma;
};

__device__ __forceinline__ int landau(const double T[6], Frame& F) {
  const double E = T[0], mx = T[1], my = T[2], pxx = T[3], pxy = T[4], pyy = T[5];
  const double disc = 9.0 * E * E - 8.0 * (mx * mx + my * my);
  if (!(E > 0.0) || !(disc >= 0.0)) return ST_NONPHYSICAL;
  const double x = 0.25 * (3.0 * E + sqrt(disc));
  double ux = mx / x, uy = my / x;
  int st = ST_LANDAU;
  for (int it = 0; it < 30; ++it) {
    const double a = E - (mx * ux + my * uy);
    const double fx = mx - (pxx * ux + pxy * uy) - a * ux;
    const double fy = my - (pxy * ux + pyy * uy) - a * uy;
    const double j00 = ux * mx - pxx - a, j01 = ux * my - pxy;
    const double j10 = uy * mx - pxy, j11 = uy * my - pyy - a;
    const double rdet = 1.0 / (j00 * j11 - j01 * j10);
    const double dx = (j01 * fy - j11 * fx) * rdet;
    const double dy = (j10 * fx - j00 * fy) * rdet;
    ux += dx;
    uy += dy;
    if (fmax(fabs(dx), fabs(dy)) < 1e-13) { st = 0; break; }
  }
  const double u2 = ux * ux + uy * uy;
  if (!(u2 < 1.0)) return ST_NONPHYSICAL;
  F.ux = ux;
  F.uy = uy;
  F.eps = E - (mx * ux + my * uy);
  F.gamma = 1.0 / sqrt(1.0 - u2);
  if (!(F.eps > 0.0)) return ST_NONPHYSICAL;
  return st;
}

// Macroscopic state of a cell: n = U_mu N^mu, theta, z (Eqs. 23-25).
struct CellState {
  double n, theta, ux, uy, z, eps, gamma;
  double g[6];
};

template <int EDF>
__device__ int cell_state(const double N[3], const double T[6], CellState& S) {
  Frame F;
  int st = landau(T, F);
  if (st & ST_NONPHYSICAL) return st;
  S.ux = F.ux;
  S.uy = F.uy;
  S.gamma = F.gamma;
  S.eps = F.eps;
  S.n = F.gamma * (N[0] - F.ux * N[1] - F.uy * N[2]);
  if (!(S.n > 0.0) || !isfinite(S.n) || !isfinite(S.eps)) return st | ST_NONPHYSICAL;
  if (EDF == EDF_MJ) {
    S.theta = S.eps / (2.0 * S.n);
    S.z = S.n / (2.0 * PI * S.theta * S.theta);
#pragma unroll
    for (int i = 0; i < 6; ++i) S.g[i] = S.z;
    return st;
  }
  const double target = 0.5 * PI * S.eps * S.eps / (S.n * S.n * S.n);
  const int zs = solve_z_from_R<EDF>(target, S.z, S.g);
  st |= zs;
  if (zs & ST_CLAMPED) S.theta = sqrt(S.n / (2.0 * PI * S.g[1]));
  else S.theta = 0.5 * S.g[1] / S.g[2] * S.eps / S.n;
  return st;
}

// --------------------------------------------- equilibrium moments (harmonic)
// Z_nk = int dp dphi f^eq p^n e^{i k phi}
//      = 2 pi n! g_{n+1}(z) theta^{n+1} gamma^n (u_x + i u_y)^k P_nk(u^2),  k <= n <= 5.
// zr/zi are indexed n(n+1)/2 + k. When nA1 / eA2 are non-negative they replace
// the degree-1 and degree-2 prefactors 2 pi g_2 theta^2 = n and
// 2 pi 2! g_3 theta^3 = eps (Eq. 25), so that the equilibrium carries the cell's
// own n and eps exactly and the collision conserves N^0 and T^{mu 0} without a
// rounding bias from the z, theta round trip.
// oi selects the expansion order's defect table (order - 2).
template <int EDF>
__device__ __forceinline__ void eq_moments(const double g[6], double theta, double ux, double uy,
                                           double gamma, double nA1, double eA2, double zr[21],
                                           double zi[21], int oi = kOrder5) {
  const double u2 = ux * ux + uy * uy;
  double wr[6], wi[6];
  wr[0] = 1.0;
  wi[0] = 0.0;
#pragma unroll
  for (int k = 1; k < 6; ++k) {
    wr[k] = wr[k - 1] * ux - wi[k - 1] * uy;
    wi[k] = wr[k - 1] * uy + wi[k - 1] * ux;
  }
  double A = 2.0 * PI * theta;  // 2 pi n! theta^{n+1} gamma^n, times g_{n+1}
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    if (n > 0) A *= n * theta * gamma;
    double An = A * g[n];
    if (n == 1 && nA1 >= 0.0) An = nA1 * gamma;
    if (n == 2 && eA2 >= 0.0) An = eA2 * gamma * gamma;
#pragma unroll
    for (int k = 0; k <= n; ++k) {
      const int i = n * (n + 1) / 2 + k;
      const double P = fma(u2, fma(u2, c_pnk[3 * i + 2], c_pnk[3 * i + 1]), c_pnk[3 * i + 0]);
      const double s = An * P;
      zr[i] = s * wr[k];
      zi[i] = s * wi[k];
    }
  }
  // The rounded projection table misses the identities that make the discrete
  // N^0, T^00 and T^0x, T^0y of f^eq equal Z_10, Z_20, Z_21 by the tiny constant
  // defects e1, e2, e3; correcting those three moments removes the resulting
  // bias (a constant error times Z would drift the conserved totals every step).
  double d10 = 0.0, d20 = 0.0, d21r = 0.0, d21i = 0.0;
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    d10 = fma(c_E[oi][EDF][n], zr[n * (n + 1) / 2], d10);
    d20 = fma(c_E[oi][EDF][6 + n], zr[n * (n + 1) / 2], d20);
  }
#pragma unroll
  for (int n = 1; n < 6; ++n) {
    d21r = fma(c_E[oi][EDF][12 + n], zr[n * (n + 1) / 2 + 1], d21r);
    d21i = fma(c_E[oi][EDF][12 + n], zi[n * (n + 1) / 2 + 1], d21i);
  }
  zr[1] -= d10;
  zr[3] -= d20;
  zr[4] -= d21r;
  zi[4] -= d21i;
}

// Discrete equilibrium of one shell s at the 12 directions (order index oi =
// N - 2; the fifth order by default):
//   f^eq_{ds} = sum_k R^c_k cos(k phi_d) + R^s_k sin(k phi_d),
//   R^{c|s}_k = sum_{n>=k} Q^(k)_{s n} Re|Im Z_nk,
// evaluated with the 12-point symmetries phi -> phi + pi (odd k flip sign) and
// phi -> pi - phi.
template <int EDF>
__device__ __forceinline__ void feq_shell(int s, const double zr[21], const double zi[21],
                                          double fe[12], int oi = kOrder5) {
  double Rc[6], Rs[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double ac = 0.0, as = 0.0;
#pragma unroll
    for (int n = k; n < 6; ++n) {
      const double q = c_Q[oi][EDF][qoff(k) + s * (6 - k) + (n - k)];
      ac = fma(q, zr[n * (n + 1) / 2 + k], ac);
      as = fma(q, zi[n * (n + 1) / 2 + k], as);
    }
    Rc[k] = ac;
    Rs[k] = as;
  }
  const double h = SQRT3_2;
  // even harmonics (period pi)
  const double t1 = Rc[0] + Rc[4], t2 = fma(-0.5, Rc[4], Rc[0]), h2 = 0.5 * Rc[2];
  const double Ec0 = t1 + Rc[2], Ec3 = t1 - Rc[2], Ec1 = t2 + h2, Ec2 = t2 - h2;
  const double Es1 = h * (Rs[2] + Rs[4]), Es2 = h * (Rs[2] - Rs[4]);
  const double E0 = Ec0, E1 = Ec1 + Es1, E2 = Ec2 + Es2, E3 = Ec3, E4 = Ec2 - Es2, E5 = Ec1 - Es1;
  // odd harmonics (antiperiodic in pi)
  const double Oc0 = Rc[1] + Rc[3] + Rc[5], Oc1 = h * (Rc[1] - Rc[5]),
               Oc2 = fma(0.5, Rc[1] + Rc[5], -Rc[3]);
  const double Os1 = fma(0.5, Rs[1] + Rs[5], Rs[3]), Os2 = h * (Rs[1] - Rs[5]),
               Os3 = Rs[1] - Rs[3] + Rs[5];
  const double O0 = Oc0, O1 = Oc1 + Os1, O2 = Oc2 + Os2, O3 = Os3, O4 = Os2 - Oc2, O5 = Os1 - Oc1;
  fe[0] = E0 + O0; fe[6] = E0 - O0;
  fe[1] = E1 + O1; fe[7] = E1 - O1;
  fe[2] = E2 + O2; fe[8] = E2 - O2;
  fe[3] = E3 + O3; fe[9] = E3 - O3;
  fe[4] = E4 + O4; fe[10] = E4 - O4;
  fe[5] = E5 + O5; fe[11] = E5 - O5;
}

// ------------------------------------------------------------------ moments
// Harmonic sums of a 12-vector v over the directions: sum v, sum cos v,
// sum sin v, sum cos2 v, sum sin2 v (pairs d, d+6 folded first).
struct Harm {
  double h0, c1, s1, c2, s2;
};

__device__ __forceinline__ Harm harmonics(const double v[12], bool need2) {
  double e[6], o[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    e[d] = v[d] + v[d + 6];
    o[d] = v[d] - v[d + 6];
  }
  const double h = SQRT3_2;
  Harm H;
  H.h0 = ((e[0] + e[1]) + (e[2] + e[3])) + (e[4] + e[5]);
  H.c1 = fma(h, o[1] - o[5], fma(0.5, o[2] - o[4], o[0]));
  H.s1 = fma(h, o[2] + o[4], fma(0.5, o[1] + o[5], o[3]));
  if (need2) {
    H.c2 = fma(0.5, (e[1] - e[2]) + (e[5] - e[4]), e[0] - e[3]);
    H.s2 = h * ((e[1] + e[2]) - (e[4] + e[5]));
  } else {
    H.c2 = H.s2 = 0.0;
  }
  return H;
}

}  // namespace rlbm
