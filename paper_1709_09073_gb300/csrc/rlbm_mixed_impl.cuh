// Mixed-precision step: FP32 / BF16 / FP16 storage, FP32 streaming, equilibrium
// and relaxation carried out on deviations f - fref from each domain's rest
// reference equilibrium, and double-float (an unevaluated pair of FP32 numbers,
// about 48 bits) for the quantities that set conservation: the totals N^mu,
// T^{mu nu}, the Landau-frame residual (Eq. 21), gamma, n, eps and the degree-1
// and degree-2 equilibrium moments.
//
// GB300 executes FP64 at 1/64 of the FP32 rate, so the kernel issues no FP64
// instruction: the 72-term moment sums run in FP32 on the small deviations
// (their rounding error is relative to the deviation, not to f), the Landau
// solve is FP32 Newton followed by one correction with a double-float residual,
// and the equilibrium moments that the collision must reproduce exactly for N^0
// and T^{mu 0} (Z_1k = n gamma (u_x + i u_y)^k P_1k, Z_2k = eps gamma^2
// (u_x + i u_y)^k P_2k) are formed from the double-float n and eps.
//
// This header holds the kernels and their host helpers; each storage format is
// instantiated in a translation unit of its own (rlbm_mixed_<storage>.cu) so
// that the units compile in parallel, and rlbm_mixed.cu dispatches to them.
// Every unit that includes it has its own copy of the constant tables and
// uploads it (upload_mixed_tables) before its first launch.
#pragma once
#include <cuda_runtime.h>

#include "rlbm_dfloat.cuh"
#include "rlbm_kernels.cuh"
#include "rlbm_tma.cuh"

namespace rlbm {

// ------------------------------------------------------------- FP32 tables
static __constant__ float c_pf[3][6] = {RLBM_PF_MJ_INIT, RLBM_PF_FD_INIT, RLBM_PF_BE_INIT};
static __constant__ float c_Qf[3][126] = {RLBM_QF_MJ_INIT, RLBM_QF_FD_INIT, RLBM_QF_BE_INIT};
// exact defects of the FP32 tables in the conserved moments (see eq_moments)
static __constant__ float c_Ef[3][18] = {RLBM_EF_MJ_INIT, RLBM_EF_FD_INIT, RLBM_EF_BE_INIT};
static __constant__ float c_p2f[3][6];
static __constant__ float c_pnkf[63];
// terms of the power series of Li_nu(x), |x| <= 1/4
#ifndef RLBM_SERIES_TERMS
#define RLBM_SERIES_TERMS 12  // the first term left out is below 2^-24 of g_1 for |x| <= 1/4
#endif
constexpr int kSerF = RLBM_SERIES_TERMS, kExpBEf = 16, kExpFDf = 26;
static __constant__ float c_invpowf[6 * kSerF];
static __constant__ float c_be_expf[6 * kExpBEf];
static __constant__ float c_fd_expf[6 * kExpFDf];
static __constant__ float c_be_logcoeff[6];
static __constant__ float c_be_harmf[6];
static __constant__ float c_g_zcf[6];

constexpr float kPIf = 3.14159265358979f;
// sqrt(3)/2 = kH + kHl: FP32 value and its residual. Products with sqrt(3)/2
// take both parts (two FMAs): with kH alone every moment and synthesis that
// pairs directions at +-30 degrees would shrink by the same 1.8e-8 each step,
// a steady sink of momentum (a Taylor-Green flow decayed 1e-5 too fast in 500
// steps).
constexpr float kH = 0.866025403784438647f;
constexpr float kHl = (float)(0.866025403784438647 - (double)kH);
__device__ __forceinline__ float mul_h(float x) { return fmaf(kH, x, kHl * x); }
__device__ __forceinline__ float fma_h(float x, float y) { return fmaf(kH, x, fmaf(kHl, x, y)); }
constexpr float kRZCf = (float)RLBM_R_ZC;
constexpr float kZCf = 0.9999999f;

// --------------------------------------------------- FP32 EDF integrals g_nu
// sum_{k>=1} x^k k^{-nu}, nu = 1..6, |x| <= 1/4. Fully unrolled, so that the
// coefficients are immediate constant operands. Rolled, each term loaded its
// six coefficients first; unrolling made the FD and BE steps 14 % and 5 % faster.
__device__ __forceinline__ void li_series6f(float x, float g[6]) {
  float xk = 1.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) g[i] = 0.0f;
#pragma unroll
  for (int k = 1; k <= kSerF; ++k) {
    xk *= x;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = fmaf(xk, c_invpowf[i * kSerF + k - 1], g[i]);
  }
}

template <int EDF>
__device__ void g_allf(float z, float g[6]) {
  if (EDF == EDF_MJ) {
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = z;
    return;
  }
  if (EDF == EDF_BE) {
    if (z <= 0.25f) { li_series6f(z, g); return; }
    const float mu = logf(z);
    float mk = 1.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < kExpBEf; ++k) {
#pragma unroll
      for (int i = 0; i < 6; ++i) g[i] = fmaf(mk, c_be_expf[i * kExpBEf + k], g[i]);
      mk *= mu;
    }
    const float lnm = logf(-mu);
    float mp = 1.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      g[i] = fmaf(mp, fmaf(-c_be_logcoeff[i], lnm, c_be_harmf[i]), g[i]);
      mp *= mu;
    }
    return;
  }
  if (z <= 0.25f) {
    li_series6f(-z, g);
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = -g[i];
    return;
  }
  if (z <= 4.0f) {
    const float mu = logf(z);
    float mk = 1.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = 0.0f;
#pragma unroll 2
    for (int k = 0; k < kExpFDf; ++k) {
#pragma unroll
      for (int i = 0; i < 6; ++i) g[i] = fmaf(mk, c_fd_expf[i * kExpFDf + k], g[i]);
      mk *= mu;
    }
    return;
  }
  li_series6f(-1.0f / z, g);
  const float L = logf(z);
  const float eta2 = 0.822467033f, eta4 = 0.947032829f, eta6 = 0.985551091f;
  const float L2 = L * L, L3 = L2 * L, L4 = L3 * L, L5 = L4 * L, L6 = L5 * L;
  // the inversion formula's polynomial in L, products and sums written out
  g[0] = -g[0] + L;
  g[1] = g[1] + fmaf(L2, 0.5f, 2.0f * eta2);
  g[2] = -g[2] + fmaf(L3, 1.0f / 6.0f, (2.0f * eta2) * L);
  g[3] = g[3] + fmaf(L4, 1.0f / 24.0f, fmaf(eta2, L2, 2.0f * eta4));
  g[4] = -g[4] + fmaf(L5, 1.0f / 120.0f, fmaf(eta2 / 3.0f, L3, (2.0f * eta4) * L));
  g[5] = g[5] + fmaf(L6, 1.0f / 720.0f, fmaf(eta2 / 12.0f, L4, fmaf(eta4, L2, 2.0f * eta6)));
}

// g_1, g_2, g_3 alone (g[0..2] of g_allf), what the Newton iterations below
// need: in the series range three series instead of six.
template <int EDF>
__device__ __forceinline__ void g123f(float z, float g[3]) {
  if (EDF != EDF_MJ && z <= 0.25f) {
    const float x = EDF == EDF_BE ? z : -z;
    float xk = 1.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
    for (int k = 1; k <= kSerF; ++k) {
      xk *= x;
      s1 = fmaf(xk, c_invpowf[k - 1], s1);
      s2 = fmaf(xk, c_invpowf[kSerF + k - 1], s2);
      s3 = fmaf(xk, c_invpowf[2 * kSerF + k - 1], s3);
    }
    const float sg = EDF == EDF_BE ? 1.0f : -1.0f;
    g[0] = sg * s1;
    g[1] = sg * s2;
    g[2] = sg * s3;
    return;
  }
  float g6[6];
  g_allf<EDF>(z, g6);
  g[0] = g6[0];
  g[1] = g6[1];
  g[2] = g6[2];
}

// A Newton step d in mu leaves an error of about C d^2, with C = |F''/(2F')| of
// the equation solved. Computed with arbitrary-precision polylogs, C is at most
// 0.23 for FD (z from 0.17 to 30) and about 0.12/(1 - z) for BE (0.24 at
// z = 0.5, 13 at z = 0.99), for both solves below. So a Newton step with
// d^2 C_bound < 1e-9 (C_bound = 0.25, or 0.25/(1 - z) for BE) is accepted
// without evaluating the equation again: the result is within 1e-9 of the root.
template <int EDF>
__device__ __forceinline__ bool newton_done(float d, float z) {
  const float cb = EDF == EDF_BE ? 0.25f / (1.0f - z) : 0.25f;
  return d * d * cb < 1e-9f;
}

// Fugacity from g_3^2/g_2^3 = target (Eq. 25), FP32 safeguarded Newton in mu = ln z.
// Start: the series g_nu = z + s z^2/2^nu + z^3/3^nu + s z^4/4^nu ... (s = -1 FD,
// +1 BE) make w = 1/target = g_2^3/g_3^2 a power series in z; inverting it gives
// mu = ln w - s w/2 + (119/1728) w^2 - s (85/6912) w^3 + O(w^4), off by 1.4e-6 in
// mu at z = 0.17, so one Newton step reaches the FP32 floor (newton_done accepts
// it). The iterations evaluate g_1..g_3 alone; all six g_nu are evaluated once,
// at the converged mu (the last step applied).
template <int EDF>
__device__ int solve_z_R_f(float target, float& z, float g[6]) {
  if (EDF == EDF_BE && target < kRZCf) {
    z = kZCf;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = c_g_zcf[i];
    return ST_CLAMPED;
  }
  float lo = -40.0f, hi = (EDF == EDF_BE) ? -1.0e-7f : 40.0f;
  const float lt = logf(target);
  float mu = -lt;
  {
    const float w = 1.0f / target;
    if (w < 0.5f) {
      constexpr float kS = EDF == EDF_BE ? 1.0f : -1.0f;
      mu = fmaf(fmaf(fmaf(-kS * (85.0f / 6912.0f), w, 119.0f / 1728.0f), w, -0.5f * kS), w, mu);
    }
  }
  mu = fminf(fmaxf(mu, lo + 1e-3f), hi);
  int st = ST_ZSOLVE;
  float dprev = INFINITY;
  for (int it = 0; it < 40; ++it) {
    float gi[3];
    const float ze = expf(mu);
    g123f<EDF>(ze, gi);
    const float F = logf(gi[2] * gi[2] / (gi[1] * gi[1] * gi[1])) - lt;
    if (F == 0.0f) {
      st = 0;
      break;
    }
    const float dF = 2.0f * gi[1] / gi[2] - 3.0f * gi[0] / gi[1];
    if (F > 0.0f) lo = mu; else hi = mu;
    float mn = mu - F / dF;
    const bool newton = mn >= lo && mn <= hi;
    if (!newton) mn = 0.5f * (lo + hi);
    const float d = fabsf(mn - mu);
    mu = mn;
    if (d <= 4e-7f * fmaxf(1.0f, fabsf(mu)) || (newton && newton_done<EDF>(d, ze)) ||
        (d < 1e-4f && d >= dprev)) {
      st = 0;
      break;
    }
    dprev = d;
  }
  z = expf(mu);
  g_allf<EDF>(z, g);
  return st;
}

// Fugacity from (n, theta): n = 2 pi theta^2 g_2(z), FP32 safeguarded Newton in
// mu = ln z. Start: inverting G = g_2(z) = z -+ z^2/4 + z^3/9 -+ ... (G = n / (2 pi
// theta^2)) gives mu = ln G +- G/4 - (5/288) G^2 +- G^3/288 + O(G^4) (upper signs
// FD, lower BE) for small G. Convergence as in solve_z_R_f.
template <int EDF>
__device__ int solve_z_nt_f(float n, float theta, float& z, float g[6]) {
  const float G = n / (2.0f * kPIf * theta * theta);
  if (EDF == EDF_MJ) {
    z = G;
    g_allf<EDF>(z, g);
    return 0;
  }
  if (EDF == EDF_BE && G >= c_g_zcf[1]) {
    z = kZCf;
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = c_g_zcf[i];
    return ST_CLAMPED;
  }
  float lo = -40.0f, hi = (EDF == EDF_BE) ? -1.0e-7f : 40.0f;
  const float lG = logf(G);
  float mu = lG;
  if (G < 0.5f) {
    constexpr float kS = EDF == EDF_BE ? -1.0f : 1.0f;
    mu = fmaf(fmaf(fmaf(kS / 288.0f, G, -5.0f / 288.0f), G, 0.25f * kS), G, mu);
  }
  mu = fminf(fmaxf(mu, lo + 1e-3f), hi);
  float dprev = INFINITY;
  int st = ST_ZSOLVE;
  for (int it = 0; it < 40; ++it) {
    float gi[3];
    const float ze = expf(mu);
    g123f<EDF>(ze, gi);
    const float F = logf(gi[1]) - lG;
    if (F == 0.0f) {
      st = 0;
      break;
    }
    const float dF = gi[0] / gi[1];
    if (F < 0.0f) lo = mu; else hi = mu;
    float mn = mu - F / dF;
    const bool newton = mn >= lo && mn <= hi;
    if (!newton) mn = 0.5f * (lo + hi);
    const float d = fabsf(mn - mu);
    mu = mn;
    if (d <= 4e-7f * fmaxf(1.0f, fabsf(mu)) || (newton && newton_done<EDF>(d, ze)) ||
        (d < 1e-4f && d >= dprev)) {
      st = 0;
      break;
    }
    dprev = d;
  }
  z = expf(mu);
  g_allf<EDF>(z, g);
  return st;
}

// ------------------------------------------------------------- Landau frame
// T^a_b U^b = eps U^a (Eq. 21) as m - Pi u = (T00 - m.u) u. FP32 Newton from the
// ideal-fluid estimate, then one Newton correction whose residual is evaluated
// in double-float (the FP32 Jacobian only scales the small correction), which
// brings u to ~1e-15. eps, gamma follow in double-float. T = {T00, T01, T02,
// T11, T12, T22}.
__device__ __forceinline__ int landau_df(const df T[6], df& ux, df& uy, df& eps, df& gamma) {
  // every product that meets a sum is an explicit FMA (or the sum a rounded
  // intrinsic), so each kernel that inlines this gets the same roundings
  const float E = T[0].hi, mx = T[1].hi, my = T[2].hi, pxx = T[3].hi, pxy = T[4].hi, pyy = T[5].hi;
  const float disc = fmaf(9.0f * E, E, -8.0f * fmaf(mx, mx, __fmul_rn(my, my)));
  if (!(E > 0.0f) || !(disc >= 0.0f)) return ST_NONPHYSICAL;
  const float x = 0.25f * fmaf(3.0f, E, sqrtf(disc));
  float fu = mx / x, fv = my / x;
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const float a = fmaf(-mx, fu, fmaf(-my, fv, E));
    const float fx = fmaf(-a, fu, fmaf(-pxx, fu, fmaf(-pxy, fv, mx)));
    const float fy = fmaf(-a, fv, fmaf(-pxy, fu, fmaf(-pyy, fv, my)));
    const float j00 = __fsub_rn(fmaf(fu, mx, -pxx), a), j01 = fmaf(fu, my, -pxy), j10 = fmaf(fv, mx, -pxy),
                j11 = __fsub_rn(fmaf(fv, my, -pyy), a);
    const float rdet = 1.0f / fmaf(j00, j11, -__fmul_rn(j01, j10));
    fu = fmaf(fmaf(j01, fy, -__fmul_rn(j11, fx)), rdet, fu);
    fv = fmaf(fmaf(j10, fx, -__fmul_rn(j00, fy)), rdet, fv);
  }
  if (!(fmaf(fu, fu, __fmul_rn(fv, fv)) < 1.0f)) return ST_NONPHYSICAL;
  {
    const df a = df_sub(T[0], df_add(df_mul(T[1], fu), df_mul(T[2], fv)));
    const df rx = df_sub(df_sub(T[1], df_add(df_mul(T[3], fu), df_mul(T[4], fv))), df_mul(a, fu));
    const df ry = df_sub(df_sub(T[2], df_add(df_mul(T[4], fu), df_mul(T[5], fv))), df_mul(a, fv));
    const float af = a.hi;
    const float j00 = __fsub_rn(fmaf(fu, mx, -pxx), af), j01 = fmaf(fu, my, -pxy), j10 = fmaf(fv, mx, -pxy),
                j11 = __fsub_rn(fmaf(fv, my, -pyy), af);
    const float rdet = 1.0f / fmaf(j00, j11, -__fmul_rn(j01, j10));
    const float gx = df_to_float(rx), gy = df_to_float(ry);
    ux = two_sum(fu, __fmul_rn(fmaf(j01, gy, -__fmul_rn(j11, gx)), rdet));
    uy = two_sum(fv, __fmul_rn(fmaf(j10, gx, -__fmul_rn(j00, gy)), rdet));
  }
  eps = df_sub(T[0], df_add(df_mul(T[1], ux), df_mul(T[2], uy)));
  const df w = df_sub(df_make(1.0f, 0.0f), df_add(df_mul(ux, ux), df_mul(uy, uy)));
  if (!(w.hi > 0.0f) || !(eps.hi > 0.0f)) return ST_NONPHYSICAL;
  gamma = df_rsqrt(w);
  return 0;
}

// Relaxation rate of direction d, gamma (1 - v_d . u) / tau (Eq. 3), with the
// roundings written out (see landau_df).
__device__ __forceinline__ float relax_rate(int d, float gam, float ux, float uy, float itau) {
  const float vu = fmaf((float)dcos(d), ux, __fmul_rn((float)dsin(d), uy));
  return __fmul_rn(__fmul_rn(gam, __fsub_rn(1.0f, vu)), itau);
}

// FP32 harmonic sums of a 12-vector (pairs d, d+6 folded first).
struct HarmF {
  float h0, c1, s1, c2, s2;
};

__device__ __forceinline__ HarmF harmonics_f(const float v[12]) {
  float e[6], o[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    e[d] = v[d] + v[d + 6];
    o[d] = v[d] - v[d + 6];
  }
  HarmF H;
  H.h0 = ((e[0] + e[1]) + (e[2] + e[3])) + (e[4] + e[5]);
  H.c1 = fma_h(o[1] - o[5], fmaf(0.5f, o[2] - o[4], o[0]));
  H.s1 = fma_h(o[2] + o[4], fmaf(0.5f, o[1] + o[5], o[3]));
  H.c2 = fmaf(0.5f, (e[1] - e[2]) + (e[5] - e[4]), e[0] - e[3]);
  H.s2 = mul_h((e[1] + e[2]) - (e[4] + e[5]));
  return H;
}

// FP32 deviation of the equilibrium from fref for shell s (12 directions):
// R^{c|s}_k = sum_n Qf^(k)_{s n} dZ_nk (+ rres_s in R^c_0), then the folded
// 12-point synthesis (same symmetries as the FP64 form).
template <int EDF>
__device__ __forceinline__ void dfeq_shell(int s, float rres, const float zr[21], const float zi[21],
                                           float fe[12]) {
  float Rc[6], Rs[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float ac = 0.0f, as = 0.0f;
#pragma unroll
    for (int n = k; n < 6; ++n) {
      const float q = c_Qf[EDF][qoff(k) + s * (6 - k) + (n - k)];
      ac = fmaf(q, zr[n * (n + 1) / 2 + k], ac);
      as = fmaf(q, zi[n * (n + 1) / 2 + k], as);
    }
    Rc[k] = ac;
    Rs[k] = as;
  }
  Rc[0] += rres;
  const float t1 = Rc[0] + Rc[4], t2 = fmaf(-0.5f, Rc[4], Rc[0]);
  const float Ec0 = t1 + Rc[2], Ec3 = t1 - Rc[2], Ec1 = fmaf(0.5f, Rc[2], t2), Ec2 = fmaf(-0.5f, Rc[2], t2);
  const float Es1 = mul_h(Rs[2] + Rs[4]), Es2 = mul_h(Rs[2] - Rs[4]);
  const float E0 = Ec0, E1 = Ec1 + Es1, E2 = Ec2 + Es2, E3 = Ec3, E4 = Ec2 - Es2, E5 = Ec1 - Es1;
  const float Oc0 = Rc[1] + Rc[3] + Rc[5], Oc1 = mul_h(Rc[1] - Rc[5]), Oc2 = fmaf(0.5f, Rc[1] + Rc[5], -Rc[3]);
  const float Os1 = fmaf(0.5f, Rs[1] + Rs[5], Rs[3]), Os2 = mul_h(Rs[1] - Rs[5]), Os3 = Rs[1] - Rs[3] + Rs[5];
  const float O0 = Oc0, O1 = Oc1 + Os1, O2 = Oc2 + Os2, O3 = Os3, O4 = Os2 - Oc2, O5 = Os1 - Oc1;
  fe[0] = E0 + O0; fe[6] = E0 - O0;
  fe[1] = E1 + O1; fe[7] = E1 - O1;
  fe[2] = E2 + O2; fe[8] = E2 - O2;
  fe[3] = E3 + O3; fe[9] = E3 - O3;
  fe[4] = E4 + O4; fe[10] = E4 - O4;
  fe[5] = E5 + O5; fe[11] = E5 - O5;
}

// FP32 equilibrium-moment deviations dZ_nk = Z_nk - Z_ref (Appendix, harmonic
// form). When An1, An2 >= 0 they replace the degree-1 and degree-2 prefactors
// (n gamma and eps gamma^2 from the double-float state); the caller then sets
// the conserved isotropic entries dZ_10, dZ_20 itself.
template <int EDF>
__device__ __forceinline__ void dz_moments(const DomDev& D, const float g[6], float theta, float ux, float uy,
                                           float gam, float An1, float An2, float zr[21], float zi[21]) {
  // products that meet sums are explicit FMAs (see landau_df)
  const float u2 = fmaf(ux, ux, __fmul_rn(uy, uy));
  float wr[6], wi[6];
  wr[0] = 1.0f;
  wi[0] = 0.0f;
#pragma unroll
  for (int k = 1; k < 6; ++k) {
    wr[k] = fmaf(wr[k - 1], ux, -__fmul_rn(wi[k - 1], uy));
    wi[k] = fmaf(wr[k - 1], uy, __fmul_rn(wi[k - 1], ux));
  }
  float A = 2.0f * kPIf * theta;
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    if (n > 0) A *= (float)n * theta * gam;
    float An = A * g[n];
    if (n == 1 && An1 >= 0.0f) An = An1;
    if (n == 2 && An2 >= 0.0f) An = An2;
#pragma unroll
    for (int k = 0; k <= n; ++k) {
      const int i = n * (n + 1) / 2 + k;
      const float P = fmaf(u2, fmaf(u2, c_pnkf[3 * i + 2], c_pnkf[3 * i + 1]), c_pnkf[3 * i + 0]);
      if (k == 0) {
        zr[i] = fmaf(An, P, -D.zref_f[n]);  // the isotropic moments as deviations from the reference
        zi[i] = 0.0f;
      } else {
        const float sc = __fmul_rn(An, P);
        zr[i] = __fmul_rn(sc, wr[k]);
        zi[i] = __fmul_rn(sc, wi[k]);
      }
    }
  }
}

// Halo writer of the mixed step: copies of the cell's post-collision values
// (FP32 deviations held in its shared-memory column col[q * kThreads]) and, at
// fixed-T walls, the
// FP32 equilibrium deviation of the wall ghost. Reading the copies back from
// global memory instead would put a read-after-write round trip to L2 on every
// edge warp, which costs more than keeping the column up to date.
template <int EDF, class S>
__device__ __noinline__ void write_halo_mixed(const DomDev& D, int x, int y, typename S::T* __restrict__ fout,
                                              const float* col, bool have_state, float n, float ux, float uy,
                                              float gam, unsigned& st, bool images) {
  int hx[8], hy[8], wall[8];
  const int cnt = halo_targets(D, x, y, hx, hy, wall, images);
  for (int i = 0; i < cnt; ++i) {
    const long long h = cell_rel(D, hx[i], hy[i]);
    if (wall[i] < 0 || !have_state) {
      for (int q = 0; q < 72; ++q) {
        fout[q * kBlkW + h] = S::encf(col[q * kThreads], D, q % 6);
      }
    } else {
      const float tw = D.t_wall_f[wall[i]];
      float z, g[6];
      st |= solve_z_nt_f<EDF>(n, tw, z, g);
      float zr[21], zi[21];
      dz_moments<EDF>(D, g, tw, ux, uy, gam, -1.0f, -1.0f, zr, zi);
#pragma unroll 1
      for (int s = 0; s < 6; ++s) {
        float fe[12];
        dfeq_shell<EDF>(s, D.rres[s], zr, zi, fe);
        for (int d = 0; d < 12; ++d) fout[(6 * d + s) * kBlkW + h] = S::encf(fe[d], D, s);
      }
    }
  }
}

constexpr size_t kSmemF = 72 * kThreads * sizeof(float);  // the shared-memory column of a block

#ifndef RLBM_MIXED_MIN_BLOCKS
// resident blocks per SM the register budget must allow: 640 threads (96
// registers, no spills; 20 warps per SM). Measured against 512 threads (128
// registers) and 768 (80 registers, spills): 2 % faster than the first on every
// workload, 12 % faster than the second.
#define RLBM_MIXED_MIN_BLOCKS (640 / kThreads)
#endif
// 1: at the start of a tile one thread asks L2 for the tile's own blocks in rows
// y0-1 .. y0+kTileH (one contiguous segment per row), so that the pull's later
// directions find them in L2
#ifndef RLBM_MIXED_L2_PREFETCH
#define RLBM_MIXED_L2_PREFETCH 1
#endif
// 1: only warps holding an edge cell keep the relaxed values in the column (a
// second copy of the relaxation loop); 0: every warp keeps them (one loop)
#ifndef RLBM_MIXED_EDGE_WARPS
#define RLBM_MIXED_EDGE_WARPS 0
#endif

// Relaxation (Eq. 3) of one cell's 72 pulled deviations in its column, shell
// by shell, stored to fout; kKeep: the relaxed values also go back into the
// column (warps holding an edge cell, whose halo writer reads them there).
template <int EDF, class S, bool kKeep>
__device__ __forceinline__ void relax_cell(const DomDev& D, const float zr[21], const float zi[21], const float om[12],
                                           float* smf, int tid, long long c, typename S::T* __restrict__ fout) {
#pragma unroll 1
  for (int s = 0; s < 6; ++s) {
    float fe[12];
    dfeq_shell<EDF>(s, D.rres[s], zr, zi, fe);
#pragma unroll
    for (int d = 0; d < 12; ++d) {
      const int q = 6 * d + s;
      const float v = smf[q * kThreads + tid];
      const float r = fmaf(om[d], fe[d] - v, v);
      if constexpr (kKeep) smf[q * kThreads + tid] = r;
      fout[q * kBlkW + c] = S::encf(r, D, s);
    }
  }
}

// Collision of one cell (Eqs. 20-25, 10-11 and 3) from its pulled FP32
// deviations, held in the thread's shared-memory column smf[q * kThreads + tid],
// and the shell sums A_d = sum_s p_s dv_{6d+s}, B_d = sum_s p_s^2 dv_{6d+s} of
// each direction; stores f* to fout, writes the cell's halo images and returns
// its status bits. Called by the active lanes of a warp (the lanes of cells
// inside the domain). kImages: also write the periodic halo images (the
// TMA-staged step reads them; the L1 pull wraps instead). kHalo, the launch's
// halo work (StepArgs::halo): 0 none (every side periodic or exchanged), 1 wall
// equilibria only (every other side a fixed-T wall), 2 also copies (zero-gradient
// sides). Below 2, with kImages = false, no halo cell copies the cell's relaxed
// values, so they need not go back to the column.
template <int EDF, class S, bool kImages, int kHalo = 2>
__device__ __forceinline__ unsigned collide_mixed(const DomDev& D, int x, int y, long long c, const float A[12],
                                                  const float B[12], float* smf, int tid,
                                                  typename S::T* __restrict__ fout) {
  // a warp with no cell on an edge that has halo cells to write skips the halo
  // writer (uniform per warp)
  const bool edge = kImages ? (x == 0 || x == D.nx - 1 || y == 0 || y == D.ny - 1)
                            : kHalo > 0 && ((x == 0 && bc_writes_halo(D.bc[0])) ||
                                        (x == D.nx - 1 && bc_writes_halo(D.bc[1])) ||
                                        (y == 0 && bc_writes_halo(D.bc[2])) ||
                                        (y == D.ny - 1 && bc_writes_halo(D.bc[3])));
  const bool edge_warp = __any_sync(__activemask(), edge);
  const HarmF ha = harmonics_f(A), hb = harmonics_f(B);
  // moment totals in double-float: reference moments + FP32 deviation sums
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
    // conserved equilibrium moments from the double-float state: Z_1k from
    // n gamma, Z_2k from eps gamma^2 (a clamped BE state relaxes to its own
    // equilibrium energy 4 pi theta^3 g_3(z_c))
    const df nG = df_mul(n, gam);
    df eG2 = df_mul(df_mul(eps, gam), gam);
    if (st & ST_CLAMPED) eG2 = df_make(4.0f * kPIf * theta * theta * theta * g[2] * gf * gf, 0.0f);
    float zr[21], zi[21];
    dz_moments<EDF>(D, g, theta, uxf, uyf, gf, nG.hi, eG2.hi, zr, zi);
    // Z_20 = eps gamma^2 (1 + u^2/2), all in double-float
    const df u2h = df_scale(df_add(df_mul(ux, ux), df_mul(uy, uy)), 0.5f);
    const df dz10 = df_sub(nG, df_make(D.z1_hl[0], D.z1_hl[1]));
    const df dz20 = df_sub(df_add(eG2, df_mul(eG2, u2h)), df_make(D.z2_hl[0], D.z2_hl[1]));
    zr[1] = df_to_float(dz10);
    zr[3] = df_to_float(dz20);
    // Z_21 = (3/2) eps gamma^2 (u_x + i u_y) (Appendix; the rest state has none),
    // also from the double-float state rather than from FP32 eps gamma^2
    const df e15 = df_mul(eG2, 1.5f);
    zr[4] = df_to_float(df_mul(e15, ux));
    zi[4] = df_to_float(df_mul(e15, uy));
    // remove the FP32 tables' defects in N^0, T^00, T^0x, T^0y (FP32 suffices:
    // the corrections are ~1e-8 of the moments)
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
    // constant tau, or the local tau = 4 (eta/s) / theta + 0.2546 of Sec. 3.5
    float itau = D.inv_tau_f;
    if (D.eta_s_f > 0.0f) itau = 1.0f / (4.0f * D.eta_s_f / theta + 0.2546f);
    float om[12];
#pragma unroll
    for (int d = 0; d < 12; ++d) om[d] = relax_rate(d, gf, uxf, uyf, itau);
    if constexpr (!kImages && kHalo < 2) {
      relax_cell<EDF, S, false>(D, zr, zi, om, smf, tid, c, fout);
    } else {
#if RLBM_MIXED_EDGE_WARPS
      if (edge_warp) relax_cell<EDF, S, true>(D, zr, zi, om, smf, tid, c, fout);
      else relax_cell<EDF, S, false>(D, zr, zi, om, smf, tid, c, fout);
#else
      relax_cell<EDF, S, true>(D, zr, zi, om, smf, tid, c, fout);
#endif
    }
  } else {
    for (int q = 0; q < 72; ++q) fout[q * kBlkW + c] = S::encf(smf[q * kThreads + tid], D, q % 6);
  }
  if (kImages || kHalo > 0)
    if (edge_warp) write_halo_mixed<EDF, S>(D, x, y, fout, smf + tid, ok, nf, uxf, uyf, gf, st, kImages);
  return st;
}

// Ask L2 for a tile's own blocks in rows y0-1 .. y0+kTileH of every plane: one
// contiguous segment per row, one bulk prefetch each.
template <class S>
__device__ __forceinline__ void prefetch_tile_l2(const DomDev& D, const Tile& tl, const typename S::T* fin) {
  const int r1 = min(tl.y0 + kTileH, D.ny);
  for (int r = tl.y0 - 1; r <= r1; ++r) {
    const typename S::T* p = fin + cell_rel(D, tl.x0, r);  // lane 0, plane 0 of the tile's block
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)),
                 "r"((unsigned)(kBlk * sizeof(typename S::T)))
                 : "memory");
  }
}

// One tile of the step (32 x 4 cells, or a packed ragged block): pull,
// collide, store (the thread's cell).
template <int EDF, class S, int kHalo>
__device__ __forceinline__ void step_tile_mixed(const StepArgs& a, int t, float* smf, int tid) {
  const Tile tl = a.tiles[t];
  const DomDev& D = a.doms[tl.dom];
  int x, y;
  if (!tile_cell(tl, threadIdx.x, threadIdx.y, x, y) || x >= D.nx || y >= D.ny) return;
  const typename S::T* __restrict__ fin = static_cast<const typename S::T*>(a.fin) + D.off;
  typename S::T* __restrict__ fout = static_cast<typename S::T*>(a.fout) + D.off;
#if RLBM_MIXED_L2_PREFETCH
  // (a packed tile uses at most half of each block it would fetch: not worth it)
  if (tid == 0 && tl.w == 0) prefetch_tile_l2<S>(D, tl, fin);
#endif
  const long long c = cell_rel(D, x, y);
  const Nbr nb = neighbours(D, x, y);
  // pull (FP32, deviation form) with the FP32 deviation moment sums
  float A[12], B[12], pc[6], p2c[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    pc[s] = c_pf[EDF][s];
    p2c[s] = c_p2f[EDF][s];
  }
#define RLBM_PULL_DIR(d)                                                        \
  {                                                                             \
    float a_ = 0.0f, b_ = 0.0f;                                                 \
    _Pragma("unroll") for (int s = 0; s < 6; ++s) {                             \
      const float v = S::decf(pull_one<d, float, S>(fin + c + (6 * d + s) * kBlkW, nb), D, s); \
      smf[(6 * d + s) * kThreads + tid] = v;                                    \
      a_ = fmaf(v, pc[s], a_);                                                  \
      b_ = fmaf(v, p2c[s], b_);                                                 \
    }                                                                           \
    A[d] = a_;                                                                  \
    B[d] = b_;                                                                  \
  }
  RLBM_PULL_DIR(0) RLBM_PULL_DIR(1) RLBM_PULL_DIR(2) RLBM_PULL_DIR(3)
  RLBM_PULL_DIR(4) RLBM_PULL_DIR(5) RLBM_PULL_DIR(6) RLBM_PULL_DIR(7)
  RLBM_PULL_DIR(8) RLBM_PULL_DIR(9) RLBM_PULL_DIR(10) RLBM_PULL_DIR(11)
#undef RLBM_PULL_DIR
  const unsigned st = collide_mixed<EDF, S, false, kHalo>(D, x, y, c, A, B, smf, tid, fout);
  if (st) atomicOr(a.status, st);
}

// kHalo = StepArgs::halo (see collide_mixed): 0 no halo writer, 0 and 1 no copy
// of the relaxed values into the column.
template <int EDF, class S, int kHalo>
__global__ void __launch_bounds__(kThreads, RLBM_MIXED_MIN_BLOCKS) k_step_mixed(StepArgs a) {
  extern __shared__ float smf[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    step_tile_mixed<EDF, S, kHalo>(a, t, smf, tid);
  }
}

// ------------------------------------------- TMA-staged variant of the step
// Per 32 x 4 tile and direction d, one TMA box brings the six shell planes of d
// for the tile's block of 32 cells and the blocks either side, rows y0-1 ..
// y0+kTileH, into shared memory (a box {32 lanes, 6 planes, 3 blocks, kTileH + 2 rows} of the
// 4D tensor {32, 72, nblk, ny + 2}); the bilinear pull reads its four
// neighbours there at fixed offsets (x - 1 of lane 0 and x + 1 of lane 31 in
// the neighbouring blocks). A ring of kStages boxes keeps the next directions --
// and, while a tile collides, the next tile's first directions -- in flight.
// The arithmetic is the same as k_step_mixed's, so the two variants give
// identical results.
template <class S>
struct TmaBox {
  using T = typename S::T;
  static constexpr int kPlane = kBlkW;                        // a plane's 32 lanes
  static constexpr int kBlock = kBoxPlanes * kPlane;          // six planes of one block
  static constexpr int kRow = kBoxBlocks * kBlock;            // three blocks of one row
  static constexpr unsigned kBytes = (unsigned)(kBoxElems * sizeof(T));
  static constexpr int kStageElems = kBoxElems;
};
constexpr int kStages = 3;  // ring depth in directions (a divisor of 12)

template <class S>
constexpr size_t tma_smem_bytes() {
  return kStages * (size_t)TmaBox<S>::kBytes + 72 * kThreads * sizeof(float) + kStages * sizeof(uint64_t);
}

// Issue the box of direction d of tile t into its ring stage (one thread).
template <class S>
__device__ __forceinline__ void tma_issue(const StepArgs& a, int t, int d, unsigned char* ring, uint64_t* bar) {
  const Tile tl = a.tiles[t];
  const void* map = static_cast<const unsigned char*>(a.tmaps) + (size_t)tl.dom * kTensorMapBytes;
  const int k = d % kStages;
  mbar_expect_tx(&bar[k], TmaBox<S>::kBytes);
  // lanes from 0, planes from 6d, blocks from the one left of the tile's
  // (x0 / 32 + 1 holds x0), rows from y = y0 - 1 (row index y0)
  tma_load_4d(ring + k * TmaBox<S>::kBytes, map, 0, 6 * d, tl.x0 / kBlkW, tl.y0, &bar[k]);
}

// Pull of direction d from its staged box; `cell` points at the cell's own
// value in shell 0 of that stage, oxm / oxp are the offsets of x - 1 / x + 1
// there (same weights and order of operations as pull_one), col at the
// thread's shared-memory column.
template <int d, class S>
__device__ __forceinline__ void pull_dir_staged(const typename S::T* cell, int oxm, int oxp, const DomDev& D,
                                                const float pc[6], const float p2c[6], float* col, float& A,
                                                float& B) {
  using TB = TmaBox<S>;
  constexpr double cx = dcos(d), cy = dsin(d);
  constexpr int sx = sgnd(cx), sy = sgnd(cy);
  constexpr double ax = dabs(cx), ay = dabs(cy);
  constexpr float axr = (float)ax, ayr = (float)ay;
  constexpr float w1 = axr * ayr, w2 = (1.0f - axr) * ayr, w3 = axr * (1.0f - ayr),
                  w4 = (1.0f - axr) * (1.0f - ayr);
  const int ox = sx > 0 ? oxm : (sx < 0 ? oxp : 0);
  constexpr int oy = -sy * TB::kRow;
  float a_ = 0.0f, b_ = 0.0f;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const typename S::T* pl = cell + s * TB::kPlane;
    float v;
    if (ax == 0.0 || ay == 0.0) {
      v = S::raw(pl[ox + oy]);
    } else {
      const float v1 = S::raw(pl[ox + oy]), v2 = S::raw(pl[oy]), v3 = S::raw(pl[ox]), v4 = S::raw(pl[0]);
      v = fmaf(w1, v1, fmaf(w2, v2, fmaf(w3, v3, w4 * v4)));
    }
    v = S::decf(v, D, s);
    col[(6 * d + s) * kThreads] = v;
    a_ = fmaf(v, pc[s], a_);
    b_ = fmaf(v, p2c[s], b_);
  }
  A = a_;
  B = b_;
}

template <int EDF, class S>
__global__ void __launch_bounds__(kThreads, RLBM_MIXED_MIN_BLOCKS) k_step_mixed_tma(StepArgs a) {
  using T = typename S::T;
  using TB = TmaBox<S>;
  extern __shared__ __align__(128) unsigned char smt[];
  unsigned char* ring = smt;
  float* smf = reinterpret_cast<float*>(smt + kStages * TB::kBytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smt + kStages * TB::kBytes + 72 * kThreads * sizeof(float));
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (blockIdx.x >= a.ntiles) return;  // whole block
  const unsigned long long wait_ns = a.wait_ns ? a.wait_ns : kDefaultWaitNs;
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < kStages; ++k) mbar_init(&bar[k], 1);
    fence_barrier_init();
  }
  __syncthreads();
  // thread 0 tracks the loads in flight per stage (for the drain on a timeout)
  unsigned inflight = 0, issued[kStages] = {};
  if (tid == 0) {
#pragma unroll
    for (int d = 0; d < kStages; ++d) {
      tma_issue<S>(a, blockIdx.x, d, ring, bar);
      inflight |= 1u << d;
      ++issued[d];
    }
  }
  // the cell's own value in shell 0 of stage 0 (row ty + 1, middle block, lane
  // tx), the offsets of its x neighbours, and its column
  const T* cell0 = reinterpret_cast<const T*>(ring) + (threadIdx.y + 1) * TB::kRow + TB::kBlock + threadIdx.x;
  const int oxm = threadIdx.x > 0 ? -1 : -TB::kBlock + (kBlkW - 1);
  const int oxp = threadIdx.x < kBlkW - 1 ? 1 : TB::kBlock - (kBlkW - 1);
  float* col = smf + tid;
  float pc[6], p2c[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    pc[s] = c_pf[EDF][s];
    p2c[s] = c_p2f[EDF][s];
  }
  unsigned it = 0;  // tiles done by this block: stage uses so far = it * 12 / kStages + d / kStages
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++it) {
    const Tile tl = a.tiles[t];
    const DomDev& D = a.doms[tl.dom];
    const int x = tl.x0 + threadIdx.x, y = tl.y0 + threadIdx.y;
    const int tnext = t + gridDim.x;
    const unsigned use0 = it * (12 / kStages);
    float A[12], B[12];
    // every lane pulls (lanes outside the domain read the box's padding and
    // fill only their own column, which is never stored)
#define RLBM_STAGED_DIR(d)                                                                      \
  {                                                                                             \
    constexpr int k_ = (d) % kStages;                                                           \
    const bool ok_ = mbar_wait(&bar[k_], (use0 + (d) / kStages) & 1, wait_ns);                  \
    pull_dir_staged<d, S>(cell0 + k_ * TB::kStageElems, oxm, oxp, D, pc, p2c, col, A[d], B[d]); \
    if (__syncthreads_or(!ok_)) goto timed_out;                                                 \
    if (tid == 0) {                                                                             \
      inflight &= ~(1u << k_);                                                                  \
      const int tt_ = (d) + kStages < 12 ? t : tnext;                                           \
      if (tt_ < a.ntiles) {                                                                     \
        tma_issue<S>(a, tt_, ((d) + kStages) % 12, ring, bar);                                  \
        inflight |= 1u << k_;                                                                   \
        ++issued[k_];                                                                           \
      }                                                                                         \
    }                                                                                           \
  }
    RLBM_STAGED_DIR(0) RLBM_STAGED_DIR(1) RLBM_STAGED_DIR(2) RLBM_STAGED_DIR(3)
    RLBM_STAGED_DIR(4) RLBM_STAGED_DIR(5) RLBM_STAGED_DIR(6) RLBM_STAGED_DIR(7)
    RLBM_STAGED_DIR(8) RLBM_STAGED_DIR(9) RLBM_STAGED_DIR(10) RLBM_STAGED_DIR(11)
#undef RLBM_STAGED_DIR
    if (x < D.nx && y < D.ny) {
      T* __restrict__ fout = static_cast<T*>(a.fout) + D.off;
      const unsigned st = collide_mixed<EDF, S, true>(D, x, y, cell_rel(D, x, y), A, B, smf, tid, fout);
      if (st) atomicOr(a.status, st);
    }
  }
  return;
timed_out:
  // a copy did not land in time: report it, let the copies still in flight
  // finish (bounded by the default limit, whatever the limit of the waits
  // above) so that none writes shared memory after exit, return
  if (tid == 0) {
    atomicOr(a.status, ST_TIMEOUT);
#pragma unroll
    for (int k = 0; k < kStages; ++k)
      if (inflight & (1u << k)) mbar_wait(&bar[k], (issued[k] - 1) & 1);
  }
}

// Macroscopic fields (n, theta, ux, uy, z) of a mixed storage's populations in
// the collision's own arithmetic -- the FP32 pull and deviation sums, the
// double-float totals and Landau frame (Eqs. 20-25), the FP32 fugacity solve --
// written as FP64 (the double-float values exactly). It runs on the FP32 pipe;
// the FP64 read-out k_fields, at 1/64 of that rate, serves the diagnostics.
template <int EDF, class S>
__global__ void __launch_bounds__(kThreads) k_fields_mixed(FieldsArgs a) {
  int dom, x, y;
  cell_of_launch(a.tiles, a.dom, dom, x, y);
  const DomDev& D = a.doms[dom];
  if (x >= D.nx || y >= D.ny) return;
  const typename S::T* __restrict__ f = static_cast<const typename S::T*>(a.f) + D.off;
  const long long c = cell_rel(D, x, y);
  float A[12], B[12];
  {
    float pc[6], p2c[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      pc[s] = c_pf[EDF][s];
      p2c[s] = c_p2f[EDF][s];
    }
    const Nbr nb = neighbours(D, x, y);
    const bool streamed = a.streamed != 0;
#define RLBM_FIELDS_DIR(d)                                                                       \
  {                                                                                              \
    float a_ = 0.0f, b_ = 0.0f;                                                                  \
    _Pragma("unroll") for (int s = 0; s < 6; ++s) {                                              \
      const typename S::T* pl = f + c + (6 * d + s) * kBlkW;                                     \
      const float r = streamed ? pull_one<d, float, S>(pl, nb) : S::raw(pl[0]);                  \
      const float v = S::decf(r, D, s);                                                          \
      a_ = fmaf(v, pc[s], a_);                                                                   \
      b_ = fmaf(v, p2c[s], b_);                                                                  \
    }                                                                                            \
    A[d] = a_;                                                                                   \
    B[d] = b_;                                                                                   \
  }
    RLBM_FIELDS_DIR(0) RLBM_FIELDS_DIR(1) RLBM_FIELDS_DIR(2) RLBM_FIELDS_DIR(3)
    RLBM_FIELDS_DIR(4) RLBM_FIELDS_DIR(5) RLBM_FIELDS_DIR(6) RLBM_FIELDS_DIR(7)
    RLBM_FIELDS_DIR(8) RLBM_FIELDS_DIR(9) RLBM_FIELDS_DIR(10) RLBM_FIELDS_DIR(11)
#undef RLBM_FIELDS_DIR
  }
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
  double on = nan(""), oth = nan(""), oux = nan(""), ouy = nan(""), oz = nan("");
  if (!(st & ST_NONPHYSICAL)) {
    const float nf = df_to_float(n), ef = df_to_float(eps);
    float theta, z, g[6];
    if (EDF == EDF_MJ) {
      theta = ef / (2.0f * nf);
      z = nf / (2.0f * kPIf * theta * theta);
    } else {
      const float target = 0.5f * kPIf * ef * ef / (nf * nf * nf);
      const int zs = solve_z_R_f<EDF>(target, z, g);
      st |= zs;
      if (zs & ST_CLAMPED) theta = sqrtf(nf / (2.0f * kPIf * g[1]));
      else theta = 0.5f * g[1] / g[2] * ef / nf;
    }
    on = (double)n.hi + (double)n.lo;
    oux = (double)ux.hi + (double)ux.lo;
    ouy = (double)uy.hi + (double)uy.lo;
    oth = theta;
    oz = z;
  }
  const long long i = (a.tiles ? D.foff : 0) + (long long)y * D.nx + x;
  if (a.n) a.n[i] = on;
  if (a.theta) a.theta[i] = oth;
  if (a.ux) a.ux[i] = oux;
  if (a.uy) a.uy[i] = ouy;
  if (a.z) a.z[i] = oz;
  if (st) atomicOr(a.status, st);
}

// The mixed storages' read-out: the fields in the collision's arithmetic, or
// the FP64 kernel when diagnostics are asked for.
template <class S>
cudaError_t launch_fields_mixed_t(int edf, const FieldsArgs& a, int nx, int ny, cudaStream_t s) {
  if (a.diag) return launch_fields_t<S>(edf, a, nx, ny, s);
  const dim3 grid = launch_grid(a.tiles, a.ntiles, nx, ny);
  switch (edf) {
    case EDF_MJ: k_fields_mixed<EDF_MJ, S><<<grid, dim3(kTileW, kTileH), 0, s>>>(a); break;
    case EDF_FD: k_fields_mixed<EDF_FD, S><<<grid, dim3(kTileW, kTileH), 0, s>>>(a); break;
    default: k_fields_mixed<EDF_BE, S><<<grid, dim3(kTileW, kTileH), 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

// f = f^eq of the given fields in a mixed storage (time zero), halo included:
// the collision's FP32 equilibrium deviations (dz_moments, dfeq_shell, with the
// tables' conserved-moment defects removed) from the FP64 input fields. Its
// rounding is that of every collision of the mixed step, and it runs on the
// FP32 pipe (an FP64 initialiser costs as much as ten mixed steps on GB300).
template <int EDF, class S>
__global__ void __launch_bounds__(kThreads) k_init_mixed(InitArgs a) {
  extern __shared__ float smi[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  int dom, x, y;
  cell_of_launch(a.tiles, a.dom, dom, x, y);
  const DomDev& D = a.doms[dom];
  if (x >= D.nx || y >= D.ny) return;
  const long long i = (a.tiles ? D.foff : 0) + (long long)y * D.nx + x;
  const float theta = (float)a.theta[i], ux = (float)a.ux[i], uy = (float)a.uy[i];
  unsigned st = 0;
  float z, n, g[6];
  if (a.kind == 1) {
    z = (float)a.a[i];
    g_allf<EDF>(z, g);
    n = 2.0f * kPIf * theta * theta * g[1];
  } else {
    n = (float)a.a[i];
    st |= (theta > 0.0f && n > 0.0f) ? solve_z_nt_f<EDF>(n, theta, z, g) : 0;
  }
  const float u2 = ux * ux + uy * uy;
  const bool ok = (u2 < 1.0f) && (theta > 0.0f) && (n > 0.0f) && isfinite(z) && isfinite(u2);
  if (!ok) st |= ST_NONPHYSICAL;
  const float gam = ok ? 1.0f / sqrtf(1.0f - u2) : 1.0f;
  typename S::T* __restrict__ f = static_cast<typename S::T*>(a.f) + D.off;
  const long long c = cell_rel(D, x, y);
  float* col = smi + tid;
  if (ok) {
    float zr[21], zi[21];
    dz_moments<EDF>(D, g, theta, ux, uy, gam, -1.0f, -1.0f, zr, zi);
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
#pragma unroll 1
    for (int s = 0; s < 6; ++s) {
      float fe[12];
      dfeq_shell<EDF>(s, D.rres[s], zr, zi, fe);
#pragma unroll
      for (int d = 0; d < 12; ++d) {
        const int q = 6 * d + s;
        col[q * kThreads] = fe[d];
        f[q * kBlkW + c] = S::encf(fe[d], D, s);
      }
    }
  } else {
    for (int q = 0; q < 72; ++q) {
      col[q * kThreads] = __int_as_float(0x7fc00000);  // NaN
      f[q * kBlkW + c] = S::encf(col[q * kThreads], D, q % 6);
    }
  }
  write_halo_mixed<EDF, S>(D, x, y, f, col, ok, n, ux, uy, gam, st, true);
  if (st) atomicOr(a.status, st);
}

template <class S>
cudaError_t launch_init_mixed_t(int edf, const InitArgs& a, int nx, int ny, cudaStream_t s) {
  const dim3 grid = launch_grid(a.tiles, a.ntiles, nx, ny);
  switch (edf) {
    case EDF_MJ: k_init_mixed<EDF_MJ, S><<<grid, dim3(kTileW, kTileH), kSmemF, s>>>(a); break;
    case EDF_FD: k_init_mixed<EDF_FD, S><<<grid, dim3(kTileW, kTileH), kSmemF, s>>>(a); break;
    default: k_init_mixed<EDF_BE, S><<<grid, dim3(kTileW, kTileH), kSmemF, s>>>(a); break;
  }
  return cudaGetLastError();
}

// Reference rest equilibrium of every domain (FP64), its FP32 rounding and
// the reference moments, written into the device descriptors.
template <int EDF>
__global__ void k_prepare_refs(DomDev* doms, int ndom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndom) return;
  DomDev& D = doms[i];
  double z, g[6];
  solve_z_from_n_theta<EDF>(D.ref_n, D.ref_theta, z, g);
  double fact = 1.0, th = D.ref_theta, thp = th;
  for (int n = 0; n < 6; ++n) {
    if (n > 0) { fact *= n; thp *= th; }
    D.zref[n] = 2.0 * PI * fact * g[n] * thp * c_pnk[3 * (n * (n + 1) / 2)];
  }
  double n0 = 0.0, t00 = 0.0;
  for (int s = 0; s < 6; ++s) {
    double fe = 0.0;
    for (int n = 0; n < 6; ++n) fe += c_Q[kOrder5][EDF][qoff(0) + s * 6 + n] * D.zref[n];
    const float ff = (float)fe;
    D.fref[s] = ff;
    D.rres[s] = (float)(fe - (double)ff);
    const float as = (float)((double)ff * D.scale);
    D.a_s[s] = as;
    D.b_s[s] = 1.0f / as;
    n0 += 12.0 * (double)ff * c_p[EDF][s];
    t00 += 12.0 * (double)ff * c_p2[EDF][s];
  }
  D.n0ref = n0;
  D.t00ref = t00;
  double r1 = 0.0, r2 = 0.0;
  for (int s = 0; s < 6; ++s) {
    r1 += 12.0 * (double)D.rres[s] * (double)c_pf[EDF][s];
    r2 += 12.0 * (double)D.rres[s] * (double)c_p2f[EDF][s];
  }
  D.zeff1 = n0 + r1;
  D.zeff2 = t00 + r2;
  const double v4[4] = {D.n0ref, D.t00ref, D.zeff1, D.zeff2};
  float* pairs[4] = {D.n0_hl, D.t00_hl, D.z1_hl, D.z2_hl};
  for (int k = 0; k < 4; ++k) {
    pairs[k][0] = (float)v4[k];
    pairs[k][1] = (float)(v4[k] - (double)pairs[k][0]);
  }
  for (int n = 0; n < 6; ++n) D.zref_f[n] = (float)D.zref[n];
}

// ------------------------------------------------------------- launchers
static const double h_p2[3][6] = {RLBM_P2_MJ_INIT, RLBM_P2_FD_INIT, RLBM_P2_BE_INIT};
static const double h_pnk[63] = RLBM_PNK_INIT;
static const double h_invpow[6 * RLBM_NSERIES] = RLBM_INVPOW_INIT;
static const double h_be_exp[6 * RLBM_NEXP] = RLBM_BE_EXP_INIT;
static const double h_fd_exp[6 * RLBM_NEXP] = RLBM_FD_EXP_INIT;
static const double h_be_logcoef[6] = RLBM_BE_LOGCOEF_INIT;
static const double h_be_harm[6] = RLBM_BE_HARM_INIT;
static const double h_g_zc[6] = RLBM_G_ZC_INIT;

template <class S, int EDF>
static cudaError_t prepare_tma_t() {
  cudaError_t e = cudaFuncSetAttribute(k_step_mixed_tma<EDF, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tma_smem_bytes<S>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_step_mixed_tma<EDF, S>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

template <class S, int EDF>
static cudaError_t prepare_mixed_t() {
  cudaError_t e = cudaFuncSetAttribute(k_init_mixed<EDF, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemF);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_step_mixed<EDF, S, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemF);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_step_mixed<EDF, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemF);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_step_mixed<EDF, S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemF);
}

template <class S>
static cudaError_t prepare_s() {
  cudaError_t e;
  if ((e = prepare_mixed_t<S, EDF_MJ>())) return e;
  if ((e = prepare_mixed_t<S, EDF_FD>())) return e;
  if ((e = prepare_mixed_t<S, EDF_BE>())) return e;
  if ((e = prepare_tma_t<S, EDF_MJ>())) return e;
  if ((e = prepare_tma_t<S, EDF_FD>())) return e;
  if ((e = prepare_tma_t<S, EDF_BE>())) return e;
  if ((e = prepare_common_t<S, EDF_MJ>())) return e;
  if ((e = prepare_common_t<S, EDF_FD>())) return e;
  return prepare_common_t<S, EDF_BE>();
}

// Upload the FP32 tables of this translation unit (converted once from the FP64
// tables).
static cudaError_t upload_mixed_tables() {
  float p2f[3][6], pnk[63], inv[6 * kSerF], be[6 * kExpBEf], fd[6 * kExpFDf], lc[6], hm[6], gz[6];
  for (int e = 0; e < 3; ++e)
    for (int s = 0; s < 6; ++s) p2f[e][s] = (float)h_p2[e][s];
  for (int i = 0; i < 63; ++i) pnk[i] = (float)h_pnk[i];
  for (int nu = 0; nu < 6; ++nu) {
    for (int k = 0; k < kSerF; ++k) inv[nu * kSerF + k] = (float)h_invpow[nu * RLBM_NSERIES + k];
    for (int k = 0; k < kExpBEf; ++k) be[nu * kExpBEf + k] = (float)h_be_exp[nu * RLBM_NEXP + k];
    for (int k = 0; k < kExpFDf; ++k) fd[nu * kExpFDf + k] = (float)h_fd_exp[nu * RLBM_NEXP + k];
    lc[nu] = (float)h_be_logcoef[nu];
    hm[nu] = (float)h_be_harm[nu];
    gz[nu] = (float)h_g_zc[nu];
  }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_p2f, p2f, sizeof(p2f)))) return e;
  if ((e = cudaMemcpyToSymbol(c_pnkf, pnk, sizeof(pnk)))) return e;
  if ((e = cudaMemcpyToSymbol(c_invpowf, inv, sizeof(inv)))) return e;
  if ((e = cudaMemcpyToSymbol(c_be_expf, be, sizeof(be)))) return e;
  if ((e = cudaMemcpyToSymbol(c_fd_expf, fd, sizeof(fd)))) return e;
  if ((e = cudaMemcpyToSymbol(c_be_logcoeff, lc, sizeof(lc)))) return e;
  if ((e = cudaMemcpyToSymbol(c_be_harmf, hm, sizeof(hm)))) return e;
  return cudaMemcpyToSymbol(c_g_zcf, gz, sizeof(gz));
}


template <class S>
static cudaError_t step_s(int edf, const StepArgs& a, int grid, cudaStream_t s) {
  if (a.tmaps) {  // TMA-staged variant; without descriptors the pull goes through L1
    const size_t sm = tma_smem_bytes<S>();
    switch (edf) {
      case EDF_MJ: k_step_mixed_tma<EDF_MJ, S><<<grid, dim3(kTileW, kTileH), sm, s>>>(a); break;
      case EDF_FD: k_step_mixed_tma<EDF_FD, S><<<grid, dim3(kTileW, kTileH), sm, s>>>(a); break;
      default: k_step_mixed_tma<EDF_BE, S><<<grid, dim3(kTileW, kTileH), sm, s>>>(a); break;
    }
    return cudaGetLastError();
  }
  const dim3 blk(kTileW, kTileH);
#define RLBM_STEP_L1(H)                                                           \
  switch (edf) {                                                                  \
    case EDF_MJ: k_step_mixed<EDF_MJ, S, H><<<grid, blk, kSmemF, s>>>(a); break; \
    case EDF_FD: k_step_mixed<EDF_FD, S, H><<<grid, blk, kSmemF, s>>>(a); break; \
    default: k_step_mixed<EDF_BE, S, H><<<grid, blk, kSmemF, s>>>(a); break;     \
  }
  if (a.halo == 0) {
    RLBM_STEP_L1(0)
  } else if (a.halo == 1) {
    RLBM_STEP_L1(1)
  } else {
    RLBM_STEP_L1(2)
  }
#undef RLBM_STEP_L1
  return cudaGetLastError();
}

// The launchers of one storage format, exported by its translation unit.
struct MixedUnit {
  cudaError_t (*prepare)();
  cudaError_t (*step)(int edf, const StepArgs& a, int grid, cudaStream_t s);
  cudaError_t (*init)(int edf, const InitArgs& a, int nx, int ny, cudaStream_t s);
  cudaError_t (*fields)(int edf, const FieldsArgs& a, int nx, int ny, cudaStream_t s);
  cudaError_t (*copy)(const CopyArgs& a, cudaStream_t s);
};

// Tables of this unit, shared-memory limits of its kernels.
template <class S>
static cudaError_t prepare_unit() {
  cudaError_t e = upload_mixed_tables();
  return e != cudaSuccess ? e : prepare_s<S>();
}

template <class S>
constexpr MixedUnit mixed_unit() {
  return MixedUnit{&prepare_unit<S>, &step_s<S>, &launch_init_mixed_t<S>, &launch_fields_mixed_t<S>,
                   &launch_copy_t<S>};
}

extern const MixedUnit kMixedF32, kMixedF32Dev, kMixedBF16, kMixedF16;

}  // namespace rlbm
