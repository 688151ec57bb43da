/*
 * Oracle for the fully dissipative 2D ultra-relativistic lattice Boltzmann
 * method (arXiv:1709.09073). TEST INFRASTRUCTURE ONLY: a plain, slow FP64 CPU
 * restatement of the paper used to check the CUDA path; only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Every function follows one passage of the paper (cited in its comment) and
 * is written for a reader checking it against the paper by eye: no blocking,
 * no fusion, FP64 throughout. Where the paper is silent, the reading used is
 * stated next to the code.
 *
 * Parity status of each part (what pins it, in tests/test_oracle_*.py):
 *   quadrature tables      pinned: printed nodes/weights (Sec. 2.4), Gauss-Laguerre,
 *                          moment identities, degree-10 exactness
 *   orc_g                  pinned: mpmath polylog at many points
 *   orc_eq_moments         pinned: the Appendix closed forms I_2^{mnq}; brute-force 2D integrals
 *   orc_feq                pinned: Fig. 1 errors (18.5 % / 1.8 %), moment reproduction
 *   orc_landau/orc_state   pinned: numpy eigen-decomposition; equilibrium round trip
 *   orc_step               pinned: conservation of N^0, T^{mu 0}; rest state fixed point;
 *                          mirror/rotation symmetry; Taylor-Green viscosity law (Eq. 31)
 *   orc_diagnostics        pinned: zero at equilibrium; pi^{x..x} against the Appendix moments;
 *                          heat flux by the conductivity law kappa = 3 tau g_3 / (2 g_2), Sec. 3.3
 *   orc_feq_order          pinned: moments of degree <= N reproduced; equals the order-N
 *                          expansion of Fig. 1 (orc_expansion_at) at the nodes
 *   local tau (eta_s)      pinned: a uniform-theta state equals the constant-tau run
 *   orc_step_rows,         pinned: slabs stepped with their neighbours' edge rows equal
 *   orc_edge_row           orc_step of the whole domain bit for bit
 */
#include "rlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "quadrature_tables.h"

#define PI 3.14159265358979323846264338327950288
#define Z_C (1.0 - 1.0e-7) /* BE reference fugacity z_c = 1 - 10^-7, Eq. (15) */
#define NPHI 256           /* trapezoid points for the angular moment integrals */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Compensated (Neumaier) summation step. */
static void neumaier_add(double *sum, double *comp, double x) {
  double t = *sum + x;
  if (fabs(*sum) >= fabs(x)) *comp += (*sum - t) + x;
  else *comp += (x - t) + *sum;
  *sum = t;
}

/* ------------------------------------------------------------------ lattice */

/* d2v72 (Sec. 2.4): 12 directions phi_d = d pi/6 (roots of sin 6 phi) times the
 * six shell momenta of the radial Gauss rule of each weight function. The
 * direction cosines are the exact values {0, +-1/2, +-sqrt(3)/2, +-1}. */
void orc_lattice(int edf, double p[6], double w[6], double cphi[12], double sphi[12]) {
  const double h = 0.5 * sqrt(3.0);
  const double c[12] = {1.0, h, 0.5, 0.0, -0.5, -h, -1.0, -h, -0.5, 0.0, 0.5, h};
  const double s[12] = {0.0, 0.5, h, 1.0, h, 0.5, 0.0, -0.5, -h, -1.0, -h, -0.5};
  for (int i = 0; i < 6; ++i) {
    if (p) p[i] = ORC_SHELL_P[edf][i];
    if (w) w[i] = ORC_SHELL_W[edf][i];
  }
  for (int d = 0; d < 12; ++d) {
    if (cphi) cphi[d] = c[d];
    if (sphi) sphi[d] = s[d];
  }
}

/* ------------------------------------------------------------- polylogarithms */

/* Bernoulli numbers B_{2j}, j = 0..15 (B_0 = 1), as exact rationals. The
 * expansions below never ask beyond B_30 (NAN if they did). */
static double bernoulli_even(int j) {
  if (j < 0 || j > 15) return NAN;
  static const double num[16] = {1.0, 1.0, -1.0, 1.0, -1.0, 5.0, -691.0, 7.0, -3617.0, 43867.0,
                                 -174611.0, 854513.0, -236364091.0, 8553103.0, -23749461029.0,
                                 8615841276005.0};
  static const double den[16] = {1.0, 6.0, 30.0, 42.0, 30.0, 66.0, 2730.0, 6.0, 510.0, 798.0,
                                 330.0, 138.0, 2730.0, 6.0, 870.0, 14322.0};
  return num[j] / den[j];
}

/* Riemann zeta at an integer s != 1 (s <= 7): zeta(-m) = -B_{m+1}/(m+1), zeta(0) = -1/2. */
static double zeta_int(int s) {
  static const double zpos[8] = {0, 0, 1.6449340668482264365, 1.2020569031595942854,
                                 1.0823232337111381915, 1.0369277551433699263,
                                 1.0173430619844491397, 1.0083492773819228268};
  if (s >= 2) return zpos[s];
  if (s == 0) return -0.5;
  int m = -s; /* s = -m, m >= 1 */
  if ((m + 1) % 2) return 0.0; /* B_odd = 0 beyond B_1 */
  return -bernoulli_even((m + 1) / 2) / (double)(m + 1);
}

/* Dirichlet eta at an integer s: eta(1) = ln 2, eta(s) = (1 - 2^{1-s}) zeta(s). */
static double eta_int(int s) {
  if (s == 1) return log(2.0);
  return (1.0 - ldexp(1.0, 1 - s)) * zeta_int(s);
}

/* Li_nu(x) for |x| <= 1/2 by its defining power series sum x^k / k^nu. */
static double li_series(int nu, double x) {
  double sum = 0.0, xk = 1.0;
  for (int k = 1; k < 200; ++k) {
    xk *= x;
    double t = xk / pow((double)k, (double)nu);
    sum += t;
    if (fabs(t) < 1e-20 * fabs(sum)) break;
  }
  return sum;
}

/* g_nu(z) of Eq. (12). MJ: z. BE: Li_nu(z) for 0 <= z < 1. FD: -Li_nu(-z), z >= 0.
 * Near |x| = 1 the standard expansions in mu = ln z are used:
 *   Li_nu(e^mu)   = sum_{k != nu-1} zeta(nu-k) mu^k/k! + mu^{nu-1}/(nu-1)! [H_{nu-1} - ln(-mu)]
 *   -Li_nu(-e^mu) = sum_k eta(nu-k) mu^k/k!                         (|mu| < pi)
 * and for FD with z > 2 the inversion formula
 *   -Li_nu(-z) = (-1)^nu Li_nu(-1/z) + (ln z)^nu/nu! + 2 sum_{j<=nu/2} eta(2j)(ln z)^{nu-2j}/(nu-2j)! */
double orc_g(int edf, int nu, double z) {
  if (edf == ORC_MJ) return z;
  if (edf == ORC_BE) {
    if (!(z < 1.0) || z < 0.0) return NAN;
    if (z <= 0.5) return li_series(nu, z);
    double mu = log(z);
    double sum = 0.0, term = 1.0; /* term = mu^k / k!; |mu| < ln 2 so 30 terms suffice */
    for (int k = 0; k <= 30; ++k) {
      if (k > 0) term *= mu / k;
      if (k == nu - 1) {
        double H = 0.0;
        for (int j = 1; j <= nu - 1; ++j) H += 1.0 / j;
        sum += term * (H - log(-mu));
      } else {
        sum += zeta_int(nu - k) * term;
      }
    }
    return sum;
  }
  /* FD */
  if (z < 0.0) return NAN;
  if (z <= 0.5) return -li_series(nu, -z);
  if (z <= 2.0) {
    double mu = log(z);
    double sum = 0.0, term = 1.0;
    for (int k = 0; k <= 30; ++k) {
      if (k > 0) term *= mu / k;
      sum += eta_int(nu - k) * term;
    }
    return sum;
  }
  double L = log(z);
  double r = ((nu % 2) ? -1.0 : 1.0) * li_series(nu, -1.0 / z);
  double fact = 1.0;
  for (int j = 2; j <= nu; ++j) fact *= j;
  r += pow(L, nu) / fact;
  for (int j = 1; 2 * j <= nu; ++j) {
    double f2 = 1.0;
    for (int i = 2; i <= nu - 2 * j; ++i) f2 *= i;
    r += 2.0 * eta_int(2 * j) * pow(L, nu - 2 * j) / f2;
  }
  return r;
}

/* ------------------------------------------------------------ Landau frame */

/* Eq. (21): T^a_b U^b = eps U^a with T^a_b = T^{ag} eta_{gb}, eta = diag(1,-1,-1),
 * solved with the power method the paper names. Reading (the paper gives no
 * start vector or stopping rule): start from U = (1, 0, 0); each iterate is
 * scaled to (1, u); stop when the change of u is 0 or no longer decreases
 * below 1e-13 (the floating-point noise floor); at most 400 iterations. */
int orc_landau(const double T[6], double *eps, double U[3], int *iters) {
  const double A[3][3] = {{T[0], -T[1], -T[2]}, {T[1], -T[3], -T[4]}, {T[2], -T[4], -T[5]}};
  double ux = 0.0, uy = 0.0, dprev = INFINITY;
  int st = 0, it;
  for (it = 1; it <= 400; ++it) {
    double y0 = A[0][0] + A[0][1] * ux + A[0][2] * uy;
    double y1 = A[1][0] + A[1][1] * ux + A[1][2] * uy;
    double y2 = A[2][0] + A[2][1] * ux + A[2][2] * uy;
    if (!(y0 > 0.0)) { st |= ORC_E_NONPHYSICAL; break; }
    double nx = y1 / y0, ny = y2 / y0;
    double d = fmax(fabs(nx - ux), fabs(ny - uy));
    ux = nx;
    uy = ny;
    if (d == 0.0) break;
    if (d < 1e-13 && d >= dprev) break;
    dprev = d;
  }
  if (it > 400) st |= ORC_W_LANDAU_MAXITER;
  if (iters) *iters = it;
  double u2 = ux * ux + uy * uy;
  if (!(u2 < 1.0)) { st |= ORC_E_NONPHYSICAL; u2 = 0.0; ux = uy = 0.0; }
  double g = 1.0 / sqrt(1.0 - u2);
  U[0] = g; U[1] = g * ux; U[2] = g * uy;
  /* eps = U_a T^{ab} U_b with U_a = eta_ab U^b */
  *eps = T[0] * U[0] * U[0] - 2.0 * T[1] * U[0] * U[1] - 2.0 * T[2] * U[0] * U[2] +
         T[3] * U[1] * U[1] + 2.0 * T[4] * U[1] * U[2] + T[5] * U[2] * U[2];
  return st;
}

/* ------------------------------------------------------- state (n, theta, z) */

/* R(z) = g_3(z)^2 / g_2(z)^3, which equals (pi/2) eps^2 / n^3 by Eq. (25). */
static double R_of_mu(int edf, double mu) {
  double z = exp(mu);
  double g2 = orc_g(edf, 2, z), g3 = orc_g(edf, 3, z);
  return g3 * g3 / (g2 * g2 * g2);
}

/* Solve h(mu) = target for a decreasing h by bisection on [lo, hi] to the last bit. */
static double bisect_decreasing(int edf, int which, double target, double lo, double hi, double theta2) {
  for (int i = 0; i < 200; ++i) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double v;
    if (which == 0) v = R_of_mu(edf, mid);
    else v = -orc_g(edf, 2, exp(mid)); /* g_2 increasing -> -g_2 decreasing */
    (void)theta2;
    if (v > target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Fugacity from (n, theta) with n = 2 pi theta^2 g_2(z), Eq. (25). */
int orc_z_from_n_theta(int edf, double n, double theta, double *z) {
  double g2t = n / (2.0 * PI * theta * theta);
  if (!(g2t > 0.0) || !isfinite(g2t)) { *z = NAN; return ORC_E_NONPHYSICAL; }
  if (edf == ORC_MJ) { *z = g2t; return 0; }
  double hi = (edf == ORC_BE) ? log(Z_C) : 60.0;
  if (edf == ORC_BE && g2t >= orc_g(ORC_BE, 2, Z_C)) { *z = Z_C; return ORC_W_CLAMPED_FUGACITY; }
  double mu = bisect_decreasing(edf, 1, -g2t, -60.0, hi, 0.0);
  *z = exp(mu);
  return 0;
}

/* Macroscopic state, Eqs. (21)-(25): Landau solve, n = U_mu N^mu, then
 *   MJ:    g_nu = z, so theta = eps/(2n) and z = n/(2 pi theta^2);
 *   FD/BE: (reading; the paper does not say how z is found) z solves
 *          g_3^2/g_2^3 = (pi/2) eps^2/n^3 and theta = (1/2)(g_2/g_3)(eps/n), Eq. (24).
 *   BE clamp (reading): if the target lies below R(z_c), z = z_c, n is kept and
 *          theta follows from n = 2 pi theta^2 g_2(z_c); flagged as a warning. */
int orc_state(int edf, const double N[3], const double T[6], double out[6]) {
  double eps, U[3];
  int st = orc_landau(T, &eps, U, NULL);
  double n = U[0] * N[0] - U[1] * N[1] - U[2] * N[2];
  double ux = U[1] / U[0], uy = U[2] / U[0];
  double theta, z;
  if (!(n > 0.0) || !(eps > 0.0) || !isfinite(n) || !isfinite(eps)) {
    st |= ORC_E_NONPHYSICAL;
    theta = z = NAN;
  } else if (edf == ORC_MJ) {
    theta = eps / (2.0 * n);
    z = n / (2.0 * PI * theta * theta);
  } else {
    double target = 0.5 * PI * eps * eps / (n * n * n);
    if (edf == ORC_BE && target < R_of_mu(ORC_BE, log(Z_C))) {
      z = Z_C;
      theta = sqrt(n / (2.0 * PI * orc_g(ORC_BE, 2, Z_C)));
      st |= ORC_W_CLAMPED_FUGACITY;
    } else {
      double hi = (edf == ORC_BE) ? log(Z_C) : 60.0;
      double mu = bisect_decreasing(edf, 0, target, -60.0, hi, 0.0);
      z = exp(mu);
      theta = 0.5 * orc_g(edf, 2, z) / orc_g(edf, 3, z) * eps / n;
    }
  }
  out[0] = n; out[1] = theta; out[2] = ux; out[3] = uy; out[4] = z; out[5] = eps;
  return st;
}

/* ----------------------------------------------------- equilibrium moments */



void orc_basis(int n[36], int k[36], int c[36]) {
  int a = 0;
  for (int nn = 0; nn <= 5; ++nn)
    for (int kk = 0; kk <= nn; ++kk)
      for (int cc = 0; cc <= (kk > 0 ? 1 : 0); ++cc) {
        n[a] = nn; k[a] = kk; c[a] = cc; ++a;
      }
}

static int basis_n[36], basis_k[36], basis_c[36];
static double trap_cos[NPHI], trap_sin[NPHI], trap_trig[36][NPHI];
static int tables_ready;

/* Basis list and the trapezoid's trigonometric table, built once. */
static void ensure_tables(void) {
#pragma omp critical(orc_tables)
  {
    if (!tables_ready) {
      orc_basis(basis_n, basis_k, basis_c);
      for (int j = 0; j < NPHI; ++j) {
        double ph = 2.0 * PI * j / NPHI;
        trap_cos[j] = cos(ph);
        trap_sin[j] = sin(ph);
        for (int a = 0; a < 36; ++a)
          trap_trig[a][j] = basis_c[a] ? sin(basis_k[a] * ph) : cos(basis_k[a] * ph);
      }
      tables_ready = 1;
    }
  }
}

/* Appendix: the moments of f^eq on the light cone separate into a radial EDF
 * integral and an angular one,
 *   int dp dphi f^eq p^n trig(k phi)
 *     = Gamma(n+1) g_{n+1}(z) theta^{n+1} int dphi trig(k phi) / [gamma (1 - v.u)]^{n+1},
 * (the identity before Eq. A.2). The angular integral of this smooth periodic
 * function is taken with the NPHI-point trapezoid rule, which is exact to
 * round-off for |u| <= 0.95. */
/* The Appendix closed forms I_2^{m a b} = int d^2p/p^0 f^eq p^m (p^x)^a (p^y)^b,
 * m + a + b <= 5, as printed (56 forms). tg2 and tg3 stand for theta^2 g_2(z)
 * and theta^3 g_3(z); the caller may set them from n and eps through Eq. (25)
 * (tg2 = n / (2 pi), tg3 = eps / (4 pi)). */
static double pw(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

static void appendix_I2(int edf, double tg2, double tg3, double th, double ux, double uy, double z,
                        double I[6][6][6]) {
  const double pi = PI;
  const double u2 = ux * ux + uy * uy, gam = 1.0 / sqrt(1.0 - u2);
  const double g1 = orc_g(edf, 1, z), g2 = orc_g(edf, 2, z), g3 = orc_g(edf, 3, z);
  const double g4 = orc_g(edf, 4, z), g5 = orc_g(edf, 5, z), g6 = orc_g(edf, 6, z);
  (void)g2;
  (void)g3;
  I[0][0][0] = 2*pi*th*g1;
  I[1][0][0] = 2*pi*tg2*gam;
  I[2][0][0] = 2*pi*tg3*(2 + u2)*pw(gam, 2);
  I[3][0][0] = 6*pi*pw(th, 4)*g4*(2 + 3*u2)*pw(gam, 3);
  I[4][0][0] = 6*pi*(8 + 24*u2 + 3*pw(u2, 2))*pw(th, 5)*g5*pw(gam, 4);
  I[0][1][0] = 2*pi*tg2*ux*gam;
  I[0][2][0] = 2*pi*tg3*(1 - u2 + 3*ux*ux)*pw(gam, 2);
  I[0][3][0] = 6*pi*pw(th, 4)*g4*(3*(1 - u2)*ux + 5*pw(ux, 3))*pw(gam, 3);
  I[0][4][0] = 6*pi*(3 + 3*pw(u2, 2) + 30*pw(ux, 2) + 35*pw(ux, 4) - 6*u2*(1 + 5*pw(ux, 2)))*pw(th, 5)*g5*pw(gam, 4);
  I[0][0][1] = 2*pi*tg2*uy*gam;
  I[0][0][2] = 2*pi*tg3*(1 - u2 + 3*uy*uy)*pw(gam, 2);
  I[0][0][3] = 6*pi*pw(th, 4)*g4*(3*(1 - u2)*uy + 5*pw(uy, 3))*pw(gam, 3);
  I[0][0][4] = 6*pi*(3 + 3*pw(u2, 2) + 30*pw(uy, 2) + 35*pw(uy, 4) - 6*u2*(1 + 5*pw(uy, 2)))*pw(th, 5)*g5*pw(gam, 4);
  I[2][2][0] = 6*pi*(4 - 3*u2 - pw(u2, 2) + 5*pw(ux, 2)*(6 + u2))*pw(th, 5)*g5*pw(gam, 4);
  I[1][2][0] = 6*pi*pw(th, 4)*g4*((1 - u2) + 5*ux*ux)*pw(gam, 3);
  I[2][0][2] = 6*pi*(4 - 3*u2 - pw(u2, 2) + 5*pw(uy, 2)*(6 + u2))*pw(th, 5)*g5*pw(gam, 4);
  I[1][0][2] = 6*pi*pw(th, 4)*g4*((1 - u2) + 5*uy*uy)*pw(gam, 3);
  I[0][2][2] = 6*pi*((1 - u2) + 4*(1 - u2)*u2 + 35*pw(ux, 2)*pw(uy, 2))*pw(th, 5)*g5*pw(gam, 4);
  I[0][3][1] = 30*pi*pw(th, 5)*g5*(3*(1 - u2) + 7*pw(ux, 2))*ux*uy*pw(gam, 4);
  I[2][1][1] = 30*pi*(6 + u2)*pw(th, 5)*g5*ux*uy*pw(gam, 4);
  I[0][1][1] = 6*pi*tg3*ux*uy*pw(gam, 2);
  I[1][1][1] = 6*pi*pw(th, 4)*g4*(5*ux*uy)*pw(gam, 3);
  I[1][3][0] = -30*pi*ux*(-3 + 3*u2 - 7*pw(ux, 2))*pw(th, 5)*g5*pw(gam, 4);
  I[3][1][0] = 30*pi*(4 + 3*u2)*pw(th, 5)*ux*g5*pw(gam, 4);
  I[1][1][0] = 6*pi*tg3*ux*pw(gam, 2);
  I[1][0][1] = 6*pi*tg3*uy*pw(gam, 2);
  I[0][1][3] = 30*pi*pw(th, 5)*g5*(3*(1 - u2) + 7*pw(uy, 2))*ux*uy*pw(gam, 4);
  I[1][0][3] = -30*pi*uy*(-3 + 3*u2 - 7*pw(uy, 2))*pw(th, 5)*g5*pw(gam, 4);
  I[1][2][1] = -30*pi*(-1 + u2 - 7*pw(ux, 2))*uy*pw(th, 5)*g5*pw(gam, 4);
  I[2][0][1] = 6*pi*pw(th, 4)*g4*(4 + u2)*uy*pw(gam, 3);
  I[3][0][1] = 30*pi*(4 + 3*u2)*pw(th, 5)*uy*g5*pw(gam, 4);
  I[0][2][1] = 6*pi*pw(th, 4)*g4*((1 - u2) + 5*ux*ux)*uy*pw(gam, 3);
  I[1][1][2] = -30*pi*(-1 + u2 - 7*pw(uy, 2))*ux*pw(th, 5)*g5*pw(gam, 4);
  I[2][1][0] = 6*pi*pw(th, 4)*g4*(4 + u2)*ux*pw(gam, 3);
  I[0][1][2] = 6*pi*pw(th, 4)*g4*((1 - u2) + 5*uy*uy)*ux*pw(gam, 3);
  I[0][5][0] = 30*pi*ux*(15*pw((1 - u2), 2) + 70*pw(ux, 2)*(1 - u2) + 63*pw(ux, 4))*pw(th, 6)*g6*pw(gam, 5);
  I[0][0][5] = 30*pi*uy*(15*pw((1 - u2), 2) + 70*pw(uy, 2)*(1 - u2) + 63*pw(uy, 4))*pw(th, 6)*g6*pw(gam, 5);
  I[5][0][0] = 30*pi*(8 + 40*u2 + 15*pw(u2, 2))*pw(th, 6)*g6*pw(gam, 5);
  I[2][3][0] = 30*pi*ux*(18 - 3*pw(u2, 2) + 56*pw(ux, 2) + u2*(-15 + 7*pw(ux, 2)))*pw(th, 6)*g6*pw(gam, 5);
  I[2][0][3] = 30*pi*uy*(18 - 3*pw(u2, 2) + 56*pw(uy, 2) + u2*(-15 + 7*pw(uy, 2)))*pw(th, 6)*g6*pw(gam, 5);
  I[0][4][1] = 90*pi*(pw((1 - u2), 2) + 14*pw(ux, 2)*(1 - u2) + 21*pw(ux, 4))*uy*pw(th, 6)*g6*pw(gam, 5);
  I[2][2][1] = -30*pi*(-6*(1 - u2) - u2*(1 - u2) - 56*pw(ux, 2) + u2*(-7*pw(ux, 2)))*uy*pw(th, 6)*g6*pw(gam, 5);
  I[0][1][4] = 90*pi*(pw((1 - u2), 2) + 14*pw(uy, 2)*(1 - u2) + 21*pw(uy, 4))*ux*pw(th, 6)*g6*pw(gam, 5);
  I[0][3][2] = -30*pi*ux*(pw(ux, 2)*(-1 + 4*u2 - 63*pw(uy, 2)) + 3*(-1 + (-5 + 6*u2)*pw(uy, 2)))*pw(th, 6)*g6*pw(gam, 5);
  I[2][1][2] = -30*pi*(-6*(1 - u2) - u2*(1 - u2) - 56*pw(uy, 2) + u2*(-7*pw(uy, 2)))*ux*pw(th, 6)*g6*pw(gam, 5);
  I[4][1][0] = 90*pi*ux*(8 + 12*u2 + pw(u2, 2))*pw(th, 6)*g6*pw(gam, 5);
  I[0][2][3] = -30*pi*uy*(pw(uy, 2)*(-1 + 4*u2 - 63*pw(ux, 2)) + 3*(-1 + (-5 + 6*u2)*pw(ux, 2)))*pw(th, 6)*g6*pw(gam, 5);
  I[4][0][1] = 90*pi*uy*(8 + 12*u2 + pw(u2, 2))*pw(th, 6)*g6*pw(gam, 5);
  I[1][4][0] = 90*pi*(pw((1 - u2), 2) + 14*pw(ux, 2)*(1 - u2) + 21*pw(ux, 4))*pw(th, 6)*g6*pw(gam, 5);
  I[3][2][0] = -30*pi*(-4*(1 - u2) - 3*u2*(1 - u2) - 42*pw(ux, 2) + u2*(-21*pw(ux, 2)))*pw(th, 6)*g6*pw(gam, 5);
  I[1][0][4] = 90*pi*(pw((1 - u2), 2) + 14*pw(uy, 2)*(1 - u2) + 21*pw(uy, 4))*pw(th, 6)*g6*pw(gam, 5);
  I[3][0][2] = -30*pi*(-4*(1 - u2) - 3*u2*(1 - u2) - 42*pw(uy, 2) + u2*(-21*pw(uy, 2)))*pw(th, 6)*g6*pw(gam, 5);
  I[1][2][2] = -30*pi*(-1 + u2 - 6*u2*(1 - u2) - 63*pw(ux, 2)*pw(uy, 2))*pw(th, 6)*g6*pw(gam, 5);
  I[1][3][1] = -630*pi*ux*(-1 + u2 - 3*pw(ux, 2))*uy*pw(th, 6)*g6*pw(gam, 5);
  I[3][1][1] = 315*pi*(2 + u2)*pw(th, 6)*g6*2*ux*uy*pw(gam, 5);
  I[1][1][3] = -630*pi*uy*(-1 + u2 - 3*pw(uy, 2))*ux*pw(th, 6)*g6*pw(gam, 5);
}

/* Harmonic moments int dp dphi f^eq p^n trig(k phi) from the monomial closed
 * forms: p^n e^{i k phi} = p^{n-k} (p^x + i p^y)^k, expanded binomially. */
static void harmonic_from_I2(const double I[6][6][6], double M[36]) {
  for (int a = 0; a < 36; ++a) {
    const int n = basis_n[a], k = basis_k[a], c = basis_c[a];
    double sum = 0.0, binom = 1.0;
    for (int j = 0; j <= k; ++j) {
      if (j > 0) binom = binom * (k - j + 1) / j;
      /* i^j: real for even j (sign (-1)^(j/2)), imaginary for odd j (sign (-1)^((j-1)/2)) */
      if ((j % 2 == 0) == (c == 0)) {
        const double sign = ((j / 2) % 2) ? -1.0 : 1.0;
        sum += sign * binom * I[n - k][k - j][j];
      }
    }
    M[a] = sum;
  }
}

/* The 36 equilibrium moments in the harmonic basis from the Appendix closed
 * forms (the paper's own route to the projections, Eq. 11). */
void orc_eq_moments(int edf, double theta, double ux, double uy, double z, double M[36]) {
  orc_eq_moments_ne(edf, -1.0, -1.0, theta, ux, uy, z, M);
}

/* As orc_eq_moments, with the degree-1 and degree-2 radial factors written
 * through Eq. (25) from the given n and eps (ignored when negative), so that the
 * collision reproduces the cell's own n and eps exactly, up to rounding. */
void orc_eq_moments_ne(int edf, double n, double eps, double theta, double ux, double uy, double z,
                       double M[36]) {
  ensure_tables();
  double I[6][6][6];
  const double tg2 = n >= 0.0 ? n / (2.0 * PI) : theta * theta * orc_g(edf, 2, z);
  const double tg3 = eps >= 0.0 ? eps / (4.0 * PI) : theta * theta * theta * orc_g(edf, 3, z);
  memset(I, 0, sizeof(I));
  appendix_I2(edf, tg2, tg3, theta, ux, uy, z, I);
  harmonic_from_I2(I, M);
}

/* The same moments by direct quadrature of their definition: the radial EDF
 * integral Gamma(n+1) g_{n+1}(z) theta^{n+1} (identity before Eq. A.2) times the
 * angular integral of trig(k phi) / [gamma (1 - v.u)]^{n+1} with the NPHI-point
 * trapezoid rule (exact to round-off for |u| <= 0.95). A check of the closed
 * forms that uses nothing from them. */
void orc_eq_moments_quad(int edf, double theta, double ux, double uy, double z, double M[36]) {
  ensure_tables();
  double gamma = 1.0 / sqrt(1.0 - ux * ux - uy * uy);
  double ang[36], comp[36];
  for (int a = 0; a < 36; ++a) ang[a] = comp[a] = 0.0;
  for (int j = 0; j < NPHI; ++j) {
    double r = 1.0 / (gamma * (1.0 - ux * trap_cos[j] - uy * trap_sin[j]));
    double rp[7];
    rp[0] = 1.0;
    for (int e = 1; e <= 6; ++e) rp[e] = rp[e - 1] * r;
    for (int a = 0; a < 36; ++a) neumaier_add(&ang[a], &comp[a], trap_trig[a][j] * rp[basis_n[a] + 1]);
  }
  for (int a = 0; a < 36; ++a) {
    double fact = 1.0;
    for (int i = 2; i <= basis_n[a]; ++i) fact *= i;
    M[a] = fact * orc_g(edf, basis_n[a] + 1, z) * pow(theta, basis_n[a] + 1) * (2.0 * PI / NPHI) *
           (ang[a] + comp[a]);
  }
}

/* ------------------------------------------------ discrete equilibrium f^eq */

/* Gram matrix of the basis p^n trig(k phi) under the d2v72 weights, its
 * Cholesky factor and the basis values at the 72 nodes, per EDF (built once). */
static double gram_G[3][36][36];
static double gram_L[3][36][36];
static double node_phi[3][72][36];
static int gram_ready[3];

static void ensure_gram(int edf) {
  ensure_tables();
#pragma omp critical(orc_gram)
  {
    if (!gram_ready[edf]) {
      double p[6], w[6], cphi[12], sphi[12];
      orc_lattice(edf, p, w, cphi, sphi);
      /* basis value at node q = 6d + s: p_s^n trig(k phi_d); trig(k phi_d) is
       * read from the exact direction table at index k d mod 12 */
      for (int d = 0; d < 12; ++d)
        for (int s = 0; s < 6; ++s)
          for (int a = 0; a < 36; ++a) {
            int j = (basis_k[a] * d) % 12;
            node_phi[edf][6 * d + s][a] = pow(p[s], basis_n[a]) * (basis_c[a] ? sphi[j] : cphi[j]);
          }
      double G[36][36];
      for (int a = 0; a < 36; ++a)
        for (int b = 0; b < 36; ++b) {
          /* compensated: G is used for every cell, so its rounding must not bias the
           * equilibrium's moments */
          double sum = 0.0, comp = 0.0;
          for (int q = 0; q < 72; ++q) neumaier_add(&sum, &comp, w[q % 6] * node_phi[edf][q][a] * node_phi[edf][q][b]);
          G[a][b] = sum + comp;
          gram_G[edf][a][b] = sum + comp;
        }
      /* Cholesky G = L L^T */
      double (*L)[36] = gram_L[edf];
      memset(L, 0, sizeof(double) * 36 * 36);
      for (int j = 0; j < 36; ++j) {
        double sum = G[j][j];
        for (int k = 0; k < j; ++k) sum -= L[j][k] * L[j][k];
        L[j][j] = sqrt(sum);
        for (int i = j + 1; i < 36; ++i) {
          double t = G[i][j];
          for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
          L[i][j] = t / L[j][j];
        }
      }
      gram_ready[edf] = 1;
    }
  }
}

/* Solve L L^T x = b (forward then backward substitution). */
static void cholesky_solve(const double (*L)[36], const double b[36], double x[36]) {
  double y[36];
  for (int i = 0; i < 36; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = 35; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 36; ++k) s -= L[k][i] * x[k];
    x[i] = s / L[i][i];
  }
}

/* Eqs. (10)-(11) read as an orthogonal projection (the 36 relativistic
 * polynomials P^{i..}, P^{i..0} of degree <= 5 span the same space as
 * p^n {cos, sin}(k phi), 0 <= k <= n <= 5, and are orthonormal under
 * int d^2p/p^0 omega): f^eq_i = w_i sum_ab phi_a(p_i) (G^{-1})_ab M_b with the
 * continuous moments M_b of f^eq. The quadrature is exact to degree 10, so the
 * discrete f^eq reproduces every moment of degree <= 5. */
void orc_feq(int edf, double theta, double ux, double uy, double z, double feq[72]) {
  orc_feq_ne(edf, -1.0, -1.0, theta, ux, uy, z, feq);
}

void orc_feq_ne(int edf, double n, double eps, double theta, double ux, double uy, double z,
                double feq[72]) {
  ensure_gram(edf);
  double M[36], c[36], r[36], dc[36];
  orc_eq_moments_ne(edf, n, eps, theta, ux, uy, z, M);
  const double (*L)[36] = (const double (*)[36])gram_L[edf];
  const double (*G)[36] = (const double (*)[36])gram_G[edf];
  /* G c = M by Cholesky, then one step of iterative refinement (r = M - G c,
   * G dc = r, c += dc): the refined c reproduces the moments M to rounding, so
   * the discrete equilibrium carries no systematic defect in N^0, T^{mu 0}. */
  cholesky_solve(L, M, c);
  for (int i = 0; i < 36; ++i) {
    double sum = M[i];
    for (int k = 0; k < 36; ++k) sum -= G[i][k] * c[k];
    r[i] = sum;
  }
  cholesky_solve(L, r, dc);
  for (int i = 0; i < 36; ++i) c[i] += dc[i];
  double w[6];
  orc_lattice(edf, NULL, w, NULL, NULL);
  for (int q = 0; q < 72; ++q) {
    /* compensated: the terms cancel strongly on the outer shells */
    double v = 0.0, cv = 0.0;
    for (int a = 0; a < 36; ++a) neumaier_add(&v, &cv, node_phi[edf][q][a] * c[a]);
    feq[q] = w[q % 6] * (v + cv);
  }
}

/* Order-N equilibrium (Eq. 10 truncated at N, Sec. 3.5): the same least-squares
 * projection as orc_feq_ne restricted to the basis functions with n <= N. The
 * Gram matrix of the retained functions is solved by Gaussian elimination with
 * partial pivoting, then one refinement step. */
void orc_feq_order(int edf, int order, double n, double eps, double theta, double ux, double uy, double z,
                   double feq[72]) {
  if (order <= 0 || order >= 5) {
    orc_feq_ne(edf, n, eps, theta, ux, uy, z, feq);
    return;
  }
  ensure_gram(edf);
  int nb = 0, idx[36];
  for (int a = 0; a < 36; ++a)
    if (basis_n[a] <= order) idx[nb++] = a;
  double M[36], w[6];
  orc_eq_moments_ne(edf, n, eps, theta, ux, uy, z, M);
  orc_lattice(edf, NULL, w, NULL, NULL);
  double G[36][36], A[36][37], c[36] = {0}, r[36];
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      double sum = 0.0;
      for (int q = 0; q < 72; ++q) sum += w[q % 6] * node_phi[edf][q][idx[i]] * node_phi[edf][q][idx[j]];
      G[i][j] = sum;
    }
  for (int pass = 0; pass < 2; ++pass) {
    /* right-hand side: the moments (pass 0), then the residual M - G c (pass 1) */
    for (int i = 0; i < nb; ++i) {
      double rhs = M[idx[i]];
      if (pass)
        for (int j = 0; j < nb; ++j) rhs -= G[i][j] * c[j];
      for (int j = 0; j < nb; ++j) A[i][j] = G[i][j];
      A[i][nb] = rhs;
    }
    for (int col = 0; col < nb; ++col) {
      int piv = col;
      for (int rr = col + 1; rr < nb; ++rr)
        if (fabs(A[rr][col]) > fabs(A[piv][col])) piv = rr;
      for (int j = 0; j <= nb; ++j) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
      for (int rr = col + 1; rr < nb; ++rr) {
        double m = A[rr][col] / A[col][col];
        for (int j = col; j <= nb; ++j) A[rr][j] -= m * A[col][j];
      }
    }
    for (int i = nb - 1; i >= 0; --i) {
      double sum = A[i][nb];
      for (int j = i + 1; j < nb; ++j) sum -= A[i][j] * r[j];
      r[i] = sum / A[i][i];
    }
    for (int i = 0; i < nb; ++i) c[i] += r[i];
  }
  for (int q = 0; q < 72; ++q) {
    double v = 0.0, cv = 0.0;
    for (int i = 0; i < nb; ++i) neumaier_add(&v, &cv, node_phi[edf][q][idx[i]] * c[i]);
    feq[q] = w[q % 6] * (v + cv);
  }
}

/* Value of the order-N expansion of Eq. (10) at an arbitrary momentum (p, phi):
 * omega(p) times the projection of f^eq/omega onto the polynomials of degree
 * <= N (the basis functions with n <= N), N = 1..5. Used for Fig. 1. */
double orc_expansion_at(int edf, int order, double theta, double ux, double uy, double z,
                        double p, double phi) {
  ensure_gram(edf);
  int nb = 0, idx[36];
  for (int a = 0; a < 36; ++a)
    if (basis_n[a] <= order) idx[nb++] = a;
  double M[36], w[6];
  orc_eq_moments(edf, theta, ux, uy, z, M);
  orc_lattice(edf, NULL, w, NULL, NULL);
  /* Gram of the retained functions, solved by Gaussian elimination with pivoting */
  double G[36][37];
  for (int i = 0; i < nb; ++i) {
    for (int j = 0; j < nb; ++j) {
      double sum = 0.0;
      for (int q = 0; q < 72; ++q) sum += w[q % 6] * node_phi[edf][q][idx[i]] * node_phi[edf][q][idx[j]];
      G[i][j] = sum;
    }
    G[i][nb] = M[idx[i]];
  }
  for (int col = 0; col < nb; ++col) {
    int piv = col;
    for (int r = col + 1; r < nb; ++r)
      if (fabs(G[r][col]) > fabs(G[piv][col])) piv = r;
    for (int j = 0; j <= nb; ++j) { double t = G[col][j]; G[col][j] = G[piv][j]; G[piv][j] = t; }
    for (int r = col + 1; r < nb; ++r) {
      double m = G[r][col] / G[col][col];
      for (int j = col; j <= nb; ++j) G[r][j] -= m * G[col][j];
    }
  }
  double c[36];
  for (int i = nb - 1; i >= 0; --i) {
    double sum = G[i][nb];
    for (int j = i + 1; j < nb; ++j) sum -= G[i][j] * c[j];
    c[i] = sum / G[i][i];
  }
  double v = 0.0;
  for (int i = 0; i < nb; ++i) {
    int a = idx[i];
    v += c[i] * pow(p, basis_n[a]) * (basis_c[a] ? sin(basis_k[a] * phi) : cos(basis_k[a] * phi));
  }
  double omega;
  if (edf == ORC_MJ) omega = exp(-p) / (2.0 * PI);
  else if (edf == ORC_FD) omega = 1.0 / (exp(p) + 1.0);
  else omega = 1.0 / (exp(p) / Z_C - 1.0);
  return omega * v;
}

/* N^mu = sum_i f_i p^mu_i and T^{mu nu} = sum_i f_i p^mu_i p^nu_i, Eqs. (20), (22).
 * The sums are compensated (Neumaier): the momentum components cancel between
 * opposite directions, and a plain sum would leave an error of one unit of the
 * energy density in them, i.e. an error in u that does not shrink with u. */
void orc_moments72(int edf, const double f[72], double N[3], double T[6]) {
  double p[6], cphi[12], sphi[12];
  orc_lattice(edf, p, NULL, cphi, sphi);
  double sN[3] = {0, 0, 0}, cN[3] = {0, 0, 0}, sT[6] = {0, 0, 0, 0, 0, 0}, cT[6] = {0, 0, 0, 0, 0, 0};
  for (int d = 0; d < 12; ++d)
    for (int s = 0; s < 6; ++s) {
      double v = f[6 * d + s];
      double p0 = p[s], px = p[s] * cphi[d], py = p[s] * sphi[d];
      neumaier_add(&sN[0], &cN[0], v * p0);
      neumaier_add(&sN[1], &cN[1], v * px);
      neumaier_add(&sN[2], &cN[2], v * py);
      neumaier_add(&sT[0], &cT[0], v * p0 * p0);
      neumaier_add(&sT[1], &cT[1], v * p0 * px);
      neumaier_add(&sT[2], &cT[2], v * p0 * py);
      neumaier_add(&sT[3], &cT[3], v * px * px);
      neumaier_add(&sT[4], &cT[4], v * px * py);
      neumaier_add(&sT[5], &cT[5], v * py * py);
    }
  for (int i = 0; i < 3; ++i) N[i] = sN[i] + cN[i];
  for (int i = 0; i < 6; ++i) T[i] = sT[i] + cT[i];
}

/* ------------------------------------------------------- streaming and BCs */

typedef struct {
  const orc_domain *dom;
  const double *f;
  double *ghost_x; /* [2][ny][72] fixed-T wall ghosts at x = -1, x = nx */
  double *ghost_y; /* [2][nx][72] at y = -1, y = ny */
  const double *row_lo, *row_hi; /* given rows y = -1, y = ny as [72][nx + 2] (x = -1..nx), or NULL */
} orc_ctx;

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Population q of the post-collision state at (x, y), possibly outside the
 * domain. Reading of the boundary conditions (one ghost layer):
 *   periodic       wrap around;
 *   zero-gradient  the ghost copies the nearest edge cell (the open ends);
 *   fixed-T wall   the ghost holds f^eq(n_b, u_b, theta_wall), (n_b, u_b) being
 *                  the pre-collision state of the adjacent fluid cell at the
 *                  current time ("zeroth order extrapolation", Sec. 3.3).
 * At a corner outside both axes an x wall takes precedence over a y wall. */
static double fetch(const orc_ctx *c, int q, int x, int y) {
  const orc_domain *D = c->dom;
  int nx = D->nx, ny = D->ny, gx = 0, gy = 0;
  if (x < 0 || x >= nx) {
    if (D->bc_xlo == ORC_PERIODIC) x = ((x % nx) + nx) % nx;
    else gx = (x < 0) ? -1 : 1;
  }
  if (y < 0 || y >= ny) {
    if (D->bc_ylo == ORC_PERIODIC) y = ((y % ny) + ny) % ny;
    else gy = (y < 0) ? -1 : 1;
  }
  int xc = clampi(x, 0, nx - 1), yc = clampi(y, 0, ny - 1);
  /* a row beyond a slab edge, given by the neighbouring slab (x ghosts included) */
  const double *row = gy < 0 ? c->row_lo : (gy > 0 ? c->row_hi : NULL);
  if (row) return row[(size_t)q * (nx + 2) + (gx ? (gx < 0 ? 0 : nx + 1) : xc + 1)];
  if (gx) {
    int bc = gx < 0 ? D->bc_xlo : D->bc_xhi;
    if (bc >= ORC_FIXED_T_WALL) return c->ghost_x[((gx < 0 ? 0 : 1) * ny + yc) * 72 + q];
  }
  if (gy) {
    int bc = gy < 0 ? D->bc_ylo : D->bc_yhi;
    if (bc >= ORC_FIXED_T_WALL) return c->ghost_y[((gy < 0 ? 0 : 1) * nx + xc) * 72 + q];
  }
  return c->f[((size_t)q * ny + yc) * nx + xc];
}

/* Bilinear interpolated streaming, Eqs. (17)-(18): off-axis directions pull
 * from the four grid points around x - v_i with weights |v_x||v_y|,
 * (1-|v_x|)|v_y|, |v_x|(1-|v_y|), (1-|v_x|)(1-|v_y|); the bar positions are read
 * as the grid neighbours x - sgn(v_x), y - sgn(v_y). Axis directions shift by one cell. */
static void pull_cell(const orc_ctx *c, int edf, int x, int y, double f[72]) {
  double cphi[12], sphi[12];
  orc_lattice(edf, NULL, NULL, cphi, sphi);
  for (int d = 0; d < 12; ++d) {
    int sx = (cphi[d] > 0) - (cphi[d] < 0), sy = (sphi[d] > 0) - (sphi[d] < 0);
    double ax = fabs(cphi[d]), ay = fabs(sphi[d]);
    for (int s = 0; s < 6; ++s) {
      int q = 6 * d + s;
      if (ax == 0.0 || ay == 0.0) {
        f[q] = fetch(c, q, x - sx, y - sy);
      } else {
        f[q] = ax * ay * fetch(c, q, x - sx, y - sy) + (1.0 - ax) * ay * fetch(c, q, x, y - sy) +
               ax * (1.0 - ay) * fetch(c, q, x - sx, y) + (1.0 - ax) * (1.0 - ay) * fetch(c, q, x, y);
      }
    }
  }
}

static int has_vwall(const orc_domain *D) {
  return D->bc_xlo == ORC_VELOCITY_WALL || D->bc_xhi == ORC_VELOCITY_WALL ||
         D->bc_ylo == ORC_VELOCITY_WALL || D->bc_yhi == ORC_VELOCITY_WALL;
}

/* Relaxation time of a cell: constant, or the local tau of Sec. 3.5. */
static double cell_tau(const orc_domain *D, double theta) {
  return D->eta_s > 0.0 ? 4.0 * D->eta_s / theta + 0.2546 : D->tau;
}

/* The equilibrium a cell relaxes towards: order-N f^eq of its Landau state
 * (n, eps, theta, z) at the velocity shifted by the body force, u + a tau
 * (Sec. 3.4; no shift without a force). Also returns the shifted velocity. */
static void collision_feq(const orc_domain *D, int cs, const double m[6], double feq[72], double *uxe,
                          double *uye) {
  int edf = D->edf;
  double tau = cell_tau(D, m[1]);
  *uxe = m[2] + D->accel_x * tau;
  *uye = m[3] + D->accel_y * tau;
  /* degree-1/2 moments from the cell's n and eps (Eq. 25); a clamped BE state
   * uses the equilibrium's own eps = 4 pi theta^3 g_3(z_c) */
  double eps_eq = (cs & ORC_W_CLAMPED_FUGACITY) ? 4.0 * PI * m[1] * m[1] * m[1] * orc_g(edf, 3, m[4]) : m[5];
  orc_feq_order(edf, D->order, m[0], eps_eq, m[1], *uxe, *uye, m[4], feq);
}

/* Ghost populations of the walls from the previous step: fixed-T walls from
 * the pre-collision state (n, u) of the adjacent cell; velocity walls from
 * f^eq(n_wall, 0, theta_wall) + (f* - f^eq) of the adjacent cell, f* its
 * post-collision populations (f_in) and f^eq the equilibrium it relaxed
 * towards, at the force-shifted velocity u + a tau (from its full state in
 * macro_in). Measured against the shifted equilibrium the wall sits on the
 * ghost node; against the unshifted one the forcing part of f* - f^eq would
 * read as a slip (the channel profile's zero moves out by 0.17 cells). */
static int build_wall_ghosts(const orc_domain *D, const double *macro_in, const double *f_in, double *gxs,
                             double *gys) {
  int nx = D->nx, ny = D->ny, st = 0;
  size_t plane = (size_t)nx * ny;
  int full = has_vwall(D);
  int pn = 0, pux = full ? 2 : 1, puy = full ? 3 : 2;
  for (int axis = 0; axis < 2; ++axis)
    for (int side = 0; side < 2; ++side) {
      int bc = axis == 0 ? (side ? D->bc_xhi : D->bc_xlo) : (side ? D->bc_yhi : D->bc_ylo);
      if (bc != ORC_FIXED_T_WALL && bc != ORC_VELOCITY_WALL) continue;
      double tw = axis == 0 ? (side ? D->t_wall_xhi : D->t_wall_xlo) : (side ? D->t_wall_yhi : D->t_wall_ylo);
      int len = axis == 0 ? ny : nx;
      double *out = axis == 0 ? gxs : gys;
      for (int j = 0; j < len; ++j) {
        int x = axis == 0 ? (side ? nx - 1 : 0) : j, y = axis == 0 ? j : (side ? ny - 1 : 0);
        size_t i = (size_t)y * nx + x;
        double *g = out + ((size_t)side * len + j) * 72, z;
        if (bc == ORC_FIXED_T_WALL) {
          double n = macro_in[pn * plane + i], ux = macro_in[pux * plane + i], uy = macro_in[puy * plane + i];
          st |= orc_z_from_n_theta(D->edf, n, tw, &z);
          orc_feq_order(D->edf, D->order, -1.0, -1.0, tw, ux, uy, z, g);
        } else {
          double m[6], feqb[72];
          for (int k = 0; k < 6; ++k) m[k] = macro_in[k * plane + i];
          st |= orc_z_from_n_theta(D->edf, D->n_wall, tw, &z);
          orc_feq_order(D->edf, D->order, -1.0, -1.0, tw, 0.0, 0.0, z, g);
          double uxe, uye;
          collision_feq(D, 0, m, feqb, &uxe, &uye);
          for (int q = 0; q < 72; ++q) g[q] += f_in[q * plane + i] - feqb[q];
        }
      }
    }
  return st;
}

static int has_wall(const orc_domain *D) {
  return D->bc_xlo >= ORC_FIXED_T_WALL || D->bc_xhi >= ORC_FIXED_T_WALL ||
         D->bc_ylo >= ORC_FIXED_T_WALL || D->bc_yhi >= ORC_FIXED_T_WALL;
}

static int check_domain(const orc_domain *D) {
  if (D->nx < 1 || D->ny < 1 || D->edf < 0 || D->edf > 2) return -1;
  if ((D->bc_xlo == ORC_PERIODIC) != (D->bc_xhi == ORC_PERIODIC)) return -1;
  if ((D->bc_ylo == ORC_PERIODIC) != (D->bc_yhi == ORC_PERIODIC)) return -1;
  return 0;
}

/* ------------------------------------------------------------------ step */

/* One step: stream (pull), moments, Landau state, f^eq, and the discrete
 * Anderson-Witting relaxation of Eq. (3) with delta t = 1:
 *   f*_i = f_i - gamma (1 - v_i.u) (f_i - f^eq_i) / tau.
 * A cell whose state is non-physical is left unrelaxed and flagged. */
static int step_impl(const orc_domain *D, const double *f_in, const double *macro_in, const double *row_lo,
                     const double *row_hi, double *f_out, double *macro_out) {
  if (check_domain(D)) return -1;
  int nx = D->nx, ny = D->ny, edf = D->edf, st = 0;
  size_t plane = (size_t)nx * ny;
  ensure_gram(edf);
  orc_ctx c = {D, f_in, NULL, NULL, row_lo, row_hi};
  if (has_wall(D)) {
    if (!macro_in) return -1;
    c.ghost_x = (double *)malloc(sizeof(double) * 2 * ny * 72);
    c.ghost_y = (double *)malloc(sizeof(double) * 2 * nx * 72);
    st |= build_wall_ghosts(D, macro_in, f_in, c.ghost_x, c.ghost_y);
  }
  double cphi[12], sphi[12];
  orc_lattice(edf, NULL, NULL, cphi, sphi);
#pragma omp parallel for collapse(2) reduction(| : st) schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      double f[72], feq[72], N[3], T[6], m[6];
      pull_cell(&c, edf, x, y, f);
      orc_moments72(edf, f, N, T);
      int cs = orc_state(edf, N, T, m);
      st |= cs;
      size_t i = (size_t)y * nx + x;
      if (cs & ORC_E_NONPHYSICAL) {
        for (int q = 0; q < 72; ++q) f_out[q * plane + i] = f[q];
      } else {
        /* the equilibrium of the (force-shifted) state; the local relaxation
         * time of Sec. 3.5 from the cell's temperature */
        double uxe, uye;
        collision_feq(D, cs, m, feq, &uxe, &uye);
        double gamma = 1.0 / sqrt(1.0 - uxe * uxe - uye * uye);
        double tau = cell_tau(D, m[1]);
        for (int d = 0; d < 12; ++d) {
          double om = gamma * (1.0 - (cphi[d] * uxe + sphi[d] * uye)) / tau;
          for (int s = 0; s < 6; ++s) {
            int q = 6 * d + s;
            f_out[q * plane + i] = f[q] - om * (f[q] - feq[q]);
          }
        }
      }
      if (macro_out)
        for (int j = 0; j < 6; ++j) macro_out[j * plane + i] = m[j];
    }
  }
  free(c.ghost_x);
  free(c.ghost_y);
  return st;
}

int orc_step(const orc_domain *D, const double *f_in, const double *macro_in, double *f_out,
             double *macro_out) {
  return step_impl(D, f_in, macro_in, NULL, NULL, f_out, macro_out);
}

/* One step of a slab of a larger domain cut along y: the rows just below and
 * above the slab (y = -1 and y = ny; NULL = use the slab's own y boundary
 * condition) are given as [72][nx + 2] arrays of post-collision populations,
 * x = -1..nx, i.e. with the x ghost values the owning slab computed. Everything
 * else is orc_step. Used to check a y-slab decomposition against the whole
 * domain. */
int orc_step_rows(const orc_domain *D, const double *f_in, const double *macro_in, const double *row_lo,
                  const double *row_hi, double *f_out, double *macro_out) {
  return step_impl(D, f_in, macro_in, row_lo, row_hi, f_out, macro_out);
}

/* Row y = 0 (side 0) or y = ny - 1 (side 1) of the post-collision state as a
 * neighbouring slab reads it: [72][nx + 2], x = -1..nx, the x ghosts taken from
 * the x boundary conditions (a wall ghost from macro_in, the pre-collision
 * state of the edge cell, as in orc_step). */
int orc_edge_row(const orc_domain *D, const double *f, const double *macro_in, int side, double *row) {
  if (check_domain(D) || (side != 0 && side != 1)) return -1;
  int nx = D->nx, ny = D->ny, st = 0;
  orc_ctx c = {D, f, NULL, NULL, NULL, NULL};
  if (D->bc_xlo >= ORC_FIXED_T_WALL || D->bc_xhi >= ORC_FIXED_T_WALL) {
    if (!macro_in) return -1;
    c.ghost_x = (double *)malloc(sizeof(double) * 2 * ny * 72);
    c.ghost_y = (double *)malloc(sizeof(double) * 2 * nx * 72);
    st |= build_wall_ghosts(D, macro_in, f, c.ghost_x, c.ghost_y);
  }
  int y = side ? ny - 1 : 0;
  for (int q = 0; q < 72; ++q)
    for (int x = -1; x <= nx; ++x) row[(size_t)q * (nx + 2) + x + 1] = fetch(&c, q, x, y);
  free(c.ghost_x);
  free(c.ghost_y);
  return st;
}

/* Initial state f = f^eq of the given fields (the time-zero convention: an
 * equilibrium is its own post-collision state). */
int orc_init(const orc_domain *D, int kind, const double *a, const double *theta,
             const double *ux, const double *uy, double *f, double *macro_out) {
  if (check_domain(D)) return -1;
  int nx = D->nx, ny = D->ny, edf = D->edf, st = 0;
  size_t plane = (size_t)nx * ny;
  ensure_gram(edf);
#pragma omp parallel for collapse(2) reduction(| : st) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      double z, n, feq[72];
      if (kind == ORC_INIT_Z_THETA) {
        z = a[i];
        n = 2.0 * PI * theta[i] * theta[i] * orc_g(edf, 2, z);
      } else {
        n = a[i];
        st |= orc_z_from_n_theta(edf, n, theta[i], &z);
      }
      if (!(ux[i] * ux[i] + uy[i] * uy[i] < 1.0) || !(theta[i] > 0.0) || !(n > 0.0)) {
        st |= ORC_E_NONPHYSICAL;
      }
      orc_feq_order(edf, D->order, -1.0, -1.0, theta[i], ux[i], uy[i], z, feq);
      for (int q = 0; q < 72; ++q) f[q * plane + i] = feq[q];
      if (macro_out) {
        macro_out[i] = n;
        macro_out[plane + i] = ux[i];
        macro_out[2 * plane + i] = uy[i];
      }
    }
  return st;
}

int orc_fields(const orc_domain *D, const double *f_in, const double *macro_in, int streamed,
               double *out) {
  if (check_domain(D)) return -1;
  int nx = D->nx, ny = D->ny, edf = D->edf, st = 0;
  size_t plane = (size_t)nx * ny;
  orc_ctx c = {D, f_in, NULL, NULL};
  if (streamed && has_wall(D)) {
    if (!macro_in) return -1;
    c.ghost_x = (double *)malloc(sizeof(double) * 2 * ny * 72);
    c.ghost_y = (double *)malloc(sizeof(double) * 2 * nx * 72);
    st |= build_wall_ghosts(D, macro_in, f_in, c.ghost_x, c.ghost_y);
  }
#pragma omp parallel for collapse(2) reduction(| : st) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      double f[72], N[3], T[6], m[6];
      size_t i = (size_t)y * nx + x;
      if (streamed) pull_cell(&c, edf, x, y, f);
      else
        for (int q = 0; q < 72; ++q) f[q] = f_in[q * plane + i];
      orc_moments72(edf, f, N, T);
      st |= orc_state(edf, N, T, m);
      for (int j = 0; j < 6; ++j) out[j * plane + i] = m[j];
    }
  free(c.ghost_x);
  free(c.ghost_y);
  return st;
}

/* Diagnostic fields [7][ny][nx]: the heat flux of the Eckart-Landau
 * correspondence (Sec. 3.3), q^a = (3 theta g_3(z) / g_2(z)) (n U^a - N^a),
 * a = 0, x, y, with U = gamma (1, u_x, u_y); and the diagonal components of
 * the non-equilibrium tensors of Sec. 3.1, pi^{x..x} = sum_i (f_i - f^eq_i)
 * (p_i cos phi_i)^k for k = 2..5, f^eq_i being the discrete fifth-order
 * equilibrium of the cell's Landau state (the one orc_step relaxes towards).
 * f is pulled first when streamed. Non-physical cells give NaN. */
int orc_diagnostics(const orc_domain *D, const double *f_in, const double *macro_in, int streamed,
                    double *out) {
  if (check_domain(D)) return -1;
  int nx = D->nx, ny = D->ny, edf = D->edf, st = 0;
  size_t plane = (size_t)nx * ny;
  ensure_gram(edf);
  orc_ctx c = {D, f_in, NULL, NULL, NULL, NULL};
  if (streamed && has_wall(D)) {
    if (!macro_in) return -1;
    c.ghost_x = (double *)malloc(sizeof(double) * 2 * ny * 72);
    c.ghost_y = (double *)malloc(sizeof(double) * 2 * nx * 72);
    st |= build_wall_ghosts(D, macro_in, f_in, c.ghost_x, c.ghost_y);
  }
  double p[6], cphi[12], sphi[12];
  orc_lattice(edf, p, NULL, cphi, sphi);
#pragma omp parallel for collapse(2) reduction(| : st) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      double f[72], feq[72], N[3], T[6], m[6], o[7];
      size_t i = (size_t)y * nx + x;
      if (streamed) pull_cell(&c, edf, x, y, f);
      else
        for (int q = 0; q < 72; ++q) f[q] = f_in[q * plane + i];
      orc_moments72(edf, f, N, T);
      int cs = orc_state(edf, N, T, m);
      st |= cs;
      if (cs & ORC_E_NONPHYSICAL) {
        for (int k = 0; k < 7; ++k) o[k] = NAN;
      } else {
        double n = m[0], theta = m[1], ux = m[2], uy = m[3], z = m[4];
        double gamma = 1.0 / sqrt(1.0 - ux * ux - uy * uy);
        double hq = 3.0 * theta * orc_g(edf, 3, z) / orc_g(edf, 2, z);
        o[0] = hq * (n * gamma - N[0]);
        o[1] = hq * (n * gamma * ux - N[1]);
        o[2] = hq * (n * gamma * uy - N[2]);
        double eps_eq = (cs & ORC_W_CLAMPED_FUGACITY) ? 4.0 * PI * theta * theta * theta * orc_g(edf, 3, z) : m[5];
        orc_feq_order(edf, D->order, n, eps_eq, theta, ux, uy, z, feq);
        for (int k = 2; k <= 5; ++k) {
          double sum = 0.0;
          for (int d = 0; d < 12; ++d)
            for (int s = 0; s < 6; ++s) {
              int q = 6 * d + s;
              sum += (f[q] - feq[q]) * pow(p[s] * cphi[d], k);
            }
          o[k + 1] = sum;
        }
      }
      for (int k = 0; k < 7; ++k) out[k * plane + i] = o[k];
    }
  free(c.ghost_x);
  free(c.ghost_y);
  return st;
}
