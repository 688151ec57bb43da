/*
 * Oracle for the fully dissipative 2D ultra-relativistic lattice Boltzmann
 * method (Coelho, Mendoza, Doria, Herrmann, arXiv:1709.09073).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, FP64 CPU restatement of the
 * method, written from the paper, used to check the CUDA implementation. Only
 * the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it. It shares no code, header or table with the CUDA path.
 *
 * Layout (the same as the library's public C ABI, because results are compared
 * element by element): populations are structure-of-arrays f[q][y][x], with
 * q = 6*d + s, direction d = 0..11 at phi_d = d*pi/6 and shell s = 0..5
 * (ascending momentum). Macroscopic fields are row-major [y][x].
 */
#ifndef RLBM_ORACLE_H
#define RLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NDIR 12
#define ORC_NSHELL 6
#define ORC_Q 72
#define ORC_NBASIS 36

enum { ORC_MJ = 0, ORC_FD = 1, ORC_BE = 2 };
enum { ORC_PERIODIC = 0, ORC_ZERO_GRADIENT = 1, ORC_FIXED_T_WALL = 2, ORC_VELOCITY_WALL = 3 };
enum { ORC_INIT_N_THETA = 0, ORC_INIT_Z_THETA = 1 };

/* status bits (OR-ed over cells) */
#define ORC_W_LANDAU_MAXITER 1
#define ORC_W_CLAMPED_FUGACITY 2
#define ORC_E_NONPHYSICAL 4
#define ORC_E_ZSOLVE 8

typedef struct {
  int nx, ny;
  double tau;
  int edf;
  int bc_xlo, bc_xhi, bc_ylo, bc_yhi; /* periodic must be set on both sides of an axis */
  double t_wall_xlo, t_wall_xhi, t_wall_ylo, t_wall_yhi;
  int order;    /* expansion order N of Eq. (10), 2..5 (0 is read as 5) */
  double eta_s; /* > 0: local relaxation time tau = 4 (eta/s) / theta + 0.2546 (Sec. 3.5) */
  double accel_x, accel_y; /* body acceleration a: the collision uses u + a tau (Sec. 3.4) */
  double n_wall;           /* density of ORC_VELOCITY_WALL sides (their theta: t_wall) */
} orc_domain;
/* ORC_VELOCITY_WALL (Sec. 3.4, Poiseuille): a wall at rest whose ghost holds
 * f^eq(n_wall, u = 0, theta_wall) plus the non-equilibrium part f* - f^eq of
 * the adjacent fluid cell's last collision (f^eq at its force-shifted velocity,
 * the one it relaxed towards). A domain with such a side passes
 * orc_step the full previous state (the 6 planes n, theta, ux, uy, z, eps of
 * orc_step's macro_out) as macro_in instead of (n, ux, uy). */

/* Lattice: shell momenta p[6], per-vector weights w[6] and direction cosines. */
void orc_lattice(int edf, double p[6], double w[6], double cphi[12], double sphi[12]);

/* EDF integral g_nu(z), Eq. (12): z for MJ, -Li_nu(-z) for FD, Li_nu(z) for BE. */
double orc_g(int edf, int nu, double z);

/* Landau-Lifshitz frame, Eq. (21): power method on T^a_b. T = {T00,T01,T02,T11,T12,T22}.
 * Returns status bits; writes eps and U^mu (U^mu U_mu = 1, U^0 > 0). */
int orc_landau(const double T[6], double *eps, double U[3], int *iters);

/* Macroscopic state from N^mu and T^{mu nu}: Eqs. (21)-(25) and the fugacity
 * reading for FD/BE. Writes n, theta, ux, uy, z, eps. Returns status bits. */
int orc_state(int edf, const double N[3], const double T[6], double out[6]);

/* Fugacity from (n, theta): solves n = 2 pi theta^2 g_2(z), Eq. (25). */
int orc_z_from_n_theta(int edf, double n, double theta, double *z);

/* The 36 equilibrium moments int dp dphi f^eq p^n {cos,sin}(k phi), basis order
 * of orc_basis, from the Appendix closed forms I_2^{mnq}. */
void orc_eq_moments(int edf, double theta, double ux, double uy, double z, double M[36]);

/* The same moments by trapezoidal angular quadrature of their definition. */
void orc_eq_moments_quad(int edf, double theta, double ux, double uy, double z, double M[36]);

/* Same with the degree-1 and degree-2 radial factors taken from n and eps via
 * Eq. (25) (n/(2 pi) and eps/(2 pi)); a negative n or eps is ignored. */
void orc_eq_moments_ne(int edf, double n, double eps, double theta, double ux, double uy, double z,
                       double M[36]);

/* Basis function list: for a in 0..35, n[a], k[a], c[a] (c = 0 cos, 1 sin). */
void orc_basis(int n[36], int k[36], int c[36]);

/* Discrete fifth-order equilibrium f^eq_q (projection onto degree <= 5), Eqs. (10)-(11). */
void orc_feq(int edf, double theta, double ux, double uy, double z, double feq[72]);

/* Same with n and eps fixing the degree-1 and degree-2 moments (Eq. 25). */
void orc_feq_ne(int edf, double n, double eps, double theta, double ux, double uy, double z,
                double feq[72]);

/* The order-N equilibrium (N = 2..5): projection of f^eq / omega onto the basis
 * functions of degree <= N only; n or eps < 0 as for orc_eq_moments_ne. */
void orc_feq_order(int edf, int order, double n, double eps, double theta, double ux, double uy, double z,
                   double feq[72]);

/* Value of the order-N expansion (N = 1..5) at an arbitrary momentum (Fig. 1). */
double orc_expansion_at(int edf, int order, double theta, double ux, double uy, double z,
                        double p, double phi);

/* Moments N^mu, T^{mu nu} of 72 populations, Eqs. (20)-(22). */
void orc_moments72(int edf, const double f[72], double N[3], double T[6]);

/* One time step of one domain: pull-stream (Eqs. 17-18, with the boundary
 * ghosts), then Anderson-Witting relaxation (Eq. 3).
 * macro_in: [3][ny][nx] (n, ux, uy) pre-collision state of the previous step
 * (needed only for fixed-T walls; may be NULL otherwise). macro_out: [6][ny][nx]
 * (n, theta, ux, uy, z, eps) of the streamed populations, may be NULL. */
int orc_step(const orc_domain *dom, const double *f_in, const double *macro_in, double *f_out,
             double *macro_out);
/* y-slab decomposition: a step of a slab whose outside rows ([72][nx + 2],
 * x = -1..nx, NULL = own boundary condition) are given, and the extraction of
 * a slab's bottom (side 0) or top (side 1) row as its neighbour reads it. */
int orc_step_rows(const orc_domain *D, const double *f_in, const double *macro_in, const double *row_lo,
                  const double *row_hi, double *f_out, double *macro_out);
int orc_edge_row(const orc_domain *D, const double *f, const double *macro_in, int side, double *row);

/* Initialise f = f^eq from fields a (n or z, per kind), theta, ux, uy.
 * macro_out [3][ny][nx] receives (n, ux, uy), may be NULL. */
int orc_init(const orc_domain *dom, int kind, const double *a, const double *theta,
             const double *ux, const double *uy, double *f, double *macro_out);

/* Macroscopic fields of the stored populations: streamed = 1 pulls first (the
 * state the next collision relaxes), 0 takes the stored populations as they are.
 * out: [6][ny][nx] (n, theta, ux, uy, z, eps). */
int orc_fields(const orc_domain *dom, const double *f, const double *macro_in, int streamed,
               double *out);
/* heat flux q^0, q^x, q^y and diagonal non-equilibrium tensors of orders 2..5, [7][ny][nx] */
int orc_diagnostics(const orc_domain *D, const double *f_in, const double *macro_in, int streamed,
                    double *out);

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int orc_num_threads(void);
/* Threads for later calls (n > 0); the timing of the CPU baseline runs it at 1. */
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
