/*
 * rlbm.h -- C ABI of the GB300 (sm_103a) implementation of the fully
 * dissipative two-dimensional ultra-relativistic lattice Boltzmann method of
 * Coelho, Mendoza, Doria and Herrmann, arXiv:1709.09073.
 *
 * The library advances populations f_i on the d2v72 quadrature (12 directions
 * phi_d = d pi/6 times 6 energy shells, Sec. 2.4) with the fused per-cell
 * update of the paper: bilinear interpolated pull-streaming (Eqs. 17-18),
 * moments N^mu and T^{mu nu} (Eqs. 20, 22), the Landau-frame eigenproblem
 * T^a_b U^b = eps U^a (Eq. 21), temperature and fugacity (Eqs. 24-25), the
 * fifth-order expansion of the Maxwell-Juttner, Fermi-Dirac or Bose-Einstein
 * equilibrium (Eqs. 10-11, Appendix) and Anderson-Witting relaxation (Eq. 3).
 *
 * Conventions shared by every call
 *  - Units: delta t = delta x = c = k_B = 1; theta = T/T_0 (Sec. 2.3).
 *  - Population index q = 6 d + s: direction d = 0..11 (phi_d = d pi/6,
 *    counter-clockwise from +x), shell s = 0..5 (ascending momentum).
 *  - Macroscopic field arrays are row-major [ny][nx] FP64 (index y*nx + x),
 *    on the host or on the device as the `on_device` argument says.
 *  - Device memory: the caller allocates ONE workspace of
 *    rlbm_workspace_bytes(config) bytes (256-byte aligned) and keeps it alive
 *    until rlbm_destroy; the library allocates no device memory of its own
 *    (rlbm_step_noalloc, at the end, uses a fixed static array instead).
 *    The handle (host memory) and a captured CUDA graph belong to the library.
 *  - Streams: every call is ordered on config->cuda_stream (a cudaStream_t;
 *    NULL = the legacy default stream). rlbm_step is asynchronous; calls that
 *    return data to host memory synchronise that stream before returning.
 *  - Return codes: 0 = success, > 0 = warning bits (the call completed),
 *    < 0 = error (nothing was done, or the device state is unspecified for
 *    RLBM_E_CUDA). rlbm_status_string() describes any code.
 *  - Threads: a handle must not be used by two host threads at once.
 */
#ifndef RLBM_H
#define RLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlbm_ctx *rlbm_handle;

/* Equilibrium distribution, Eq. (7): xi = 0 (MJ), 1 (FD), -1 (BE). Every
 * domain of one handle uses the same EDF. */
typedef enum { RLBM_MJ = 0, RLBM_FD = 1, RLBM_BE = 2 } rlbm_edf;

/* Storage of the populations in HBM.
 *  RLBM_F64      FP64 populations, FP64 arithmetic throughout (the plain method).
 *  RLBM_F32      FP32 populations; FP32 streaming, equilibrium and relaxation;
 *                moments and Landau solve in FP64-class precision.
 *  RLBM_BF16DEV, RLBM_F16DEV
 *                relative deviations h = (f / f_ref - 1) / scale from the rest
 *                equilibrium f_ref(ref_n, ref_theta) of each domain, stored in
 *                BF16 or FP16; arithmetic as for RLBM_F32.
 *  RLBM_F32DEV   the deviation f - f_ref itself in FP32 (scale unused);
 *                arithmetic as for RLBM_F32. */
typedef enum { RLBM_F64 = 0, RLBM_F32 = 1, RLBM_BF16DEV = 2, RLBM_F16DEV = 3, RLBM_F32DEV = 4 } rlbm_storage;

/* Boundary condition of one side (one ghost layer; Sec. 3):
 *  RLBM_PERIODIC       wrap-around (must be set on both sides of an axis);
 *  RLBM_ZERO_GRADIENT  the ghost copies the adjacent edge cell (open ends);
 *  RLBM_FIXED_T_WALL   the ghost holds f^eq(n_b, u_b, theta_wall) with n_b, u_b
 *                      the pre-collision state of the adjacent fluid cell at the
 *                      current time (zeroth-order extrapolation, Sec. 3.3).
 *  RLBM_VELOCITY_WALL  a wall at rest (Sec. 3.4, Poiseuille flow): the ghost holds
 *                      f^eq(n_wall, u = 0, theta_wall) plus the non-equilibrium part
 *                      f* - f^eq of the adjacent fluid cell's last collision
 *                      (non-equilibrium extrapolation). FP64 storage only; all such
 *                      sides of a domain share one theta_wall.
 *  RLBM_EXCHANGED      y sides only: the ghost row is supplied by the caller
 *                      (rlbm_unpack_ghost_rows, the face of a neighbouring y-slab)
 *                      and the library never writes it. It must be supplied
 *                      before every step and before a streamed read-out.
 *  At a corner outside both axes an x-side wall takes precedence over a y-side wall. */
typedef enum {
  RLBM_PERIODIC = 0,
  RLBM_ZERO_GRADIENT = 1,
  RLBM_FIXED_T_WALL = 2,
  RLBM_VELOCITY_WALL = 3,
  RLBM_EXCHANGED = 4
} rlbm_bc;

/* Meaning of the first field given to rlbm_init. */
typedef enum { RLBM_INIT_N_THETA = 0, RLBM_INIT_Z_THETA = 1 } rlbm_init_kind;

typedef struct {
  int nx, ny;                 /* lattice size, >= 1 each */
  double tau;                 /* relaxation time (Eq. 3), > 0 */
  int bc_xlo, bc_xhi, bc_ylo, bc_yhi;                /* rlbm_bc */
  double t_wall_xlo, t_wall_xhi, t_wall_ylo, t_wall_yhi; /* wall theta, if a wall */
  double ref_n, ref_theta;    /* reference rest equilibrium of the mixed storages */
  double scale;               /* deviation scale of the 16-bit *DEV storages (> 0) */
  double eta_s;               /* > 0: local relaxation time tau = 4 eta_s / theta + 0.2546
                                 from each cell's temperature (Sec. 3.5; tau above is then
                                 unused); 0: constant tau */
  double accel_x, accel_y;    /* body acceleration a (Sec. 3.4): the collision relaxes towards
                                 f^eq at u + a tau; FP64 storage only when non-zero */
  double n_wall;              /* density of the RLBM_VELOCITY_WALL sides (> 0 if any) */
} rlbm_domain;

typedef struct {
  int ndomains;               /* >= 1 independent domains, advanced together */
  const rlbm_domain *domains; /* host array of ndomains descriptors (copied) */
  int edf;                    /* rlbm_edf */
  int storage;                /* rlbm_storage */
  int order;                  /* expansion order N of Eq. (10): 2..5 with RLBM_F64
                                 storage (Sec. 3.5 order comparison), 5 otherwise */
  void *device_buffer;        /* caller-owned workspace, rlbm_workspace_bytes() */
  size_t buffer_bytes;
  void *cuda_stream;          /* cudaStream_t or NULL */
} rlbm_config;

/* Status codes. Warnings are bits that may be OR-ed together. */
#define RLBM_OK 0
#define RLBM_W_LANDAU_MAXITER 1     /* Landau solve hit its iteration cap in some cell */
#define RLBM_W_CLAMPED_FUGACITY 2   /* BE state beyond z_c clamped to z_c (n kept) */
#define RLBM_W_NONPHYSICAL 4        /* some cell had |u|>=1, n<=0, eps<=0 or a non-finite
                                       moment; it was streamed but not relaxed */
#define RLBM_W_ZSOLVE 8             /* fugacity solve (FD/BE) did not converge in some cell */
#define RLBM_W_DEVICE_TIMEOUT 16    /* a bounded wait inside a kernel gave up (a copy did not
                                       arrive within a second); that step's results are invalid */
#define RLBM_E_ARG (-1)             /* invalid argument */
#define RLBM_E_CUDA (-2)            /* a CUDA call failed */
#define RLBM_E_STATE (-3)           /* call out of order (e.g. step before init) */
#define RLBM_E_UNSUPPORTED (-4)     /* valid but unsupported combination */
#define RLBM_E_NOBUFFER (-5)        /* device buffer missing, misaligned or too small */

/* Bytes of device workspace the configuration needs (0 if the config is invalid).
 * Holds two halo-padded population copies, the device descriptor and tile
 * tables, a status word and a host-transfer staging area. */
size_t rlbm_workspace_bytes(const rlbm_config *config);

/* The tile work list a handle of this configuration would walk (host only, no
 * device work; the paper has no counterpart): packed = 0 the plain list of
 * 32 x 4 tiles (TMA-staged and FP64 steps, initialisers, read-outs), packed = 1
 * the list of the mixed L1 step, where each domain's ragged last x block of
 * w <= 16 cells is one tile per 4 * (32 / w) rows, a warp covering 32 / w rows
 * of w cells. Writes up to max_tiles quadruples (domain, x0, y0, w) to `out`
 * (host, int[4 * max_tiles]; may be null) and returns the number of tiles, or
 * RLBM_E_ARG for an invalid configuration. */
int rlbm_layout_tiles(const rlbm_config *config, int packed, int *out, int max_tiles);

/* Create a handle over the caller's workspace. Copies the descriptors; uploads
 * the tables; does not initialise populations. *out = NULL on error. */
int rlbm_create(const rlbm_config *config, rlbm_handle *out);

/* Set domain `domain` to the equilibrium f = f^eq of the given fields (time 0;
 * an equilibrium is its own post-collision state). kind = RLBM_INIT_N_THETA:
 * a = n; RLBM_INIT_Z_THETA: a = fugacity z (MJ: z = n / (2 pi theta^2), Eq. 25).
 * Fields are [ny][nx] FP64 on host (on_device = 0) or device (1). Every domain
 * must be initialised before the first rlbm_step. Returns warning bits of the
 * fugacity solve, or an error. FP64 storage evaluates the fifth-order
 * equilibrium (Eqs. 10-11) in FP64; the mixed storages in the collision's own
 * FP32 deviation arithmetic. */
int rlbm_init(rlbm_handle h, int domain, int kind, const double *a, const double *theta,
              const double *ux, const double *uy, int on_device);

/* rlbm_init for every domain of the handle in one kernel launch: each field
 * array holds the domains' [ny][nx] fields one after the other in domain
 * order (sum of nx * ny values, FP64, host or device per on_device; host
 * fields are staged through the spare population copy). Returns the warning
 * bits of this call, RLBM_E_ARG, RLBM_E_UNSUPPORTED or RLBM_E_CUDA. */
int rlbm_init_all(rlbm_handle h, int kind, const double *a, const double *theta, const double *ux,
                  const double *uy, int on_device);

/* Advance every domain by nsteps >= 0 fused stream-collide steps (Eqs. 3,
 * 17-18), asynchronously on the handle's stream (replayed from a captured CUDA
 * graph). Returns RLBM_OK or an error; per-cell warnings accumulate on the
 * device and are read by rlbm_sync_status. */
int rlbm_step(rlbm_handle h, int nsteps);

/* Macroscopic fields of domain `domain`: streamed = 1 gives the state of the
 * populations after streaming the stored post-collision populations (what the
 * next step relaxes); streamed = 0 takes the stored populations as they are.
 * Writes n, theta, ux, uy and, when non-NULL, z (each [ny][nx] FP64, host or
 * device per on_device). Host outputs are complete on return. */
int rlbm_moments(rlbm_handle h, int domain, int streamed, double *n, double *theta, double *ux,
                 double *uy, double *z, int on_device);

/* rlbm_moments for every domain in one kernel launch: outputs packed as the
 * fields of rlbm_init_all (z may be NULL). Every domain must be initialised
 * (RLBM_E_STATE otherwise). */
int rlbm_moments_all(rlbm_handle h, int streamed, double *n, double *theta, double *ux, double *uy,
                     double *z, int on_device);

/* Diagnostic fields of domain `domain` (streamed as for rlbm_moments), FP64
 * [7][ny][nx] into `out` (host or device per on_device): the heat flux
 * q^0, q^x, q^y = (3 theta g_3(z) / g_2(z)) (n U^a - N^a) (Sec. 3.3, the
 * Eckart-Landau correspondence) and the diagonal non-equilibrium tensors
 * pi^{xx}, pi^{xxx}, pi^{xxxx}, pi^{xxxxx} = sum_i (f_i - f^eq_i) (p_i^x)^k
 * (Sec. 3.1), f^eq being the fifth-order equilibrium of the cell's Landau
 * state. Non-physical cells give NaN. Host outputs are complete on return. */
int rlbm_diagnostics(rlbm_handle h, int domain, int streamed, double *out, int on_device);

/* Raw state of domain `domain` for checkpoint/resume: the stored populations
 * including the one-cell halo ring (periodic images, which the mixed L1 step
 * does not store, are filled from the interior first), as FP64 [72][ny+2][nx+2] (index
 * (q*(ny+2) + y+1)*(nx+2) + x+1 for x in -1..nx, y in -1..ny), converted from
 * the storage format. rlbm_set_populations writes them back (rounded to the
 * storage format); a resumed run then continues bit-for-bit. */
int rlbm_get_populations(rlbm_handle h, int domain, double *f, int on_device);
int rlbm_set_populations(rlbm_handle h, int domain, const double *f, int on_device);

/* ---- y-slab halo rows ----------------------------------------------------
 * One domain too large for one GPU is cut into y-slabs, one handle (or one
 * domain of a handle) each, whose y sides that border another slab are given
 * RLBM_ZERO_GRADIENT. The pull of the interpolated streaming (Eqs. 17-18)
 * reaches one row: row 0 reads the ghost row y = -1 only in the 30 planes
 * q = 6..35 (directions d = 1..5, v_y > 0) and row ny-1 reads y = ny only in
 * q = 42..71 (d = 7..11, v_y < 0). Before every rlbm_step (and after
 * rlbm_init) each slab therefore packs its two edge rows, sends them to its y
 * neighbours (NCCL, a peer copy, or a plain device copy for slabs on one GPU)
 * and unpacks what it receives into its ghost rows. Slabs stepped this way
 * reproduce the undivided domain bit for bit.
 *
 * A packed face is [30][nx + 2] elements of the handle's storage type in its
 * storage encoding (index k*(nx + 2) + x + 1 for x in -1..nx, plane 6 + k or
 * 42 + k), so slabs that exchange rows must share nx, storage, ref_n,
 * ref_theta and scale. rlbm_edge_row_bytes gives its size (0 for bad
 * arguments). */
size_t rlbm_edge_row_bytes(rlbm_handle h, int domain);

/* Pack the current post-collision edge rows of `domain` into device buffers:
 * `lo` <- row 0, planes 42..71 (what the slab below reads), `hi` <- row ny-1,
 * planes 6..35 (what the slab above reads), each with its two x ghost values.
 * Either pointer may be NULL (that face is skipped); non-NULL ones are device
 * memory of rlbm_edge_row_bytes() bytes, aligned to the element size. Runs on
 * the handle's stream (one kernel launch), asynchronously. RLBM_E_STATE for an
 * uninitialised domain. */
int rlbm_pack_edge_rows(rlbm_handle h, int domain, void *lo, void *hi);

/* Write received edge rows into the ghost rows of `domain`: `lo` (the top row
 * of the slab below, planes 6..35) into y = -1, `hi` (the bottom row of the
 * slab above, planes 42..71) into y = ny. The other planes of the ghost rows
 * are left as they are. Pointers, sizes and errors as for
 * rlbm_pack_edge_rows; asynchronous on the handle's stream. */
int rlbm_unpack_ghost_rows(rlbm_handle h, int domain, const void *lo, const void *hi);

/* Autotune the launch of the step kernel on the current state (left unchanged):
 * time `repeats` launches of each candidate -- every kernel variant the handle
 * has (rlbm_select_kernel) with one block per 32 x 4 tile or a persistent grid
 * of k x (SM count) blocks, k in {1, 2, 3, 4, 6, 8} -- and keep the fastest for
 * later rlbm_step calls (the captured step graphs are rebuilt). Every domain
 * must be initialised. Returns the chosen grid size (> 0) or an error; device
 * warnings raised while timing are discarded. */
int rlbm_tune(rlbm_handle h, int repeats);

/* Launch the step kernel with `grid` blocks in later rlbm_step calls: a
 * persistent grid, each block walking the tile list with stride `grid`, or
 * one block per tile for grid = 0 (the default). The mixed L1 step walks a
 * list in which each domain's ragged last block of w <= 16 cells is packed,
 * 32 / w rows per warp; the other kernels walk 32 x 4 tiles. rlbm_tune sets it
 * as well. Returns the grid now in use (grid >= 0) or RLBM_E_ARG. */
int rlbm_set_grid(rlbm_handle h, int grid);

/* Variants of the mixed-precision step kernel; both compute the same update
 * with the same arithmetic in the same order (identical results).
 *  RLBM_KERNEL_L1   each thread pulls its bilinear neighbours from global
 *                   memory through L1 and stores its 72 values (default);
 *  RLBM_KERNEL_TMA  a ring of TMA boxes (one direction's six shell planes of
 *                   the tile's block of 32 cells and its two neighbours, rows
 *                   y0-1 .. y0+4 of a 32 x 4 tile) staged in shared memory, every wait for a
 *                   copy bounded (rlbm_set_wait_limit). Needs the driver's
 *                   tensor-map encoder. */
#define RLBM_KERNEL_L1 0
#define RLBM_KERNEL_TMA 1

/* Select the step kernel variant (kernel >= 0) or query it (kernel < 0).
 * Returns the variant now in use, RLBM_E_ARG for an unknown variant, or
 * RLBM_E_UNSUPPORTED for RLBM_KERNEL_TMA on FP64 storage (it has one step
 * kernel) or without TMA descriptors. rlbm_tune may change the selection. */
int rlbm_select_kernel(rlbm_handle h, int kernel);

/* Time limit of every wait of the TMA-staged step (RLBM_KERNEL_TMA) for a
 * copy to land, in seconds; 0 or less restores the default of one second. A
 * wait that runs out ends the step early with RLBM_W_DEVICE_TIMEOUT set (the
 * step's results are then invalid; the handle stays usable), after letting the
 * copies still in flight land (bounded by the default limit). Limits under a
 * microsecond poll without suspending, so they run out on the first copy not
 * yet landed: a failure-detection test uses that. The paper has no
 * counterpart. Returns RLBM_OK or RLBM_E_ARG (NaN). */
int rlbm_set_wait_limit(rlbm_handle h, double seconds);

/* Measured FMA throughput of this GPU (the current device): the FP64 and FP32
 * flop rates (FMA = 2 flops) of an FMA-chain kernel over every SM, best of
 * three timed launches, and the SM count. These are the compute ceilings of
 * the step kernels' roofline; the paper has no counterpart (it is a property
 * of the machine, not of the method). Outputs are host pointers (sm_count may
 * be null). Takes about two seconds; synchronises the device's work it
 * launches. Returns RLBM_OK, RLBM_E_ARG or RLBM_E_CUDA. */
int rlbm_pipe_peaks(double *fp64_flops, double *fp32_flops, int *sm_count);

/* Wait for the handle's stream, return the warning bits accumulated since the
 * last call (and clear them), or RLBM_E_CUDA. */
int rlbm_sync_status(rlbm_handle h);

/* Release the handle (and its CUDA graph). The workspace stays the caller's. */
int rlbm_destroy(rlbm_handle h);

/* Static text for any status code or warning bit set. */
const char *rlbm_status_string(int code);

/* Cells x steps executed by the last rlbm_step call and kernel launches it
 * issued (for throughput accounting). */
int rlbm_last_step_info(rlbm_handle h, long long *cell_updates, int *kernel_launches);

/* ---- Fixed-scratch step (no allocation) ----------------------------------
 * The paper has no counterpart to this entry point: it is a service of the
 * library for callers that cannot call cudaMalloc -- a host application whose
 * own allocator has reserved the device memory and hands out nothing more, or
 * code on a latency-critical path where cudaMalloc/cudaFree are banned because
 * they can synchronise the whole device.
 *
 * Advances ONE domain by nsteps >= 0 steps of the plain method (FP64 storage
 * and arithmetic, fifth order; the same step kernel as rlbm_step with
 * RLBM_F64) without a handle or workspace and without allocating anything:
 * no cudaMalloc, cudaFree or allocating library routine is called.
 *  - domain: host descriptor, checked as rlbm_create checks it (ref_n,
 *    ref_theta, scale ignored; eta_s > 0 selects the local tau; RLBM_EXCHANGED
 *    sides are refused, having no face to receive); edf: rlbm_edf.
 *  - f_in, f_out: caller-owned DEVICE buffers, FP64 [72][ny+2][nx+2] with the
 *    halo ring -- the layout of rlbm_get_populations -- holding the stored
 *    post-collision populations before and after the steps. The halo of f_in
 *    must be the one a step left (e.g. a checkpoint taken with
 *    rlbm_get_populations(..., on_device = 1) or a previous f_out). f_out may
 *    equal f_in. Neither is retained after the call.
 *  - cuda_stream: cudaStream_t the work is ordered on (NULL = legacy default
 *    stream). The call is asynchronous unless `warnings` is non-NULL: then it
 *    waits for the stream and stores this call's warning bits (RLBM_W_*) there.
 *  - Scratch: all working memory (two halo-padded copies, descriptor, tile
 *    list, status word) lives in one file-scope device array of
 *    RLBM_NOALLOC_SCRATCH_BYTES (32 MiB), which the CUDA runtime reserves on
 *    every GPU where the library's module is loaded and holds until the
 *    process exits. A domain fits when 1.5 KB + 16 * ceil(nx/32) * ceil(ny/4)
 *    + 2 * 8 * (ny + 2) * nblk * 2304 <= 32 MiB, nblk = floor((nx + 32) / 32)
 *    + 1 blocks of 32 cells per row (about 148 x 148 cells); a larger one
 *    returns RLBM_E_SCRATCH before any device work.
 *  - First call on each device: it looks up the array's device address
 *    (cudaGetSymbolAddress) and sets the step kernel's shared-memory limit.
 *    Make that first call before any stream capture begins.
 *  - Sharing: every call on a device uses the same array, which keeps the last
 *    call's contents (the status word is cleared at the start of each call).
 *    Calls whose work overlaps on the GPU -- different streams, or host threads
 *    that do not order their calls -- race on it and give undefined results.
 * Returns RLBM_OK, RLBM_E_ARG, RLBM_E_SCRATCH, RLBM_E_UNSUPPORTED (device
 * ordinal >= 64) or RLBM_E_CUDA. */
#define RLBM_E_SCRATCH (-6)               /* domain too large for the fixed scratch */
#define RLBM_NOALLOC_SCRATCH_BYTES (32u << 20)
int rlbm_step_noalloc(const rlbm_domain *domain, int edf, int nsteps, const double *f_in,
                      double *f_out, void *cuda_stream, unsigned *warnings);

#ifdef __cplusplus
}
#endif
#endif /* RLBM_H */
