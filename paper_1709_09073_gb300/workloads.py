"""Seeded synthetic inputs: domain descriptions and initial macroscopic fields.

This module holds only input recipes (geometry, relaxation times, boundary
conditions and the initial n/z, theta, u fields); it performs none of the
method's arithmetic and imports neither the CUDA library nor the oracle, so the
same inputs feed both. Every workload mirrors an experiment of Sec. 3 of
arXiv:1709.09073 at the sizes the benchmark uses.
"""
from dataclasses import dataclass, field

import numpy as np

MJ, FD, BE = 0, 1, 2
PERIODIC, ZERO_GRADIENT, FIXED_T_WALL, VELOCITY_WALL, EXCHANGED = 0, 1, 2, 3, 4
INIT_N_THETA, INIT_Z_THETA = 0, 1
Z_C = 1.0 - 1.0e-7  # BE reference fugacity, Eq. (15)


@dataclass
class DomainSpec:
    nx: int
    ny: int
    tau: float
    edf: int = MJ
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)  # xlo, xhi, ylo, yhi
    t_wall: tuple = (1.0, 1.0, 1.0, 1.0)
    ref_n: float = 1.0       # reference equilibrium of the deviation storage formats
    ref_theta: float = 1.0
    scale: float = 1.0       # per-domain scale of the deviation storage formats
    eta_s: float = 0.0       # > 0: local tau = 4 eta_s / theta + 0.2546 (Sec. 3.5)
    accel: tuple = (0.0, 0.0)  # body acceleration (Sec. 3.4 forcing)
    n_wall: float = 1.0      # density of velocity walls


@dataclass
class InitialState:
    kind: int                # INIT_N_THETA: a = n;  INIT_Z_THETA: a = z
    a: np.ndarray            # [ny][nx]
    theta: np.ndarray
    ux: np.ndarray
    uy: np.ndarray


@dataclass
class Workload:
    name: str
    domains: list
    init: list               # one InitialState per domain
    steps: int
    meta: dict = field(default_factory=dict)

    @property
    def cells(self):
        return sum(d.nx * d.ny for d in self.domains)


def _grid(nx, ny):
    x = np.broadcast_to(np.arange(nx, dtype=np.float64)[None, :], (ny, nx))
    y = np.broadcast_to(np.arange(ny, dtype=np.float64)[:, None], (ny, nx))
    return x, y


def taylor_green_state(L, u0):
    """Taylor-Green vortex, Eqs. (27)-(28): n = 1, theta = 1, evaluated at integer (x, y)."""
    x, y = _grid(L, L)
    k = 2.0 * np.pi / L
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    one = np.ones((L, L))
    return InitialState(INIT_N_THETA, one.copy(), one.copy(), ux, uy)


def taylor_green(L=64, u0=0.01, tau=0.9, steps=500, edf=MJ):
    """Single periodic Taylor-Green domain (default: 64 x 64, tau = 0.9, 500 steps)."""
    return Workload("taylor_green_%dx%d_%s" % (L, L, "MJ FD BE".split()[edf]),
                    [DomainSpec(L, L, tau, edf)], [taylor_green_state(L, u0)], steps,
                    {"u0": u0})


# Riemann problem: quasi-1D, left pressure 5.4, right 2.2, u = 0, at the weight
# function's reference fugacity (z = 1 for MJ and FD, z = z_c for BE); the
# temperature follows from P = eps/2 = 2 pi theta^3 g_3(z), Eq. (25):
#   theta = (P / (2 pi g_3(z)))^(1/3), with g_3 = 1 (MJ), 3 zeta(3)/4 (FD), Li_3(z_c) (BE).
RIEMANN_THETA = {
    MJ: (0.95076086513236252, 0.70482441164894412),
    FD: (0.98418301806156748, 0.72960114588178238),
    BE: (0.89418965540560981, 0.66288666360503771),
}
RIEMANN_Z = {MJ: 1.0, FD: 1.0, BE: Z_C}


def riemann(edf=MJ, nx=2048, ny=4, tau=0.6, steps=1000):
    """Riemann problem, Sec. 3.1 geometry: zero-gradient ends in x, periodic in y."""
    x, _ = _grid(nx, ny)
    th_l, th_r = RIEMANN_THETA[edf]
    theta = np.where(x < nx // 2, th_l, th_r)
    z = np.full((ny, nx), RIEMANN_Z[edf])
    zero = np.zeros((ny, nx))
    bc = (ZERO_GRADIENT, ZERO_GRADIENT, PERIODIC, PERIODIC)
    return Workload("riemann_%dx%d_%s" % (nx, ny, "MJ FD BE".split()[edf]),
                    [DomainSpec(nx, ny, tau, edf, bc)],
                    [InitialState(INIT_Z_THETA, z, theta, zero, zero.copy())], steps)


def hot_spot(L=8192, sigma=64.0, peak=0.5, tau=0.8, steps=2000, edf=BE):
    """Hot-spot relaxation (Sec. 3.5 experiment, Gaussian profile): n = 1, u = 0,
    theta = 1 + peak exp(-r^2 / (2 sigma^2)) about the domain centre, periodic."""
    x, y = _grid(L, L)
    r2 = (x - L // 2) ** 2 + (y - L // 2) ** 2
    theta = 1.0 + peak * np.exp(-r2 / (2.0 * sigma * sigma))
    one = np.ones((L, L))
    zero = np.zeros((L, L))
    return Workload("hot_spot_%dx%d_%s" % (L, L, "MJ FD BE".split()[edf]),
                    [DomainSpec(L, L, tau, edf)],
                    [InitialState(INIT_N_THETA, one, theta, zero, zero.copy())], steps,
                    {"sigma": sigma})


def hot_spot_step(L=512, radius=32.0, th_in=1.5, th_out=0.5, eta_s=0.5, steps=100, edf=MJ):
    """Hot-spot relaxation of the order comparison (Sec. 3.5): n = 1, u = 0,
    theta = th_in inside the disc of the given radius about the centre and
    th_out outside; open (zero-gradient) borders; local tau = 4 eta_s / theta
    + 0.2546."""
    x, y = _grid(L, L)
    r2 = (x - L // 2) ** 2 + (y - L // 2) ** 2
    theta = np.where(r2 <= radius * radius, th_in, th_out).astype(np.float64)
    one = np.ones((L, L))
    zero = np.zeros((L, L))
    zg = (ZERO_GRADIENT,) * 4
    spec = DomainSpec(L, L, 1.0, edf, zg, eta_s=eta_s)
    return Workload("hot_spot_step_%dx%d_%s" % (L, L, "MJ FD BE".split()[edf]), [spec],
                    [InitialState(INIT_N_THETA, one, theta, zero, zero.copy())], steps,
                    {"radius": radius})


def batched_taylor_green(n_domains=256, side_lo=32, side_hi=512, seed=20260101, steps=200,
                         tau_lo=0.55, tau_hi=2.0, edf=MJ):
    """Many periodic Taylor-Green domains of uneven size (a viscosity sweep over tau,
    Sec. 3.2): sides uniform in [side_lo, side_hi], amplitudes uniform in [0.005, 0.05]."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=n_domains)
    amps = rng.uniform(0.005, 0.05, size=n_domains)
    taus = np.linspace(tau_lo, tau_hi, n_domains)
    doms, inits = [], []
    for L, a, t in zip(sides, amps, taus):
        doms.append(DomainSpec(int(L), int(L), float(t), edf))
        inits.append(taylor_green_state(int(L), float(a)))
    return Workload("batched_taylor_green_x%d_%s" % (n_domains, "MJ FD BE".split()[edf]), doms, inits,
                    steps, {"seed": seed, "sides": sides.tolist(), "amps": amps.tolist()})


def fourier_state(nx, ny, th_cold, th_hot):
    """Fourier flow, Sec. 3.3: n = 1, u = 0, linear initial temperature profile."""
    x, _ = _grid(nx, ny)
    theta = th_cold + x * (th_hot - th_cold) / nx
    one = np.ones((ny, nx))
    zero = np.zeros((ny, nx))
    return InitialState(INIT_N_THETA, one, theta, zero, zero.copy())


def batched_fourier(n_domains=64, nx=1024, ny=256, tau_lo=0.6, tau_hi=1.5, th_cold=0.95,
                    th_hot=1.05, steps=200, edf=FD, scale=1.0):
    """Many Fourier-flow domains (a conductivity sweep over tau, Sec. 3.3): fixed-T walls
    at x = -1 (cold) and x = nx (hot), periodic in y."""
    taus = np.linspace(tau_lo, tau_hi, n_domains)
    bc = (FIXED_T_WALL, FIXED_T_WALL, PERIODIC, PERIODIC)
    doms = [DomainSpec(nx, ny, float(t), edf, bc, (th_cold, th_hot, 1.0, 1.0), 1.0, 1.0, scale)
            for t in taus]
    inits = [fourier_state(nx, ny, th_cold, th_hot) for _ in taus]
    return Workload("batched_fourier_x%d_%dx%d_%s" % (n_domains, nx, ny, "MJ FD BE".split()[edf]),
                    doms, inits, steps)


def random_domain_state(nx, ny, seed, edf=MJ, u_amp=0.1, th_amp=0.1):
    """Smooth random fields for parity tests: n, theta near 1, |u| <= u_amp."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    def smooth():
        out = np.zeros((ny, nx))
        for _ in range(3):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            out += rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
        return out / 3.0
    n = 1.0 + 0.1 * smooth()
    theta = 1.0 + th_amp * smooth()
    ux = u_amp * smooth()
    uy = u_amp * smooth()
    return InitialState(INIT_N_THETA, n, theta, ux, uy)
