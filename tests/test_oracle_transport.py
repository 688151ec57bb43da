"""Transport coefficients of the oracle against closed forms derived from the
method itself (Sec. 3.2 viscosity, Sec. 3.3 conductivity, Sec. 3.4 grid
convergence). None of these goes through the oracle's own formulas.

Numerical viscosity of the interpolated streaming (Eqs. 17-18). Linear
interpolation between two nodes at fractional distance a spreads a population
like a diffusion of coefficient a(1 - a)/2 per step along that axis; the
bilinear pull is the product of two such 1-D interpolations, so population d
diffuses with the diagonal tensor D_d = diag(|v_x|(1-|v_x|), |v_y|(1-|v_y|))/2
(zero for the four axis directions; 1/8 along the component 1/2 and
(sqrt(3)/2 - 3/4)/2 along the component sqrt(3)/2). Taking the first
moment p^0 p^x of that diffusion over the linear response of the equilibrium
to a shear velocity, the radial integrals cancel against the momentum density
eps + P (for every EDF), and the extra kinematic viscosity is the angular
average of D_d weighted by the squared velocity component along the flow:
  shear u_x(y) (along a lattice axis):     sum_d cos^2(phi_d) D_d,yy / 6 = sqrt(3)/24,
  shear along a diagonal (the Taylor-Green vortex is a sum of two):
                                            (sqrt(3) - 1)/12.
With the usual (tau - 1/2)/4 of the relaxation, the two offsets delta in
nu = (tau - delta)/4 are 1/2 - sqrt(3)/6 = 0.21132 (axis) and
(5 - 2 sqrt(3))/6 = 0.25598 (diagonal). The paper's fitted 0.2546 (Sec. 3.2)
is the diagonal one measured at the amplitude u_0 = 0.1, where the decay is
no longer linear.

Heat conductivity. First-order Chapman-Enskog expansion of the
Anderson-Witting equation (Eq. 3) about a fluid at rest with a temperature
gradient along x and uniform pressure (dP = 0 fixes d ln z = -3 (g_3/g_2)
d ln T through P = 2 pi T^3 g_3(z), Eq. 25) gives the particle diffusion
current, and with h_E = 3 T g_3/g_2 the heat flux q^x = -kappa dT/dx with
  kappa = (3/2) tau n (g_3/g_2) (3 g_1 g_3 / g_2^2 - 2),
the integrals int p^k f(1 -+ f) dp reducing to T^k Gamma(k) g_{k-1} by parts.
The moment this needs (p/2 at rest, degree one) lies in the span of the
fifth-order expansion, so the discrete model has the same coefficient. For MJ
(g_nu = z) it is 1.5 tau n, the printed a_MJ = 1.4999998; for FD and BE it
differs from the printed kappa g_2/g_3 = 1.5 tau by the factor
n (3 g_1 g_3/g_2^2 - 2), which is 1 only where g_1 g_3 = g_2^2 (MJ, or the
classical limit z -> 0): about 0.94 (FD) and 1.06 (BE) at the channel's
fugacity z ~ 0.16. g_1 is taken here in closed form: ln(1 + z) (FD),
-ln(1 - z) (BE)."""
import math

import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W

DELTA_AXIS = 0.5 - math.sqrt(3.0) / 6.0             # shear along a lattice axis
DELTA_DIAG = (5.0 - 2.0 * math.sqrt(3.0)) / 6.0     # shear along a diagonal (Taylor-Green)


def _wave_decay(orc, kind, L, tau, edf=W.MJ, amp=1e-4, efolds=0.6):
    """Kinematic viscosity from the decay of one low-amplitude shear wave: the
    amplitude's log over `efolds` e-foldings after a short start-up transient,
    divided by k^2. kind 'axis': u_x = A sin(2 pi y / L) on an L x 1 column;
    'diag': u = A (1, -1)/sqrt(2) sin(2 pi (x + y)/L) on L x L."""
    if kind == "axis":
        nx, ny = 1, L
        x, y = np.zeros((L, 1)), np.arange(L, dtype=float)[:, None]
        ph = 2 * math.pi * y / L
        ux, uy = amp * np.sin(ph), np.zeros((L, 1))
        k2 = (2 * math.pi / L) ** 2
        proj = lambda o: 2 * np.mean(o[2] * np.sin(ph))
    else:
        nx = ny = L
        y, x = np.mgrid[0:L, 0:L].astype(float)
        ph = 2 * math.pi * (x + y) / L
        ux, uy = amp * np.sin(ph) / math.sqrt(2), -amp * np.sin(ph) / math.sqrt(2)
        k2 = 2 * (2 * math.pi / L) ** 2
        proj = lambda o: 2 * np.mean((o[2] - o[3]) / math.sqrt(2) * np.sin(ph))
    dom = orc.domain(nx, ny, tau, edf)
    one = np.ones((ny, nx))
    f, m, _ = orc.init(dom, W.INIT_N_THETA, one, one, ux, uy)
    steps = int(efolds / ((tau - 0.25) / 4 * k2))
    f, m, _ = orc.run(dom, f, m, max(4, int(8 * tau)))
    a0 = proj(orc.fields(dom, f, m, streamed=False)[0])
    f, m, _ = orc.run(dom, f, m, steps)
    a1 = proj(orc.fields(dom, f, m, streamed=False)[0])
    return math.log(a0 / a1) / steps / k2, k2


def _delta_extrapolated(orc, kind, sizes, tau, edf=W.MJ):
    """Offset delta of nu = (tau - delta)/4, with the O(k^2) lattice correction
    of the decay rate removed by Richardson extrapolation over two sizes."""
    (nu1, k1), (nu2, k2) = (_wave_decay(orc, kind, L, tau, edf) for L in sizes)
    nu = nu2 - (nu1 - nu2) * k2 / (k1 - k2)
    return tau - 4.0 * nu


@pytest.mark.parametrize("tau", [0.8, 1.4])
def test_shear_viscosity_closed_forms(orc, tau):
    """Axis and diagonal shear waves (MJ) decay with the closed-form numerical
    viscosities of the bilinear streaming, and their excess viscosities stand
    in the ratio sqrt(3)/(2 (sqrt(3) - 1)) = 1.1830."""
    d_axis = _delta_extrapolated(orc, "axis", (64, 128), tau)
    d_diag = _delta_extrapolated(orc, "diag", (32, 64), tau)
    print("tau %.1f: delta axis %.5f (closed form %.5f), diagonal %.5f (%.5f)"
          % (tau, d_axis, DELTA_AXIS, d_diag, DELTA_DIAG))
    assert abs(d_axis - DELTA_AXIS) <= 3e-4
    assert abs(d_diag - DELTA_DIAG) <= 3e-4
    ratio = (0.5 - d_axis) / (0.5 - d_diag)
    assert abs(ratio - math.sqrt(3.0) / (2.0 * (math.sqrt(3.0) - 1.0))) <= 2e-3


@pytest.mark.parametrize("edf", [W.FD, W.BE])
def test_shear_viscosity_is_edf_independent(orc, edf):
    """The numerical viscosity does not depend on the distribution (the radial
    integrals cancel): FD and BE axis shear waves give the same offset as MJ."""
    d = _delta_extrapolated(orc, "axis", (32, 64), 1.1, edf)
    assert abs(d - DELTA_AXIS) <= 5e-4, d


def test_taylor_green_paper_protocol(orc):
    """Sec. 3.2 as printed: sigma_{u^2} of the Taylor-Green vortex at u_0 = 0.1,
    fitted over the decay the paper follows (sigma falls by e^-3.7, as in 45000
    steps at L = 512, tau = 0.8). On 64^2 the fit gives delta within 1e-3 of the
    printed 0.2546 (delta_nu = -0.2454); the low-amplitude limit is the closed
    form 0.25598 (test above)."""
    L, tau, u0 = 64, 0.8, 0.1
    wl = W.taylor_green(L=L, u0=u0, tau=tau, steps=0)
    d, s = wl.domains[0], wl.init[0]
    dom = orc.domain(d.nx, d.ny, d.tau, d.edf)
    f, macro, _ = orc.init(dom, s.kind, s.a, s.theta, s.ux, s.uy)
    nu0 = (tau - 0.2546) / 4
    total = int(3.7 * L * L / (16 * math.pi ** 2 * nu0))
    every = total // 12
    ts, sig = [], []
    for i in range(13):
        if i:
            f, macro, _ = orc.run(dom, f, macro, every)
        out, _ = orc.fields(dom, f, macro, streamed=False)
        u2 = out[2] ** 2 + out[3] ** 2
        ts.append(i * every)
        sig.append(math.sqrt(np.mean((u2 - u2.mean()) ** 2)))
    slope = np.polyfit(ts[1:], np.log(sig[1:]), 1)[0]
    nu = -slope * L * L / (16 * math.pi ** 2)
    delta = tau - 4 * nu
    print("Taylor-Green u0 = 0.1: delta %.5f (printed 0.2546)" % delta)
    assert abs(delta - 0.2546) <= 1e-3


def _poiseuille_error(orc, L, nu_ref, tau=3.0, a=1e-8, edf=W.MJ):
    """Steady forced channel (Sec. 3.4) of width L between velocity walls at the
    ghost rows y = -1 and y = L; eps_u against u_ref = a/(2 nu_ref) (y+1)(L-y)."""
    bc = (W.PERIODIC, W.PERIODIC, W.VELOCITY_WALL, W.VELOCITY_WALL)
    dom = orc.domain(1, L, tau, edf, bc, accel=(a, 0.0), n_wall=1.0)
    y = np.arange(L, dtype=float)
    guess = a / (2 * nu_ref) * (y + 1) * (L - y)   # start near the answer
    one, zero = np.ones((L, 1)), np.zeros((L, 1))
    f, m, _ = orc.init(dom, W.INIT_N_THETA, one, one, guess[:, None], zero)
    f, m, _ = orc.run(dom, f, m, int(6 * (L + 1) ** 2 / nu_ref) + 2000)
    ux = orc.fields(dom, f, m, streamed=False)[0][2][:, 0]
    f2, m2, _ = orc.run(dom, f, m, 500)
    ux2 = orc.fields(dom, f2, m2, streamed=False)[0][2][:, 0]
    assert np.max(np.abs(ux2 - ux)) <= 1e-10 * np.max(np.abs(ux))   # steady
    return math.sqrt(np.sum((ux - guess) ** 2) / np.sum(guess ** 2))


def test_poiseuille_grid_convergence(orc):
    """Sec. 3.4 (tau = 3, a = 1e-8): against the axis-shear viscosity (the
    channel is a shear along a lattice axis) eps_u falls as L^-2 (fitted slope
    -2 +- 0.1 over L = 8..64; the paper prints -2.037). Against the Taylor-Green
    law nu = (tau - 0.2546)/4 the paper uses as reference, eps_u stays at the
    1.6 % the two viscosities differ by: that reference cannot give the slope."""
    tau = 3.0
    nu_axis = (tau - DELTA_AXIS) / 4
    sizes = (8, 16, 32, 64)
    errs = [_poiseuille_error(orc, L, nu_axis, tau) for L in sizes]
    slope = np.polyfit(np.log(sizes), np.log(errs), 1)[0]
    print("eps_u", ["%.3e" % e for e in errs], "slope %.3f" % slope)
    assert abs(slope + 2.0) <= 0.1
    assert errs[-1] <= 2e-4
    e_tg = _poiseuille_error(orc, 32, (tau - 0.2546) / 4, tau)
    assert 0.01 <= e_tg <= 0.02


def _kappa(orc, edf, nx, steps, tau, dts=(5e-4, 1e-3, 1.5e-3)):
    """Sec. 3.3 measurement: slope of <q^x> against <F(dT)> over three wall
    temperature differences, F = -[(1 + u^2 gamma^2) dT/dx + T gamma (d(gamma u)/dt
    + u d(gamma u)/dx)], averages over the inner 7/8 of the channel. Returns the
    slope and the channel's mean n and z."""
    pts = []
    for dT in dts:
        thL, thR = 1 - dT / 2, 1 + dT / 2
        dom = orc.domain(nx, 2, tau, edf, (W.FIXED_T_WALL, W.FIXED_T_WALL, W.PERIODIC, W.PERIODIC),
                         (thL, thR, 1.0, 1.0))
        st = W.fourier_state(nx, 2, thL, thR)
        f, m, _ = orc.init(dom, st.kind, st.a, st.theta, st.ux, st.uy)
        f, m, _ = orc.run(dom, f, m, steps - 1)
        prev = orc.fields(dom, f, m, True)[0]
        f, m, _ = orc.run(dom, f, m, 1)
        fl = orc.fields(dom, f, m, True)[0]
        d = orc.diagnostics(dom, f, m, True)[0]
        th, ux = fl[1], fl[2]
        g, g0 = 1 / np.sqrt(1 - ux ** 2), 1 / np.sqrt(1 - prev[2] ** 2)
        F = -((1 + ux ** 2 * g ** 2) * np.gradient(th, axis=1)
              + th * g * ((g * ux - g0 * prev[2]) + ux * np.gradient(g * ux, axis=1)))
        core = slice(nx // 16, nx - nx // 16)
        pts.append((F[:, core].mean(), d[1][:, core].mean(), fl[0][:, core].mean(), fl[4][:, core].mean()))
    slope = np.polyfit([p[0] for p in pts], [p[1] for p in pts], 1)[0]
    return slope, np.mean([p[2] for p in pts]), np.mean([p[3] for p in pts])


def _g1(edf, z):
    return z if edf == W.MJ else (math.log1p(z) if edf == W.FD else -math.log1p(-z))


@pytest.mark.parametrize("edf", [W.MJ, W.FD, W.BE])
def test_conductivity_chapman_enskog(orc, edf):
    """kappa of a 256 x 2 Fourier channel (1000 steps, tau = 0.8) equals the
    Chapman-Enskog coefficient (3/2) tau n (g_3/g_2)(3 g_1 g_3/g_2^2 - 2) to 1e-4
    for MJ, FD and BE. For MJ this is the printed law kappa g_2/g_3 = 1.5 tau
    (a_MJ = 1.4999998); for FD and BE the printed law misses by the factor
    n (3 g_1 g_3/g_2^2 - 2), more than 5 % here."""
    tau = 0.8
    kappa, n, z = _kappa(orc, edf, 256, 1000, tau)
    g1, g2, g3 = _g1(edf, z), orc.g(edf, 2, z), orc.g(edf, 3, z)
    factor = 3.0 * g1 * g3 / g2 ** 2 - 2.0
    kappa_ce = 1.5 * tau * n * (g3 / g2) * factor
    print("edf %d: kappa %.6f, Chapman-Enskog %.6f, ratio %.6f; printed-law ratio %.5f (n %.5f z %.5f)"
          % (edf, kappa, kappa_ce, kappa / kappa_ce, kappa / (1.5 * tau * g3 / g2), n, z))
    assert abs(kappa / kappa_ce - 1.0) <= 1e-4
    if edf == W.MJ:
        assert abs(kappa * g2 / g3 / tau - 1.5) <= 1e-4
    else:
        assert abs(n * factor - 1.0) >= 0.05
