"""Pins of the oracle's EDF integrals, equilibrium moments and discrete
fifth-order equilibrium (Secs. 2.3, 2.5 and the Appendix)."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Z_C = 1.0 - 1.0e-7


def _appendix():
    forms = {}
    with open(os.path.join(GOLDEN, "appendix_I2.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, expr = line.split(":", 1)
            forms[tuple(int(ch) for ch in key.strip())] = expr.strip()
    assert len(forms) == 56
    return forms


def _closed_form(orc, edf, expr, th, ux, uy, z):
    env = dict(pi=math.pi, th=th, ux=ux, uy=uy, u2=ux * ux + uy * uy,
               gam=1.0 / math.sqrt(1.0 - ux * ux - uy * uy))
    for nu in range(1, 7):
        env["g%d" % nu] = orc.g(edf, nu, z)
    return eval(expr, {"__builtins__": {}}, env)


def _trig_coeffs(n, q):
    """cos^n sin^q = a0 + sum_k a_k cos k phi + b_k sin k phi (exact via FFT)."""
    N = 32
    ph = 2 * np.pi * np.arange(N) / N
    F = np.fft.rfft(np.cos(ph) ** n * np.sin(ph) ** q) / N
    a = {0: F[0].real}
    b = {}
    for k in range(1, n + q + 1):
        a[k] = 2 * F[k].real
        b[k] = -2 * F[k].imag
    return a, b


def _I2_from_oracle(orc, edf, m, n, q, th, ux, uy, z, quad=True):
    """I_2^{mnq} rebuilt from the oracle's harmonic moments: by default those of the
    direct angular quadrature, which uses nothing of the closed forms."""
    M = orc.eq_moments_quad(edf, th, ux, uy, z) if quad else orc.eq_moments(edf, th, ux, uy, z)
    bn, bk, bc = orc.basis()
    idx = {(int(bn[i]), int(bk[i]), int(bc[i])): i for i in range(36)}
    d = m + n + q
    a, b = _trig_coeffs(n, q)
    val = a[0] * M[idx[(d, 0, 0)]]
    for k in range(1, n + q + 1):
        val += a[k] * M[idx[(d, k, 0)]] + b[k] * M[idx[(d, k, 1)]]
    return val


CASES = [
    (0, 1.0, 0.0, 0.0, 1 / (2 * math.pi)),
    (0, 1.3, 0.4, -0.25, 0.2),
    (1, 0.9, -0.3, 0.5, 1.0),
    (1, 1.1, 0.05, 0.02, 0.16),
    (2, 1.2, 0.2, 0.35, 0.5),
    (2, 0.8, -0.1, 0.0, Z_C),
]


@pytest.mark.parametrize("nu", range(1, 7))
def test_polylog_against_mpmath(orc, nu):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for z in [1e-6, 0.05, 0.3, 0.5, 0.500001, 0.8, 0.99, 0.999999, Z_C]:
        ref = float(mp.polylog(nu, z))
        assert abs(orc.g(2, nu, z) - ref) <= 2e-15 * abs(ref), ("BE", nu, z)
    for z in [1e-6, 0.05, 0.3, 0.5, 0.7, 1.0, 1.9, 2.0, 2.5, 10.0, 1e3]:
        ref = float(-mp.polylog(nu, -z))
        assert abs(orc.g(1, nu, z) - ref) <= 2e-15 * abs(ref), ("FD", nu, z)
    assert orc.g(0, nu, 0.37) == 0.37


@pytest.mark.parametrize("edf,th,ux,uy,z", CASES)
def test_closed_form_moments_equal_quadrature(orc, edf, th, ux, uy, z):
    """The oracle's harmonic moments from the Appendix closed forms equal those of
    the direct angular quadrature of their definition."""
    a = orc.eq_moments(edf, th, ux, uy, z)
    b = orc.eq_moments_quad(edf, th, ux, uy, z)
    bn, _, _ = orc.basis()
    for i in range(36):
        scale = abs(b[[j for j in range(36) if bn[j] == bn[i]][0]])
        assert abs(a[i] - b[i]) <= 2e-14 * scale, (i, a[i], b[i])


@pytest.mark.parametrize("edf,th,ux,uy,z", CASES)
def test_moments_match_appendix_closed_forms(orc, edf, th, ux, uy, z):
    """All 56 printed I_2^{mnq} against the oracle's angular-quadrature moments."""
    for (m, n, q), expr in _appendix().items():
        ref = _closed_form(orc, edf, expr, th, ux, uy, z)
        got = _I2_from_oracle(orc, edf, m, n, q, th, ux, uy, z)
        scale = abs(_closed_form(orc, edf, _appendix()[(m + n + q, 0, 0)], th, ux, uy, z))
        assert abs(got - ref) <= 1e-12 * scale, ((m, n, q), got, ref)


@pytest.mark.parametrize("edf,mnq", [(0, (0, 0, 0)), (1, (1, 1, 0)), (2, (0, 2, 1)), (1, (0, 0, 5)),
                                     (0, (2, 1, 1))])
def test_moments_brute_force_2d_integral(orc, edf, mnq):
    """Direct 2D momentum integral of the EDF of Eq. (8) on a tiny case."""
    from scipy import integrate
    th, ux, uy, z = 1.1, 0.3, -0.2, 0.4
    gam = 1 / math.sqrt(1 - ux * ux - uy * uy)
    xi = {0: 0.0, 1: 1.0, 2: -1.0}[edf]
    m, n, q = mnq

    def inner(ph):
        a = gam * (1 - ux * math.cos(ph) - uy * math.sin(ph)) / th
        fn = lambda p: p ** (m + n + q) * math.cos(ph) ** n * math.sin(ph) ** q * (
            z * math.exp(-p * a) / (1 + xi * z * math.exp(-p * a)))
        return integrate.quad(fn, 0, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]

    ref = integrate.quad(inner, 0, 2 * math.pi, epsabs=0, epsrel=1e-12, limit=200)[0]
    got = _I2_from_oracle(orc, edf, m, n, q, th, ux, uy, z, quad=False)
    scale = _I2_from_oracle(orc, edf, m + n + q, 0, 0, th, ux, uy, z)
    assert abs(got - ref) <= 1e-9 * abs(scale)


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_discrete_feq_reproduces_all_moments(orc, edf):
    """Eq. (16) with f^eq: sum_i f^eq_i p^m (p^x)^n (p^y)^q = I_2^{mnq} for all 56 forms."""
    rng = np.random.default_rng(7 + edf)
    p, w, c, s = orc.lattice(edf)
    P, C, S = np.tile(p, 12), np.repeat(c, 6), np.repeat(s, 6)
    for _ in range(4):
        th = rng.uniform(0.7, 1.4)
        u = rng.uniform(0, 0.6)
        a = rng.uniform(0, 2 * math.pi)
        ux, uy = u * math.cos(a), u * math.sin(a)
        z = {0: 1 / (2 * math.pi), 1: rng.uniform(0.1, 1.5), 2: rng.uniform(0.05, 0.9)}[edf]
        fe = orc.feq(edf, th, ux, uy, z)
        for (m, n, q), expr in _appendix().items():
            ref = _closed_form(orc, edf, expr, th, ux, uy, z)
            disc = np.sum(fe * P ** m * (P * C) ** n * (P * S) ** q)
            scale = abs(_closed_form(orc, edf, _appendix()[(m + n + q, 0, 0)], th, ux, uy, z))
            assert abs(disc - ref) <= 1e-12 * scale, ((m, n, q), disc, ref)


def test_fig1_expansion_errors(orc):
    """Sec. 2.3 / Fig. 1: MJ, theta = 1, beta = 0.6, p = (1, 0): 2nd order 18.5 %, 5th 1.8 %."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fig1_errors.txt")) if not l.startswith("#")]
    z = 1 / (2 * math.pi)
    exact = z * math.exp(-1.0 / math.sqrt(1 - 0.36) * (1 - 0.6))
    for order, pct in rows:
        v = orc.expansion_at(0, int(order), 1.0, 0.6, 0.0, z, 1.0, 0.0)
        rel = abs(v - exact) / exact * 100
        assert abs(rel - float(pct)) < 0.05, (order, rel, pct)
    # the orders converge toward the exact EDF (Fig. 1, right panel)
    errs = [abs(orc.expansion_at(0, o, 1.0, 0.6, 0.0, z, 1.0, 0.0) - exact) for o in (2, 3, 4, 5)]
    assert errs[3] < errs[0]


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_density_and_energy_closed_forms(orc, edf):
    """Eq. (25): the discrete f^eq gives n = 2 pi theta^2 g_2(z), eps = 2P = 4 pi theta^3 g_3(z)."""
    for th, ux, uy, z in [(1.0, 0.0, 0.0, 0.3), (1.25, 0.3, 0.1, 0.6), (0.85, -0.2, 0.4, 0.12)]:
        if edf == 0:
            z = 0.7
        fe = orc.feq(edf, th, ux, uy, z)
        N, T = orc.moments72(edf, fe)
        out, st = orc.state(edf, N, T)
        n_ref = 2 * math.pi * th ** 2 * orc.g(edf, 2, z)
        e_ref = 4 * math.pi * th ** 3 * orc.g(edf, 3, z)
        assert abs(out[0] - n_ref) <= 1e-13 * n_ref
        assert abs(out[5] - e_ref) <= 1e-13 * e_ref
        # MJ at rest: eps = 2P = 2 n T
        if edf == 0:
            assert abs(out[5] - 2 * out[0] * out[1]) <= 1e-13 * out[5]


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_feq_is_a_perfect_fluid_in_any_frame(orc, edf):
    """Lorentz covariance of the lowest equilibrium moments. For a state
    (theta, u, z) the discrete f^eq carries N^mu = n U^mu and T^{mu nu} =
    (eps + P) U^mu U^nu - P eta^{mu nu}, with the rest-frame n = 2 pi theta^2
    g_2(z) and eps = 2P = 4 pi theta^3 g_3(z) (Eq. 25). This checks the boosted
    moments through the perfect-fluid form alone, not the Appendix formulas."""
    p, w, c, s = orc.lattice(edf)
    P = np.tile(p, 12)
    pv = [P, P * np.repeat(c, 6), P * np.repeat(s, 6)]
    eta = np.diag([1.0, -1.0, -1.0])
    for th, ux, uy, z in [(1.0, 0.3, -0.2, 0.4), (0.8, -0.55, 0.1, 0.2), (1.3, 0.05, 0.62, 0.7)]:
        fe = orc.feq(edf, th, ux, uy, z)
        gam = 1.0 / math.sqrt(1.0 - ux * ux - uy * uy)
        U = np.array([gam, gam * ux, gam * uy])
        n = 2 * math.pi * th ** 2 * orc.g(edf, 2, z)
        eps = 4 * math.pi * th ** 3 * orc.g(edf, 3, z)
        pr = eps / 2
        for a in range(3):
            assert abs(np.sum(fe * pv[a]) - n * U[a]) <= 1e-13 * n * gam, (a, th, ux, uy)
            for b in range(3):
                ref = (eps + pr) * U[a] * U[b] - pr * eta[a, b]
                assert abs(np.sum(fe * pv[a] * pv[b]) - ref) <= 1e-12 * (eps + pr) * gam ** 2, (a, b)
