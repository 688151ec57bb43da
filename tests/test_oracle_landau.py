"""Pins of the oracle's Landau-frame solve and macroscopic state (Eqs. 21-25)."""
import math

import numpy as np
import pytest

Z_C = 1.0 - 1.0e-7


def _random_T(orc, edf, rng, amp):
    p, w, c, s = orc.lattice(edf)
    fe = orc.feq(edf, rng.uniform(0.8, 1.3), rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4),
                 {0: 0.16, 1: 0.5, 2: 0.5}[edf])
    f = fe * (1 + amp * rng.uniform(-1, 1, 72))
    return orc.moments72(edf, f)


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_landau_matches_numpy_eig(orc, edf):
    """The timelike eigenpair of T^a_b = T^{ag} eta_gb from numpy.linalg.eig."""
    rng = np.random.default_rng(11 + edf)
    eta = np.diag([1.0, -1.0, -1.0])
    for _ in range(20):
        N, T = _random_T(orc, edf, rng, 0.3)
        Tm = np.array([[T[0], T[1], T[2]], [T[1], T[3], T[4]], [T[2], T[4], T[5]]])
        vals, vecs = np.linalg.eig(Tm @ eta)
        # the energy eigenvalue is the one with a timelike eigenvector
        best = None
        for i in range(3):
            v = vecs[:, i].real
            nrm = v @ eta @ v
            if nrm > 0:
                best = (vals[i].real, v / math.sqrt(nrm) * np.sign(v[0]))
        assert best is not None
        eps, U, st, it = orc.landau(T)
        assert st == 0
        assert abs(eps - best[0]) <= 1e-13 * abs(best[0])
        np.testing.assert_allclose(U, best[1], rtol=0, atol=1e-12)
        # U is normalised, future-pointing
        assert abs(U[0] ** 2 - U[1] ** 2 - U[2] ** 2 - 1) < 1e-13 and U[0] > 0


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("umax,tol", [(0.5, 1e-13), (0.8, 1e-11)])
def test_state_round_trip(orc, edf, umax, tol):
    """(n, theta, u) -> f^eq -> N, T -> Landau state gives the same state back.
    At high Lorentz factor the FP64 round-off of the 72-term sums grows (the
    energy comes from U_a T^{ab} U_b, which cancels like gamma^4), hence the
    looser bound for |u| up to 0.8."""
    rng = np.random.default_rng(3 + edf)
    for _ in range(12):
        th = rng.uniform(0.7, 1.5)
        u = rng.uniform(0, umax)
        a = rng.uniform(0, 2 * math.pi)
        ux, uy = u * math.cos(a), u * math.sin(a)
        n = rng.uniform(0.3, 2.0)
        z, st = orc.z_from_n_theta(edf, n, th)
        if edf == 2 and st:
            continue
        fe = orc.feq(edf, th, ux, uy, z)
        N, T = orc.moments72(edf, fe)
        out, st = orc.state(edf, N, T)
        assert st == 0
        assert abs(out[0] - n) <= tol * n
        assert abs(out[1] - th) <= 2 * tol * th
        assert abs(out[2] - ux) <= tol and abs(out[3] - uy) <= tol
        assert abs(out[4] - z) <= 4 * tol * z


def test_be_fugacity_clamp(orc):
    """BE reading: a state below R(z_c) is clamped to z = z_c, keeping n, and flagged.
    A mixture of two z_c equilibria at different temperatures lies below R(z_c)
    (the Riemann problem at constant fugacity produces such states)."""
    fe = orc.feq(2, 1.0, 0.0, 0.0, Z_C) + orc.feq(2, 0.7, 0.0, 0.0, Z_C)
    N, T = orc.moments72(2, fe)
    out, st = orc.state(2, N, T)
    assert st & orc.W_CLAMPED_FUGACITY
    assert out[4] == Z_C
    assert abs(out[0] - 2 * math.pi * out[1] ** 2 * orc.g(2, 2, Z_C)) <= 1e-13 * out[0]
    # an equilibrium just inside the bound is not clamped
    fe = orc.feq(2, 1.0, 0.0, 0.0, 1.0 - 1e-6)
    out, st = orc.state(2, *orc.moments72(2, fe))
    assert st == 0 and abs(out[4] - (1.0 - 1e-6)) < 1e-12


def test_nonphysical_flagged(orc):
    """A tensor with no timelike energy eigenvector is flagged, not solved."""
    T = np.array([1.0, 2.0, 0.0, 1.0, 0.0, 0.0])
    out, st = orc.state(0, np.array([1.0, 0.0, 0.0]), T)
    assert st & orc.E_NONPHYSICAL
