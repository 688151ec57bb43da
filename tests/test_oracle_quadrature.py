"""Pins of the oracle's d2v72 quadrature (Sec. 2.4) against what the paper and
the mathematics fix: the printed nodes/weights, Gauss-Laguerre, the FD moment
identities and the degree-10 exactness of Eq. (16)."""
import math
import os

import numpy as np
import pytest
from scipy.special import beta as B

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _printed():
    rows = {}
    with open(os.path.join(GOLDEN, "quadrature_printed.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            e, s, p, w = line.split()
            rows.setdefault(e, []).append((int(s), p, w))
    return rows


def _digits_match(value, printed):
    """True when the printed decimal string is value rounded or truncated to its
    digits (the paper's BE w_2 = 5.510286e-1 is the truncation of 0.55102865...)."""
    mant = printed.lower().split("e")[0]
    dec = len(mant.split(".")[1]) if "." in mant else 0
    exp = int(printed.lower().split("e")[1]) if "e" in printed.lower() else 0
    scaled = value / 10.0 ** exp
    return abs(scaled - float(mant)) <= 1.0 * 10.0 ** (-dec) * (1 + 1e-9)


@pytest.mark.parametrize("name,edf", [("MJ", 0), ("BE", 2)])
def test_printed_nodes_and_weights(orc, name, edf):
    p, w, _, _ = orc.lattice(edf)
    for s, ps, ws in _printed()[name]:
        assert _digits_match(p[s - 1], ps), (name, s, p[s - 1], ps)
        assert _digits_match(w[s - 1], ws), (name, s, w[s - 1], ws)


def test_mj_is_gauss_laguerre(orc):
    """MJ shells are the 6-point Gauss-Laguerre rule; w_s = w_GL / 12 (omega = e^-p / 2 pi)."""
    x, wl = np.polynomial.laguerre.laggauss(6)
    p, w, _, _ = orc.lattice(orc.MJ)
    np.testing.assert_allclose(p, x, rtol=1e-14)
    np.testing.assert_allclose(w, wl / 12.0, rtol=1e-13)


def _radial_moment(edf, k):
    """int_0^inf p^k omega(p) dp for the weight functions of Eqs. (13)-(15)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    if edf == 0:
        return float(mp.factorial(k) / (2 * mp.pi))
    if edf == 1:
        return float(mp.factorial(k) * (mp.log(2) if k == 0 else mp.altzeta(k + 1)))
    return float(mp.factorial(k) * mp.polylog(k + 1, 1 - mp.mpf(10) ** -7))


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_radial_exactness_degree_11(orc, edf):
    """sum_s lambda_s p_s^k equals the radial moment for k <= 11 (6-node Gauss)."""
    p, w, _, _ = orc.lattice(edf)
    lam = w * 12.0 / (2.0 * math.pi)
    for k in range(12):
        exact = _radial_moment(edf, k)
        assert abs(np.sum(lam * p ** k) - exact) <= 1e-13 * exact, (edf, k)


def test_fd_weight_sum(orc):
    """12 sum_s w_s = 2 pi ln 2 for omega = 1/(e^p + 1)."""
    _, w, _, _ = orc.lattice(orc.FD)
    assert abs(12 * np.sum(w) - 2 * math.pi * math.log(2)) < 1e-14


def _angular(b, c):
    """int_0^{2 pi} cos^b sin^c dphi (Beta function closed form)."""
    if b % 2 or c % 2:
        return 0.0
    return 2.0 * B((b + 1) / 2.0, (c + 1) / 2.0)


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_d2v72_exact_to_degree_10(orc, edf):
    """Eq. (16): sum_i w_i (p^0)^a (p^x)^b (p^y)^c = int d^2p/p^0 omega (...) for a+b+c <= 10."""
    p, w, cphi, sphi = orc.lattice(edf)
    P = np.tile(p, 12)
    W = np.tile(w, 12)
    C = np.repeat(cphi, 6)
    S = np.repeat(sphi, 6)
    worst = 0.0
    for a in range(11):
        for b in range(11 - a):
            for c in range(11 - a - b):
                deg = a + b + c
                disc = np.sum(W * P ** deg * C ** b * S ** c)
                cont = _radial_moment(edf, deg) * _angular(b, c)
                scale = _radial_moment(edf, deg) * 2 * math.pi
                worst = max(worst, abs(disc - cont) / scale)
    assert worst < 1e-13, worst
