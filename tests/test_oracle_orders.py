"""Pins of the oracle's lower expansion orders (Eq. 10 truncated at N = 2..4,
Sec. 3.5) and of the local relaxation time tau = 4 (eta/s) / theta + 0.2546:
the discrete order-N equilibrium reproduces every equilibrium moment of degree
<= N (Appendix closed forms) and equals the order-N expansion of Fig. 1 at
the nodes; a step with eta/s relaxes each cell at the rate its own temperature
sets."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W

STATES = [(1.0, 0.05, -0.02, 0.3), (1.3, 0.3, 0.2, 0.12), (0.8, -0.45, 0.1, 0.05)]


def _node_basis(orc, edf):
    p, w, c, s = orc.lattice(edf)
    bn, bk, bc = orc.basis()
    d = np.repeat(np.arange(12), 6)
    P = np.tile(p, 12)
    phi = d * np.pi / 6
    B = np.array([P ** bn[a] * (np.sin(bk[a] * phi) if bc[a] else np.cos(bk[a] * phi)) for a in range(36)])
    return B, bn, np.tile(w, 12), P, phi


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_order_n_reproduces_moments_up_to_degree_n(orc, edf, order):
    B, bn, w, P, phi = _node_basis(orc, edf)
    for th, ux, uy, z in STATES:
        if edf == 2:
            z = min(z, 0.5)
        f = orc.feq_order(edf, order, th, ux, uy, z)
        M = orc.eq_moments(edf, th, ux, uy, z)
        got = B @ f
        for a in range(36):
            if bn[a] <= order:
                assert abs(got[a] - M[a]) <= 1e-12 * (abs(M[a]) + np.max(np.abs(M[bn == bn[a]]))), (a, order)
    if order < 5:  # the truncation is real: some degree-(N+1) moment is missed
        f = orc.feq_order(edf, order, 1.3, 0.3, 0.2, 0.12 if edf < 2 else 0.12)
        M = orc.eq_moments(edf, 1.3, 0.3, 0.2, 0.12)
        sel = bn == order + 1
        assert np.max(np.abs((B @ f)[sel] - M[sel])) > 1e-6 * np.max(np.abs(M[sel]))


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_order_n_equals_the_expansion_of_fig1_at_the_nodes(orc, edf, order):
    B, bn, w, P, phi = _node_basis(orc, edf)
    zc = 1.0 - 1e-7
    omega = {0: lambda p: np.exp(-p) / (2 * np.pi), 1: lambda p: 1.0 / (np.exp(p) + 1.0),
             2: lambda p: 1.0 / (np.exp(p) / zc - 1.0)}[edf]
    th, ux, uy, z = 1.2, 0.25, -0.15, 0.2
    f = orc.feq_order(edf, order, th, ux, uy, z)
    for q in range(72):
        e = orc.expansion_at(edf, order, th, ux, uy, z, P[q], phi[q])
        assert abs(f[q] - w[q] * e / omega(P[q])) <= 1e-11 * abs(f).max(), q


def test_local_relaxation_time(orc):
    """One step with eta/s = 0.5: per cell, (f_local - f_pulled) / (f_tau1 - f_pulled)
    = 1 / tau(theta) with tau = 4 eta_s / theta + 0.2546 (theta of the pulled state)."""
    nx, ny, eta = 10, 7, 0.5
    init = W.random_domain_state(nx, ny, 5, 0, u_amp=0.08, th_amp=0.3)
    def one(tau, eta_s=0.0):
        dom = orc.domain(nx, ny, tau, 0, eta_s=eta_s)
        f, m, _ = orc.init(dom, init.kind, init.a, init.theta, init.ux, init.uy)
        f1, _, _ = orc.step(dom, f, m)
        return dom, f, m, f1
    dom, f0, m0, f_loc = one(1.0, eta)
    _, _, _, f_1 = one(1.0)
    _, _, _, f_pull = one(1e30)
    theta = orc.fields(dom, f0, m0, streamed=True)[0][1]
    tau = 4 * eta / theta + 0.2546
    a, b = f_loc - f_pull, f_1 - f_pull
    q = np.argmax(np.abs(b), axis=0)
    yy, xx = np.indices((ny, nx))
    ratio = a[q, yy, xx] / b[q, yy, xx]
    assert np.max(np.abs(ratio * tau - 1.0)) <= 1e-9
    assert np.ptp(tau) > 0.1  # the temperatures differ enough for tau to vary
