"""Pins of the oracle's diagnostic fields (heat flux, Sec. 3.3; diagonal
non-equilibrium tensors, Sec. 3.1) against facts that do not go through them:
they vanish at equilibrium; pi^{x..x} equals the raw moment minus the
Appendix closed-form equilibrium moment (cos^k expanded in harmonics), and
pi^{xx} minus the perfect-fluid stress P + (eps + P) gamma^2 u_x^2 with P = eps/2;
the heat flux is orthogonal to U (q^mu U_mu = 0, since n = U_mu N^mu). The
conductivity it gives in a Fourier flow is pinned in test_oracle_transport.py."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W

# cos^k(phi) = sum_j A[k][j] cos(j phi)
COS_POW = {2: {0: 0.5, 2: 0.5}, 3: {1: 0.75, 3: 0.25}, 4: {0: 0.375, 2: 0.5, 4: 0.125},
           5: {1: 0.625, 3: 0.3125, 5: 0.0625}}


def _state(orc, edf, steps):
    spec = W.DomainSpec(14, 9, 0.8, edf, (W.FIXED_T_WALL, W.FIXED_T_WALL, W.PERIODIC, W.PERIODIC),
                        (0.96, 1.05, 1.0, 1.0))
    init = W.random_domain_state(14, 9, 90 + edf, edf, u_amp=0.12, th_amp=0.1)
    dom = orc.domain(spec.nx, spec.ny, spec.tau, edf, spec.bc, spec.t_wall)
    f, m, _ = orc.init(dom, init.kind, init.a, init.theta, init.ux, init.uy)
    f, m, _ = orc.run(dom, f, m, steps)
    return dom, f, m


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_zero_at_equilibrium(orc, edf):
    dom, f, m = _state(orc, edf, 0)
    d, st = orc.diagnostics(dom, f, m, streamed=False)
    p, w, c, s = orc.lattice(edf)
    for k in range(2, 6):
        scale = np.max(np.abs(np.einsum("qyx,q->yx", f, np.abs(np.tile(p, 12) * np.repeat(c, 6)) ** k)))
        assert np.max(np.abs(d[k + 1])) <= 1e-13 * scale, k
    fl, _ = orc.fields(dom, f, m, streamed=False)
    assert np.max(np.abs(d[:3])) <= 1e-13 * np.max(fl[0] * fl[1])


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_pi_against_closed_forms_and_q_orthogonal_to_u(orc, edf):
    dom, f, m = _state(orc, edf, 4)
    d, st = orc.diagnostics(dom, f, m, streamed=False)
    fl, _ = orc.fields(dom, f, m, streamed=False)
    p, w, c, s = orc.lattice(edf)
    P, C = np.tile(p, 12), np.repeat(c, 6)
    bn, bk, bc = orc.basis()
    idx = {(int(bn[a]), int(bk[a])): a for a in range(36) if bc[a] == 0}
    for y in range(dom.ny):
        for x in range(dom.nx):
            n, th, ux, uy, z, eps = fl[:, y, x]
            M = orc.eq_moments(edf, th, ux, uy, z)
            for k in range(2, 6):
                raw = np.sum(f[:, y, x] * (P * C) ** k)
                eq = sum(a * M[idx[(k, j)]] for j, a in COS_POW[k].items())
                scale = np.sum(f[:, y, x] * np.abs(P * C) ** k)
                assert abs(d[k + 1, y, x] - (raw - eq)) <= 1e-12 * scale, (k, x, y)
            # second order against the perfect-fluid stress of a conformal gas
            g2 = 1.0 / (1.0 - ux * ux - uy * uy)
            txx = np.sum(f[:, y, x] * (P * C) ** 2)
            assert abs(d[3, y, x] - (txx - (eps / 2 + 1.5 * eps * g2 * ux * ux))) <= 1e-12 * txx
            # Landau frame: n = U_mu N^mu, hence q^mu U_mu = 0 (metric +,-,-)
            qU = np.sqrt(g2) * (d[0, y, x] - d[1, y, x] * ux - d[2, y, x] * uy)
            # (q is a difference of O(h_E n) terms: bound relative to h_E n)
            assert abs(qU) <= 1e-13 * 3.0 * th * n
    # the states are genuinely out of equilibrium
    assert np.max(np.abs(d[3])) > 1e-6 and np.max(np.abs(d[1])) > 1e-7


@pytest.mark.parametrize("edf", [0, 2])
def test_heat_flux_from_raw_moments_and_enthalpy(orc, edf):
    """q^a = h_E (n U^a - N^a) with h_E = (eps + P)/n = 3 eps / (2 n) from the
    state's n and eps, and N^a summed from the populations directly."""
    dom, f, m = _state(orc, edf, 3)
    d, _ = orc.diagnostics(dom, f, m, streamed=False)
    fl, _ = orc.fields(dom, f, m, streamed=False)
    p, w, c, s = orc.lattice(edf)
    P, C, S = np.tile(p, 12), np.repeat(c, 6), np.repeat(s, 6)
    N = np.stack([np.einsum("qyx,q->yx", f, P), np.einsum("qyx,q->yx", f, P * C),
                  np.einsum("qyx,q->yx", f, P * S)])
    n, th, ux, uy, z, eps = fl
    gam = 1.0 / np.sqrt(1.0 - ux ** 2 - uy ** 2)
    U = np.stack([gam, gam * ux, gam * uy])
    want = 1.5 * eps / n * (n * U - N)
    assert np.max(np.abs(d[:3] - want)) <= 1e-12 * np.max(1.5 * eps)
