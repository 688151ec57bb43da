"""Pins of the oracle's time step: streaming (Eqs. 17-18), relaxation (Eq. 3),
boundary ghosts, conservation and symmetry. The viscosity law is pinned in
test_oracle_transport.py."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W


def _conserved(orc, edf, f):
    """Global N^0 and T^{mu 0}: the densities that streaming transports."""
    p, w, c, s = orc.lattice(edf)
    P, C, S = np.tile(p, 12), np.repeat(c, 6), np.repeat(s, 6)
    fs = f.reshape(72, -1).sum(axis=1)
    return np.array([np.sum(fs * P), np.sum(fs * P * P), np.sum(fs * P * P * C), np.sum(fs * P * P * S)])


def _perturbed(orc, dom, seed, amp=0.05):
    st = W.random_domain_state(dom.nx, dom.ny, seed, dom.edf)
    f, macro, _ = orc.init(dom, st.kind, st.a, st.theta, st.ux, st.uy)
    rng = np.random.default_rng(seed)
    return f * (1 + amp * rng.uniform(-1, 1, f.shape)), macro


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_collision_conserves_N0_and_T_mu0(orc, edf):
    """Derived from Eq. (3) with Eqs. (21)-(23): the change of N^0 is prop. to
    U_nu(N^nu - n U^nu) = 0 and of T^{mu 0} to U_nu(T^{mu nu} - T_E^{mu nu}) = 0."""
    dom = orc.domain(9, 7, 0.7, edf)
    f, macro = _perturbed(orc, dom, 5 + edf)
    c0 = _conserved(orc, edf, f)
    f1, _, st = orc.step(dom, f, macro)
    assert st == 0
    c1 = _conserved(orc, edf, f1)
    assert np.max(np.abs(c1 - c0)) <= 2e-15 * np.max(np.abs(c0)) * 8


def test_periodic_conservation_over_steps(orc):
    dom = orc.domain(16, 12, 0.8, 0)
    f, macro = _perturbed(orc, dom, 9)
    c0 = _conserved(orc, 0, f)
    f, macro, st = orc.run(dom, f, macro, 20)
    assert st == 0
    assert np.max(np.abs(_conserved(orc, 0, f) - c0)) <= 1e-13 * np.max(np.abs(c0))


@pytest.mark.parametrize("edf", [0, 1, 2])
def test_rest_state_is_fixed_point(orc, edf):
    dom = orc.domain(6, 5, 0.9, edf)
    one = np.ones((5, 6))
    f0, m0, _ = orc.init(dom, orc.INIT_N_THETA, one, one * 1.1, 0 * one, 0 * one)
    f1, mo, st = orc.step(dom, f0, m0)
    assert st == 0
    assert np.max(np.abs(f1 - f0)) <= 1e-14 * np.max(f0)
    assert np.max(np.abs(mo[0] - 1)) < 1e-14 and np.max(np.abs(mo[1] - 1.1)) < 1e-14
    assert np.max(np.abs(mo[2:4])) < 1e-15


def test_streaming_reproduces_linear_fields(orc):
    """Bilinear interpolation is exact for linear fields: with no relaxation
    (tau huge) an interior cell must receive the value at x - v_i (Eqs. 17-18)."""
    nx, ny = 12, 10
    dom = orc.domain(nx, ny, 1e300, 0, (orc.ZERO_GRADIENT,) * 4)
    st = W.random_domain_state(nx, ny, 1)
    f0, macro, _ = orc.init(dom, st.kind, st.a, st.theta, st.ux, st.uy)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    rng = np.random.default_rng(2)
    coef = rng.uniform(0.5, 1.5, (72, 3))
    lin = np.stack([coef[q, 0] + 0.01 * coef[q, 1] * x + 0.02 * coef[q, 2] * y for q in range(72)])
    f1, _, _ = orc.step(dom, lin * np.mean(f0), macro)
    _, _, c, s = orc.lattice(0)
    for d in range(12):
        for sh in range(6):
            q = 6 * d + sh
            expect = (coef[q, 0] + 0.01 * coef[q, 1] * (x - c[d]) + 0.02 * coef[q, 2] * (y - s[d])) * np.mean(f0)
            np.testing.assert_allclose(f1[q, 1:-1, 1:-1], np.broadcast_to(expect, (ny, nx))[1:-1, 1:-1],
                                       rtol=1e-14)


def test_mirror_and_rotation_symmetry(orc):
    """The stencil and collision commute with x -> -x (d -> 6-d) and with a 90
    degree rotation (d -> d+3): symmetric initial states stay symmetric."""
    L = 10
    dom = orc.domain(L, L, 0.75, 0)
    x, y = np.meshgrid(np.arange(L), np.arange(L))
    # fields symmetric under the mirror x -> L-1-x
    n = 1 + 0.05 * np.cos(2 * np.pi * (x - (L - 1) / 2) / L) * np.sin(2 * np.pi * y / L + 0.3)
    th = 1 + 0.04 * np.cos(4 * np.pi * (x - (L - 1) / 2) / L)
    ux = 0.05 * np.sin(2 * np.pi * (x - (L - 1) / 2) / L) * np.cos(2 * np.pi * y / L)
    uy = 0.03 * np.cos(2 * np.pi * (x - (L - 1) / 2) / L)
    f, macro, _ = orc.init(dom, orc.INIT_N_THETA, n, th, ux, uy)
    f, macro, st = orc.run(dom, f, macro, 5)
    mir = [6 * ((6 - d) % 12) + s for d in range(12) for s in range(6)]
    fm = f[mir][:, :, ::-1]
    assert np.max(np.abs(fm - f)) <= 1e-13 * np.max(f)
    # rotation: take an arbitrary state, rotate it, step both, compare
    st0 = W.random_domain_state(L, L, 4)
    f, macro, _ = orc.init(dom, st0.kind, st0.a, st0.theta, st0.ux, st0.uy)

    # explicit index mapping, independent of numpy rotation conventions
    def rotate_explicit(g):
        out = np.empty_like(g)
        for d in range(12):
            for s_ in range(6):
                src = g[6 * d + s_]
                dst = np.empty_like(src)
                for yy in range(L):
                    for xx in range(L):
                        dst[xx, L - 1 - yy] = src[yy, xx]  # (x, y) -> (L-1-y, x)
                out[6 * ((d + 3) % 12) + s_] = dst
        return out
    fr = rotate_explicit(f)
    f1, _, _ = orc.step(dom, f, macro)
    fr1, _, _ = orc.step(dom, fr, None)
    assert np.max(np.abs(rotate_explicit(f1) - fr1)) <= 1e-13 * np.max(f1)


@pytest.mark.parametrize("edf", [0, 1])
def test_uniform_state_with_zero_gradient_and_walls(orc, edf):
    """A uniform rest state stays put with open (zero-gradient) ends and with
    fixed-T walls at the fluid's own temperature."""
    nx, ny = 7, 4
    one = np.ones((ny, nx))
    for bc in [(orc.ZERO_GRADIENT, orc.ZERO_GRADIENT, orc.PERIODIC, orc.PERIODIC),
               (orc.FIXED_T_WALL, orc.FIXED_T_WALL, orc.PERIODIC, orc.PERIODIC),
               (orc.FIXED_T_WALL, orc.ZERO_GRADIENT, orc.FIXED_T_WALL, orc.ZERO_GRADIENT)]:
        dom = orc.domain(nx, ny, 0.8, edf, bc, (1.05, 1.05, 1.05, 1.05))
        f0, m0, _ = orc.init(dom, orc.INIT_N_THETA, one, one * 1.05, 0 * one, 0 * one)
        f, m, st = orc.run(dom, f0, m0, 3)
        assert st == 0
        assert np.max(np.abs(f - f0)) <= 1e-13 * np.max(f0)


def test_hot_wall_heats_fluid(orc):
    """With a hotter wall the energy density of the fluid grows (Fourier setup, Sec. 3.3)."""
    nx, ny = 8, 2
    one = np.ones((ny, nx))
    dom = orc.domain(nx, ny, 0.8, 0, (orc.FIXED_T_WALL, orc.FIXED_T_WALL, orc.PERIODIC, orc.PERIODIC),
                     (1.0, 1.2, 1.0, 1.0))
    f0, m0, _ = orc.init(dom, orc.INIT_N_THETA, one, one, 0 * one, 0 * one)
    f, m, st = orc.run(dom, f0, m0, 10)
    out, _ = orc.fields(dom, f, m)
    assert out[1][:, -1].mean() > 1.0 + 1e-4      # next to the hot wall
    assert abs(out[1][:, 0].mean() - 1.0) < out[1][:, -1].mean() - 1.0
