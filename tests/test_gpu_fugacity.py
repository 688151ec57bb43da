"""Parity away from the dilute limit, where the fugacity solves leave their
power-series branch (Eq. 25; the states of the other parity tests sit near
z = 0.17). Fermi-Dirac states around z = 0.6, 2 and 8 take the expansion in
ln z and, beyond z = 4, the inversion formula; Bose-Einstein states around
z = 0.5 and 0.9 take the expansion about z = 1. The fields start from (z,
theta) with smooth gradients and a small velocity, between fixed-temperature
walls in x (whose ghosts solve n = 2 pi theta^2 g_2(z) for z). Each runs 20 steps
in FP64 (bound 1e-12) and in FP32 deviations taken about the mean state (bound
1e-5 on n, theta and u), against the FP64 oracle. As in the other parity tests the
velocity error is normwise, max|du| / max|u|. The flow is a shear that keeps
|u| of 0.05 to 0.09 after 20 steps, over 2 % gradients of z and theta. The FP32
path leaves an absolute velocity error of about 3e-7 at these densities (n = 3 to
23, measured on a smaller domain), which would be 1.6e-5 of a flow of |u| = 0.02."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W

pytestmark = pytest.mark.gpu
NX, NY, STEPS = 32, 32, 20
CASES = [(W.FD, 0.17), (W.FD, 0.6), (W.FD, 2.0), (W.FD, 8.0), (W.BE, 0.5), (W.BE, 0.9)]


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1709_09073_gb300 import build, rlbm
    build.build()
    rlbm.load()
    return rlbm


def _state(edf, z0, seed):
    base = W.random_domain_state(NX, NY, seed, edf, u_amp=0.2, th_amp=0.02)
    z = z0 * (1.0 + 0.2 * (base.a - 1.0))  # z0 (1 +- 2 %)
    if edf == W.BE:
        z = np.minimum(z, 0.97)
    return W.InitialState(W.INIT_Z_THETA, z, base.theta, base.ux, base.uy)


def _oracle(orc, spec, init, steps):
    dom = orc.domain(spec.nx, spec.ny, spec.tau, spec.edf, spec.bc, spec.t_wall)
    f, m, st0 = orc.init(dom, init.kind, init.a, init.theta, init.ux, init.uy)
    f, m, st = orc.run(dom, f, m, steps)
    out, st2 = orc.fields(dom, f, m)
    return out, st0 | st | st2


def _errors(g, ref):
    n, th, ux, uy, z = g
    e_n = np.max(np.abs(n / ref[0] - 1))
    e_t = np.max(np.abs(th / ref[1] - 1))
    umax = max(np.max(np.abs(ref[2])), np.max(np.abs(ref[3])))
    e_u = max(np.max(np.abs(ux - ref[2])), np.max(np.abs(uy - ref[3]))) / umax
    e_z = np.max(np.abs(z / ref[4] - 1))
    return e_n, e_t, e_u, e_z


@pytest.mark.parametrize("edf,z0", CASES)
@pytest.mark.parametrize("storage,tol", [(0, 1e-12), (4, 1e-5)])
def test_degenerate_states_match_the_oracle(R, orc, edf, z0, storage, tol):
    init = _state(edf, z0, 90 + int(10 * z0) + edf)
    spec0 = W.DomainSpec(NX, NY, 0.9, edf, (W.FIXED_T_WALL, W.FIXED_T_WALL, W.PERIODIC, W.PERIODIC),
                         (0.97, 1.03, 1.0, 1.0))
    ref, st_ref = _oracle(orc, spec0, init, STEPS)
    assert st_ref & orc.E_NONPHYSICAL == 0
    # the deviation storage about the mean state of the oracle's initial fields
    f0, _ = _oracle(orc, spec0, init, 0)
    spec = W.DomainSpec(NX, NY, 0.9, edf, spec0.bc, spec0.t_wall,
                        ref_n=float(np.mean(f0[0])), ref_theta=float(np.mean(f0[1])))
    sim = R.Simulation([spec], edf=edf, storage=storage)
    st = sim.init(0, init)
    sim.step(STEPS)
    st |= sim.sync_status()
    got = sim.moments(0)
    sim.close()
    errs = _errors(got, ref)
    print("edf %d z0 %.1f storage %d: n %.2e theta %.2e u %.2e z %.2e" % ((edf, z0, storage) + errs))
    assert st & R.RLBM_W_NONPHYSICAL == 0
    assert max(errs[:3]) <= tol, errs
    assert errs[3] <= 10 * tol, errs
