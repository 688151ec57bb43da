"""rlbm_step_noalloc, the fixed-scratch FP64 step, against rlbm_step.

The file name makes pytest collect it last: the entry point's scratch array is
set up by its first call on a device and shared by every later call, so the
check must hold after the other tests have used the GPU as well as alone in a
fresh process. Both calls go through the C ABI (the ctypes binding)."""
import ctypes

import numpy as np
import pytest

from paper_1709_09073_gb300 import rlbm, workloads as W

TOL = 1e-12  # FP64 parity tolerance of the GPU tests, relative to max |f|

WALLS_Y = (W.PERIODIC, W.PERIODIC, W.FIXED_T_WALL, W.FIXED_T_WALL)
OPEN_X = (W.ZERO_GRADIENT, W.ZERO_GRADIENT, W.PERIODIC, W.PERIODIC)
PERIODIC = (W.PERIODIC,) * 4

CASES = [
    # (edf, bc, nx, ny): ragged tiles with walls, open ends, and the largest square that fits
    (W.FD, WALLS_Y, 45, 19),
    (W.BE, OPEN_X, 37, 11),
    (W.MJ, PERIODIC, 160, 160),
]


def _checkpoint(sim, spec, torch):
    """Device copy of the handle's populations, halo included ([72][ny+2][nx+2])."""
    f = torch.empty((72, spec.ny + 2, spec.nx + 2), dtype=torch.float64, device="cuda")
    rlbm._check(rlbm.load().rlbm_get_populations(sim.h, 0, ctypes.c_void_p(f.data_ptr()), 1))
    return f


def _rel_err(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.all(np.isfinite(a))
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.gpu
@pytest.mark.parametrize("edf,bc,nx,ny", CASES)
def test_noalloc_matches_rlbm_step_on_two_calls_in_a_row(edf, bc, nx, ny):
    torch = pytest.importorskip("torch")
    spec = W.DomainSpec(nx=nx, ny=ny, tau=0.8, edf=edf, bc=bc, t_wall=(1.0, 1.0, 1.08, 0.95))
    sim = rlbm.Simulation([spec], edf=edf, storage=rlbm.RLBM_F64)
    assert sim.init(0, W.random_domain_state(nx, ny, seed=nx * 1000 + ny, edf=edf, u_amp=0.05,
                                             th_amp=0.05)) == 0
    sim.step(3)
    f0 = _checkpoint(sim, spec, torch)
    f0_kept = f0.clone()

    # first call: out of place, 4 steps
    f1 = torch.full_like(f0, float("nan"))
    w1 = rlbm.step_noalloc(spec, edf, 4, f0, f1, stream=sim.stream)
    sim.step(4)
    g1 = _checkpoint(sim, spec, torch)

    # second call in a row: in place, 5 steps, on the previous call's output
    f2 = f1.clone()
    w2 = rlbm.step_noalloc(spec, edf, 5, f2, f2, stream=sim.stream)
    sim.step(5)
    g2 = _checkpoint(sim, spec, torch)
    torch.cuda.synchronize()

    assert w1 == 0 and w2 == 0
    assert sim.sync_status() == 0
    assert _rel_err(f1, g1) <= TOL
    assert _rel_err(f2, g2) <= TOL
    assert torch.equal(f0, f0_kept)  # an out-of-place call leaves its input alone
    sim.close()


def test_noalloc_rejects_domains_beyond_the_scratch():
    """Host-side check: an oversize domain is refused before any device work."""
    L = rlbm.load()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    for nx, ny in [(1024, 1024), (168, 168), (1 << 21, 1)]:
        dom = rlbm.make_domains([W.DomainSpec(nx=nx, ny=ny, tau=1.0)])
        r = L.rlbm_step_noalloc(dom, rlbm.RLBM_MJ, 1, fake, fake, None, None)
        assert r == rlbm.RLBM_E_SCRATCH, (nx, ny, r)
    assert b"fixed scratch" in L.rlbm_status_string(rlbm.RLBM_E_SCRATCH)
    # argument errors come before the size check
    bad = rlbm.make_domains([W.DomainSpec(nx=0, ny=4, tau=1.0)])
    assert L.rlbm_step_noalloc(bad, rlbm.RLBM_MJ, 1, fake, fake, None, None) == rlbm.RLBM_E_ARG
    ok = rlbm.make_domains([W.DomainSpec(nx=8, ny=8, tau=1.0)])
    assert L.rlbm_step_noalloc(ok, 7, 1, fake, fake, None, None) == rlbm.RLBM_E_ARG
    assert L.rlbm_step_noalloc(ok, rlbm.RLBM_MJ, -1, fake, fake, None, None) == rlbm.RLBM_E_ARG
    assert L.rlbm_step_noalloc(ok, rlbm.RLBM_MJ, 1, None, fake, None, None) == rlbm.RLBM_E_ARG
