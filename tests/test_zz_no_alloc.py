"""rlbm_step_noalloc, the fixed-scratch FP64 step, against rlbm_step.

The file name makes pytest collect it last: the entry point's scratch array is
set up by its first call on a device and shared by every later call, so the
check must hold after the other tests have used the GPU as well as alone in a
fresh process (one case runs in a child process whose first library call is
the entry point itself, before any handle exists). Both calls go through the C ABI (the ctypes binding)."""
import ctypes
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from paper_1709_09073_gb300 import rlbm, workloads as W

TOL = 1e-12  # FP64 parity tolerance of the GPU tests, relative to max |f|

WALLS_Y = (W.PERIODIC, W.PERIODIC, W.FIXED_T_WALL, W.FIXED_T_WALL)
OPEN_X = (W.ZERO_GRADIENT, W.ZERO_GRADIENT, W.PERIODIC, W.PERIODIC)
PERIODIC = (W.PERIODIC,) * 4

VWALLS_Y = (W.PERIODIC, W.PERIODIC, W.VELOCITY_WALL, W.VELOCITY_WALL)

CASES = [
    # (edf, bc, nx, ny, extra): ragged tiles with walls, open ends, the largest
    # square that fits, and velocity walls with a body force and the local tau
    # (Secs. 3.4, 3.5), whose descriptor fields the entry point fills itself
    (W.FD, WALLS_Y, 45, 19, {}),
    (W.BE, OPEN_X, 37, 11, {}),
    (W.MJ, PERIODIC, 148, 148, {}),
    (W.FD, VWALLS_Y, 40, 12, {"accel": (2e-4, -1e-4), "eta_s": 0.2, "n_wall": 1.03}),
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
@pytest.mark.parametrize("edf,bc,nx,ny,extra", CASES)
def test_noalloc_matches_rlbm_step_on_two_calls_in_a_row(edf, bc, nx, ny, extra):
    torch = pytest.importorskip("torch")
    tw = (1.0, 1.0, 1.08, 1.08) if bc == VWALLS_Y else (1.0, 1.0, 1.08, 0.95)
    spec = W.DomainSpec(nx=nx, ny=ny, tau=0.8, edf=edf, bc=bc, t_wall=tw, **extra)
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
    # the local-tau parameter is checked as rlbm_create checks it
    for eta in (-0.1, float("nan"), float("inf")):
        d = rlbm.make_domains([W.DomainSpec(nx=8, ny=8, tau=1.0, eta_s=eta)])
        assert L.rlbm_step_noalloc(d, rlbm.RLBM_MJ, 1, fake, fake, None, None) == rlbm.RLBM_E_ARG, eta


def test_noalloc_binding_checks_its_tensors():
    """Host-side check: the binding refuses buffers the copy kernels would
    overrun (wrong shape, type or device) before it calls the library."""
    torch = pytest.importorskip("torch")
    spec = W.DomainSpec(nx=8, ny=6, tau=1.0)
    good = torch.zeros((72, 8, 10), dtype=torch.float64)  # host tensor: refused as not CUDA
    for bad in (good, good.float(), torch.zeros((72, 8, 9), dtype=torch.float64), None):
        with pytest.raises(ValueError):
            rlbm.step_noalloc(spec, rlbm.RLBM_MJ, 1, bad, good)
        with pytest.raises(ValueError):
            rlbm.step_noalloc(spec, rlbm.RLBM_MJ, 1, good, bad)


CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_1709_09073_gb300 import build, rlbm, workloads as W
build.build()
rlbm.load()
f0 = np.load(INPUT)
spec = W.DomainSpec(nx=f0.shape[2] - 2, ny=f0.shape[1] - 2, tau=0.9, edf=W.BE)
torch.cuda.set_device(0)
fin = torch.from_numpy(f0).cuda()
fout = torch.full_like(fin, float("nan"))
# the library's first call in this process, before any handle exists: the
# entry point looks up its scratch array here
w = rlbm.step_noalloc(spec, W.BE, 6, fin, fout)
assert w == 0, w
np.save(OUTPUT, fout.cpu().numpy())
sim = rlbm.Simulation([spec], edf=W.BE, storage=rlbm.RLBM_F64)
sim.set_populations(0, f0)
sim.step(6)
np.save(OUTPUT2, sim.get_populations(0))
sim.close()
"""


@pytest.mark.gpu
def test_noalloc_first_call_in_a_fresh_process(orc):
    """The entry point as the first library call of a process (no handle, no
    other kernel of the library before it), on a checkpoint built on the host from the
    oracle's initial state: it matches rlbm_step, and the interior matches the
    oracle's own steps, both to 1e-12."""
    pytest.importorskip("torch")
    nx, ny, steps = 29, 13, 6
    dom = orc.domain(nx, ny, 0.9, W.BE)
    st = W.random_domain_state(nx, ny, seed=321, edf=W.BE, u_amp=0.05, th_amp=0.05)
    f, m, _ = orc.init(dom, st.kind, st.a, st.theta, st.ux, st.uy)
    ckpt = np.pad(f, ((0, 0), (1, 1), (1, 1)), mode="wrap")  # periodic halo ring
    f_ref, _, _ = orc.run(dom, f, m, steps)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as tmp:
        paths = [os.path.join(tmp, n) for n in ("in.npy", "out.npy", "step.npy")]
        np.save(paths[0], ckpt)
        code = "ROOT=%r; INPUT=%r; OUTPUT=%r; OUTPUT2=%r\n" % (root, *paths) + CHILD
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
        out, via_step = np.load(paths[1]), np.load(paths[2])
    scale = np.max(np.abs(via_step))
    assert np.all(np.isfinite(out))
    assert np.max(np.abs(out - via_step)) <= TOL * scale
    assert np.max(np.abs(out[:, 1:-1, 1:-1] - f_ref)) <= TOL * np.max(np.abs(f_ref))
