"""Parity of the benchmark workloads with the FP64 oracle.

* Downscaled twins that the oracle runs whole: a 128 x 128 Bose-Einstein hot
  spot (sigma = 4, 200 steps) in the FP32 storages, and two 128 x 32
  Fermi-Dirac Fourier-flow domains with fixed-temperature walls (200 steps) in
  the 16-bit deviation storages. The oracle's BE/FD step costs 7-12 us per
  cell (its fugacity solve is a bisection), which sets these sizes.
* Full-size runs in the launch configuration the benchmark times (autotuned
  grid and kernel, CUDA-graph replay), checked on samples the oracle can
  compute one by one: the 8192 x 8192 hot spot at selected cells (the oracle
  runs a patch around each cell whose border, zero-gradient, cannot reach the
  centre within the steps taken) plus its conservation and mirror symmetry, and
  the 256-domain batched Taylor-Green workload on whole small domains.

Bounds: n and theta relative, u normwise (max|du| / max|u|), 1e-5 for the FP32
storages; the 16-bit formats hold the deviation to 2^-9 (BF16) and 2^-12 (FP16)
relative, so their bounds follow from that precision (reported, not 1e-5)."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W
from test_gpu_fp64 import errors, oracle_fields, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1709_09073_gb300 import build, rlbm
    build.build()
    rlbm.load()
    return rlbm


@pytest.mark.parametrize("stname,code", [("f32dev", 4), ("f32", 1)])
def test_hot_spot_twin_be(R, orc, stname, code):
    wl = W.hot_spot(L=128, sigma=4.0, steps=200)
    spec, init = wl.domains[0], wl.init[0]
    sim, outs, st = run_gpu(R, [spec], [init], wl.steps, storage=code)
    ref, _ = oracle_fields(orc, spec, init, wl.steps)
    errs = errors(outs[0], ref)
    print("hot spot 128 BE %s 200: n %.2e theta %.2e u %.2e z %.2e" % ((stname,) + tuple(errs)))
    assert (st & (R.RLBM_W_NONPHYSICAL | R.RLBM_W_ZSOLVE)) == 0
    assert max(errs[:3]) <= 1e-5, errs


@pytest.mark.parametrize("stname,code,tol", [("f16dev", 3, 2e-3), ("bf16dev", 2, 2e-2)])
def test_fourier_twin_fd(R, orc, stname, code, tol):
    wl = W.batched_fourier(n_domains=2, nx=128, ny=32, steps=200)
    sim, outs, st = run_gpu(R, wl.domains, wl.init, wl.steps, storage=code)
    assert (st & R.RLBM_W_NONPHYSICAL) == 0
    for i, (spec, init) in enumerate(zip(wl.domains, wl.init)):
        ref, _ = oracle_fields(orc, spec, init, wl.steps)
        n, th, ux, uy, z = outs[i]
        e_n = np.max(np.abs(n - ref[0]) / ref[0])
        e_t = np.max(np.abs(th - ref[1]) / ref[1])
        # the flow stays nearly at rest: absolute velocity error (c = 1)
        e_u = max(np.max(np.abs(ux - ref[2])), np.max(np.abs(uy - ref[3])))
        print("fourier FD %s dom %d: n %.2e theta %.2e |du| %.2e" % (stname, i, e_n, e_t, e_u))
        assert max(e_n, e_t) <= tol, (i, e_n, e_t)
        assert e_u <= tol, (i, e_u)
        # the walls set the temperature profile: monotone from cold to hot in x
        prof = th.mean(axis=0)
        assert prof[0] < prof[-1]


def _patch_reference(orc, spec, init, cx, cy, steps):
    """Oracle fields at cell (cx, cy) after `steps` steps, from a patch of the
    periodic initial state around it with zero-gradient borders: the border
    error moves at most one cell per step, so the centre is exact when the
    half-width exceeds the step count."""
    h = steps + 2
    xs = np.arange(cx - h, cx + h + 1) % spec.nx
    ys = np.arange(cy - h, cy + h + 1) % spec.ny
    sub = lambda a: a[np.ix_(ys, xs)]
    zg = (W.ZERO_GRADIENT,) * 4
    pspec = W.DomainSpec(2 * h + 1, 2 * h + 1, spec.tau, spec.edf, zg)
    pinit = W.InitialState(init.kind, sub(init.a), sub(init.theta), sub(init.ux), sub(init.uy))
    ref, _ = oracle_fields(orc, pspec, pinit, steps)
    return [r[h, h] for r in ref], max(np.max(np.abs(ref[2])), np.max(np.abs(ref[3])))


def test_hot_spot_full_size_sampled(R, orc):
    """8192^2 BE hot spot, FP32 deviations, autotuned launch, 20 steps."""
    import torch
    steps = 20
    wl = W.hot_spot(L=8192, steps=steps)
    spec, init = wl.domains[0], wl.init[0]
    sim = R.Simulation([spec], edf=spec.edf, storage=R.RLBM_F32DEV)
    assert sim.init(0, init) == 0
    sim.tune(1)
    sim.step(steps)
    st = sim.sync_status()
    assert (st & (R.RLBM_W_NONPHYSICAL | R.RLBM_W_ZSOLVE)) == 0
    n, th, ux, uy, _ = sim.moments(0, on_device=True)
    c = spec.nx // 2
    for (x, y) in [(c, c), (c + 40, c - 25), (c - 90, c + 3), (17, 5000)]:
        ref, umax = _patch_reference(orc, spec, init, x, y, steps)
        g = [float(a[y, x]) for a in (n, th, ux, uy)]
        e_n = abs(g[0] - ref[0]) / ref[0]
        e_t = abs(g[1] - ref[1]) / ref[1]
        e_u = max(abs(g[2] - ref[2]), abs(g[3] - ref[3])) / max(umax, 1e-300)
        print("hot spot 8192 cell (%d, %d): n %.2e theta %.2e u %.2e" % (x, y, e_n, e_t, e_u))
        assert max(e_n, e_t) <= 1e-5 and (e_u <= 1e-5 or umax < 1e-12), (x, y, e_n, e_t, e_u)
    # mirror symmetry about the centre and the diagonal (rounding-level)
    t = th.double()
    core = t[c - 300:c + 301, c - 300:c + 301]
    assert torch.max(torch.abs(core - torch.flip(core, [1]))).item() <= 1e-6
    assert torch.max(torch.abs(core - core.T)).item() <= 1e-6
    del n, th, ux, uy, t, core
    sim.close()


def test_batched_taylor_green_full_size_sampled(R, orc):
    """The 256-domain benchmark batch in FP32 deviations, autotuned launch, 50
    steps: the four smallest domains agree with the oracle whole."""
    steps = 50
    wl = W.batched_taylor_green()
    sim = R.Simulation(wl.domains, edf=0, storage=R.RLBM_F32DEV)
    for i, s in enumerate(wl.init):
        assert sim.init(i, s) == 0
    sim.tune(1)
    sim.step(steps)
    assert sim.sync_status() == 0
    small = sorted(range(len(wl.domains)), key=lambda i: wl.domains[i].nx * wl.domains[i].ny)[:4]
    for i in small:
        ref, _ = oracle_fields(orc, wl.domains[i], wl.init[i], steps)
        errs = errors(sim.moments(i), ref)
        print("batched TG domain %d (%dx%d): n %.2e theta %.2e u %.2e" % (
            (i, wl.domains[i].nx, wl.domains[i].ny) + tuple(errs[:3])))
        assert max(errs[:3]) <= 1e-5, (i, errs)
    sim.close()
