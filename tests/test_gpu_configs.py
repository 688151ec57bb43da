"""Parity of the benchmark workloads with the FP64 oracle.

* Downscaled twins that the oracle runs whole: a 128 x 128 Bose-Einstein hot
  spot (sigma = 4, 200 steps) in the FP32 storages, and two 128 x 32
  Fermi-Dirac Fourier-flow domains with fixed-temperature walls (200 steps) in
  the 16-bit deviation storages. The oracle's BE/FD step costs 7-12 us per
  cell (its fugacity solve is a bisection), which sets these sizes.
* Full-size runs in the launch configuration the benchmark times (autotuned
  grid and kernel, CUDA-graph replay), checked on samples the oracle can
  compute one by one: the 8192 x 8192 hot spot at selected cells after 60
  steps, plus its mirror symmetry, and the 256-domain batched Taylor-Green
  workload after the benchmark's 200 steps, on cells of its largest domains,
  on both sides of domain-to-domain seams of the tile work list, on one whole
  128^2-class domain and on its four smallest domains whole. A sampled cell's
  oracle value comes from its light cone: the periodic initial state around it,
  stepped with one ring of cells cropped after every step (a cell's state after
  k steps depends only on cells within k of it, so the ring the zero-gradient
  border has touched is always the one cropped).

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


def _cone_reference(orc, spec, init, cx, cy, steps):
    """Oracle fields (streamed) at cell (cx, cy) of a periodic domain after
    `steps` steps, from its light cone (see the module docstring); also the
    largest |u| of the final 3 x 3 patch."""
    h = steps + 1
    xs = np.arange(cx - h, cx + h + 1) % spec.nx
    ys = np.arange(cy - h, cy + h + 1) % spec.ny
    sub = lambda a: np.ascontiguousarray(a[np.ix_(ys, xs)])
    zg = (W.ZERO_GRADIENT,) * 4
    side = 2 * h + 1
    dom = orc.domain(side, side, spec.tau, spec.edf, zg)
    f, _, _ = orc.init(dom, init.kind, sub(init.a), sub(init.theta), sub(init.ux), sub(init.uy))
    for _ in range(steps):
        f, _, _ = orc.step(dom, f, None)
        f = np.ascontiguousarray(f[:, 1:-1, 1:-1])
        side -= 2
        dom = orc.domain(side, side, spec.tau, spec.edf, zg)
    ref, _ = orc.fields(dom, f, None, streamed=True)
    return [r[1, 1] for r in ref], max(np.max(np.abs(ref[2])), np.max(np.abs(ref[3])))


def _check_cell(label, fields, ref, umax, tol=1e-5):
    g = [float(a) for a in fields]
    e_n = abs(g[0] - ref[0]) / ref[0]
    e_t = abs(g[1] - ref[1]) / ref[1]
    e_u = max(abs(g[2] - ref[2]), abs(g[3] - ref[3])) / max(umax, 1e-300)
    print("%s: n %.2e theta %.2e u %.2e" % (label, e_n, e_t, e_u))
    assert max(e_n, e_t) <= tol and (e_u <= tol or umax < 1e-12), (label, e_n, e_t, e_u)


def test_hot_spot_full_size_sampled(R, orc):
    """8192^2 BE hot spot, FP32 deviations, autotuned launch, 60 steps."""
    import torch
    steps = 60
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
    for (x, y) in [(c, c), (c + 40, c - 25), (c - 90, c + 3), (c + 31, c + 32), (17, 5000)]:
        ref, umax = _cone_reference(orc, spec, init, x, y, steps)
        _check_cell("hot spot 8192 cell (%d, %d)" % (x, y), [a[y, x] for a in (n, th, ux, uy)], ref, umax)
    # mirror symmetry about the centre and the diagonal (rounding-level)
    t = th.double()
    core = t[c - 300:c + 301, c - 300:c + 301]
    assert torch.max(torch.abs(core - torch.flip(core, [1]))).item() <= 1e-6
    assert torch.max(torch.abs(core - core.T)).item() <= 1e-6
    del n, th, ux, uy, t, core
    sim.close()


def test_batched_taylor_green_full_size_sampled(R, orc):
    """The 256-domain benchmark batch in FP32 deviations, autotuned launch,
    after the benchmark's 200 steps: a cell of each of the two largest domains
    at a corner of four tiles, the cells on both sides of three domain-to-domain
    seams of the work list (the last cell of a domain and the first of the
    next), one whole domain of about 128^2, and the four smallest domains whole."""
    steps = 200
    wl = W.batched_taylor_green()
    sim = R.Simulation(wl.domains, edf=0, storage=R.RLBM_F32DEV)
    for i, s in enumerate(wl.init):
        assert sim.init(i, s) == 0
    sim.tune(1)
    sim.step(steps)
    assert sim.sync_status() == 0
    fields = {}

    def at(i, x, y):
        if i not in fields:
            fields[i] = sim.moments(i)
        return [a[y, x] for a in fields[i][:4]]

    area = [d.nx * d.ny for d in wl.domains]
    order = sorted(range(len(area)), key=lambda i: area[i])
    for i in order[-2:]:
        d = wl.domains[i]
        for (x, y) in [(31, 3)]:
            ref, umax = _cone_reference(orc, d, wl.init[i], x, y, steps)
            _check_cell("batch domain %d (%dx%d) cell (%d, %d)" % (i, d.nx, d.ny, x, y), at(i, x, y), ref, umax)
    for i in (0, 127, 254):
        a, b = wl.domains[i], wl.domains[i + 1]
        for j, (x, y) in ((i, (a.nx - 1, a.ny - 1)), (i + 1, (0, 0))):
            ref, umax = _cone_reference(orc, wl.domains[j], wl.init[j], x, y, steps)
            _check_cell("seam %d|%d: domain %d cell (%d, %d)" % (i, i + 1, j, x, y), at(j, x, y), ref, umax)
    mid = min(range(len(area)), key=lambda i: abs(area[i] - 128 * 128))
    for i in [mid] + order[:4]:
        ref, _ = oracle_fields(orc, wl.domains[i], wl.init[i], steps)
        errs = errors(sim.moments(i), ref)
        print("batched TG domain %d (%dx%d): n %.2e theta %.2e u %.2e" % (
            (i, wl.domains[i].nx, wl.domains[i].ny) + tuple(errs[:3])))
        assert max(errs[:3]) <= 1e-5, (i, errs)
    sim.close()
