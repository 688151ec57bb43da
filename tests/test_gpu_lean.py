"""The lean variants of the mixed step (RLBM_KERNEL_LEAN: one cell per thread;
RLBM_KERNEL_LEAN2: two adjacent cells of a row per thread) and the staged one
(RLBM_KERNEL_STAGED: TMA-staged tiles, populations in registers, next tile
loading during the collision) against the L1 variant. They carry out the same arithmetic in the same order, so the
populations, halo ring included, must be bit-identical: for every mixed
storage and EDF, on ragged walled domains (odd widths put the last cell pair
across the right edge), on domains one to three cells wide, with the local
relaxation time of Sec. 3.5, and on a batch of uneven domains under the grid
the tuner picks."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W

pytestmark = pytest.mark.gpu
STORAGES = {"f32": 1, "f32dev": 4, "f16dev": 3, "bf16dev": 2}


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1709_09073_gb300 import build, rlbm
    build.build()
    rlbm.load()
    return rlbm


def _populations(R, specs, inits, storage, kernel, steps, grid_tune=False, grid=None):
    sim = R.Simulation(specs, edf=specs[0].edf, storage=storage)
    for i, s in enumerate(inits):
        sim.init(i, s)
    if grid_tune:
        sim.tune(1)
    if kernel == R.RLBM_KERNEL_STAGED and any(d.nx < 4 for d in specs) and storage in (1, 4):
        sim.close()
        return None, None  # no TMA descriptors for FP32 domains under 4 cells wide
    assert sim.select_kernel(kernel) == kernel
    sim.step(steps)
    st = sim.sync_status()
    out = [sim.get_populations(i) for i in range(len(specs))]
    sim.close()
    return out, st


def _same(R, specs, inits, storage, steps, grid_tune=False):
    ref, s_ref = _populations(R, specs, inits, storage, R.RLBM_KERNEL_L1, steps, grid_tune)
    for kernel in (R.RLBM_KERNEL_LEAN, R.RLBM_KERNEL_LEAN2, R.RLBM_KERNEL_STAGED):
        out, s_out = _populations(R, specs, inits, storage, kernel, steps, grid_tune)
        if out is None:
            continue
        assert s_out == s_ref, (kernel, s_out, s_ref)
        for i, (a, b) in enumerate(zip(ref, out)):
            assert np.array_equal(a, b, equal_nan=True), (kernel, i, np.nanmax(np.abs(a - b)))


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("stname", list(STORAGES))
def test_lean_matches_l1_bitwise(R, edf, stname):
    spec = W.DomainSpec(37, 11, 0.8, edf, (W.FIXED_T_WALL, W.ZERO_GRADIENT, W.ZERO_GRADIENT, W.FIXED_T_WALL),
                        (0.97, 1.0, 1.0, 1.03))
    init = W.random_domain_state(37, 11, 50 + edf, edf, u_amp=0.05)
    _same(R, [spec], [init], STORAGES[stname], 12)


@pytest.mark.parametrize("nx", [1, 2, 3, 32, 33, 63])
def test_lean_narrow_and_ragged_widths(R, nx):
    specs = [W.DomainSpec(nx, 9, 0.9, 0), W.DomainSpec(nx, 6, 1.2, 0, (1, 1, 2, 2), (1.0, 1.0, 0.98, 1.02))]
    inits = [W.random_domain_state(nx, s.ny, 60 + i) for i, s in enumerate(specs)]
    _same(R, specs, inits, 4, 7)


def test_lean_local_tau(R):
    spec = W.DomainSpec(45, 14, 0.9, 1, (W.FIXED_T_WALL, W.FIXED_T_WALL, W.PERIODIC, W.PERIODIC),
                        (0.9, 1.1, 1.0, 1.0), eta_s=0.3)
    init = W.random_domain_state(45, 14, 77, 1, u_amp=0.05, th_amp=0.15)
    _same(R, [spec], [init], 4, 9)


def test_lean_matches_l1_on_a_tuned_batch(R):
    specs = [W.DomainSpec(33, 17, 0.7, 0), W.DomainSpec(64, 8, 1.3, 0, (1, 1, 0, 0)),
             W.DomainSpec(101, 40, 0.9, 0, (2, 2, 0, 0), (0.95, 1.05, 1, 1)),
             W.DomainSpec(6, 7, 1.1, 0), W.DomainSpec(130, 3, 2.0, 0, (0, 0, 1, 1)),
             W.DomainSpec(1, 5, 0.8, 0), W.DomainSpec(97, 66, 0.6, 0)]
    inits = [W.random_domain_state(s.nx, s.ny, 40 + i) for i, s in enumerate(specs)]
    _same(R, specs, inits, 4, 9, grid_tune=True)


@pytest.mark.parametrize("grid", [1, 3, 7])
def test_staged_persistent_grids(R, grid):
    """The staged kernel with persistent grids of a few blocks (each block walks
    many tiles, interior and edge ones alternating, so the next-tile loads
    overlap collisions) against the L1 variant, bit for bit."""
    specs = [W.DomainSpec(97, 30, 0.9, 1, (2, 2, 0, 0), (0.96, 1.04, 1, 1)), W.DomainSpec(130, 21, 1.4, 1),
             W.DomainSpec(40, 9, 0.7, 1, (1, 1, 1, 1))]
    inits = [W.random_domain_state(s.nx, s.ny, 90 + i, 1, u_amp=0.05) for i, s in enumerate(specs)]
    outs = []
    for kernel in (R.RLBM_KERNEL_L1, R.RLBM_KERNEL_STAGED):
        sim = R.Simulation(specs, edf=1, storage=4)
        for i, s in enumerate(inits):
            sim.init(i, s)
        assert sim.select_kernel(kernel) == kernel
        sim.set_grid(grid)
        sim.step(8)
        assert sim.sync_status() == 0
        outs.append([sim.get_populations(i) for i in range(len(specs))])
        sim.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
