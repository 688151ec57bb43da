"""The TMA-staged variant of the mixed step (RLBM_KERNEL_TMA) against the L1
variant: the same arithmetic, so the populations (halo ring included) must be
bit-identical, for every mixed storage and EDF, on ragged walled domains, on
domains one to three cells wide, with the local relaxation time, and on a batch
of uneven domains under the persistent grid the tuner may pick or a fixed
one. Also the bounded copy waits: a limit that runs out is reported and the
handle recovers."""
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


def _populations(R, specs, inits, storage, kernel, steps, grid_tune=False):
    sim = R.Simulation(specs, edf=specs[0].edf, storage=storage)
    for i, s in enumerate(inits):
        sim.init(i, s)
    if grid_tune:
        sim.tune(1)
    assert sim.select_kernel(kernel) == kernel
    sim.step(steps)
    st = sim.sync_status()
    out = [sim.get_populations(i) for i in range(len(specs))]
    sim.close()
    return out, st


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("stname", list(STORAGES))
def test_tma_matches_l1_bitwise(R, edf, stname):
    spec = W.DomainSpec(37, 11, 0.8, edf, (W.FIXED_T_WALL, W.FIXED_T_WALL, W.PERIODIC, W.PERIODIC),
                        (0.97, 1.03, 1.0, 1.0))
    init = W.random_domain_state(37, 11, 50 + edf, edf, u_amp=0.05)
    a, sa = _populations(R, [spec], [init], STORAGES[stname], R.RLBM_KERNEL_L1, 12)
    b, sb = _populations(R, [spec], [init], STORAGES[stname], R.RLBM_KERNEL_TMA, 12)
    assert sa == sb and (sa & R.RLBM_W_DEVICE_TIMEOUT) == 0
    assert np.array_equal(a[0], b[0])


@pytest.mark.parametrize("nx", [1, 2, 3, 16, 17, 31, 33, 48, 63])
def test_tma_matches_l1_on_narrow_and_ragged_widths(R, nx):
    """The L1 step walks packed tiles (a last block of w <= 16 cells, 32/w rows per
    warp) and wraps across periodic sides; the TMA step walks 32 x 4 tiles and
    reads the stored halo images: w = 1, 2, 3, 16 packed, 17 and 31 not, and
    periodic x with walls in y, zero-gradient x with walls, periodic both ways."""
    specs = [W.DomainSpec(nx, 9, 0.9, 0), W.DomainSpec(nx, 6, 1.2, 0, (1, 1, 2, 2), (1.0, 1.0, 0.98, 1.02)),
             W.DomainSpec(nx, 13, 0.8, 0, (0, 0, 2, 2), (1.0, 1.0, 1.03, 0.97))]
    inits = [W.random_domain_state(nx, s.ny, 60 + i) for i, s in enumerate(specs)]
    a, _ = _populations(R, specs, inits, 4, R.RLBM_KERNEL_L1, 7)
    b, st = _populations(R, specs, inits, 4, R.RLBM_KERNEL_TMA, 7)
    assert st == 0
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_tma_matches_l1_with_local_tau(R):
    spec = W.DomainSpec(45, 14, 0.9, 1, (W.FIXED_T_WALL, W.FIXED_T_WALL, W.PERIODIC, W.PERIODIC),
                        (0.9, 1.1, 1.0, 1.0), eta_s=0.3)
    init = W.random_domain_state(45, 14, 77, 1, u_amp=0.05, th_amp=0.15)
    a, _ = _populations(R, [spec], [init], 4, R.RLBM_KERNEL_L1, 9)
    b, _ = _populations(R, [spec], [init], 4, R.RLBM_KERNEL_TMA, 9)
    assert np.array_equal(a[0], b[0])


@pytest.mark.parametrize("grid", [1, 3, 7])
def test_tma_matches_l1_on_fixed_persistent_grids(R, grid):
    specs = [W.DomainSpec(97, 30, 0.9, 1, (2, 2, 0, 0), (0.96, 1.04, 1, 1)), W.DomainSpec(130, 21, 1.4, 1),
             W.DomainSpec(40, 9, 0.7, 1, (1, 1, 1, 1))]
    inits = [W.random_domain_state(s.nx, s.ny, 90 + i, 1, u_amp=0.05) for i, s in enumerate(specs)]
    outs = []
    for kernel in (R.RLBM_KERNEL_L1, R.RLBM_KERNEL_TMA):
        sim = R.Simulation(specs, edf=1, storage=4)
        for i, s in enumerate(inits):
            sim.init(i, s)
        assert sim.select_kernel(kernel) == kernel
        assert sim.set_grid(grid) == grid
        sim.step(8)
        assert sim.sync_status() == 0
        outs.append([sim.get_populations(i) for i in range(len(specs))])
        sim.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_tma_matches_l1_on_a_tuned_batch(R):
    specs = [W.DomainSpec(33, 17, 0.7, 0), W.DomainSpec(64, 8, 1.3, 0, (1, 1, 0, 0)),
             W.DomainSpec(101, 40, 0.9, 0, (2, 2, 0, 0), (0.95, 1.05, 1, 1)),
             W.DomainSpec(6, 7, 1.1, 0), W.DomainSpec(130, 3, 2.0, 0, (0, 0, 1, 1))]
    inits = [W.random_domain_state(s.nx, s.ny, 40 + i) for i, s in enumerate(specs)]
    a, _ = _populations(R, specs, inits, 4, R.RLBM_KERNEL_L1, 9, grid_tune=True)
    b, st = _populations(R, specs, inits, 4, R.RLBM_KERNEL_TMA, 9, grid_tune=True)
    assert st == 0
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_kernel_selection_rules(R):
    sim = R.Simulation([W.DomainSpec(16, 8, 0.9, 0)], storage=R.RLBM_F64)
    assert sim.select_kernel() == R.RLBM_KERNEL_L1
    with pytest.raises(R.RlbmError):
        sim.select_kernel(R.RLBM_KERNEL_TMA)  # FP64 storage has no staged variant
    sim.close()
    narrow = R.Simulation([W.DomainSpec(3, 8, 0.9, 0)], storage=R.RLBM_F32DEV)
    assert narrow.select_kernel(R.RLBM_KERNEL_TMA) == R.RLBM_KERNEL_TMA  # any width: boxes span whole blocks
    with pytest.raises(R.RlbmError):
        narrow.select_kernel(7)
    narrow.close()
    sim = R.Simulation([W.DomainSpec(64, 16, 0.9, 0)], storage=R.RLBM_F32DEV)
    sim.init(0, W.random_domain_state(64, 16, 1))
    assert sim.tune(1) > 0 and sim.select_kernel() in (R.RLBM_KERNEL_L1, R.RLBM_KERNEL_TMA)
    sim.close()


def test_copy_wait_limit_runs_out_and_the_handle_recovers(R):
    """Failure detection without a fault: with the TMA variant's copy-wait limit
    set to one nanosecond (polling, so the first copy still in flight runs it
    out) a step ends early with RLBM_W_DEVICE_TIMEOUT and no other effect on the
    context. With the default limit restored and the domain initialised again,
    the next steps are clean and bit-identical to the L1 variant."""
    spec = W.DomainSpec(512, 64, 0.9, 0)
    init = W.random_domain_state(512, 64, 31, 0, u_amp=0.05)
    ref, s_ref = _populations(R, [spec], [init], 4, R.RLBM_KERNEL_L1, 5)
    sim = R.Simulation([spec], edf=0, storage=4)
    sim.init(0, init)
    assert sim.select_kernel(R.RLBM_KERNEL_TMA) == R.RLBM_KERNEL_TMA
    sim.set_wait_limit(1e-9)
    sim.step(1)
    st = sim.sync_status()
    assert st & R.RLBM_W_DEVICE_TIMEOUT, st
    assert "timed out" in R.status_string(st)
    sim.set_wait_limit(0)          # back to the default of one second
    sim.init(0, init)              # the interrupted step left no valid state
    sim.step(5)
    st2 = sim.sync_status()
    out = sim.get_populations(0)
    sim.close()
    assert st2 == s_ref == 0
    assert np.array_equal(out, ref[0])


@pytest.mark.parametrize("edf", [0, 1])
def test_tma_matches_l1_on_a_periodic_batch(R, edf):
    """A handle whose domains are all periodic launches the L1 step without its
    halo writer (nothing to write: the pull wraps); the TMA step writes and
    reads the periodic images. Ragged, packed and one-cell-wide domains."""
    specs = [W.DomainSpec(37, 11, 0.8, edf), W.DomainSpec(5, 9, 1.1, edf), W.DomainSpec(64, 4, 0.7, edf),
             W.DomainSpec(1, 3, 0.9, edf), W.DomainSpec(50, 21, 1.6, edf)]
    inits = [W.random_domain_state(s.nx, s.ny, 70 + i, edf, u_amp=0.05) for i, s in enumerate(specs)]
    for stname, storage in STORAGES.items():
        a, _ = _populations(R, specs, inits, storage, R.RLBM_KERNEL_L1, 9)
        b, st = _populations(R, specs, inits, storage, R.RLBM_KERNEL_TMA, 9)
        assert st == 0, stname
        for x, y in zip(a, b):
            assert np.array_equal(x, y), stname
