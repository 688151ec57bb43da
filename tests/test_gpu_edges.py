"""Degenerate cases of the step on the GPU.

* A single periodic cell is a uniform fluid: streaming (Eqs. 17-18) hands
  every population back to its own cell and the equilibrium start is a fixed
  point of the collision (Eq. 3), so its fields stay the initial ones -- to
  1e-13 in FP64 and 1e-6 in FP32 deviations -- for the three statistics.
* A single cell boxed in by fixed-temperature walls, and one-row and
  one-column domains, agree with the oracle to 1e-12.
* Zero steps change nothing and launch nothing.
* A domain narrower than 4 cells runs both step variants (the TMA boxes
  span whole 32-cell blocks)."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W
from test_gpu_fp64 import errors, oracle_fields, run_gpu

pytestmark = pytest.mark.gpu
P, WALL = W.PERIODIC, W.FIXED_T_WALL


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1709_09073_gb300 import build, rlbm
    build.build()
    rlbm.load()
    return rlbm


@pytest.mark.parametrize("storage,tol", [(0, 1e-13), (4, 1e-6)])
@pytest.mark.parametrize("edf", [0, 1, 2])
def test_single_periodic_cell_is_a_fixed_point(R, edf, storage, tol):
    spec = W.DomainSpec(1, 1, 0.9, edf)
    init = W.random_domain_state(1, 1, 60 + edf, edf, u_amp=0.1)
    sim, outs, st = run_gpu(R, [spec], [init], 25, storage=storage)
    n, th, ux, uy, _ = outs[0]
    assert (st & R.RLBM_W_NONPHYSICAL) == 0
    assert abs(n[0, 0] - init.a[0, 0]) <= tol * init.a[0, 0]
    assert abs(th[0, 0] - init.theta[0, 0]) <= tol * init.theta[0, 0]
    assert max(abs(ux[0, 0] - init.ux[0, 0]), abs(uy[0, 0] - init.uy[0, 0])) <= tol
    sim.close()


@pytest.mark.parametrize("nx,ny,bc,tw", [
    (1, 1, (WALL, WALL, WALL, WALL), (0.96, 1.03, 1.01, 0.99)),
    (9, 1, (WALL, WALL, P, P), (0.97, 1.04, 1.0, 1.0)),
    (1, 9, (P, P, WALL, WALL), (1.0, 1.0, 1.04, 0.97)),
])
@pytest.mark.parametrize("edf", [0, 2])
def test_thin_domains_match_the_oracle(R, orc, edf, nx, ny, bc, tw):
    spec = W.DomainSpec(nx, ny, 0.8, edf, bc, tw)
    init = W.random_domain_state(nx, ny, 61 + edf, edf, u_amp=0.05)
    sim, outs, st = run_gpu(R, [spec], [init], 12)
    ref, _ = oracle_fields(orc, spec, init, 12)
    e = errors(outs[0], ref)
    assert (st & R.RLBM_W_NONPHYSICAL) == 0
    assert max(e[:3]) <= 1e-12, e
    sim.close()


def test_zero_steps_change_nothing(R):
    spec = W.DomainSpec(13, 6, 0.9, 0, (WALL, WALL, P, P), (0.97, 1.04, 1.0, 1.0))
    sim = R.Simulation([spec], storage=R.RLBM_F32DEV)
    sim.init(0, W.random_domain_state(13, 6, 62))
    before = sim.get_populations(0)
    assert sim.step(0) == 0
    assert sim.last_step_info() == (0, 0)
    assert np.array_equal(sim.get_populations(0), before)
    sim.close()


def test_narrow_domain_runs_both_variants(R):
    sim = R.Simulation([W.DomainSpec(3, 8, 0.9, 0)], storage=R.RLBM_F32DEV)
    sim.init(0, W.random_domain_state(3, 8, 63))
    assert sim.select_kernel() == R.RLBM_KERNEL_L1
    sim.step(2)
    assert sim.select_kernel(R.RLBM_KERNEL_TMA) == R.RLBM_KERNEL_TMA
    sim.step(2)
    assert sim.sync_status() == 0
    sim.close()
