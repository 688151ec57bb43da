"""Mixed-precision CUDA path (FP32 / BF16 / FP16 deviation storage, FP32
streaming and collision, FP64 totals and Landau solve) against the FP64 oracle.

Bound for FP32 storage: per-field relative error <= 1e-5 (n, theta relative;
u normwise max|du|/max|u|), the mixed-path requirement. The 16-bit deviation
formats keep relative precision 2^-9 (BF16) and 2^-12 (FP16) of the deviation
f/fref - 1 per stored value; their bounds below follow from that precision and
are reported, not claimed to meet 1e-5 (BF16 cannot)."""
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


# storage: (code, tolerance after the run)
STORAGE = {"f32": (1, 1e-5), "f32dev": (4, 1e-5), "f16dev": (3, 1e-3), "bf16dev": (2, 1e-2)}


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("stname", list(STORAGE))
def test_mixed_parity_small(R, orc, edf, stname):
    code, tol = STORAGE[stname]
    bc, tw = (2, 2, 0, 0), (0.97, 1.03, 1.0, 1.0)
    spec = W.DomainSpec(37, 11, 0.8, edf, bc, tw)
    init = W.random_domain_state(37, 11, 21, edf, u_amp=0.05)
    steps = 40
    sim, outs, st = run_gpu(R, [spec], [init], steps, storage=code)
    ref, _ = oracle_fields(orc, spec, init, steps)
    assert (st & R.RLBM_W_NONPHYSICAL) == 0
    errs = errors(outs[0], ref)
    print("mixed %s edf %d: n %.2e theta %.2e u %.2e z %.2e" % ((stname, edf) + tuple(errs)))
    assert max(errs[:3]) <= tol, errs


@pytest.mark.parametrize("stname", ["f32", "f32dev"])
def test_mixed_taylor_green_64(R, orc, stname):
    """Taylor-Green 64 x 64, MJ, 500 steps, FP32 populations or FP32 deviations.
    Raw FP32 populations round each stored f to 6e-8 f every step; the momentum
    they carry then has absolute noise ~1e-8 per step, which over 500 steps reaches
    ~1.5e-5 of max|u| = 0.01: n and theta meet 1e-5, u needs the deviation
    encoding (FP32 deviations round to 6e-8 of f - f_ref) to meet it."""
    code = STORAGE[stname][0]
    wl = W.taylor_green(L=64, u0=0.01, tau=0.9, steps=500)
    sim, outs, st = run_gpu(R, wl.domains, wl.init, wl.steps, storage=code)
    ref, _ = oracle_fields(orc, wl.domains[0], wl.init[0], wl.steps)
    errs = errors(outs[0], ref)
    print("mixed %s TG64 500: n %.2e theta %.2e u %.2e z %.2e" % ((stname,) + tuple(errs)))
    assert st == 0
    assert max(errs[:2]) <= 1e-5, errs
    assert errs[2] <= (1e-5 if stname == "f32dev" else 3e-5), errs


def test_mixed_conservation_periodic(R):
    """The FP32 path still conserves the global N^0 and T^{mu 0} to FP32 storage
    rounding (no drift from the collision) on a periodic domain."""
    spec = W.DomainSpec(48, 40, 0.7, 0)
    init = W.random_domain_state(48, 40, 6, 0, u_amp=0.08)
    sim = R.Simulation([spec], storage=1)
    sim.init(0, init)
    from oracle import oracle as O
    p, w, c, s = O.lattice(0)
    P, C, S = np.tile(p, 12), np.repeat(c, 6), np.repeat(s, 6)
    def cons():
        f = sim.get_populations(0)[:, 1:-1, 1:-1].reshape(72, -1).sum(axis=1)
        return np.array([np.sum(f * P), np.sum(f * P * P), np.sum(f * P * P * C), np.sum(f * P * P * S)])
    c0 = cons()
    sim.step(200)
    c1 = cons()
    scale = np.abs(c0[:2]).max()
    assert np.max(np.abs(c1 - c0)) <= 2e-6 * scale, (c1 - c0) / scale
