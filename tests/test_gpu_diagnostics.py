"""Diagnostic fields of the CUDA path (rlbm_diagnostics through the C ABI)
against the oracle: heat flux q^0, q^x, q^y and the diagonal non-equilibrium
tensors pi^{x..x}, orders 2-5, on a walled domain after a few steps. Errors
are measured against each field's natural scale (h_E n for q, the raw moment
sum f |p^x|^k for pi): 1e-12 for FP64 storage, 1e-5 for FP32 deviations."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W
from test_gpu_fp64 import run_gpu

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


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("storage,tol", [(0, 1e-12), (4, 1e-5)])
@pytest.mark.parametrize("streamed", [True, False])
def test_diagnostics_match_oracle(R, orc, edf, storage, tol, streamed):
    spec = W.DomainSpec(37, 11, 0.8, edf, (W.FIXED_T_WALL, W.FIXED_T_WALL, W.PERIODIC, W.PERIODIC),
                        (0.96, 1.05, 1.0, 1.0))
    init = W.random_domain_state(37, 11, 60 + edf, edf, u_amp=0.1)
    steps = 7
    sim, _, st = run_gpu(R, [spec], [init], steps, storage=storage, streamed=streamed)
    assert (st & R.RLBM_W_NONPHYSICAL) == 0
    g = sim.diagnostics(0, streamed=streamed)
    dom = orc.domain(spec.nx, spec.ny, spec.tau, edf, spec.bc, spec.t_wall)
    f, m, _ = orc.init(dom, init.kind, init.a, init.theta, init.ux, init.uy)
    f, m, _ = orc.run(dom, f, m, steps)
    ref, _ = orc.diagnostics(dom, f, m, streamed=streamed)
    fl, _ = orc.fields(dom, f, m, streamed=streamed)
    p, w, c, s = orc.lattice(edf)
    PC = np.abs(np.tile(p, 12) * np.repeat(c, 6))
    hq = np.max(3.0 * fl[1] * fl[0])
    for k, name in enumerate(R.Simulation.DIAGNOSTICS):
        if k < 3:
            scale = hq
        else:
            scale = np.max(np.einsum("qyx,q->yx", np.abs(f), PC ** (k - 1)))
        err = np.max(np.abs(g[name] - ref[k])) / scale
        print("edf %d storage %d streamed %d %s: %.2e" % (edf, storage, streamed, name, err))
        assert err <= tol, (name, err)
    sim.close()
