"""rlbm_init_all / rlbm_moments_all (every domain in one launch, fields packed
domain after domain) against the per-domain rlbm_init / rlbm_moments: the same
kernels' arithmetic, so the populations and fields must be bit-identical, from
host and from device fields, for every storage. The mixed storages initialise
in the collision's FP32 deviation arithmetic: the stored equilibrium returns
its input fields (n, theta relative, u absolute) to within FP32 rounding."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W

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


def _batch(edf):
    specs = [W.DomainSpec(33, 17, 0.7, edf), W.DomainSpec(64, 8, 1.3, edf, (1, 1, 0, 0)),
             W.DomainSpec(101, 40, 0.9, edf, (2, 2, 0, 0), (0.95, 1.05, 1, 1)),
             W.DomainSpec(1, 5, 0.8, edf), W.DomainSpec(6, 7, 1.1, edf, (0, 0, 2, 2), (1, 1, 1.02, 0.99))]
    inits = [W.random_domain_state(s.nx, s.ny, 80 + i, edf, u_amp=0.08) for i, s in enumerate(specs)]
    return specs, inits


def _packed(inits):
    return [np.concatenate([getattr(s, k).reshape(-1) for s in inits]) for k in ("a", "theta", "ux", "uy")]


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("storage", [0, 1, 4, 2, 3])
@pytest.mark.parametrize("on_device", [False, True])
def test_batched_init_and_moments_match_per_domain(R, edf, storage, on_device):
    import torch
    specs, inits = _batch(edf)
    one = R.Simulation(specs, edf=edf, storage=storage)
    st1 = 0
    for i, s in enumerate(inits):
        st1 |= one.init(i, s)
    allh = R.Simulation(specs, edf=edf, storage=storage)
    packed = _packed(inits)
    if on_device:
        packed = [torch.from_numpy(p).cuda() for p in packed]
    st2 = allh.init_all(inits[0].kind, *packed)
    assert st1 == st2
    for i in range(len(specs)):
        assert np.array_equal(one.get_populations(i), allh.get_populations(i), equal_nan=True), i
    one.step(3)
    allh.step(3)
    ref = [one.moments(i) for i in range(len(specs))]
    if on_device:
        n = sum(d.nx * d.ny for d in specs)
        out = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(5)]
        got = [o.cpu().numpy() for o in allh.moments_all(out=out)]
    else:
        got = allh.moments_all()
    for k in range(5):
        want = np.concatenate([r[k].reshape(-1) for r in ref])
        assert np.array_equal(got[k], want, equal_nan=True), k
    one.close()
    allh.close()


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("storage", [1, 4])
def test_mixed_init_returns_its_fields(R, edf, storage):
    specs, inits = _batch(edf)
    sim = R.Simulation(specs, edf=edf, storage=storage)
    assert sim.init_all(inits[0].kind, *_packed(inits)) == 0
    for i, s in enumerate(inits):
        n, th, ux, uy, z = sim.moments(i, streamed=False)
        assert np.max(np.abs(n / s.a - 1)) <= 1e-6
        assert np.max(np.abs(th / s.theta - 1)) <= 1e-6
        assert max(np.max(np.abs(ux - s.ux)), np.max(np.abs(uy - s.uy))) <= 1e-6
    sim.close()


def test_batched_calls_check_their_arguments(R):
    specs, inits = _batch(0)
    sim = R.Simulation(specs, edf=0, storage=4)
    with pytest.raises(R.RlbmError):
        sim.moments_all()                                  # nothing initialised yet
    short = [p[:-1] for p in _packed(inits)]
    with pytest.raises(ValueError):
        sim.init_all(0, *short)
    sim.close()


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("streamed", [True, False])
def test_mixed_readout_matches_fp64_readout(R, edf, streamed):
    """The mixed storages read their fields in the collision's arithmetic (FP32
    pull and sums, double-float totals and Landau frame): the same populations
    read by the FP64 kernel (through an FP64 handle holding them) agree to
    FP32-rounding level."""
    specs, inits = _batch(edf)
    sim = R.Simulation(specs, edf=edf, storage=4)
    sim.init_all(inits[0].kind, *_packed(inits))
    sim.step(5)
    ref = R.Simulation(specs, edf=edf, storage=0)
    for i in range(len(specs)):
        ref.set_populations(i, sim.get_populations(i))
    for i in range(len(specs)):
        a = sim.moments(i, streamed=streamed)
        b = ref.moments(i, streamed=streamed)
        assert np.max(np.abs(a[0] / b[0] - 1)) <= 1e-6
        assert np.max(np.abs(a[1] / b[1] - 1)) <= 1e-6
        umax = max(np.max(np.abs(b[2])), np.max(np.abs(b[3])))
        assert max(np.max(np.abs(a[2] - b[2])), np.max(np.abs(a[3] - b[3]))) <= 1e-6 * umax
        assert np.max(np.abs(a[4] / b[4] - 1)) <= 1e-5
    sim.close()
    ref.close()
