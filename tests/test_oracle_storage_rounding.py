"""The error floor of 16-bit population storage, measured on the oracle alone.

The compressed configuration stores every population as a 16-bit deviation
from a per-domain reference equilibrium (here f^eq(n = 1, theta = 1, u = 0)),
h = (f - f_ref) / f_ref, rounded once per step. Applying exactly that rounding
to the FP64 oracle's state after every step of a Fermi-Dirac Fourier flow
(walls at theta = 0.95 and 1.05) isolates the error the format itself causes,
with no GPU arithmetic involved. A rounding of unit roundoff u perturbs each
population by up to u |f - f_ref|; with |f - f_ref| / f of order 0.1 (a 5 %
temperature range reaches the high-momentum shells strongly) the 72 roundings
of a cell add noise of order u / 100 to its conserved moments every step, and
the moments carry it forward as a random walk that diffusion only partly
smooths. So:

* FP32 (u = 2^-24) stays far inside the 1e-5 per-field bound;
* FP16 (u = 2^-11) ends above 1e-5 after 200 steps, and BF16 (u = 2^-8)
  about eight times higher: with this reference no 16-bit encoding can meet
  1e-5, since a scale per domain or per shell does not change a float's
  relative precision.
The GPU's measured errors of the 16-bit storages sit above this floor, since
there the fixed-temperature wall ghosts are also stored in 16 bits."""
import numpy as np
import pytest

from paper_1709_09073_gb300 import workloads as W


def _round_f16(h):
    return h.astype(np.float16).astype(np.float64)


def _round_bf16(h):
    b = h.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000   # round to nearest even, keep the top 16 bits
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _round_f32(h):
    return h.astype(np.float32).astype(np.float64)


def _errors(orc, rounding, steps=200, nx=96, ny=8):
    wl = W.batched_fourier(n_domains=1, nx=nx, ny=ny, steps=steps, edf=W.FD)
    spec, init = wl.domains[0], wl.init[0]
    dom = orc.domain(spec.nx, spec.ny, spec.tau, spec.edf, spec.bc, spec.t_wall)
    f, m, _ = orc.init(dom, init.kind, init.a, init.theta, init.ux, init.uy)
    z1, _ = orc.z_from_n_theta(W.FD, 1.0, 1.0)
    fref = orc.feq(W.FD, 1.0, 0.0, 0.0, z1)[:, None, None]
    g, mg = f.copy(), m.copy()
    for _ in range(steps):
        f, m, _ = orc.step(dom, f, m)
        m = m[[0, 2, 3]].copy()
        g, mg, _ = orc.step(dom, g, mg)
        mg = mg[[0, 2, 3]].copy()
        g = fref + rounding((g - fref) / fref) * fref
    a, _ = orc.fields(dom, f, m)
    b, _ = orc.fields(dom, g, mg)
    e_n = np.max(np.abs(b[0] / a[0] - 1))
    e_t = np.max(np.abs(b[1] / a[1] - 1))
    e_u = max(np.max(np.abs(b[2] - a[2])), np.max(np.abs(b[3] - a[3])))
    return max(e_n, e_t, e_u)


def test_rounding_helpers():
    # BF16 keeps 8 significant bits: spacing 2^-7 at 1, relative error <= 2^-8
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 3 * 2.0 ** -8, -0.3])
    r = _round_bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0                    # a tie goes to the even neighbour
    assert r[2] == 1.0 + 2.0 ** -7
    assert r[3] == 1.0 + 2.0 ** -6                        # tie between 1 + 2^-7 (odd) and 1 + 2^-6
    assert abs(r[4] / -0.3 - 1) <= 2.0 ** -8
    assert _round_f16(np.array([1.0 + 2.0 ** -11]))[0] == 1.0   # FP16: 11 significant bits


def test_sixteen_bit_storage_error_floor(orc):
    e32 = _errors(orc, _round_f32)
    e16 = _errors(orc, _round_f16)
    eb16 = _errors(orc, _round_bf16)
    print("storage rounding alone after 200 steps: FP32 %.2e, FP16 %.2e, BF16 %.2e" % (e32, e16, eb16))
    assert e32 <= 1e-7
    assert 1e-5 < e16 < 1e-3
    assert 3.0 <= eb16 / e16 <= 24.0
