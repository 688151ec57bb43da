"""Pins of the CUDA path's generated constant tables (csrc/rlbm_tables.json,
written by gen/gen_tables.py alongside csrc/rlbm_tables.h) against the paper:
printed quadrature values, quadrature exactness, and the Appendix closed forms
reproduced by the harmonic moment polynomials and projection matrices."""
import json
import math
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES = os.path.join(ROOT, "paper_1709_09073_gb300", "csrc", "rlbm_tables.json")
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def tab():
    return json.load(open(TABLES))


def _printed():
    rows = {}
    for line in open(os.path.join(GOLDEN, "quadrature_printed.txt")):
        if line.startswith("#") or not line.strip():
            continue
        e, s, p, w = line.split()
        rows.setdefault(e, []).append((int(s), float(p), float(w), p, w))
    return rows


def _header_array(name):
    import re
    hdr = open(os.path.join(ROOT, "paper_1709_09073_gb300", "csrc", "rlbm_tables.h")).read()
    m = re.search(r"#define %s_INIT \{ \\\n(.*?)\n\}" % name, hdr, re.S)
    return [float(x) for x in re.findall(r"[-+0-9.e]+(?=f?,)", m.group(1))]


def _ulp_of_print(txt):
    mant = txt.lower().split("e")[0]
    dec = len(mant.split(".")[1]) if "." in mant else 0
    exp = int(txt.lower().split("e")[1]) if "e" in txt.lower() else 0
    return 10.0 ** (exp - dec)


@pytest.mark.parametrize("name,edf", [("MJ", 0), ("BE", 2)])
def test_printed_values(tab, name, edf):
    for s, p, w, ptxt, wtxt in _printed()[name]:
        assert abs(tab["p"][edf][s - 1] - p) <= _ulp_of_print(ptxt)
        assert abs(tab["w"][edf][s - 1] - w) <= _ulp_of_print(wtxt)


def test_mj_gauss_laguerre(tab):
    x, wl = np.polynomial.laguerre.laggauss(6)
    np.testing.assert_allclose(tab["p"][0], x, rtol=1e-14)
    np.testing.assert_allclose(tab["w"][0], wl / 12.0, rtol=1e-13)


def _g(edf, nu, z):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    if edf == 0:
        return z
    if edf == 1:
        return float(-mp.polylog(nu, -z))
    return float(mp.polylog(nu, z))


def _closed_forms():
    forms = {}
    for line in open(os.path.join(GOLDEN, "appendix_I2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, expr = line.split(":", 1)
        forms[tuple(int(c) for c in key.strip())] = expr.strip()
    return forms


def _harmonic_Z(tab, edf, th, ux, uy, z):
    """Z_nk of the CUDA path: 2 pi n! g_{n+1} theta^{n+1} gamma^n (ux + i uy)^k P_nk(u^2)."""
    u2 = ux * ux + uy * uy
    gam = 1 / math.sqrt(1 - u2)
    Z = {}
    for n in range(6):
        for k in range(n + 1):
            c = tab["Pnk"][n * (n + 1) // 2 + k]
            P = c[0] + u2 * (c[1] + u2 * c[2])
            Z[(n, k)] = (2 * math.pi * math.factorial(n) * _g(edf, n + 1, z) * th ** (n + 1) * gam ** n
                         * complex(ux, uy) ** k * P)
    return Z


CASES = [(0, 1.1, 0.3, -0.2, 0.16), (1, 0.9, -0.25, 0.4, 0.8), (2, 1.3, 0.1, 0.5, 0.3)]


@pytest.mark.parametrize("edf,th,ux,uy,z", CASES)
def test_moment_polynomials_match_appendix(tab, edf, th, ux, uy, z):
    Z = _harmonic_Z(tab, edf, th, ux, uy, z)
    env = dict(pi=math.pi, th=th, ux=ux, uy=uy, u2=ux * ux + uy * uy, gam=1 / math.sqrt(1 - ux * ux - uy * uy))
    for nu in range(1, 7):
        env["g%d" % nu] = _g(edf, nu, z)
    N = 32
    ph = 2 * np.pi * np.arange(N) / N
    for (m, n, q), expr in _closed_forms().items():
        d = m + n + q
        F = np.fft.rfft(np.cos(ph) ** n * np.sin(ph) ** q) / N
        val = F[0].real * Z[(d, 0)].real
        for k in range(1, n + q + 1):
            val += 2 * F[k].real * Z[(d, k)].real - 2 * F[k].imag * Z[(d, k)].imag
        ref = eval(expr, {"__builtins__": {}}, env)
        scale = abs(eval(_closed_forms()[(d, 0, 0)], {"__builtins__": {}}, env))
        assert abs(val - ref) <= 1e-13 * scale, ((m, n, q), val, ref)


@pytest.mark.parametrize("edf,th,ux,uy,z", CASES)
def test_projection_tables_reproduce_moments(tab, edf, th, ux, uy, z):
    """f^eq_ds = sum_k R^c_k cos k phi_d + R^s_k sin k phi_d with R = Q Z reproduces
    every Appendix moment through the d2v72 sums (Eqs. 10-11, 16)."""
    Z = _harmonic_Z(tab, edf, th, ux, uy, z)
    p = np.array(tab["p"][edf])
    Q = tab["Q"][edf]
    off = 0
    feq = np.zeros((12, 6))
    phi = np.arange(12) * np.pi / 6
    for k in range(6):
        for s in range(6):
            Rc = sum(Q[off + s * (6 - k) + (n - k)] * Z[(n, k)].real for n in range(k, 6))
            Rs = sum(Q[off + s * (6 - k) + (n - k)] * Z[(n, k)].imag for n in range(k, 6))
            feq[:, s] += Rc * np.cos(k * phi) + Rs * np.sin(k * phi)
        off += 6 * (6 - k)
    env = dict(pi=math.pi, th=th, ux=ux, uy=uy, u2=ux * ux + uy * uy, gam=1 / math.sqrt(1 - ux * ux - uy * uy))
    for nu in range(1, 7):
        env["g%d" % nu] = _g(edf, nu, z)
    P0 = np.broadcast_to(p[None, :], (12, 6))
    C = np.broadcast_to(np.cos(phi)[:, None], (12, 6))
    S = np.broadcast_to(np.sin(phi)[:, None], (12, 6))
    for (m, n, q), expr in _closed_forms().items():
        disc = np.sum(feq * P0 ** m * (P0 * C) ** n * (P0 * S) ** q)
        ref = eval(expr, {"__builtins__": {}}, env)
        scale = abs(eval(_closed_forms()[(m + n + q, 0, 0)], {"__builtins__": {}}, env))
        assert abs(disc - ref) <= 1e-12 * scale, ((m, n, q), disc, ref)


def test_be_clamp_constants(tab):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    zc = 1 - mp.mpf(10) ** -7
    assert abs(tab["R_zc"] - float(mp.polylog(3, zc) ** 2 / mp.polylog(2, zc) ** 3)) < 1e-15
    for nu in range(1, 7):
        assert abs(tab["g_zc"][nu - 1] - float(mp.polylog(nu, zc))) <= 1e-15 * abs(tab["g_zc"][nu - 1])


@pytest.mark.parametrize("edf", [0, 1, 2])
@pytest.mark.parametrize("kind", ["double", "float"])
def test_conservation_defect_vectors(tab, edf, kind):
    """The stored defects e1, e2, e3 are the exact residuals of the identities
    12 sum_s p_s Q0_sn = [n=1], 12 sum_s p_s^2 Q0_sn = [n=2], 6 sum_s p_s^2 Q1_sn = [n=2]
    for the rounded tables; the kernels use them to keep N^0 and T^{mu 0} exact."""
    from fractions import Fraction as Fr
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    if kind == "double":
        rnd = float
        Q = tab["Q"][edf]
        E = tab["E"][edf]
    else:
        rnd = lambda x: float(np.float32(x))
        Q = tab["Qf"][edf]
        E = tab["Ef"][edf]
    # p and p^2 exactly as the kernels store them (the p^2 table is the rounded
    # square of the exact node, read from the generated header)
    p = [Fr(rnd(x)) for x in tab["p"][edf]]
    p2 = [Fr(rnd(x)) for x in _header_array("RLBM_P2_" + "MJ FD BE".split()[edf])]
    for n in range(6):
        e1 = float(sum(12 * p[s] * Fr(Q[s * 6 + n]) for s in range(6)) - (1 if n == 1 else 0))
        e2 = float(sum(12 * p2[s] * Fr(Q[s * 6 + n]) for s in range(6)) - (1 if n == 2 else 0))
        assert abs(e1 - E[n]) <= 1e-3 * abs(e1) + 1e-30
        assert abs(e2 - E[6 + n]) <= 1e-3 * abs(e2) + 1e-30
    for n in range(1, 6):
        e3 = float(sum(6 * p2[s] * Fr(Q[36 + s * 5 + n - 1]) for s in range(6)) - (1 if n == 2 else 0))
        assert abs(e3 - E[12 + n]) <= 1e-3 * abs(e3) + 1e-30
