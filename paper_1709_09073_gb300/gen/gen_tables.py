"""Generate the constant tables of the CUDA path (csrc/rlbm_tables.h + rlbm_tables.json).

Run offline (needs mpmath and sympy); the generated header is committed, so the
build on a GPU machine needs neither. Everything is computed in 80-digit
arithmetic and rounded once to double (and float for the mixed-precision path).

 1. d2v72 radial rule (Sec. 2.4): R_6 is built by Gram-Schmidt on 1, p, ..., p^6
    under <f, g> = int f g omega dp (the inner products are the radial moments of
    the weight functions of Eqs. 13-15), its six roots are the shell momenta, and
    the radial weights solve the quadrature equations sum_s lambda_s p_s^k = m_k,
    k = 0..5. Per-vector weight w_s = (2 pi / 12) lambda_s.
 2. Projection (Eqs. 10-11): with the basis p^n {cos, sin}(k phi), 0 <= k <= n <= 5,
    the discrete Gram matrix is block diagonal (12-point trigonometric
    orthogonality): G = N_k H^(k), N_0 = 12, N_k>0 = 6, H^(k)_{nn'} = sum_s w_s p_s^{n+n'}.
    The equilibrium is f^eq_{ds} = sum_k R^c_k(s) cos k phi_d + R^s_k(s) sin k phi_d
    with R^{c|s}_k(s) = sum_{n'} Q^(k)_{s n'} M^{c|s}_{n' k} and
    Q^(k)_{s n'} = (w_s / N_k) sum_n p_s^n (H^(k))^{-1}_{n n'}.
 3. Equilibrium moments (Appendix, harmonic form): the complex moment
    Z_{nk} = int dp dphi f^eq p^n e^{i k phi}
           = 2 pi n! g_{n+1}(z) theta^{n+1} gamma^n (u_x + i u_y)^k P_{nk}(u^2),
    P_{nk} a polynomial of degree <= 2 in u^2, derived here with sympy from
    int dbeta cos(k beta)/(a - u cos beta) = 2 pi (a^2-u^2)^{-1/2} ((a - sqrt(a^2-u^2))/u)^k
    by differentiating n times in a.
 4. EDF integrals g_nu (Eq. 12) for FD/BE: power-series table k^{-nu} and the
    coefficients of the expansions in mu = ln z (zeta / eta values at integers).
"""
import json
import os

import mpmath as mp
import numpy as np
import sympy as sp

mp.mp.dps = 80
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "csrc")
NS = 6
ZC = mp.mpf(1) - mp.mpf(10) ** -7
EDFS = ("MJ", "FD", "BE")
NSERIES = 64       # power-series terms tabulated (k = 1..NSERIES)
NEXP = 48          # mu-expansion terms tabulated


def moments(edf):
    if edf == "MJ":
        return [mp.factorial(k) / (2 * mp.pi) for k in range(2 * NS + 1)]
    if edf == "FD":
        return [mp.factorial(k) * (mp.log(2) if k == 0 else mp.altzeta(k + 1)) for k in range(2 * NS + 1)]
    return [mp.factorial(k) * mp.polylog(k + 1, ZC) for k in range(2 * NS + 1)]


def radial_rule(edf):
    m = moments(edf)
    # monomial inner product <p^i, p^j> = m_{i+j}; classical Gram-Schmidt on coefficient vectors
    basis = []
    for deg in range(NS + 1):
        v = [mp.mpf(0)] * (NS + 1)
        v[deg] = mp.mpf(1)
        for b in basis:
            proj = sum(v[i] * b[j] * m[i + j] for i in range(NS + 1) for j in range(NS + 1))
            v = [v[i] - proj * b[i] for i in range(NS + 1)]
        nrm = mp.sqrt(sum(v[i] * v[j] * m[i + j] for i in range(NS + 1) for j in range(NS + 1)))
        basis.append([x / nrm for x in v])
    r6 = basis[NS]
    coeffs = [r6[NS - i] for i in range(NS + 1)]  # highest degree first
    roots = sorted(mp.re(r) for r in mp.polyroots(coeffs, maxsteps=400, extraprec=400))
    V = mp.matrix([[r ** k for r in roots] for k in range(NS)])
    lam = mp.lu_solve(V, mp.matrix(m[:NS]))
    w = [2 * mp.pi / 12 * lam[i] for i in range(NS)]
    return roots, w


def projection(p, w, order=NS - 1):
    """Projection of f^eq / omega onto the basis p^n {cos, sin}(k phi) with
    k <= n <= order (Eqs. 10-11; order 5 is the full expansion), per harmonic
    block k: Q[k][s][n - k] = w_s / N_k sum_a p_s^(n_a) (H_k^-1)[a][n - k], H_k the
    radial Gram matrix of the block. Laid out for order 5 (k, s, n'), the
    entries of degrees above `order` are zero."""
    Q = []
    for k in range(NS):
        ns = list(range(k, order + 1))
        Nk = 12 if k == 0 else 6
        if ns:
            H = mp.matrix(len(ns), len(ns))
            for a, na in enumerate(ns):
                for b, nb in enumerate(ns):
                    H[a, b] = sum(w[s] * p[s] ** (na + nb) for s in range(NS))
            Hi = H ** -1
        for s in range(NS):
            for b in range(NS - k):
                if b < len(ns):
                    Q.append(w[s] / Nk * sum(p[s] ** ns[a] * Hi[a, b] for a in range(len(ns))))
                else:
                    Q.append(mp.mpf(0))
    return Q  # ordered k, s, n'


def moment_defects(p, Q, ctype):
    """Exact defects of the rounded projection table in the conserved moments.

    With p_s and p_s^2 as stored (FP64 or FP32), the equilibrium's N^0 = sum f p
    and T^{00} = sum f p^2 should pick out exactly Z_10 and Z_20 from harmonic
    block k = 0, and T^{0x} + i T^{0y} exactly Z_21 from block k = 1. After
    rounding, column n of a block misses these identities by a tiny constant:
      e1_n = sum_s 12 p_s Q0_{sn} - [n = 1],  e2_n = sum_s 12 p_s^2 Q0_{sn} - [n = 2],
      e3_n = sum_s 6 p_s^2 Q1_{sn} - [n = 2].
    A constant defect times the equilibrium moments is a bias that the relaxation
    would turn into a drift of the conserved totals at every step; the kernels
    remove it by correcting Z_10, Z_20, Z_21 with these vectors (computed here
    exactly, in rational arithmetic on the stored values)."""
    from fractions import Fraction as Fr
    rnd = (lambda x: float(x)) if ctype == "double" else (lambda x: float(np.float32(float(x))))
    pr = [Fr(rnd(x)) for x in p]
    p2r = [Fr(rnd(x * x)) for x in p]
    Qr = [Fr(rnd(x)) for x in Q]
    e1 = [float(sum(12 * pr[s] * Qr[s * 6 + n] for s in range(6)) - (1 if n == 1 else 0)) for n in range(6)]
    e2 = [float(sum(12 * p2r[s] * Qr[s * 6 + n] for s in range(6)) - (1 if n == 2 else 0)) for n in range(6)]
    b1 = 6 * 6
    e3 = [0.0] + [float(sum(6 * p2r[s] * Qr[b1 + s * 5 + (n - 1)] for s in range(6)) - (1 if n == 2 else 0))
                  for n in range(1, 6)]
    return e1 + e2 + e3


def moment_polys():
    a, u = sp.symbols("a u", positive=True)
    out = []
    for n in range(NS):
        for k in range(n + 1):
            base = 2 * sp.pi * (a ** 2 - u ** 2) ** sp.Rational(-1, 2) * ((a - sp.sqrt(a ** 2 - u ** 2)) / u) ** k
            K = ((-1) ** n / sp.factorial(n) * sp.diff(base, a, n)).subs(a, 1)
            gam = 1 / sp.sqrt(1 - u ** 2)
            P = sp.simplify(sp.expand(K * gam ** (-(n + 1)) / (2 * sp.pi * gam ** n * u ** k)))
            v = sp.symbols("v")
            Pv = sp.Poly(sp.expand(P.subs(u, sp.sqrt(v))), v)
            c = [sp.Rational(0)] * 3
            for (e,), coef in Pv.terms():
                assert e <= 2
                c[e] = sp.Rational(coef)
            out.append([float(x) for x in c])
    return out  # ordered n, k (k <= n): index n(n+1)/2 + k


def polylog_tables():
    inv = [[float(mp.mpf(k) ** -nu) for k in range(1, NSERIES + 1)] for nu in range(1, 7)]
    be = []
    fd = []
    for nu in range(1, 7):
        rb, rf = [], []
        for k in range(NEXP):
            s = nu - k
            rb.append(0.0 if k == nu - 1 else float(mp.zeta(s) / mp.factorial(k)))
            rf.append(float((mp.log(2) if s == 1 else mp.altzeta(s)) / mp.factorial(k)))
        be.append(rb)
        fd.append(rf)
    harm = [float(mp.harmonic(nu - 1) / mp.factorial(nu - 1)) for nu in range(1, 7)]
    rfact = [float(1 / mp.factorial(nu - 1)) for nu in range(1, 7)]
    gzc = [float(mp.polylog(nu, ZC)) for nu in range(1, 7)]
    return inv, be, fd, harm, rfact, gzc


def c_arr(name, vals, ctype="double", per_line=4):
    """Emit `#define NAME_INIT { ... }` so device code can initialise __constant__ arrays."""
    # shortest decimal that reads back to the same double / float exactly
    fmt = (lambda x: repr(float(x))) if ctype == "double" else (lambda x: repr(float(np.float32(float(x)))) + "f")
    items = [fmt(v) for v in vals]
    lines = []
    for i in range(0, len(items), per_line):
        lines.append("  " + ", ".join(items[i:i + per_line]) + ", \\")
    return "/* %d x %s */\n#define %s_INIT { \\\n%s\n}\n" % (len(vals), ctype, name, "\n".join(lines))


def main():
    data = {"p": [], "w": [], "Q": []}
    hdr = ["/* Generated by paper_1709_09073_gb300/gen/gen_tables.py -- do not edit.",
           " * Constant tables of the CUDA path: d2v72 radial rule per EDF (Sec. 2.4),",
           " * harmonic-block projection matrices (Eqs. 10-11), closed-form moment",
           " * polynomials (Appendix) and polylog coefficients (Eq. 12). */",
           "#ifndef RLBM_TABLES_H", "#define RLBM_TABLES_H", ""]
    for e in EDFS:
        p, w = radial_rule(e)
        Q = projection(p, w)
        data["p"].append([float(x) for x in p])
        data["w"].append([float(x) for x in w])
        data["Q"].append([float(x) for x in Q])
        data.setdefault("Qf", []).append([float(np.float32(float(x))) for x in Q])
        E = moment_defects(p, Q, "double")
        Ef = moment_defects(p, Q, "float")
        data.setdefault("E", []).append(E)
        data.setdefault("Ef", []).append(Ef)
        hdr.append(c_arr("RLBM_P_%s" % e, p))
        hdr.append(c_arr("RLBM_W_%s" % e, w))
        hdr.append(c_arr("RLBM_P2_%s" % e, [x * x for x in p]))
        hdr.append(c_arr("RLBM_Q_%s" % e, Q))
        hdr.append(c_arr("RLBM_E_%s" % e, E))
        hdr.append(c_arr("RLBM_PF_%s" % e, p, "float"))
        hdr.append(c_arr("RLBM_WF_%s" % e, w, "float"))
        hdr.append(c_arr("RLBM_QF_%s" % e, Q, "float"))
        hdr.append(c_arr("RLBM_EF_%s" % e, Ef))
        # lower expansion orders (Sec. 3.5 order comparison), FP64 path only
        for order in (2, 3, 4):
            Qo = projection(p, w, order)
            Eo = moment_defects(p, Qo, "double")
            data.setdefault("Qo%d" % order, []).append([float(x) for x in Qo])
            data.setdefault("Eo%d" % order, []).append(Eo)
            hdr.append(c_arr("RLBM_QO%d_%s" % (order, e), Qo))
            hdr.append(c_arr("RLBM_EO%d_%s" % (order, e), Eo))
    polys = moment_polys()
    data["Pnk"] = polys
    hdr.append(c_arr("RLBM_PNK", [c for row in polys for c in row]))
    inv, be, fd, harm, rfact, gzc = polylog_tables()
    hdr.append("#define RLBM_NSERIES %d\n#define RLBM_NEXP %d" % (NSERIES, NEXP))
    hdr.append(c_arr("RLBM_INVPOW", [x for row in inv for x in row]))
    hdr.append(c_arr("RLBM_BE_EXP", [x for row in be for x in row]))
    hdr.append(c_arr("RLBM_FD_EXP", [x for row in fd for x in row]))
    hdr.append(c_arr("RLBM_BE_LOGCOEF", rfact))
    hdr.append(c_arr("RLBM_BE_HARM", harm))
    hdr.append(c_arr("RLBM_G_ZC", gzc))
    rzc = mp.polylog(3, ZC) ** 2 / mp.polylog(2, ZC) ** 3
    hdr.append("#define RLBM_R_ZC %r\n" % float(rzc))
    hdr.append("#endif")
    with open(os.path.join(CSRC, "rlbm_tables.h"), "w") as fh:
        fh.write("\n".join(hdr) + "\n")
    data["g_zc"] = gzc
    data["R_zc"] = float(rzc)
    with open(os.path.join(CSRC, "rlbm_tables.json"), "w") as fh:
        json.dump(data, fh, indent=1)
    print("wrote tables")


if __name__ == "__main__":
    main()
