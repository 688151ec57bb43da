"""Generate the oracle's d2v72 quadrature tables (oracle/quadrature_tables.h).

TEST INFRASTRUCTURE ONLY: this script belongs to the oracle, which only the
test suite, the smoke check and the CPU baseline leg of the benchmark may use.

Method (Sec. 2.4, "Gaussian Quadrature"): the quadrature equations, Eq. (16),
ask for nodes/weights exact for polynomials of degree <= 10 in (p^0, p^x, p^y).
On the light cone that factorises into
  * an angular rule: the 12 roots phi_n = n*pi/6 of sin(6 phi), each with the
    weight 2*pi/12 (exact for trigonometric degree <= 11), and
  * a radial 6-node Gauss rule for the measure omega(p) dp on [0, inf), exact
    for p^k, k <= 11, whose nodes are the roots of the sixth-order orthogonal
    polynomial R_6(p).
The radial rule is built here from the moments m_k = int_0^inf p^k omega(p) dp
by the Hankel-matrix Cholesky route to the three-term recurrence (Jacobi
matrix) and its eigen-decomposition (Golub-Welsch), in 60-digit arithmetic:
  MJ, Eq. (13):  omega = e^{-p}/(2 pi)            m_k = k!/(2 pi)
  FD, Eq. (14):  omega = 1/(e^p + 1)              m_k = k! eta(k+1)   (eta(1) = ln 2)
  BE, Eq. (15):  omega = 1/(z_c^{-1} e^p - 1)     m_k = k! Li_{k+1}(z_c), z_c = 1 - 1e-7
The per-vector weight is w_s = (2 pi / 12) * lambda_s with lambda_s the radial
Gauss weight.
"""
import os
import mpmath as mp

mp.mp.dps = 60
NS = 6
Z_C = mp.mpf(1) - mp.mpf(10) ** -7


def radial_moments(edf):
    ks = range(2 * NS + 1)
    if edf == "MJ":
        return [mp.factorial(k) / (2 * mp.pi) for k in ks]
    if edf == "FD":
        return [mp.factorial(k) * (mp.log(2) if k == 0 else mp.altzeta(k + 1)) for k in ks]
    if edf == "BE":
        return [mp.factorial(k) * mp.polylog(k + 1, Z_C) for k in ks]
    raise ValueError(edf)


def golub_welsch_from_moments(m):
    n = NS
    H = mp.matrix(n + 1, n + 1)
    for i in range(n + 1):
        for j in range(n + 1):
            H[i, j] = m[i + j]
    U = mp.cholesky(H).T  # H = U^T U, U upper triangular
    alpha = [U[j, j + 1] / U[j, j] - (U[j - 1, j] / U[j - 1, j - 1] if j > 0 else 0) for j in range(n)]
    beta = [U[j + 1, j + 1] / U[j, j] for j in range(n - 1)]
    J = mp.matrix(n, n)
    for j in range(n):
        J[j, j] = alpha[j]
        if j + 1 < n:
            J[j, j + 1] = J[j + 1, j] = beta[j]
    E, Q = mp.eigsy(J)
    order = sorted(range(n), key=lambda i: E[i])
    nodes = [E[i] for i in order]
    lam = [m[0] * Q[0, i] ** 2 for i in order]
    return nodes, lam


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "quadrature_tables.h")
    lines = [
        "/* Generated by oracle/gen_quadrature.py (60-digit Golub-Welsch from the radial",
        " * moments of each weight function, Eqs. 13-16). Oracle-only test infrastructure. */",
        "#ifndef ORC_QUADRATURE_TABLES_H",
        "#define ORC_QUADRATURE_TABLES_H",
        "/* [edf][shell]: edf 0 = MJ, 1 = FD, 2 = BE. Shell momenta p_s (ascending). */",
        "static const double ORC_SHELL_P[3][6] = {",
    ]
    tabs = {e: golub_welsch_from_moments(radial_moments(e)) for e in ("MJ", "FD", "BE")}
    for e in ("MJ", "FD", "BE"):
        lines.append("  {" + ", ".join(mp.nstr(x, 30, min_fixed=-1, max_fixed=1) for x in tabs[e][0]) + "},")
    lines.append("};")
    lines.append("/* Per-vector weights w_s = (2 pi / 12) * radial Gauss weight. */")
    lines.append("static const double ORC_SHELL_W[3][6] = {")
    for e in ("MJ", "FD", "BE"):
        lines.append("  {" + ", ".join(mp.nstr(2 * mp.pi / 12 * x, 30, min_fixed=-1, max_fixed=1) for x in tabs[e][1]) + "},")
    lines.append("};")
    lines.append("#endif")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
