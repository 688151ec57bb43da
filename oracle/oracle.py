"""ctypes binding of the FP64 CPU oracle (oracle/rlbm_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle exists to check the CUDA path. Only the
test suite, the package smoke check and the benchmark's CPU-baseline leg may
import this module; the library itself never does.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "liborc.so")
SRC = [os.path.join(HERE, "rlbm_oracle.c")]
DEPS = SRC + [os.path.join(HERE, "rlbm_oracle.h"), os.path.join(HERE, "quadrature_tables.h")]

MJ, FD, BE = 0, 1, 2
PERIODIC, ZERO_GRADIENT, FIXED_T_WALL = 0, 1, 2
INIT_N_THETA, INIT_Z_THETA = 0, 1
W_LANDAU_MAXITER, W_CLAMPED_FUGACITY, E_NONPHYSICAL, E_ZSOLVE = 1, 2, 4, 8

_lib = None


def build(force=False):
    """Compile the oracle (plain C, -O2, no FP contraction, OpenMP over rows)."""
    os.makedirs(BUILD, exist_ok=True)
    stale = force or not os.path.exists(SO) or any(
        os.path.getmtime(p) > os.path.getmtime(SO) for p in DEPS)
    if stale:
        tmp = SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-o", tmp] + SRC + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, SO)
    return SO


class Domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_double),
                ("edf", ctypes.c_int),
                ("bc_xlo", ctypes.c_int), ("bc_xhi", ctypes.c_int),
                ("bc_ylo", ctypes.c_int), ("bc_yhi", ctypes.c_int),
                ("t_wall_xlo", ctypes.c_double), ("t_wall_xhi", ctypes.c_double),
                ("t_wall_ylo", ctypes.c_double), ("t_wall_yhi", ctypes.c_double),
                ("order", ctypes.c_int), ("eta_s", ctypes.c_double),
                ("accel_x", ctypes.c_double), ("accel_y", ctypes.c_double), ("n_wall", ctypes.c_double)]

VELOCITY_WALL = 3


def domain(nx, ny, tau, edf, bc=(PERIODIC, PERIODIC, PERIODIC, PERIODIC), t_wall=(1.0, 1.0, 1.0, 1.0),
           order=5, eta_s=0.0, accel=(0.0, 0.0), n_wall=1.0):
    return Domain(nx, ny, tau, edf, *bc, *t_wall, order, eta_s, accel[0], accel[1], n_wall)


def has_velocity_wall(dom):
    return VELOCITY_WALL in (dom.bc_xlo, dom.bc_xhi, dom.bc_ylo, dom.bc_yhi)


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_lattice.argtypes = [ctypes.c_int, _D, _D, _D, _D]
        L.orc_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_g.restype = ctypes.c_double
        L.orc_landau.argtypes = [_D, _D, _D, _I]
        L.orc_state.argtypes = [ctypes.c_int, _D, _D, _D]
        L.orc_z_from_n_theta.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
        L.orc_eq_moments.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [_D]
        L.orc_eq_moments_quad.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [_D]
        L.orc_basis.argtypes = [_I, _I, _I]
        L.orc_feq.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [_D]
        L.orc_expansion_at.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 6
        L.orc_expansion_at.restype = ctypes.c_double
        L.orc_moments72.argtypes = [ctypes.c_int, _D, _D, _D]
        L.orc_step.argtypes = [ctypes.POINTER(Domain), _D, _D, _D, _D]
        L.orc_diagnostics.argtypes = [ctypes.POINTER(Domain), _D, _D, ctypes.c_int, _D]
        L.orc_feq_order.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 6 + [_D]
        L.orc_step_rows.argtypes = [ctypes.POINTER(Domain), _D, _D, _D, _D, _D, _D]
        L.orc_edge_row.argtypes = [ctypes.POINTER(Domain), _D, _D, ctypes.c_int, _D]
        L.orc_init.argtypes = [ctypes.POINTER(Domain), ctypes.c_int, _D, _D, _D, _D, _D, _D]
        L.orc_fields.argtypes = [ctypes.POINTER(Domain), _D, _D, ctypes.c_int, _D]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice(edf):
    p, w, c, s = np.zeros(6), np.zeros(6), np.zeros(12), np.zeros(12)
    lib().orc_lattice(edf, _p(p), _p(w), _p(c), _p(s))
    return p, w, c, s


def g(edf, nu, z):
    return lib().orc_g(edf, nu, z)


def landau(T):
    T = _c(T)
    eps, U, it = ctypes.c_double(), np.zeros(3), ctypes.c_int()
    st = lib().orc_landau(_p(T), ctypes.byref(eps), _p(U), ctypes.byref(it))
    return eps.value, U, st, it.value


def state(edf, N, T):
    out = np.zeros(6)
    st = lib().orc_state(edf, _p(_c(N)), _p(_c(T)), _p(out))
    return out, st


def z_from_n_theta(edf, n, theta):
    z = ctypes.c_double()
    st = lib().orc_z_from_n_theta(edf, n, theta, ctypes.byref(z))
    return z.value, st


def basis():
    n, k, c = (np.zeros(36, dtype=np.int32) for _ in range(3))
    lib().orc_basis(n.ctypes.data_as(_I), k.ctypes.data_as(_I), c.ctypes.data_as(_I))
    return n, k, c


def eq_moments(edf, theta, ux, uy, z):
    M = np.zeros(36)
    lib().orc_eq_moments(edf, theta, ux, uy, z, _p(M))
    return M


def eq_moments_quad(edf, theta, ux, uy, z):
    M = np.zeros(36)
    lib().orc_eq_moments_quad(edf, theta, ux, uy, z, _p(M))
    return M


def feq_order(edf, order, theta, ux, uy, z, n=-1.0, eps=-1.0):
    f = np.zeros(72)
    lib().orc_feq_order(edf, order, n, eps, theta, ux, uy, z, _p(f))
    return f


def feq(edf, theta, ux, uy, z):
    f = np.zeros(72)
    lib().orc_feq(edf, theta, ux, uy, z, _p(f))
    return f


def expansion_at(edf, order, theta, ux, uy, z, p, phi):
    return lib().orc_expansion_at(edf, order, theta, ux, uy, z, p, phi)


def moments72(edf, f):
    N, T = np.zeros(3), np.zeros(6)
    lib().orc_moments72(edf, _p(_c(f)), _p(N), _p(T))
    return N, T


def init(dom, kind, a, theta, ux, uy):
    nx, ny = dom.nx, dom.ny
    f = np.zeros((72, ny, nx))
    macro = np.zeros((3, ny, nx))
    st = lib().orc_init(ctypes.byref(dom), kind, _p(_c(a)), _p(_c(theta)), _p(_c(ux)), _p(_c(uy)),
                        _p(f), _p(macro))
    if st < 0:
        raise ValueError("orc_init rejected its arguments")
    return f, macro, st


def step(dom, f, macro_in=None):
    nx, ny = dom.nx, dom.ny
    fo = np.zeros((72, ny, nx))
    mo = np.zeros((6, ny, nx))
    mi = _c(macro_in) if macro_in is not None else None
    st = lib().orc_step(ctypes.byref(dom), _p(_c(f)), _p(mi), _p(fo), _p(mo))
    if st < 0:
        raise ValueError("orc_step rejected its arguments")
    return fo, mo, st


def step_rows(dom, f, macro_in, row_lo, row_hi):
    """One step of a y-slab whose outside rows (y = -1, y = ny; [72][nx + 2] or
    None for the slab's own boundary condition) come from its neighbours."""
    nx, ny = dom.nx, dom.ny
    fo = np.zeros((72, ny, nx))
    mo = np.zeros((6, ny, nx))
    mi = _c(macro_in) if macro_in is not None else None
    lo = _c(row_lo) if row_lo is not None else None
    hi = _c(row_hi) if row_hi is not None else None
    st = lib().orc_step_rows(ctypes.byref(dom), _p(_c(f)), _p(mi), _p(lo), _p(hi), _p(fo), _p(mo))
    if st < 0:
        raise ValueError("orc_step_rows rejected its arguments")
    return fo, mo, st


def edge_row(dom, f, macro_in, side):
    """Bottom (side 0) or top (side 1) row as a neighbour reads it, [72][nx + 2]."""
    row = np.zeros((72, dom.nx + 2))
    mi = _c(macro_in) if macro_in is not None else None
    st = lib().orc_edge_row(ctypes.byref(dom), _p(_c(f)), _p(mi), side, _p(row))
    if st < 0:
        raise ValueError("orc_edge_row rejected its arguments")
    return row


def run(dom, f, macro, nsteps):
    """Advance nsteps; macro is the previous state used by walls: (n, ux, uy),
    or the full 6-plane state when the domain has a velocity wall (a 3-plane
    macro, as orc_init returns, is then taken as an equilibrium start and
    completed from the populations)."""
    st_all = 0
    mo = None
    full = has_velocity_wall(dom)
    if full and (macro is None or macro.shape[0] != 6):
        macro, _ = fields(dom, f, None, streamed=False)
    for _ in range(nsteps):
        f, mo, st = step(dom, f, macro)
        st_all |= st
        macro = mo.copy() if full else mo[[0, 2, 3]].copy()
    return f, macro, st_all


def fields(dom, f, macro_in=None, streamed=True):
    nx, ny = dom.nx, dom.ny
    out = np.zeros((6, ny, nx))
    mi = _c(macro_in) if macro_in is not None else None
    st = lib().orc_fields(ctypes.byref(dom), _p(_c(f)), _p(mi), 1 if streamed else 0, _p(out))
    if st < 0:
        raise ValueError("orc_fields rejected its arguments")
    return out, st


def diagnostics(dom, f, macro_in=None, streamed=True):
    """[7][ny][nx]: q^0, q^x, q^y, pi^{xx}, pi^{xxx}, pi^{xxxx}, pi^{xxxxx}."""
    out = np.zeros((7, dom.ny, dom.nx))
    mi = _c(macro_in) if macro_in is not None else None
    st = lib().orc_diagnostics(ctypes.byref(dom), _p(_c(f)), _p(mi), 1 if streamed else 0, _p(out))
    if st < 0:
        raise ValueError("orc_diagnostics rejected its arguments")
    return out, st


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """Threads of later oracle calls (OpenMP over rows; 1 without OpenMP)."""
    lib().orc_set_num_threads(int(n))
