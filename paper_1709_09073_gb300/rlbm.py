"""Python binding of the C ABI in include/rlbm.h (argument marshalling only).

Every step of the method runs in the CUDA library librlbm.so. PyTorch provides
device memory (the workspace) and the CUDA stream. There is no fallback: if
the library cannot be loaded, every call raises.
"""
import ctypes
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librlbm.so")

RLBM_MJ, RLBM_FD, RLBM_BE = 0, 1, 2
RLBM_F64, RLBM_F32, RLBM_BF16DEV, RLBM_F16DEV, RLBM_F32DEV = 0, 1, 2, 3, 4
RLBM_PERIODIC, RLBM_ZERO_GRADIENT, RLBM_FIXED_T_WALL, RLBM_VELOCITY_WALL, RLBM_EXCHANGED = 0, 1, 2, 3, 4
RLBM_INIT_N_THETA, RLBM_INIT_Z_THETA = 0, 1
RLBM_OK = 0
RLBM_W_LANDAU_MAXITER, RLBM_W_CLAMPED_FUGACITY, RLBM_W_NONPHYSICAL, RLBM_W_ZSOLVE = 1, 2, 4, 8
RLBM_E_ARG, RLBM_E_CUDA, RLBM_E_STATE, RLBM_E_UNSUPPORTED, RLBM_E_NOBUFFER = -1, -2, -3, -4, -5
RLBM_E_SCRATCH = -6
RLBM_W_DEVICE_TIMEOUT = 16
RLBM_KERNEL_L1, RLBM_KERNEL_TMA = 0, 1
RLBM_NOALLOC_SCRATCH_BYTES = 32 << 20

EXPORTS = ["rlbm_workspace_bytes", "rlbm_create", "rlbm_init", "rlbm_step", "rlbm_moments",
           "rlbm_get_populations", "rlbm_set_populations", "rlbm_tune", "rlbm_sync_status",
           "rlbm_destroy", "rlbm_status_string", "rlbm_last_step_info", "rlbm_step_noalloc", "rlbm_diagnostics",
           "rlbm_select_kernel", "rlbm_edge_row_bytes", "rlbm_pack_edge_rows", "rlbm_unpack_ghost_rows",
           "rlbm_pipe_peaks", "rlbm_set_wait_limit", "rlbm_init_all", "rlbm_moments_all", "rlbm_set_grid",
           "rlbm_layout_tiles"]


class rlbm_domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_double),
                ("bc_xlo", ctypes.c_int), ("bc_xhi", ctypes.c_int),
                ("bc_ylo", ctypes.c_int), ("bc_yhi", ctypes.c_int),
                ("t_wall_xlo", ctypes.c_double), ("t_wall_xhi", ctypes.c_double),
                ("t_wall_ylo", ctypes.c_double), ("t_wall_yhi", ctypes.c_double),
                ("ref_n", ctypes.c_double), ("ref_theta", ctypes.c_double),
                ("scale", ctypes.c_double), ("eta_s", ctypes.c_double),
                ("accel_x", ctypes.c_double), ("accel_y", ctypes.c_double), ("n_wall", ctypes.c_double)]


class rlbm_config(ctypes.Structure):
    _fields_ = [("ndomains", ctypes.c_int), ("domains", ctypes.POINTER(rlbm_domain)),
                ("edf", ctypes.c_int), ("storage", ctypes.c_int), ("order", ctypes.c_int),
                ("device_buffer", ctypes.c_void_p), ("buffer_bytes", ctypes.c_size_t),
                ("cuda_stream", ctypes.c_void_p)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p


def load(path=None):
    """Load librlbm.so (built in-tree by paper_1709_09073_gb300.build). Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("librlbm.so not found at %s: build it with "
                           "`python -m paper_1709_09073_gb300.build` (no CPU fallback exists)" % p)
    L = ctypes.CDLL(p)
    L.rlbm_workspace_bytes.argtypes = [ctypes.POINTER(rlbm_config)]
    L.rlbm_workspace_bytes.restype = ctypes.c_size_t
    L.rlbm_layout_tiles.argtypes = [ctypes.POINTER(rlbm_config), ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    L.rlbm_layout_tiles.restype = ctypes.c_int
    L.rlbm_create.argtypes = [ctypes.POINTER(rlbm_config), ctypes.POINTER(_H)]
    L.rlbm_init.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.rlbm_step.argtypes = [_H, ctypes.c_int]
    L.rlbm_moments.argtypes = [_H, ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 5 + [ctypes.c_int]
    L.rlbm_get_populations.argtypes = [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    L.rlbm_set_populations.argtypes = [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    L.rlbm_tune.argtypes = [_H, ctypes.c_int]
    L.rlbm_select_kernel.argtypes = [_H, ctypes.c_int]
    L.rlbm_diagnostics.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    L.rlbm_sync_status.argtypes = [_H]
    L.rlbm_destroy.argtypes = [_H]
    L.rlbm_status_string.argtypes = [ctypes.c_int]
    L.rlbm_status_string.restype = ctypes.c_char_p
    L.rlbm_last_step_info.argtypes = [_H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]
    L.rlbm_edge_row_bytes.argtypes = [_H, ctypes.c_int]
    L.rlbm_edge_row_bytes.restype = ctypes.c_size_t
    L.rlbm_pack_edge_rows.argtypes = [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.rlbm_unpack_ghost_rows.argtypes = [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.rlbm_step_noalloc.argtypes = [ctypes.POINTER(rlbm_domain), ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint)]
    L.rlbm_pipe_peaks.argtypes = [_D, _D, ctypes.POINTER(ctypes.c_int)]
    L.rlbm_init_all.argtypes = [_H, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_int]
    L.rlbm_moments_all.argtypes = [_H, ctypes.c_int] + [ctypes.c_void_p] * 5 + [ctypes.c_int]
    L.rlbm_set_wait_limit.argtypes = [_H, ctypes.c_double]
    L.rlbm_set_grid.argtypes = [_H, ctypes.c_int]
    _lib = L
    return L


class RlbmError(RuntimeError):
    pass


def _check(code):
    if code < 0:
        raise RlbmError("rlbm error %d: %s" % (code, load().rlbm_status_string(code).decode()))
    return code


def make_domains(specs):
    arr = (rlbm_domain * len(specs))()
    for i, d in enumerate(specs):
        arr[i] = rlbm_domain(d.nx, d.ny, d.tau, *d.bc, *d.t_wall, d.ref_n, d.ref_theta, d.scale, d.eta_s,
                             d.accel[0], d.accel[1], d.n_wall)
    return arr


def rlbm_workspace_bytes(specs, edf, storage, order=5):
    doms = make_domains(specs)
    cfg = rlbm_config(len(specs), doms, edf, storage, order, None, 0, None)
    return load().rlbm_workspace_bytes(ctypes.byref(cfg))


def rlbm_layout_tiles(specs, edf, storage, packed):
    """The tile work list (rows of domain, x0, y0, w) a handle of these domains
    would walk: the plain 32 x 4 list, or the mixed L1 step's packed one."""
    doms = make_domains(specs)
    cfg = rlbm_config(len(specs), doms, edf, storage, 5, None, 0, None)
    n = _check(load().rlbm_layout_tiles(ctypes.byref(cfg), int(packed), None, 0))
    out = np.zeros((max(n, 1), 4), dtype=np.int32)
    _check(load().rlbm_layout_tiles(ctypes.byref(cfg), int(packed), out.ctypes.data_as(ctypes.c_void_p), n))
    return out[:n]


def _ptr(x):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr()), 1
    return x.ctypes.data_as(ctypes.c_void_p), 0


class Simulation:
    """One handle over a torch-allocated workspace; all compute in librlbm."""

    def __init__(self, specs, edf=RLBM_MJ, storage=RLBM_F64, device="cuda", stream=None, order=5):
        import torch
        self.torch = torch
        self.specs = list(specs)
        self.edf, self.storage = edf, storage
        L = load()
        self._doms = make_domains(self.specs)
        cfg = rlbm_config(len(self.specs), self._doms, edf, storage, order, None, 0, None)
        nbytes = L.rlbm_workspace_bytes(ctypes.byref(cfg))
        if nbytes == 0:
            raise RlbmError("invalid configuration")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        cfg.device_buffer = ctypes.c_void_p(self.workspace.data_ptr())
        cfg.buffer_bytes = nbytes
        cfg.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.h = _H()
        _check(L.rlbm_create(ctypes.byref(cfg), ctypes.byref(self.h)))

    def init(self, domain, state):
        """Initialise from a workloads.InitialState (host numpy or device torch fields)."""
        fields = [state.a, state.theta, state.ux, state.uy]
        if hasattr(state.a, "data_ptr"):
            ptrs = [ctypes.c_void_p(f.contiguous().data_ptr()) for f in fields]
            on_dev = 1
        else:
            fields = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
            ptrs = [f.ctypes.data_as(ctypes.c_void_p) for f in fields]
            on_dev = 0
        return _check(load().rlbm_init(self.h, domain, state.kind, *ptrs, on_dev))

    def init_all(self, kind, a, theta, ux, uy):
        """Initialise every domain at once from packed fields (the domains'
        [ny][nx] arrays one after the other): host numpy or device torch."""
        fields = [a, theta, ux, uy]
        n = sum(d.nx * d.ny for d in self.specs)
        if hasattr(a, "data_ptr"):
            for f in fields:
                if f.dtype != self.torch.float64 or not f.is_cuda or not f.is_contiguous() or f.numel() != n:
                    raise ValueError("packed fields must be contiguous float64 CUDA tensors of %d values" % n)
            ptrs, on_dev = [ctypes.c_void_p(f.data_ptr()) for f in fields], 1
        else:
            fields = [np.ascontiguousarray(f, dtype=np.float64).reshape(-1) for f in fields]
            if any(f.size != n for f in fields):
                raise ValueError("packed fields must hold %d values" % n)
            ptrs, on_dev = [f.ctypes.data_as(ctypes.c_void_p) for f in fields], 0
        return _check(load().rlbm_init_all(self.h, kind, *ptrs, on_dev))

    def moments_all(self, streamed=True, out=None):
        """n, theta, ux, uy, z of every domain, packed (see init_all): into the
        device tensors `out` if given (four or five: z is optional), else
        returned as host arrays."""
        n = sum(d.nx * d.ny for d in self.specs)
        if out is not None:
            if len(out) not in (4, 5):
                raise ValueError("outputs: n, theta, ux, uy and optionally z")
            for f in out:
                if f.dtype != self.torch.float64 or not f.is_cuda or not f.is_contiguous() or f.numel() != n:
                    raise ValueError("outputs must be contiguous float64 CUDA tensors of %d values" % n)
            ptrs = [ctypes.c_void_p(f.data_ptr()) for f in out] + ([None] if len(out) == 4 else [])
            _check(load().rlbm_moments_all(self.h, 1 if streamed else 0, *ptrs, 1))
            return out
        res = [np.empty(n) for _ in range(5)]
        _check(load().rlbm_moments_all(self.h, 1 if streamed else 0,
                                       *[r.ctypes.data_as(ctypes.c_void_p) for r in res], 0))
        return res

    def step(self, nsteps):
        return _check(load().rlbm_step(self.h, nsteps))

    def moments(self, domain, streamed=True, on_device=False):
        """Return (n, theta, ux, uy, z) as numpy arrays (or torch tensors on device)."""
        if not 0 <= domain < len(self.specs):
            dummy = np.empty(1)
            p = dummy.ctypes.data_as(ctypes.c_void_p)
            _check(load().rlbm_moments(self.h, domain, 1, p, p, p, p, p, 0))
        d = self.specs[domain]
        if on_device:
            outs = [self.torch.empty((d.ny, d.nx), dtype=self.torch.float64, device=self.workspace.device)
                    for _ in range(5)]
            ptrs = [ctypes.c_void_p(o.data_ptr()) for o in outs]
        else:
            outs = [np.empty((d.ny, d.nx)) for _ in range(5)]
            ptrs = [o.ctypes.data_as(ctypes.c_void_p) for o in outs]
        _check(load().rlbm_moments(self.h, domain, 1 if streamed else 0, *ptrs, 1 if on_device else 0))
        return outs

    DIAGNOSTICS = ("q0", "qx", "qy", "pi2", "pi3", "pi4", "pi5")

    def diagnostics(self, domain, streamed=True):
        """Heat flux q^0, q^x, q^y and the diagonal non-equilibrium tensors
        pi^{x..x} of orders 2-5, as a dict of [ny][nx] numpy arrays."""
        d = self.specs[domain]
        out = np.empty((7, d.ny, d.nx))
        _check(load().rlbm_diagnostics(self.h, domain, 1 if streamed else 0,
                                       out.ctypes.data_as(ctypes.c_void_p), 0))
        return dict(zip(self.DIAGNOSTICS, out))

    def get_populations(self, domain):
        d = self.specs[domain]
        f = np.empty((72, d.ny + 2, d.nx + 2))
        _check(load().rlbm_get_populations(self.h, domain, f.ctypes.data_as(ctypes.c_void_p), 0))
        return f

    def set_populations(self, domain, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        _check(load().rlbm_set_populations(self.h, domain, f.ctypes.data_as(ctypes.c_void_p), 0))

    # y-slab halo rows: packed faces are [30][nx + 2] device tensors of the
    # storage element type (raw storage encoding)
    _ROW_DTYPE = {RLBM_F64: "float64", RLBM_F32: "float32", RLBM_F32DEV: "float32",
                  RLBM_BF16DEV: "int16", RLBM_F16DEV: "int16"}

    def edge_row_buffer(self, domain):
        """An empty packed face for `domain` on the workspace's device."""
        n = load().rlbm_edge_row_bytes(self.h, domain)
        if n == 0:
            raise RlbmError("bad domain %d" % domain)
        dt = getattr(self.torch, self._ROW_DTYPE[self.storage])
        return self.torch.empty((30, self.specs[domain].nx + 2), dtype=dt, device=self.workspace.device)

    def pack_edge_rows(self, domain, lo, hi):
        """Bottom row (planes 42..71) into `lo`, top row (planes 6..35) into
        `hi`; either may be None. Asynchronous on the handle's stream."""
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(load().rlbm_pack_edge_rows(self.h, domain, p(lo), p(hi)))

    def unpack_ghost_rows(self, domain, lo, hi):
        """Rows received from the slab below (`lo`) and above (`hi`) into the
        ghost rows y = -1 and y = ny; either may be None."""
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(load().rlbm_unpack_ghost_rows(self.h, domain, p(lo), p(hi)))

    def tune(self, repeats=3):
        """Autotune the step launch (grid shape) on the current state; returns the grid."""
        return _check(load().rlbm_tune(self.h, repeats))

    def select_kernel(self, kernel=-1):
        """Select the mixed step variant (RLBM_KERNEL_L1 or RLBM_KERNEL_TMA) or,
        with no argument, return the one in use."""
        return _check(load().rlbm_select_kernel(self.h, kernel))

    def set_grid(self, grid=0):
        """Persistent grid of `grid` blocks for the step kernel (0: one block per tile)."""
        return _check(load().rlbm_set_grid(self.h, int(grid)))

    def set_wait_limit(self, seconds=0.0):
        """Limit of the TMA-staged step's copy waits (0: the default one second)."""
        return _check(load().rlbm_set_wait_limit(self.h, float(seconds)))

    def sync_status(self):
        return _check(load().rlbm_sync_status(self.h))

    def last_step_info(self):
        u, k = ctypes.c_longlong(), ctypes.c_int()
        _check(load().rlbm_last_step_info(self.h, ctypes.byref(u), ctypes.byref(k)))
        return u.value, k.value

    def close(self):
        if self.h:
            load().rlbm_destroy(self.h)
            self.h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_noalloc(spec, edf, nsteps, f_in, f_out, stream=None, wait=True):
    """rlbm_step_noalloc: advance one FP64 domain (DomainSpec) by nsteps from the
    device checkpoint f_in into f_out (torch float64 [72][ny+2][nx+2] on the
    GPU) using the library's fixed scratch array. Returns this call's warning
    bits when wait is true (the call then waits for the stream), else None."""
    import torch
    shape = (72, spec.ny + 2, spec.nx + 2)
    for name, t in (("f_in", f_in), ("f_out", f_out)):
        # the copy kernels trust the pointers: a wrong size, type or device would
        # make them read or write outside the caller's buffer
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError("%s must be a float64 CUDA tensor" % name)
        if t.device.index != torch.cuda.current_device():
            raise ValueError("%s must be on the current CUDA device" % name)
        if tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError("%s must be a contiguous tensor of shape %s" % (name, shape))
    dom = make_domains([spec])
    s = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    w = ctypes.c_uint(0)
    _check(load().rlbm_step_noalloc(dom, edf, nsteps, ctypes.c_void_p(f_in.data_ptr()),
                                    ctypes.c_void_p(f_out.data_ptr()), s, ctypes.byref(w) if wait else None))
    return w.value if wait else None


def pipe_peaks():
    """Measured FP64 and FP32 FMA throughput of the current GPU (flop/s, FMA =
    2) and its SM count: the compute ceilings of the roofline."""
    f64, f32, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().rlbm_pipe_peaks(ctypes.byref(f64), ctypes.byref(f32), ctypes.byref(sms)))
    return {"fp64_flops": f64.value, "fp32_flops": f32.value, "sm_count": sms.value}


def status_string(code):
    return load().rlbm_status_string(code).decode()


def from_workload(wl, storage=RLBM_F64, **kw):
    """Create a Simulation for a workloads.Workload and initialise every domain."""
    edf = wl.domains[0].edf
    sim = Simulation(wl.domains, edf=edf, storage=storage, **kw)
    kinds = {s.kind for s in wl.init}
    if len(kinds) == 1:  # one call and one launch for every domain
        packed = [np.concatenate([np.asarray(getattr(s, k), dtype=np.float64).reshape(-1) for s in wl.init])
                  for k in ("a", "theta", "ux", "uy")]
        return sim, sim.init_all(kinds.pop(), *packed)
    st = 0
    for i, s in enumerate(wl.init):
        st |= sim.init(i, s)
    return sim, st
