"""Host-side checks of the C ABI: the library builds for sm_103a, loads without a
GPU and exports every entry point that include/rlbm.h declares; the Python
binding mirrors the declared names and struct layouts. No compute calls."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(rlbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1709_09073_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["rlbm_create", "rlbm_init", "rlbm_step", "rlbm_moments", "rlbm_destroy",
              "rlbm_workspace_bytes", "rlbm_status_string", "rlbm_sync_status"]:
        assert n in names, n


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, missing


def test_library_loads_without_gpu(lib_path):
    from paper_1709_09073_gb300 import rlbm
    L = rlbm.load(lib_path)
    for n in declared_functions():
        assert hasattr(L, n), n
    assert set(rlbm.EXPORTS) <= declared_functions()
    # pure host calls: status strings and workspace sizing do not touch the GPU
    assert L.rlbm_status_string(0) == b"ok"
    assert b"argument" in L.rlbm_status_string(-1)
    # slab rows: a null handle is refused on the host
    assert L.rlbm_edge_row_bytes(None, 0) == 0
    assert L.rlbm_pack_edge_rows(None, 0, None, None) == -1
    assert L.rlbm_unpack_ghost_rows(None, 0, None, None) == -1


def test_workspace_sizing_and_validation(lib_path):
    from paper_1709_09073_gb300 import rlbm, workloads as W
    rlbm.load(lib_path)
    spec = [W.DomainSpec(64, 64, 0.9)]
    b64 = rlbm.rlbm_workspace_bytes(spec, rlbm.RLBM_MJ, rlbm.RLBM_F64)
    # two halo-padded FP64 copies: at least 2 * 72 * 66 * 66 * 8 bytes
    assert b64 >= 2 * 72 * 66 * 66 * 8
    assert b64 % 256 == 0
    # invalid: periodic on one side only, bad tau, unsupported order
    bad = [W.DomainSpec(8, 8, 0.9, bc=(0, 1, 0, 0))]
    assert rlbm.rlbm_workspace_bytes(bad, rlbm.RLBM_MJ, rlbm.RLBM_F64) == 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(8, 8, -1.0)], 0, 0) == 0
    # orders 2..5 with FP64 storage; the mixed storages carry the fifth order only
    assert rlbm.rlbm_workspace_bytes(spec, 0, 0, order=3) > 0
    assert rlbm.rlbm_workspace_bytes(spec, 0, 0, order=1) == 0
    assert rlbm.rlbm_workspace_bytes(spec, 0, 0, order=6) == 0
    assert rlbm.rlbm_workspace_bytes(spec, 0, rlbm.RLBM_F32DEV, order=3) == 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(8, 8, 0.9, eta_s=-1.0)], 0, 0) == 0
    # velocity walls and body forces: FP64 storage, one wall temperature, a wall density
    vw = (W.PERIODIC, W.PERIODIC, W.VELOCITY_WALL, W.VELOCITY_WALL)
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(4, 8, 3.0, bc=vw, accel=(1e-8, 0.0))], 0, 0) > 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(4, 8, 3.0, bc=vw)], 0, rlbm.RLBM_F32DEV) == 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(4, 8, 3.0, accel=(1e-8, 0.0))], 0, rlbm.RLBM_F32DEV) == 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(4, 8, 3.0, bc=vw, t_wall=(1, 1, 1.0, 1.1))], 0, 0) == 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(4, 8, 3.0, bc=vw, n_wall=0.0)], 0, 0) == 0
    # exchanged sides (a y-slab's faces): y sides only, never paired with a periodic side
    ex = (W.PERIODIC, W.PERIODIC, W.EXCHANGED, W.FIXED_T_WALL)
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(8, 4, 0.9, bc=ex, t_wall=(1, 1, 1, 1.02))], 0, 0) > 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(8, 4, 0.9, bc=(W.EXCHANGED, 1, 0, 0))], 0, 0) == 0
    assert rlbm.rlbm_workspace_bytes([W.DomainSpec(8, 4, 0.9, bc=(0, 0, W.EXCHANGED, 0))], 0, 0) == 0


def test_struct_layout_matches_header():
    from paper_1709_09073_gb300 import rlbm
    # rlbm_domain: 2 int + double + 4 int + 4 double + 7 double
    assert ctypes.sizeof(rlbm.rlbm_domain) == 8 + 8 + 16 + 32 + 56
    assert ctypes.sizeof(rlbm.rlbm_config) == 8 + 8 + 12 + 4 + 8 + 8 + 8
