"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/hgks.h. No compute call is made (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hgks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgks_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("hgks_mesh_create", "hgks_residual", "hgks_gmres_step", "hgks_solve_steady",
                     "hgks_mesh_destroy", "hgks_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _native.load()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_build_targets_sm103a_only():
    assert _native.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_defaults_and_error_plumbing_without_gpu():
    p = H.hgks_default_params()
    assert (p.krylov_dim, p.restarts, p.jacobi_sweeps) == (10, 3, 2)
    assert p.gamma == 1.4 and p.lin_weight == 0.025 and p.tau_eps == 0.1 and p.cfl == 10.0
    L = H.lib()
    # NULL arguments are rejected synchronously with a message, never a crash
    assert L.hgks_residual(None, C.byref(p), None, None, None, None, None) == 1
    assert b"NULL" in L.hgks_last_error()
    assert L.hgks_mesh_info(None, None) == 1
    out = C.c_void_p()
    st = L.hgks_mesh_create(None, 0, None, 0, None, None, 0, None, 0, 3, 0, C.byref(out), None)
    assert st in (1, 3)          # HGKS_ERR_ARG, or HGKS_ERR_CUDA where no device is visible
    assert out.value is None
    assert H.hgks_launch_count(reset=True) >= 0


def test_params_struct_matches_header():
    """The binding's struct mirrors the C layout (field order and sizes)."""
    src = open(os.path.join(ROOT, "include", "hgks.h")).read()
    body = src[src.index("typedef struct {\n  int32_t scheme;"):src.index("} hgks_params;")]
    ints = len(re.findall(r"int32_t ([a-z_]+);", body))
    assert ints == 10
    assert C.sizeof(H.hgks_params) == 10 * 4 + 21 * 8
    names = [f[0] for f in H.hgks_params._fields_]
    assert names[-4:] == ["Mach", "Re", "aoa_deg", "grad_relax"]
    p = H.hgks_default_params()
    assert p.Mach == 0.0 and p.Re == 0.0 and p.aoa_deg == 0.0 and p.grad_relax == 1.0


def test_batch_entry_points_reject_bad_arguments_without_gpu():
    L = H.lib()
    out = C.c_void_p()
    assert L.hgks_batch_create(None, None, 0, C.byref(out)) == 1
    assert out.value is None
    p = H.hgks_default_params()
    assert L.hgks_batch_create(None, C.byref(p), 1, C.byref(out)) == 1
    for fn, args in (("hgks_batch_residual", (None, None)), ("hgks_batch_gmres_step", (None, None, 1, None)),
                     ("hgks_batch_solve_steady", (None, 1e-8, 10, 1, None, None, None)),
                     ("hgks_batch_autotune", (None, None, None, None)), ("hgks_batch_info", (None, None)),
                     ("hgks_batch_destroy", (None,)), ("hgks_batch_set_state", (None, 0, None, None, None)),
                     ("hgks_batch_get_state", (None, 0, None, None, None, None, None))):
        assert getattr(L, fn)(*args) == 1, fn
        assert b"NULL" in L.hgks_last_error(), fn
    # hgks_batch_info_t: three int64 and three int32, padded to 8 bytes
    assert C.sizeof(H.hgks_batch_info_t) == 40


def test_server_and_dynamic_batch_entry_points_reject_bad_arguments_without_gpu():
    L = H.lib()
    out = C.c_void_p()
    assert L.hgks_server_create(0, 1 << 30, 4, None, 1, C.byref(out)) == 1
    assert L.hgks_batch_create_empty(0, 1024, 4096, 4, None, C.byref(out)) == 1
    for fn, args in (("hgks_server_destroy", (None,)), ("hgks_server_step", (None, None, None, None)),
                     ("hgks_server_status", (None, 1, None)), ("hgks_server_collect", (None, 1, None, None)),
                     ("hgks_server_info", (None, None)), ("hgks_server_cancel", (None, 1)),
                     ("hgks_batch_add", (None, None, None, None)),
                     ("hgks_batch_remove", (None, 0))):
        assert getattr(L, fn)(*args) == 1, fn
        assert b"NULL" in L.hgks_last_error(), fn
    # hgks_request_info: 2 int32, 1 int64, hgks_solve_info (24 bytes), 4 doubles
    assert C.sizeof(H.hgks_request_info) == 72
