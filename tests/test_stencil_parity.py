"""The library's non-compact stencils (csrc/mesh_setup.cpp, run on the CPU
through the test-only shim tests/host_setup/hs_shim.cpp) are the oracle's, cell
for cell and in the same order: the big stencil of Sec. 3.2 with its rings
beyond the second (boundary cells, and cells whose quadratic fit would be
singular on a regular grid), and the sub-stencils in use. Index work, so
compared exactly. CPU only."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2304_09485_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not found")
    out = str(tmp_path_factory.mktemp("hs") / "libhs.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                           "-I" + CUDA_INC, os.path.join(ROOT, "tests", "host_setup", "hs_shim.cpp"),
                           os.path.join(ROOT, "paper_2304_09485_gb300", "csrc", "mesh_setup.cpp"), "-o", out, "-ldl"])
    L = C.CDLL(out)
    L.hs_error.restype = C.c_char_p
    return L


def library_stencils(L, m):
    hexa = hasattr(m, "hex8")
    cells = np.ascontiguousarray(m.hex8 if hexa else m.tet4, dtype=np.int64)
    xyz = np.ascontiguousarray(m.xyz, dtype=np.float64)
    bf = np.ascontiguousarray(m.bface4 if hexa else m.bface3, dtype=np.int64)
    bt = np.ascontiguousarray(m.btag, dtype=np.int32)
    ps = np.ascontiguousarray(m.periodic_shift if m.periodic_shift is not None else np.zeros((0, 3)), dtype=np.float64)
    sizes = np.zeros(3, dtype=np.int64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = L.hs_build_cells(p(xyz), C.c_int64(len(xyz)), p(cells), C.c_int32(cells.shape[1]), C.c_int64(len(cells)),
                          p(bf), p(bt), C.c_int64(len(bt)), p(ps), C.c_int32(len(ps)), C.c_int(1), p(sizes))
    assert rc == 0, L.hs_error()
    N, BIG, NSUB, SUBK, BITS = len(cells), (24 if hexa else 16), (8 if hexa else 4), (3 if hexa else 6), (8 if hexa else 4)

    def get(name, dtype, rows):
        a = np.empty(rows * N, dtype=dtype)
        assert L.hs_get(name.encode(), a.ctypes.data_as(C.c_void_p), C.c_int64(a.nbytes)) == 0, name
        return a.reshape(rows, N)
    perm = get("perm", np.int64, 1)[0]
    sten, ssl, valid = get("sten", np.int32, BIG), get("ssl", np.uint32, NSUB), get("subvalid", np.uint8, 1)[0]
    big, subs = {}, {}
    for i in range(N):
        c = perm[i]
        big[c] = [int(perm[k]) for k in sten[:, i] if k >= 0]
        for mm in range(NSUB):
            if (valid[i] >> mm) & 1:
                slots = [(int(ssl[mm, i]) >> (BITS * s)) & ((1 << BITS) - 1) for s in range(SUBK)]
                # members in ascending slot order, then unused entries padded with slot 0
                used = slots[:1]
                for s in slots[1:]:
                    if s <= used[-1]:
                        break
                    used.append(s)
                subs[c, mm] = sorted(big[c][s] for s in used)
    return big, subs, NSUB


MESHES = {
    "regular cavity": lambda: I.cavity_mesh(5, jitter=0.0),
    "regular wall-clustered cavity": lambda: I.cavity_mesh(5, jitter=0.0, h_min=0.05),
    "jittered cavity": lambda: I.cavity_mesh(5),
    "regular periodic cube": lambda: I.periodic_cube_mesh(4, jitter=0.0),
    "sphere": lambda: I.sphere_mesh(4, 5, stretch=1.3),
    "regular hexahedral cavity": lambda: I.hex_cavity_mesh(4, jitter=0.0),
    "jittered hexahedral cavity": lambda: I.hex_cavity_mesh(4),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_stencils_equal_the_oracle(shim, name):
    m = MESHES[name]()
    big, subs, nsub = library_stencils(shim, m)
    om = O.OracleMesh(m)
    n = m.n_cells if hasattr(m, "hex8") else m.n_tet
    cond = I.cavity_conditions()
    om.residual(O.make_params(scheme=0, **cond), I.state_from_conditions(n, cond))
    for c in range(n):
        ob, _ = om.stencil(c)
        assert big[c] == ob.tolist(), (name, c)
        for mm in range(nsub):
            cells, ok = om.stencil(c, mm)
            assert ((c, mm) in subs) == ok, (name, c, mm)
            if ok:
                assert subs[c, mm] == sorted(cells.tolist()), (name, c, mm)
