"""The library's host-side mesh construction (csrc/mesh_setup.cpp), run on the
CPU through a test-only shim (tests/host_setup/hs_shim.cpp): cell order, face
table, stencils and the reconstruction fits of Sec. 3.1 - 3.3, checked against
closed forms and exact polynomial reproduction (not against the oracle)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_2304_09485_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_09485_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not found")
    out = str(tmp_path_factory.mktemp("hs") / "libhs.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                           "-I" + CUDA_INC, os.path.join(ROOT, "tests", "host_setup", "hs_shim.cpp"),
                           os.path.join(CSRC, "mesh_setup.cpp"), "-o", out, "-ldl"])
    L = C.CDLL(out)
    L.hs_error.restype = C.c_char_p
    L.hs_get.argtypes = [C.c_char_p, C.c_void_p, C.c_int64]
    return L


class Built:
    def __init__(self, L, m, mask=3):
        xyz = np.ascontiguousarray(m.xyz, dtype=np.float64)
        tet = np.ascontiguousarray(m.tet4, dtype=np.int64)
        bf = np.ascontiguousarray(m.bface3, dtype=np.int64).reshape(-1, 3)
        bt = np.ascontiguousarray(m.btag, dtype=np.int32)
        ps = m.periodic_shift
        psa = np.ascontiguousarray(ps if ps is not None else np.zeros((0, 3)), dtype=np.float64)
        sizes = np.zeros(3, dtype=np.int64)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        rc = L.hs_build(p(xyz), C.c_int64(len(xyz)), p(tet), C.c_int64(len(tet)), p(bf), p(bt), C.c_int64(len(bt)),
                        p(psa), C.c_int32(len(psa)), C.c_int(mask), p(sizes))
        assert rc == 0, L.hs_error()
        self.L, self.N, self.F, self.Fb = L, int(sizes[0]), int(sizes[1]), int(sizes[2])

    def get(self, name, dtype, rows=1, per="N"):
        n = rows * (self.N if per == "N" else self.F)
        a = np.empty(n, dtype=dtype)
        assert self.L.hs_get(name.encode(), a.ctypes.data_as(C.c_void_p), a.nbytes) == 0, name
        return a.reshape(rows, -1) if rows > 1 else a


def geometry(m):
    V = m.xyz[m.tet4]
    vol = np.abs(np.einsum("ij,ij->i", V[:, 1] - V[:, 0], np.cross(V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]))) / 6
    return vol, V.mean(1)


def tet_average_quadratic(xyz, tet, f):
    """Exact cell average of a quadratic: -1/20 sum over vertices + 1/5 sum over edge midpoints."""
    V = xyz[tet]
    vs = sum(f(V[:, a]) for a in range(4))
    es = sum(f(0.5 * (V[:, a] + V[:, b])) for a in range(4) for b in range(a + 1, 4))
    return -vs / 20 + es / 5


@pytest.mark.parametrize("kind", ["cavity", "periodic"])
def test_cell_order_and_face_table(shim, kind):
    m = I.cavity_mesh(3) if kind == "cavity" else I.periodic_cube_mesh(3)
    b = Built(shim, m)
    N, F = b.N, b.F
    perm = b.get("perm", np.int64)
    assert N == m.n_tet and np.array_equal(np.sort(perm), np.arange(N))
    vol, cen = geometry(m)
    np.testing.assert_allclose(b.get("vol", np.float64), vol[perm], rtol=1e-13)
    np.testing.assert_allclose(b.get("h", np.float64), np.cbrt(vol[perm]), rtol=1e-13)
    assert b.Fb == len(m.btag) and 2 * F == 4 * N + b.Fb
    fl, fr = b.get("fl", np.int32, per="F"), b.get("fr", np.int32, per="F")
    cnb, cface = b.get("cnb", np.int32, 4), b.get("cface", np.int32, 4)
    fT, fS = b.get("fT", np.float64, 9, per="F"), b.get("fS", np.float64, per="F")
    assert np.all(fl >= 0) and int((fr < 0).sum()) == b.Fb
    assert np.all(fl[fr >= 0] < fr[fr >= 0])                 # left is the lower cell
    # every (cell, slot) names its face and side; neighbours are mutual
    area_vec = np.zeros((N, 3))
    for p_ in range(4):
        f, side = cface[p_] >> 1, cface[p_] & 1
        owner = np.where(side == 0, fl[f], fr[f])
        other = np.where(side == 0, fr[f], fl[f])
        assert np.array_equal(owner, np.arange(N))
        assert np.array_equal(cnb[p_], other)
        sgn = np.where(side == 0, 1.0, -1.0)
        area_vec += (sgn * fS[f])[:, None] * fT[0:3, f].T
    for i in range(N):
        for j in cnb[:, i]:
            if j >= 0:
                assert i in cnb[:, j]
    # closed cells: the outward area vectors of each tetrahedron sum to zero
    assert np.abs(area_vec).max() <= 1e-14 * fS.max() * 10
    # face frames are orthonormal
    Tm = fT.T.reshape(F, 3, 3)
    np.testing.assert_allclose(np.einsum("fij,fkj->fik", Tm, Tm), np.broadcast_to(np.eye(3), (F, 3, 3)), atol=1e-13)
    if kind == "cavity":
        assert fS[fr < 0].sum() == pytest.approx(6.0, rel=1e-12)       # surface of the unit cube
    # the space-filling-curve order keeps neighbours close in memory
    dist = np.abs(cnb - np.arange(N)[None, :])[cnb >= 0]
    assert dist.mean() < 0.2 * N


def _quadratic(rng):
    g = rng.normal(size=3)
    Hq = rng.normal(size=(3, 3))
    Hq = Hq + Hq.T
    c0 = 1.3
    f = lambda X: c0 + X @ g + 0.5 * np.einsum("...i,ij,...j->...", X, Hq, X)
    grad = lambda X: g + X @ Hq
    return f, grad, Hq


def _scaled_coefficients(grad_c, Hq, h):
    """Coefficients of (x, y, z, x^2, y^2, z^2, xy, xz, yz) in the frame (x - centroid) / h."""
    a = np.zeros((len(h), 9))
    a[:, 0:3] = h[:, None] * grad_c
    for j in range(3):
        a[:, 3 + j] = 0.5 * h ** 2 * Hq[j, j]
    a[:, 6], a[:, 7], a[:, 8] = h ** 2 * Hq[0, 1], h ** 2 * Hq[0, 2], h ** 2 * Hq[1, 2]
    return a


@pytest.mark.parametrize("jitter", [0.1, 0.0])
def test_non_compact_fits_reproduce_quadratics_and_linear_fields(shim, jitter):
    """Eq. (polys): the big-stencil least squares returns a quadratic's coefficients
    exactly; every sub-stencil fit in use returns a linear field's gradient. Also on
    the regular grid (no jitter), whose boundary cells need more than two rings
    for a determined quadratic fit."""
    m = I.cavity_mesh(4, jitter=jitter)
    b = Built(shim, m, mask=1)
    N = b.N
    perm = b.get("perm", np.int64)
    _, cen = geometry(m)
    cen = cen[perm]
    h = b.get("h", np.float64)
    sten, X0 = b.get("sten", np.int32, 16), b.get("X0", np.float64, 9 * 16)
    rng = np.random.default_rng(3)
    f, grad, Hq = _quadratic(rng)
    Q = tet_average_quadratic(m.xyz, m.tet4, lambda X: f(X)[..., None])[:, 0][perm]
    dQ = np.where(sten >= 0, Q[np.maximum(sten, 0)] - Q[None, :], 0.0)        # [16, N]
    a = np.einsum("dkn,kn->nd", X0.reshape(9, 16, N), dQ)
    ref = _scaled_coefficients(grad(cen), Hq, h)
    # rounding, amplified by the conditioning of the wall cells' stencils; a wrong fit is off by O(h^2)
    np.testing.assert_allclose(a, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    # sub-stencils on a linear field
    gl = rng.normal(size=3)
    Ql = tet_average_quadratic(m.xyz, m.tet4, lambda X: (0.7 + X @ gl)[..., None])[:, 0][perm]
    Xs, ssl, valid = b.get("Xs", np.float64, 4 * 3 * 6), b.get("ssl", np.uint32, 4), b.get("subvalid", np.uint8)
    Xs = Xs.reshape(4, 3, 6, N)
    used = 0
    for mm in range(4):
        slots = np.stack([(ssl[mm] >> (4 * s)) & 15 for s in range(6)]).astype(np.int64)    # [6, N]
        cells = sten[slots, np.arange(N)[None, :]]
        d = np.where(cells >= 0, Ql[np.maximum(cells, 0)] - Ql[None, :], 0.0)
        bm = np.einsum("jsn,sn->nj", Xs[mm], d)
        ok = (valid >> mm) & 1 == 1
        used += int(ok.sum())
        np.testing.assert_allclose(bm[ok], (h[:, None] * gl[None, :])[ok], rtol=1e-10, atol=1e-12)
    assert used >= 3 * N                     # most sub-stencils are in use


def test_compact_fits_reproduce_quadratics_and_linear_fields(shim):
    """Eq. (compact-big-1): with exact cell averages and exact cell-averaged gradients
    the constrained least squares returns a quadratic's coefficients (cells with at
    least three face neighbours); Eq. (compact-big-2): every sub-stencil returns a
    linear field's gradient."""
    m = I.cavity_mesh(4)
    b = Built(shim, m, mask=2)
    N = b.N
    perm = b.get("perm", np.int64)
    _, cen = geometry(m)
    cen = cen[perm]
    h = b.get("h", np.float64)
    cnb = b.get("cnb", np.int32, 4)
    H0, Hm = b.get("H0", np.float64, 9 * 19).reshape(9, 19, N), b.get("Hm", np.float64, 4 * 3 * 7).reshape(4, 3, 7, N)
    rng = np.random.default_rng(5)
    f, grad, Hq = _quadratic(rng)
    Q = tet_average_quadratic(m.xyz, m.tet4, lambda X: f(X)[..., None])[:, 0][perm]
    G = grad(cen)                                              # cell-averaged gradient = gradient at the centroid
    has = cnb >= 0
    data = np.zeros((19, N))
    data[0:4] = np.where(has, Q[np.maximum(cnb, 0)] - Q[None, :], 0.0)
    data[4:7] = G.T
    for p_ in range(4):
        data[7 + 3 * p_:10 + 3 * p_] = np.where(has[p_][None, :], G[np.maximum(cnb[p_], 0)].T, 0.0)
    a = np.einsum("dcn,cn->nd", H0, data)
    full = has.sum(0) >= 3
    assert full.mean() > 0.9
    ref = _scaled_coefficients(grad(cen), Hq, h)[full]
    np.testing.assert_allclose(a[full], ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    gl = rng.normal(size=3)
    Ql = tet_average_quadratic(m.xyz, m.tet4, lambda X: (0.7 + X @ gl)[..., None])[:, 0][perm]
    for mm in range(4):
        d = np.zeros((7, N))
        d[0] = np.where(has[mm], Ql[np.maximum(cnb[mm], 0)] - Ql, 0.0)
        d[1:4] = gl[:, None]
        d[4:7] = np.where(has[mm][None, :], gl[:, None], 0.0)
        bm = np.einsum("jcn,cn->nj", Hm[mm], d)
        np.testing.assert_allclose(bm, h[:, None] * gl[None, :], rtol=1e-10, atol=1e-12)


def test_stencils_gauss_points_and_face_geometry(shim):
    """Sec. 3.1 stencils as the paper builds them (big stencil: face neighbours and
    their neighbours; sub-stencil m: the three face neighbours of its triple and the
    three other neighbours of face neighbour m), the face Gauss points (barycentric
    2/3, 1/6, 1/6 on the face shared with the slot's neighbour), normals from the
    left to the right cell, and the distances used by the viscous spectral radius."""
    m = I.cavity_mesh(4)
    b = Built(shim, m, mask=1)
    N, F = b.N, b.F
    perm = b.get("perm", np.int64)
    _, cen_c = geometry(m)
    cen = cen_c[perm]
    h = b.get("h", np.float64)
    cnb, cface = b.get("cnb", np.int32, 4), b.get("cface", np.int32, 4)
    sten, ssl, valid = b.get("sten", np.int32, 16), b.get("ssl", np.uint32, 4), b.get("subvalid", np.uint8)
    xg = b.get("xg", np.float64, 36).reshape(4, 3, 3, N)
    fT, fl, fr, fdist = (b.get("fT", np.float64, 9, per="F"), b.get("fl", np.int32, per="F"),
                         b.get("fr", np.int32, per="F"), b.get("fdist", np.float64, per="F"))
    TRIPLES = [(0, 1, 2), (0, 1, 3), (1, 2, 3), (2, 0, 3)]
    tets = m.tet4[perm]
    checked_big = checked_sub = 0
    for i in range(N):
        l1 = [int(j) for j in cnb[:, i] if j >= 0]
        ring = list(dict.fromkeys(l1 + [int(k) for j in l1 for k in cnb[:, j] if k >= 0 and k != i]))
        got = [int(k) for k in sten[:, i] if k >= 0]
        if len(ring) >= 12:
            assert got == ring, i                          # the same cells, in the same order
            checked_big += 1
        for mm in range(4):
            if not (valid[i] >> mm) & 1:
                continue
            want = [int(cnb[t, i]) for t in TRIPLES[mm] if cnb[t, i] >= 0]
            if cnb[mm, i] >= 0:
                want += [int(k) for k in cnb[:, cnb[mm, i]] if k >= 0 and k != i]
            want = set(want)
            slots = sorted(got.index(c) for c in want)
            dec = [int((ssl[mm, i] >> (4 * s)) & 15) for s in range(len(slots))]
            assert dec == slots, (i, mm)
            checked_sub += 1
        # Gauss points: on the face shared with the slot's neighbour, barycentric (2/3, 1/6, 1/6)
        Vt = m.xyz[tets[i]]
        Bm = np.vstack([Vt.T, np.ones(4)])
        for p_ in range(4):
            X = cen[i][None, :] + h[i] * xg[p_, :, :, i]                         # [3 points, 3]
            lam = np.linalg.solve(Bm, np.vstack([X.T, np.ones(3)]))            # [4 vertices, 3 points]
            zero = np.abs(lam).max(1) < 1e-12
            assert zero.sum() == 1
            np.testing.assert_allclose(np.sort(lam[~zero], axis=0), np.array([[1 / 6] * 3, [1 / 6] * 3, [2 / 3] * 3]),
                                       atol=1e-12)
            if cnb[p_, i] >= 0:                           # the vertex off the face is not in the neighbour
                assert tets[i][np.argmax(zero)] not in tets[cnb[p_, i]]
    assert checked_big > N // 2 and checked_sub > 2 * N
    # normals from left to right; distances between centroids (inside) or twice the wall distance
    inner = fr >= 0
    d = cen[fr[inner]] - cen[fl[inner]]
    assert np.all(np.einsum("ij,ji->i", d, fT[0:3, inner]) > 0)
    np.testing.assert_allclose(fdist[inner], np.linalg.norm(d, axis=1), rtol=1e-13)
    for f in np.where(~inner)[0][:50]:
        L = fl[f]
        p_ = int(np.where(cface[:, L] >> 1 == f)[0][0])
        fc = cen[L] + h[L] * xg[p_, :, :, L].mean(0)
        assert fdist[f] == pytest.approx(2 * abs((fc - cen[L]) @ fT[0:3, f]), rel=1e-12)


# ---------------------------------------------------------------------------
# hexahedral meshes (Sec. 3.1: six faces, eight corner sub-stencils)
# ---------------------------------------------------------------------------

HEX_CORNER = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
HEX_FACES = [[0, 1, 2, 3], [0, 1, 5, 4], [1, 2, 6, 5], [2, 3, 7, 6], [3, 0, 4, 7], [4, 5, 6, 7]]


class BuiltHex(Built):
    def __init__(self, L, m, mask=3):
        xyz = np.ascontiguousarray(m.xyz, dtype=np.float64)
        hx = np.ascontiguousarray(m.hex8, dtype=np.int64)
        bf = np.ascontiguousarray(m.bface4, dtype=np.int64).reshape(-1, 4)
        bt = np.ascontiguousarray(m.btag, dtype=np.int32)
        ps = m.periodic_shift
        psa = np.ascontiguousarray(ps if ps is not None else np.zeros((0, 3)), dtype=np.float64)
        sizes = np.zeros(3, dtype=np.int64)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        rc = L.hs_build_cells(p(xyz), C.c_int64(len(xyz)), p(hx), C.c_int32(8), C.c_int64(len(hx)), p(bf), p(bt),
                              C.c_int64(len(bt)), p(psa), C.c_int32(len(psa)), C.c_int(mask), p(sizes))
        assert rc == 0, L.hs_error()
        self.L, self.N, self.F, self.Fb = L, int(sizes[0]), int(sizes[1]), int(sizes[2])


def hex_average(V, f, order=5):
    """Cell averages of f and volumes of hexahedra V [n, 8, 3] by a tensor Gauss rule of the trilinear map."""
    t, w = np.polynomial.legendre.leggauss(order)
    t, w = 0.5 * (t + 1), 0.5 * w
    acc, vol = 0.0, 0.0
    sg = np.where(HEX_CORNER == 1, 1.0, -1.0)
    for a, wa in zip(t, w):
        for b, wb in zip(t, w):
            for c, wc in zip(t, w):
                r = np.array([a, b, c])
                fr = np.where(HEX_CORNER == 1, r, 1 - r)
                N = fr.prod(1)
                dN = np.stack([sg[:, e] * np.prod(np.delete(fr, e, axis=1), axis=1) for e in range(3)], 1)
                X = np.einsum("a,nad->nd", N, V)
                dj = np.linalg.det(np.einsum("ae,nad->nde", dN, V)) * wa * wb * wc
                acc = acc + dj[:, None] * f(X)
                vol = vol + dj
    return acc / vol[:, None], vol


def test_hex_cell_order_and_face_table(shim):
    m = I.hex_cavity_mesh(4, jitter=0.15)
    b = BuiltHex(shim, m)
    N, F = b.N, b.F
    perm = b.get("perm", np.int64)
    assert N == m.n_cells and np.array_equal(np.sort(perm), np.arange(N))
    cen, vol = hex_average(m.xyz[m.hex8], lambda X: X)
    np.testing.assert_allclose(b.get("vol", np.float64), vol[perm], rtol=1e-13)
    assert b.Fb == len(m.btag) and 2 * F == 6 * N + b.Fb
    cnb, cface = b.get("cnb", np.int32, 6), b.get("cface", np.int32, 6)
    fl, fr = b.get("fl", np.int32, per="F"), b.get("fr", np.int32, per="F")
    fT, fS, fw = b.get("fT", np.float64, 9, per="F"), b.get("fS", np.float64, per="F"), b.get("fw", np.float64, 4, per="F")
    area_vec = np.zeros((N, 3))
    for p_ in range(6):
        f, side = cface[p_] >> 1, cface[p_] & 1
        assert np.array_equal(np.where(side == 0, fl[f], fr[f]), np.arange(N))
        assert np.array_equal(cnb[p_], np.where(side == 0, fr[f], fl[f]))
        area_vec += (np.where(side == 0, 1.0, -1.0) * fS[f])[:, None] * fT[0:3, f].T
    assert np.abs(area_vec).max() <= 1e-15
    np.testing.assert_allclose(fw.sum(0), 1.0, rtol=0, atol=1e-15)
    assert fS[fr < 0].sum() == pytest.approx(6.0, rel=1e-12)
    inner = fr >= 0
    d = cen[perm][fr[inner]] - cen[perm][fl[inner]]
    assert np.all(np.einsum("ij,ji->i", d, fT[0:3, inner]) > 0)


def test_hex_stencils_and_gauss_points(shim):
    """Undistorted grid: an interior cell's big stencil holds its face neighbours and
    theirs (24 cells), and its eight sub-stencils are the face-neighbour triples
    across the cell's eight corners; Gauss points lie at the 2 x 2 points of the
    bilinear face with the slot's neighbour, the same points seen from both sides."""
    n = 5
    m = I.hex_cavity_mesh(n, jitter=0.0)
    b = BuiltHex(shim, m, mask=1)
    N = b.N
    perm = b.get("perm", np.int64)
    cen = hex_average(m.xyz[m.hex8], lambda X: X)[0][perm]
    hh = 1.0 / n
    sten, ssl, valid = b.get("sten", np.int32, 24), b.get("ssl", np.uint32, 8), b.get("subvalid", np.uint8)
    c = int(np.where(np.all((cen > 2 * hh) & (cen < 1 - 2 * hh), axis=1))[0][0])
    got = [int(k) for k in sten[:, c] if k >= 0]
    assert len(got) == 24
    off = {tuple(np.rint((cen[k] - cen[c]) / hh).astype(int)) for k in got}
    assert all(sum(abs(x) for x in o) in (1, 2) for o in off) and len(off) == 24
    assert valid[c] == 0xFF
    signs = set()
    for mm in range(8):
        cells = [got[(int(ssl[mm, c]) >> (8 * s)) & 255] for s in range(3)]
        o = np.rint((cen[cells] - cen[c]) / hh).astype(int)
        assert sorted(np.abs(o).sum(1)) == [1, 1, 1] and np.abs(o.sum(0)).tolist() == [1, 1, 1]
        signs.add(tuple(o.sum(0)))
    assert len(signs) == 8
    # Gauss points, jittered mesh
    mj = I.hex_cavity_mesh(3, jitter=0.15)
    bj = BuiltHex(shim, mj, mask=1)
    permj = bj.get("perm", np.int64)
    cenj = hex_average(mj.xyz[mj.hex8], lambda X: X)[0][permj]
    hj = bj.get("h", np.float64)
    xg = bj.get("xg", np.float64, 72).reshape(6, 4, 3, bj.N)
    cnb, cface = bj.get("cnb", np.int32, 6), bj.get("cface", np.int32, 6)
    hexes = mj.hex8[permj]
    gl, gh = 0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)
    for i in range(bj.N):
        for p_ in range(6):
            X = cenj[i] + hj[i] * xg[p_, :, :, i]                   # [4 points, 3]
            # the face: the quadrilateral of this cell whose bilinear 2 x 2 points are X
            hit = 0
            for F_ in HEX_FACES:
                P = mj.xyz[hexes[i][F_]]
                pts = np.array([(1 - s) * (1 - t) * P[0] + s * (1 - t) * P[1] + s * t * P[2] + (1 - s) * t * P[3]
                                for s, t in ((gl, gl), (gh, gl), (gh, gh), (gl, gh))])
                dist = np.linalg.norm(pts[:, None, :] - X[None, :, :], axis=2)
                if np.all(dist.min(0) < 1e-12) and np.all(dist.min(1) < 1e-12):
                    hit += 1
                    if cnb[p_, i] >= 0:                                # shared with the slot's neighbour
                        assert set(hexes[i][F_]) <= set(hexes[cnb[p_, i]])
            assert hit == 1, (i, p_)


def test_hex_fits_reproduce_quadratics_and_linear_fields(shim):
    """Non-compact and compact fits on jittered hexahedra: exact coefficients of a
    quadratic (cells with >= 3 face neighbours for the compact one), exact gradients
    of a linear field for every sub-stencil in use."""
    m = I.hex_cavity_mesh(5, jitter=0.15)
    b = BuiltHex(shim, m, mask=3)
    N = b.N
    perm = b.get("perm", np.int64)
    h = b.get("h", np.float64)
    rng = np.random.default_rng(7)
    f, grad, Hq = _quadratic(rng)
    Qc, _ = hex_average(m.xyz[m.hex8], lambda X: f(X)[..., None])
    Q = Qc[:, 0][perm]
    cen = hex_average(m.xyz[m.hex8], lambda X: X)[0][perm]
    ref = _scaled_coefficients(grad(cen), Hq, h)
    sten, X0 = b.get("sten", np.int32, 24), b.get("X0", np.float64, 9 * 24)
    dQ = np.where(sten >= 0, Q[np.maximum(sten, 0)] - Q[None, :], 0.0)
    a = np.einsum("dkn,kn->nd", X0.reshape(9, 24, N), dQ)
    np.testing.assert_allclose(a, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    gl = rng.normal(size=3)
    Ql = hex_average(m.xyz[m.hex8], lambda X: (0.7 + X @ gl)[..., None])[0][:, 0][perm]
    Xs, ssl, valid = b.get("Xs", np.float64, 8 * 3 * 3).reshape(8, 3, 3, N), b.get("ssl", np.uint32, 8), b.get("subvalid", np.uint8)
    used = 0
    for mm in range(8):
        slots = np.stack([(ssl[mm] >> (8 * s)) & 255 for s in range(3)]).astype(np.int64)
        cells = sten[slots, np.arange(N)[None, :]]
        d = np.where(cells >= 0, Ql[np.maximum(cells, 0)] - Ql[None, :], 0.0)
        bm = np.einsum("jsn,sn->nj", Xs[mm], d)
        ok = (valid >> mm) & 1 == 1
        used += int(ok.sum())
        np.testing.assert_allclose(bm[ok], (h[:, None] * gl[None, :])[ok], rtol=1e-10, atol=1e-12)
    assert used >= 3 * N
    # compact: data = (dQ of slots 0..5, G_i, G of slots 0..5)
    cnb = b.get("cnb", np.int32, 6)
    H0, Hm = b.get("H0", np.float64, 9 * 27).reshape(9, 27, N), b.get("Hm", np.float64, 6 * 3 * 7).reshape(6, 3, 7, N)
    G = grad(cen)
    has = cnb >= 0
    data = np.zeros((27, N))
    data[0:6] = np.where(has, Q[np.maximum(cnb, 0)] - Q[None, :], 0.0)
    data[6:9] = G.T
    for p_ in range(6):
        data[9 + 3 * p_:12 + 3 * p_] = np.where(has[p_][None, :], G[np.maximum(cnb[p_], 0)].T, 0.0)
    a = np.einsum("dcn,cn->nd", H0, data)
    full = has.sum(0) >= 3
    np.testing.assert_allclose(a[full], ref[full], rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    for mm in range(6):
        d = np.zeros((7, N))
        d[0] = np.where(has[mm], Ql[np.maximum(cnb[mm], 0)] - Ql, 0.0)
        d[1:4] = gl[:, None]
        d[4:7] = np.where(has[mm][None, :], gl[:, None], 0.0)
        np.testing.assert_allclose(np.einsum("jcn,cn->nj", Hm[mm], d), h[:, None] * gl[None, :], rtol=1e-10, atol=1e-12)


def _build_raw(L, xyz, cells, bface, btag, pshift=None, mask=3):
    """hs_build_cells on raw arrays: (status, message)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    bface = np.ascontiguousarray(bface, dtype=np.int64)
    btag = np.ascontiguousarray(btag, dtype=np.int32)
    psa = np.ascontiguousarray(pshift if pshift is not None else np.zeros((0, 3)), dtype=np.float64)
    sizes = np.zeros(3, dtype=np.int64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = L.hs_build_cells(p(xyz), C.c_int64(len(xyz)), p(cells), C.c_int32(cells.shape[1]), C.c_int64(len(cells)),
                          p(bface), p(btag), C.c_int64(len(btag)), p(psa), C.c_int32(len(psa)), C.c_int(mask), p(sizes))
    return rc, L.hs_error().decode()


def test_invalid_meshes_are_refused(shim):
    """Meshes the scheme cannot run on are refused by the host set-up with
    HGKS_ERR_MESH (2) or HGKS_ERR_ARG (1) and a message naming the fault: an
    empty mesh, an inverted or flat cell, a vertex index out of range, a face
    of three cells, a face that is neither shared, tagged nor periodic, an
    unknown tag, and a non-compact stencil with fewer than the 9 cells the
    quadratic fit needs."""
    ERR_ARG, ERR_MESH = 1, 2
    hexm = I.hex_cavity_mesh(3, jitter=0.1)
    good = (hexm.xyz, hexm.hex8, hexm.bface4, hexm.btag)
    assert _build_raw(shim, *good)[0] == 0
    # top and bottom quadrilaterals swapped: the trilinear map has detJ < 0
    inv = hexm.hex8.copy()
    inv[5] = inv[5][[4, 5, 6, 7, 0, 1, 2, 3]]
    rc, msg = _build_raw(shim, hexm.xyz, inv, hexm.bface4, hexm.btag)
    assert rc == ERR_MESH and "hexahedron 5" in msg
    # a vertex index past the vertex array
    bad = hexm.hex8.copy()
    bad[2, 3] = len(hexm.xyz)
    rc, msg = _build_raw(shim, hexm.xyz, bad, hexm.bface4, hexm.btag)
    assert rc == ERR_MESH and "out of range" in msg
    # cells of a kind the library does not have
    rc, msg = _build_raw(shim, hexm.xyz, hexm.hex8[:, :5], hexm.bface4, hexm.btag)
    assert rc == ERR_ARG and "4 or 8" in msg
    # one boundary quadrilateral dropped, no periodic shifts
    rc, msg = _build_raw(shim, hexm.xyz, hexm.hex8, hexm.bface4[1:], hexm.btag[1:])
    assert rc == ERR_MESH and msg.startswith("1 faces")
    # a boundary tag outside 1..5
    tag = hexm.btag.copy()
    tag[0] = 9
    rc, msg = _build_raw(shim, hexm.xyz, hexm.hex8, hexm.bface4, tag)
    assert rc == ERR_ARG and "tag" in msg
    # a cell listed twice: its interior faces belong to three cells
    rc, msg = _build_raw(shim, hexm.xyz, np.concatenate([hexm.hex8, hexm.hex8[13:14]]), hexm.bface4, hexm.btag)
    assert rc == ERR_MESH and "more than two" in msg

    tetm = I.cavity_mesh(2)
    flat_xyz = tetm.xyz.copy()
    t = tetm.tet4[0]
    flat_xyz[t[3]] = flat_xyz[t[0]] + 0.5 * (flat_xyz[t[1]] - flat_xyz[t[0]]) + 0.25 * (flat_xyz[t[2]] - flat_xyz[t[0]])
    rc, msg = _build_raw(shim, flat_xyz, tetm.tet4, tetm.bface3, tetm.btag)
    assert rc == ERR_MESH and "degenerate tetrahedron" in msg
    # no cells at all
    rc, msg = _build_raw(shim, tetm.xyz, np.zeros((0, 4), dtype=np.int64), np.zeros((0, 3)), np.zeros(0))
    assert rc == ERR_ARG and "empty" in msg
    # one tetrahedron, all four faces walls: no non-compact stencil
    one = np.array([[0, 1, 2, 3]])
    xyz = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    bf = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    rc, msg = _build_raw(shim, xyz, one, bf, np.full(4, I.BC_WALL_ISO), mask=1)
    assert rc == ERR_MESH and "fewer than 9" in msg
