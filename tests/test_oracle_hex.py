"""Pins of the oracle on hexahedral cells (Sec. 3.1's six-face cells and their
eight non-compact sub-stencils of three face neighbours).

The expected values come from the geometry of the trilinear cell and of the
bilinear faces computed here by other means (Gauss's theorem over the faces,
high-order quadrature of the maps), from the stencil definition of Sec. 3.1
checked on an undistorted grid, from polynomial exactness of the
reconstruction (Sec. 3), from discrete conservation and free-stream
preservation of Eq. (finite), from the design order of the scheme, and from
dense linear algebra (Sec. 4).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2304_09485_gb300 import inputs as I

GAMMA = 1.4
CORNER = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
FACES = [[0, 1, 2, 3], [0, 1, 5, 4], [1, 2, 6, 5], [2, 3, 7, 6], [3, 0, 4, 7], [4, 5, 6, 7]]


def trilinear_rule(V, order=6):
    """Points [n, q, 3] and weights w detJ [n, q] of a tensor Gauss rule of the
    trilinear map of every hexahedron V [n, 8, 3]."""
    t, w = np.polynomial.legendre.leggauss(order)
    t, w = 0.5 * (t + 1), 0.5 * w
    pts, wts = [], []
    for (a, wa), (b, wb), (c, wc) in itertools.product(zip(t, w), repeat=3):
        r = np.array([a, b, c])
        f = np.where(CORNER == 1, r, 1 - r)                          # [8, 3]
        N = f.prod(1)
        sg = np.where(CORNER == 1, 1.0, -1.0)
        dN = np.stack([sg[:, e] * np.prod(np.delete(f, e, axis=1), axis=1) for e in range(3)], 1)   # [8, 3]
        X = np.einsum("a,nad->nd", N, V)
        J = np.einsum("ae,nad->nde", dN, V)
        pts.append(X)
        wts.append(wa * wb * wc * np.linalg.det(J))
    return np.stack(pts, 1), np.stack(wts, 1)


def cell_average(V, f, order=6):
    X, W = trilinear_rule(V, order)
    vol = W.sum(1)
    return np.einsum("nq,nqc->nc", W, f(X)) / vol[:, None], vol


def bilinear_rule(P, order=6):
    """Points [q, 3] and vector area elements [q, 3] (weights included) of the
    bilinear surface through the cyclic quadrilateral P [4, 3]."""
    t, w = np.polynomial.legendre.leggauss(order)
    t, w = 0.5 * (t + 1), 0.5 * w
    X, dA = [], []
    for (s, ws), (u, wu) in itertools.product(zip(t, w), repeat=2):
        X.append((1 - s) * (1 - u) * P[0] + s * (1 - u) * P[1] + s * u * P[2] + (1 - s) * u * P[3])
        xs = (1 - u) * (P[1] - P[0]) + u * (P[2] - P[3])
        xu = (1 - s) * (P[3] - P[0]) + s * (P[2] - P[1])
        dA.append(ws * wu * np.cross(xs, xu))
    return np.array(X), np.array(dA)


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------

def test_hex_volumes_and_centroids_by_gauss_theorem():
    """|Omega| = (1/3) surface integral of x.n and its first moments
    (1/2) surface integral of x_k^2 n_k, over the cell's six bilinear faces."""
    m = I.hex_cavity_mesh(3, jitter=0.15)
    om = O.OracleMesh(m)
    vol, cen = om.vol, om.centroid
    for c in range(m.n_cells):
        V = m.xyz[m.hex8[c]]
        centre = V.mean(0)
        v, mom = 0.0, np.zeros(3)
        for f in FACES:
            X, dA = bilinear_rule(V[f])
            if np.sum(dA, 0) @ (X.mean(0) - centre) < 0:
                dA = -dA                                        # outward
            v += np.sum(np.einsum("qd,qd->q", X, dA)) / 3.0
            mom += 0.5 * np.sum(X * X * dA, 0)
        assert vol[c] == pytest.approx(v, rel=1e-13)
        np.testing.assert_allclose(cen[c], mom / v, rtol=0, atol=1e-14)
    assert vol.sum() == pytest.approx(1.0, rel=1e-14)


def test_hex_face_areas_and_normals():
    """Interior faces: n S is the vector area of the bilinear face (its four
    vertices are those the two cells share), pointing from the left cell to the
    right one; each cell's outward vector areas add up to zero."""
    m = I.hex_cavity_mesh(3, jitter=0.15)
    om = O.OracleMesh(m)
    fg = om.face_geometry()
    cen = om.centroid
    acc = np.zeros((m.n_cells, 3))
    for f in range(om.nf):
        L, R = fg["left"][f], fg["right"][f]
        nS = fg["area"][f] * fg["normal"][f]
        acc[L] += nS
        if R >= 0:
            acc[R] -= nS
            shared = np.intersect1d(m.hex8[L], m.hex8[R])
            assert shared.size == 4
            loc = [int(np.where(m.hex8[L] == v)[0][0]) for v in shared]
            cyc = next(F for F in FACES if sorted(F) == sorted(loc))
            P = m.xyz[m.hex8[L][cyc]]
            _, dA = bilinear_rule(P)
            A = dA.sum(0)
            A = A if A @ (cen[R] - cen[L]) > 0 else -A
            np.testing.assert_allclose(nS, A, rtol=0, atol=1e-15)
    assert np.abs(acc).max() <= 1e-15


def test_hex_gauss_rule_on_planar_quadrilaterals():
    """On planar (non-parallelogram) faces the 2 x 2 rule, weighted by the area
    element, integrates every quadratic exactly: one cell between a general
    planar quadrilateral and a scaled copy of it (all faces planar trapezoids)."""
    base = np.array([[0.0, 0.0, 0.0], [1.2, 0.0, 0.0], [1.0, 1.1, 0.0], [0.1, 0.9, 0.0]])
    apex = np.array([0.5, 0.4, 2.0])
    top = apex + 0.55 * (base - apex)
    xyz = np.vstack([base, top])
    hexm = I.HexMesh(xyz, np.arange(8, dtype=np.int64)[None], np.array(FACES, dtype=np.int64),
                     np.full(6, I.BC_FARFIELD, np.int32))
    om = O.OracleMesh(hexm)
    fg = om.face_geometry()
    rng = np.random.default_rng(5)
    H = rng.normal(size=(3, 3)); H = H + H.T
    a = rng.normal(size=3)
    f = lambda X: 0.7 + X @ a + np.einsum("...i,ij,...j->...", X, H, X)
    assert om.nf == 6
    for k in range(6):
        # the 2 x 2 points of a bilinear map have the mean of its four vertices
        c = fg["gp"][k].mean(0)
        P = next(xyz[F] for F in FACES if np.allclose(xyz[F].mean(0), c, rtol=0, atol=1e-13))
        X, dA = bilinear_rule(P, order=8)
        exact = np.sum(f(X) * np.linalg.norm(dA, axis=1))
        got = fg["area"][k] * np.sum(fg["gw"][k] * f(fg["gp"][k]))
        assert got == pytest.approx(exact, rel=1e-13)
        assert fg["gw"][k].sum() == pytest.approx(1.0, rel=1e-15)


# ---------------------------------------------------------------------------
# stencils (Sec. 3.1)
# ---------------------------------------------------------------------------

def test_hex_stencils_on_an_undistorted_grid():
    """Interior cell of a cube grid (local vertex labels randomly rotated): the big
    stencil is the face neighbours and theirs (24 cells: offsets e, 2e, e + e'),
    and the eight sub-stencils are the face-neighbour triples across the eight
    corners {s_x e_x, s_y e_y, s_z e_z}, one for every sign pattern."""
    n = 5
    m = I.hex_cavity_mesh(n, jitter=0.0)
    om = O.OracleMesh(m)
    cen = om.centroid
    h = 1.0 / n
    inner = np.where(np.all((cen > 2 * h) & (cen < 1 - 2 * h), axis=1))[0]
    assert inner.size == 1
    c = int(inner[0])
    big, _ = om.stencil(c)
    off = np.rint((cen[big] - cen[c]) / h).astype(int)
    expect = {tuple(s * e) for e in np.eye(3, dtype=int) for s in (1, -1, 2, -2)}
    expect |= {tuple(s1 * a + s2 * b) for a, b in itertools.combinations(np.eye(3, dtype=int), 2)
               for s1 in (1, -1) for s2 in (1, -1)}
    assert len(big) == 24 and {tuple(o) for o in off} == expect
    signs = set()
    for mm in range(8):
        sub, ok = om.stencil(c, mm)
        assert ok and len(sub) == 3
        o = np.rint((cen[sub] - cen[c]) / h).astype(int)
        assert sorted(np.abs(o).sum(1)) == [1, 1, 1] and np.abs(o.sum(0)).tolist() == [1, 1, 1]
        signs.add(tuple(o.sum(0)))
    assert len(signs) == 8


def test_hex_boundary_sub_stencils_are_dropped():
    """A corner cell has three face neighbours: only the sub-stencil across its
    interior corner has three cells; the other seven are not used."""
    m = I.hex_cavity_mesh(4, jitter=0.0)
    om = O.OracleMesh(m)
    cen = om.centroid
    c = int(np.argmin(np.linalg.norm(cen, axis=1)))
    valid = [om.stencil(c, mm)[1] for mm in range(8)]
    assert sum(valid) == 1


# ---------------------------------------------------------------------------
# reconstruction (Sec. 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [0, 1])
def test_hex_linear_fields_reproduced(scheme):
    """Linear fields are reproduced at every Gauss point, with nonlinear weights
    and characteristic variables."""
    m = I.hex_cavity_mesh(4, jitter=0.15)
    om = O.OracleMesh(m)
    rng = np.random.default_rng(23)
    A = rng.normal(size=(5, 3)) * 0.1
    b = np.array([1.0, 0.2, -0.1, 0.05, 2.5])
    f = lambda X: X @ A.T + b
    Q, _ = cell_average(m.xyz[m.hex8], f)
    G = np.repeat(A.reshape(1, 15), m.n_cells, axis=0)
    p = O.make_params(scheme=scheme, weights=0)
    for cell in rng.choice(m.n_cells, 12, replace=False):
        for slot in range(6):
            _, _, Wg, gg = om.recon_side(p, Q, G, int(cell), slot)
            gp = om.face_gauss_points(int(cell), slot)
            np.testing.assert_allclose(Wg, f(gp), rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(gg, np.repeat(A[None], 4, axis=0), rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("scheme", [0, 1])
def test_hex_quadratic_fields_reproduced_linear_weights(scheme):
    """With linear weights Eq. (weno) returns P0, exact for quadratics."""
    m = I.hex_cavity_mesh(5, jitter=0.15)
    om = O.OracleMesh(m)
    rng = np.random.default_rng(29)
    Hq = rng.normal(size=(5, 3, 3)) * 0.2
    Hq = Hq + Hq.transpose(0, 2, 1)
    A = rng.normal(size=(5, 3)) * 0.3
    b = np.array([1.0, 0.2, -0.1, 0.05, 2.5])

    def f(X):
        return X @ A.T + 0.5 * np.einsum("...i,cij,...j->...c", X, Hq, X) + b
    Q, _ = cell_average(m.xyz[m.hex8], f)
    cx, _ = cell_average(m.xyz[m.hex8], lambda X: X)             # volume centroids
    G = (np.einsum("cij,nj->nci", Hq, cx) + A[None]).reshape(-1, 15)
    p = O.make_params(scheme=scheme, weights=1)
    inner = np.where(np.all((cx > 0.3) & (cx < 0.7), axis=1))[0]
    for cell in inner[:12]:
        for slot in range(6):
            _, _, Wg, gg = om.recon_side(p, Q, G, int(cell), slot)
            gp = om.face_gauss_points(int(cell), slot)
            np.testing.assert_allclose(Wg, f(gp), rtol=1e-11, atol=1e-12)
            grad = np.einsum("cij,gj->gci", Hq, gp) + A[None]
            np.testing.assert_allclose(gg, grad, rtol=1e-9, atol=1e-10)


# ---------------------------------------------------------------------------
# residual (Eq. (finite))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [0, 1])
def test_hex_free_stream_preservation(scheme):
    m = I.hex_periodic_cube_mesh(4, jitter=0.15)
    om = O.OracleMesh(m)
    Q = I.uniform_state(m.n_cells, rho=1.1, u=0.3, v=-0.2, w=0.1, p=0.9)
    p = O.make_params(scheme=scheme)
    out = om.residual(p, Q, np.zeros((m.n_cells, 15)))
    R = out[0] if scheme == 1 else out
    assert np.abs(R).max() <= 1e-13
    if scheme == 1:
        assert np.abs(out[1]).max() <= 1e-12


@pytest.mark.parametrize("scheme,visc", [(0, 0), (1, 0), (1, 1)])
def test_hex_discrete_conservation(scheme, visc):
    m = I.hex_periodic_cube_mesh(4, jitter=0.15)
    om = O.OracleMesh(m)
    Q, G = I.smooth_state(m, amp=0.08)
    p = O.make_params(scheme=scheme, viscous=visc, mu=0.01, Pr=0.72 if visc else 1.0)
    out = om.residual(p, Q, G)
    R = out[0] if scheme else out
    scale = np.abs(R).sum(0) + 1e-3
    assert np.all(np.abs(R.sum(0)) <= 1e-13 * scale + 1e-16)
    if scheme == 1:
        assert np.abs((out[1] * om.vol[:, None]).sum(0)).max() <= 1e-13


def test_hex_closed_cavity_conserves_mass():
    """Impermeable walls: the density residuals of a closed hexahedral cavity add up to zero."""
    m = I.hex_cavity_mesh(4, jitter=0.15)
    om = O.OracleMesh(m)
    c = I.cavity_conditions(Mach=0.3, Re=100.0)
    Q, G = I.smooth_state(m, amp=0.05, base=(1.0, 0.05, -0.02, 0.03, c["p_inf"]))
    for scheme in (0, 1):
        p = O.make_params(scheme=scheme, Pr=0.72, **c)
        out = om.residual(p, Q, G)
        R = out[0] if scheme else out
        assert abs(R[:, 0].sum()) <= 1e-14 * np.abs(R[:, 0]).sum()


def bilinear_rule_batch(P, order=5):
    """bilinear_rule for a batch of quadrilaterals P [n, 4, 3]: points [n, q, 3], vector areas [n, q, 3]."""
    t, w = np.polynomial.legendre.leggauss(order)
    t, w = 0.5 * (t + 1), 0.5 * w
    X, dA = [], []
    for (s, ws), (u, wu) in itertools.product(zip(t, w), repeat=2):
        X.append((1 - s) * (1 - u) * P[:, 0] + s * (1 - u) * P[:, 1] + s * u * P[:, 2] + (1 - s) * u * P[:, 3])
        xs = (1 - u) * (P[:, 1] - P[:, 0]) + u * (P[:, 2] - P[:, 3])
        xu = (1 - s) * (P[:, 3] - P[:, 0]) + s * (P[:, 2] - P[:, 1])
        dA.append(ws * wu * np.cross(xs, xu))
    return np.stack(X, 1), np.stack(dA, 1)


def test_hex_design_order_density_wave():
    """rho = 1 + 0.2 sin(2 pi (x+y+z)/3), U = (1,1,1)/2, p = 1 solves the Euler
    equations. On planar-faced hexahedra that are not parallelepipeds, R/|Omega|
    of the cell averages approaches -(1/|Omega|) times the surface integral of
    F_Euler(Q_exact).n over the cell (cells not on the boundary): at third
    order with linear weights (P0 alone), and at least second order between the
    finer meshes with nonlinear weights and characteristic variables."""
    u0 = 0.5

    def Qx(X):
        rho = 1 + 0.2 * np.sin(2 * np.pi * X.sum(-1) / 3.0)
        return np.stack([rho, rho * u0, rho * u0, rho * u0, 1 / (GAMMA - 1) + 0.5 * rho * 3 * u0 * u0], -1)
    ns = (8, 12, 16)
    errs = {0: [], 1: []}
    for n in ns:
        m = I.hex_tilted_box_mesh(n)
        om = O.OracleMesh(m)
        V = m.xyz[m.hex8]
        Q, vol = cell_average(V, Qx)
        centre = V.mean(1)
        ex = np.zeros(m.n_cells)                    # minus the surface integral of the mass flux
        for F in FACES:
            X, dA = bilinear_rule_batch(V[:, F])
            sg = np.sign(np.einsum("nd,nd->n", dA.sum(1), X.mean(1) - centre))
            ex -= sg * np.einsum("nq,nq->n", Qx(X)[..., 0], u0 * dA.sum(-1))
        inner = np.where(np.all((om.centroid > 1.5 / n) & (om.centroid < 1 - 1.5 / n), axis=1))[0]
        for w in (0, 1):
            p = O.make_params(scheme=0, weights=w, flux_dt=1e-8, characteristic=1 - w,
                              rho_inf=1.0, u_inf=(u0, u0, u0), p_inf=1.0)
            R = om.residual(p, Q)
            err = (R[inner, 0] - ex[inner]) / vol[inner]
            errs[w].append(np.sqrt(np.mean(err ** 2)))
    ratio = np.log(np.array(ns[1:]) / np.array(ns[:-1]))
    lin = np.log(np.array(errs[1][:-1]) / np.array(errs[1][1:])) / ratio
    nonlin = np.log(np.array(errs[0][:-1]) / np.array(errs[0][1:])) / ratio
    assert np.all(lin >= 2.4), (errs, lin)
    assert nonlin[-1] >= 2.0, (errs, nonlin)


# ---------------------------------------------------------------------------
# implicit system (Sec. 4)
# ---------------------------------------------------------------------------

def test_hex_full_gmres_equals_lu():
    """GMRES with a Krylov space of the full dimension solves A x = b exactly,
    with six off-diagonal blocks per row."""
    m = I.hex_periodic_cube_mesh(3)
    om = O.OracleMesh(m)
    Q, _ = I.smooth_state(m, amp=0.1)
    p = O.make_params(scheme=0, cfl=5.0)
    diag, off = om.jacobian(p, Q)
    assert off.shape == (m.n_cells, 6, 5, 5)
    n = om.nc
    A = np.zeros((5 * n, 5 * n))
    nb = om.neighbours
    for i in range(n):
        A[5 * i:5 * i + 5, 5 * i:5 * i + 5] = diag[i]
        for q in range(6):
            if nb[i, q] >= 0:
                A[5 * i:5 * i + 5, 5 * nb[i, q]:5 * nb[i, q] + 5] += off[i, q]
    b = np.random.default_rng(43).normal(size=(n, 5))
    q = O.make_params(scheme=0, krylov_dim=5 * n, restarts=1, jacobi_sweeps=2)
    dx, _ = om.gmres(q, diag, off, b)
    x = np.linalg.solve(A, b.ravel())
    assert np.linalg.norm(dx.ravel() - x) <= 1e-10 * np.linalg.norm(x)


def test_hex_diagonal_block_is_a_multiple_of_the_identity():
    """The Euler-Jacobian part of A_ii is J(Q_i) times the sum of the cell's outward
    vector areas, zero for a closed cell: A_ii = (|Omega|/dt + sum lambda S / 2) I."""
    m = I.hex_cavity_mesh(3, jitter=0.15)
    om = O.OracleMesh(m)
    Q, _ = I.smooth_state(m, amp=0.1)
    p = O.make_params(scheme=0, cfl=5.0)
    diag, _ = om.jacobian(p, Q)
    for i in range(m.n_cells):
        d = diag[i][0, 0]
        np.testing.assert_allclose(diag[i], d * np.eye(5), rtol=0, atol=1e-13 * d)
