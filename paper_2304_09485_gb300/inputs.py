"""Seeded synthetic inputs: tetrahedral and hexahedral meshes and flow states.

This module is shared by the CUDA path's tests/benchmark and by the oracle's
tests. It holds no arithmetic of the method (no geometry of cells or faces, no
reconstruction, no flux): it only lays vertices out, connects them into
tetrahedra or hexahedra, tags boundary faces and draws seeded states.

Meshes stand in for the paper's workloads (Sec. 5.1 lid-driven cavity on
tetrahedra split from hexahedra; Sec. 5.2 flow past a sphere). The paper's own
meshes are not available; these generators reproduce their kind and size.

Boundary tags (shared vocabulary with include/hgks.h):
  1 isothermal no-slip wall at rest, 2 isothermal no-slip wall moving with the
  lid speed along +x, 3 adiabatic slip wall, 4 adiabatic no-slip wall,
  5 far field.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_WALL_ISO = 1
BC_WALL_LID = 2
BC_SLIP = 3
BC_NOSLIP_ADIA = 4
BC_FARFIELD = 5

BASE_SEED = 2304_09485


@dataclass
class Mesh:
    """A tetrahedral mesh as plain arrays (caller order)."""
    xyz: np.ndarray            # [n_vert, 3] float64
    tet4: np.ndarray           # [n_tet, 4] int64
    bface3: np.ndarray         # [n_bface, 3] int64
    btag: np.ndarray           # [n_bface] int32
    periodic_shift: np.ndarray | None = None   # [k, 3] translations, or None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_tet(self) -> int:
        return int(self.tet4.shape[0])

    @property
    def cells(self) -> np.ndarray:
        return self.tet4

    @property
    def n_cells(self) -> int:
        return int(self.tet4.shape[0])


@dataclass
class HexMesh:
    """A hexahedral mesh as plain arrays (caller order).

    Vertices of a hexahedron in the usual order: 0-3 one quadrilateral in cyclic
    order, 4-7 the opposite one with vertex 4 + a joined to vertex a; positive
    orientation ((x1 - x0) x (x3 - x0)) . (x4 - x0) > 0. Boundary quadrilaterals
    list their four vertices in cyclic order."""
    xyz: np.ndarray            # [n_vert, 3] float64
    hex8: np.ndarray           # [n_hex, 8] int64
    bface4: np.ndarray         # [n_bface, 4] int64
    btag: np.ndarray           # [n_bface] int32
    periodic_shift: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> np.ndarray:
        return self.hex8

    @property
    def n_cells(self) -> int:
        return int(self.hex8.shape[0])


def _kuhn_tets(idx):
    """Six tetrahedra of each hexahedron, all around the main diagonal.

    idx(a, b, c) returns the vertex index array of corner (a, b, c) in {0,1}^3 of
    every hexahedron. All hexahedra use the same diagonal, so neighbouring
    splits agree on every shared quadrilateral.
    """
    v0 = idx(0, 0, 0)
    v7 = idx(1, 1, 1)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for p in perms:
        c1 = [0, 0, 0]
        c1[p[0]] = 1
        c2 = list(c1)
        c2[p[1]] = 1
        tets.append(np.stack([v0, idx(*c1), idx(*c2), v7], axis=-1))
    return np.concatenate([t.reshape(-1, 4) for t in tets], axis=0)


def _signed_volume6(xyz, tet):
    a = xyz[tet[:, 0]]
    b = xyz[tet[:, 1]] - a
    c = xyz[tet[:, 2]] - a
    d = xyz[tet[:, 3]] - a
    return np.einsum("ij,ij->i", b, np.cross(c, d))


def _orient_positive(xyz, tet):
    """Swap two vertices of every negatively oriented tetrahedron."""
    s = _signed_volume6(xyz, tet)
    tet = tet.copy()
    neg = s < 0
    tet[neg, 2], tet[neg, 3] = tet[neg, 3].copy(), tet[neg, 2].copy()
    return tet


def wall_clustered_nodes(n: int, h_min: float) -> np.ndarray:
    """n + 1 nodes on [0, 1], cell sizes h_min r^min(i, n-1-i) (geometric growth
    from both walls to the middle), r found by bisection so that they sum to 1."""
    if h_min * n >= 1.0:
        return np.linspace(0.0, 1.0, n + 1)
    k = np.minimum(np.arange(n), n - 1 - np.arange(n)).astype(np.float64)
    lo, hi = 1.0, 2.0
    for _ in range(200):
        r = 0.5 * (lo + hi)
        lo, hi = (r, hi) if (h_min * r ** k).sum() < 1.0 else (lo, r)
    sz = h_min * (0.5 * (lo + hi)) ** k
    x = np.concatenate([[0.0], np.cumsum(sz)])
    return x / x[-1]


def cavity_mesh(n: int = 8, jitter: float = 0.1, seed: int = BASE_SEED + 0,
                permute: bool = True, lid_tag: int = BC_WALL_LID,
                wall_tag: int = BC_WALL_ISO, h_min: float | None = None) -> Mesh:
    """Unit cube, n^3 hexahedra, each split into 6 tetrahedra (6 n^3 cells).

    Interior vertices are moved by U(-jitter*h, +jitter*h) per axis (h the smaller
    neighbouring spacing along that axis); the order of the cells is randomly
    permuted. The lid is the face y = 1 (Sec. 5.1). With h_min, the spacing grows
    geometrically from h_min at every wall (Sec. 5.1's refined cavity mesh).
    """
    rng = np.random.default_rng(seed)
    x1 = np.linspace(0.0, 1.0, n + 1) if h_min is None else wall_clustered_nodes(n, h_min)
    sp = np.diff(x1)
    hloc = np.minimum(np.concatenate([[sp[0]], sp]), np.concatenate([sp, [sp[-1]]]))   # per node
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([I, J, K], axis=-1).reshape(-1, 3)
    xyz = x1[lat]
    interior = np.all((lat > 0) & (lat < n), axis=1)
    d = rng.uniform(-jitter, jitter, size=xyz.shape) * hloc[lat]
    xyz[interior] += d[interior]

    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    hi, hj, hk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    tet = _kuhn_tets(lambda a, b, c: vid(hi + a, hj + b, hk + c))
    tet = _orient_positive(xyz, tet)
    if permute:
        tet = tet[rng.permutation(tet.shape[0])]

    # boundary triangles: faces whose three vertices lie on one cube face
    faces = np.concatenate([tet[:, [1, 2, 3]], tet[:, [0, 2, 3]],
                            tet[:, [0, 1, 3]], tet[:, [0, 1, 2]]], axis=0)
    fl = lat[faces]                                   # [nf, 3, 3] lattice coords
    bf, bt = [], []
    for axis in range(3):
        for side in (0, n):
            on = np.all(fl[:, :, axis] == side, axis=1)
            bf.append(faces[on])
            tag = lid_tag if (axis == 1 and side == n) else wall_tag
            bt.append(np.full(on.sum(), tag, dtype=np.int32))
    bface = np.concatenate(bf).astype(np.int64)
    btag = np.concatenate(bt)
    return Mesh(xyz, tet.astype(np.int64), bface, btag, None,
                name=f"cavity{n}", meta=dict(n=n, jitter=jitter, seed=seed, h_min=h_min))


def periodic_cube_mesh(n: int = 6, jitter: float = 0.1, seed: int = BASE_SEED + 100,
                       permute: bool = True, length: float = 1.0) -> Mesh:
    """Periodic cube [0,L]^3 of n^3 Kuhn-split hexahedra, every vertex jittered.

    Periodic images of a vertex get the same jitter, so faces on opposite sides
    of the box coincide after a translation by L along one axis.
    """
    rng = np.random.default_rng(seed)
    h = length / n
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([I, J, K], axis=-1).reshape(-1, 3)
    base = rng.uniform(-jitter * h, jitter * h, size=(n, n, n, 3))
    d = base[lat[:, 0] % n, lat[:, 1] % n, lat[:, 2] % n]
    xyz = lat.astype(np.float64) * h + d

    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    hi, hj, hk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    tet = _kuhn_tets(lambda a, b, c: vid(hi + a, hj + b, hk + c))
    tet = _orient_positive(xyz, tet)
    if permute:
        tet = tet[rng.permutation(tet.shape[0])]
    return Mesh(xyz, tet.astype(np.int64), np.zeros((0, 3), np.int64),
                np.zeros(0, np.int32), np.eye(3) * length,
                name=f"periodic{n}", meta=dict(n=n, jitter=jitter, seed=seed, length=length))


# corner (a, b, c) in {0,1}^3 of the usual hexahedron vertex order
_HEX_CORNER = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                        [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])


def _hex_rotations() -> np.ndarray:
    """[24, 8] vertex relabellings of a hexahedron by the 24 rotations of a cube.

    Row r gives, for new local vertex a, the old local vertex at the corner the
    rotation moves a to: every row keeps the hexahedron positively oriented."""
    corner_id = {tuple(c): k for k, c in enumerate(_HEX_CORNER)}
    rows = []
    for perm in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
        for sg in np.ndindex(2, 2, 2):
            R = np.zeros((3, 3))
            for r in range(3):
                R[r, perm[r]] = 1.0 if sg[r] == 0 else -1.0
            if np.linalg.det(R) < 0:
                continue
            s = 2 * _HEX_CORNER - 1
            t = (s @ R.T + 1) // 2
            rows.append([corner_id[tuple(int(x) for x in v)] for v in t])
    return np.array(rows, dtype=np.int64)


def _hex_grid(n: int, vid, reorient: bool, rng) -> np.ndarray:
    hi, hj, hk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    hx = np.stack([vid(hi + c[0], hj + c[1], hk + c[2]) for c in _HEX_CORNER], axis=1)
    if reorient:
        rot = _hex_rotations()[rng.integers(0, 24, size=hx.shape[0])]
        hx = np.take_along_axis(hx, rot, axis=1)
    return hx


def hex_cavity_mesh(n: int = 6, jitter: float = 0.1, seed: int = BASE_SEED + 500,
                    permute: bool = True, reorient: bool = True, lid_tag: int = BC_WALL_LID,
                    wall_tag: int = BC_WALL_ISO) -> HexMesh:
    """Unit cube of n^3 hexahedra (Sec. 3.1's hexahedral cells), lid y = 1.

    Interior vertices are moved by U(-jitter h, +jitter h) per axis, so the faces
    are non-planar quadrilaterals; with `reorient` each hexahedron's vertices are
    relabelled by a random one of the 24 rotations of a cube (its local faces,
    and so its sub-stencils, then point along random axes); the order of the
    cells is randomly permuted."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([I, J, K], axis=-1).reshape(-1, 3)
    xyz = lat.astype(np.float64) * h
    interior = np.all((lat > 0) & (lat < n), axis=1)
    d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    xyz[interior] += d[interior]

    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    hx = _hex_grid(n, vid, reorient, rng)
    if permute:
        hx = hx[rng.permutation(hx.shape[0])]
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a, b = a.ravel(), b.ravel()
    bf, bt = [], []
    for axis in range(3):
        o1, o2 = [x for x in range(3) if x != axis]
        for side in (0, n):
            def V(u, v):
                c = [None, None, None]
                c[axis] = np.full_like(u, side)
                c[o1] = u
                c[o2] = v
                return vid(c[0], c[1], c[2])
            bf.append(np.stack([V(a, b), V(a + 1, b), V(a + 1, b + 1), V(a, b + 1)], axis=1))
            tag = lid_tag if (axis == 1 and side == n) else wall_tag
            bt.append(np.full(a.shape[0], tag, dtype=np.int32))
    return HexMesh(xyz, hx.astype(np.int64), np.concatenate(bf).astype(np.int64), np.concatenate(bt),
                   None, name=f"hexcavity{n}", meta=dict(n=n, jitter=jitter, seed=seed))


def hex_tilted_box_mesh(n: int = 6, tilt: float = 0.3, seed: int = BASE_SEED + 700,
                        permute: bool = True, reorient: bool = True,
                        tag: int = BC_FARFIELD) -> HexMesh:
    """Hexahedra between three families of tilted planes: planar faces, cells
    that are not parallelepipeds (their faces are general planar quadrilaterals).

    Plane i of family x: x = i/n + a_i (y - 1/2) + b_i (z - 1/2), a_i, b_i drawn
    from U(-tilt, tilt) / n (tilt < 1/2 keeps neighbouring planes from crossing
    inside the box), likewise for y and z; vertex (i, j, k) is the meeting
    point of planes i, j, k. Every boundary quadrilateral gets `tag`."""
    rng = np.random.default_rng(seed)
    g = np.arange(n + 1) / n
    tl = rng.uniform(-tilt, tilt, size=(3, n + 1, 2)) / n   # family, plane, two slopes
    I, J, K = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    idx = np.stack([I, J, K], axis=-1).reshape(-1, 3)
    A = np.zeros((idx.shape[0], 3, 3))
    rhs = np.zeros((idx.shape[0], 3))
    for fam in range(3):
        o1, o2 = [x for x in range(3) if x != fam]
        sl = tl[fam, idx[:, fam]]
        # x_fam - s1 x_o1 - s2 x_o2 = g - (s1 + s2) / 2
        A[:, fam, fam] = 1.0
        A[:, fam, o1] = -sl[:, 0]
        A[:, fam, o2] = -sl[:, 1]
        rhs[:, fam] = g[idx[:, fam]] - 0.5 * (sl[:, 0] + sl[:, 1])
    xyz = np.linalg.solve(A, rhs[..., None])[..., 0]

    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    hx = _hex_grid(n, vid, reorient, rng)
    if permute:
        hx = hx[rng.permutation(hx.shape[0])]
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a, b = a.ravel(), b.ravel()
    bf = []
    for axis in range(3):
        o1, o2 = [x for x in range(3) if x != axis]
        for side in (0, n):
            def V(u, v):
                c = [None, None, None]
                c[axis] = np.full_like(u, side)
                c[o1] = u
                c[o2] = v
                return vid(c[0], c[1], c[2])
            bf.append(np.stack([V(a, b), V(a + 1, b), V(a + 1, b + 1), V(a, b + 1)], axis=1))
    bf = np.concatenate(bf).astype(np.int64)
    return HexMesh(xyz, hx.astype(np.int64), bf, np.full(bf.shape[0], tag, np.int32), None,
                   name=f"hextilted{n}", meta=dict(n=n, tilt=tilt, seed=seed))


def hex_sphere_mesh(n: int = 32, layers: int = 31, r_in: float = 0.5, r_out: float = 10.0,
                    stretch: float | None = None, wall_tag: int = BC_NOSLIP_ADIA, seed: int = BASE_SEED + 800,
                    permute: bool = True) -> HexMesh:
    """Cubed-sphere O-grid of hexahedra around a sphere (Sec. 5.2's hexahedral
    sphere grids): six equiangular n x n patches on the sphere, `layers` radial
    layers stretched geometrically from r_in to r_out (first layer of the wall
    cells' tangential size times 0.36 unless `stretch` is given); inner faces
    tagged `wall_tag`, outer faces far field. 6 n^2 layers cells (n = 32,
    31 layers: 190,464, the cell count of the paper's hexahedral sphere)."""
    rng = np.random.default_rng(seed)
    g = np.arange(n + 1)
    I_, J_, K_ = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([I_, J_, K_], axis=-1).reshape(-1, 3)
    on_surf = np.any((lat == 0) | (lat == n), axis=1)
    surf = lat[on_surf]
    ns = surf.shape[0]
    sid = -np.ones((n + 1) ** 3, dtype=np.int64)
    sid[(surf[:, 0] * (n + 1) + surf[:, 1]) * (n + 1) + surf[:, 2]] = np.arange(ns)
    t = np.tan((surf.astype(np.float64) / n - 0.5) * (math.pi / 2.0))
    unit = t / np.linalg.norm(t, axis=1, keepdims=True)
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a, b = a.ravel(), b.ravel()
    quads = []
    for axis in range(3):
        for side in (0, n):
            o1, o2 = [x for x in range(3) if x != axis]

            def P(u, v):
                c = [None, None, None]
                c[axis] = np.full_like(u, side)
                c[o1] = u
                c[o2] = v
                return sid[(c[0] * (n + 1) + c[1]) * (n + 1) + c[2]]
            quads.append(np.stack([P(a, b), P(a + 1, b), P(a + 1, b + 1), P(a, b + 1)], axis=1))
    quads = np.concatenate(quads, axis=0)
    if stretch is None:
        stretch = sphere_stretch(layers, r_in, r_out, dr1=0.36 * math.pi * r_in / (2 * n))
    radii = sphere_radii(layers, r_in, r_out, stretch)
    xyz = (unit[None, :, :] * radii[:, None, None]).reshape(-1, 3)
    L = np.arange(layers)[:, None]
    lower = (L[:, :, None] * ns + quads[None, :, :]).reshape(-1, 4)
    hx = np.concatenate([lower, lower + ns], axis=1)
    # orient every hexahedron positively (the quads' cyclic direction depends on the patch)
    x = xyz[hx]
    neg = np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 3] - x[:, 0]), x[:, 4] - x[:, 0]) < 0
    hx[neg] = hx[neg][:, [0, 3, 2, 1, 4, 7, 6, 5]]
    if permute:
        hx = hx[rng.permutation(hx.shape[0])]
    bface = np.concatenate([quads, quads + layers * ns], axis=0).astype(np.int64)
    btag = np.concatenate([np.full(len(quads), wall_tag, np.int32), np.full(len(quads), BC_FARFIELD, np.int32)])
    return HexMesh(xyz, hx.astype(np.int64), bface, btag, None, name=f"hexsphere{n}x{layers}",
                   meta=dict(n=n, layers=layers, r_in=r_in, r_out=r_out, stretch=stretch))


def hex_periodic_cube_mesh(n: int = 4, jitter: float = 0.1, seed: int = BASE_SEED + 600,
                           permute: bool = True, reorient: bool = True, length: float = 1.0) -> HexMesh:
    """Periodic cube [0,L]^3 of n^3 hexahedra, every vertex jittered (periodic
    images of a vertex move together)."""
    rng = np.random.default_rng(seed)
    h = length / n
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([I, J, K], axis=-1).reshape(-1, 3)
    base = rng.uniform(-jitter * h, jitter * h, size=(n, n, n, 3))
    xyz = lat.astype(np.float64) * h + base[lat[:, 0] % n, lat[:, 1] % n, lat[:, 2] % n]

    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    hx = _hex_grid(n, vid, reorient, rng)
    if permute:
        hx = hx[rng.permutation(hx.shape[0])]
    return HexMesh(xyz, hx.astype(np.int64), np.zeros((0, 4), np.int64), np.zeros(0, np.int32),
                   np.eye(3) * length, name=f"hexperiodic{n}", meta=dict(n=n, jitter=jitter, seed=seed))


def sphere_radii(layers: int, r_in: float, r_out: float, stretch: float) -> np.ndarray:
    """Radii of a geometric O-grid: first spacing dr1, ratio `stretch`, r_out reached."""
    if stretch == 1.0:
        return np.linspace(r_in, r_out, layers + 1)
    dr1 = (r_out - r_in) * (stretch - 1.0) / (stretch ** layers - 1.0)
    l = np.arange(layers + 1, dtype=np.float64)
    return r_in + dr1 * (stretch ** l - 1.0) / (stretch - 1.0)


def sphere_mesh(n: int = 32, layers: int = 64, r_in: float = 0.5, r_out: float = 10.0,
                stretch: float = 1.08, wall_tag: int = BC_SLIP, seed: int = BASE_SEED + 1,
                permute: bool = True) -> Mesh:
    """Cubed-sphere O-grid around a sphere, split into tetrahedra.

    Six n x n patches (equiangular) on the sphere, `layers` radial layers. Each
    surface quadrilateral is cut along its shorter diagonal (at the eight cube
    corners, where three patches meet at 120 degrees, this gives the corner vertex
    six triangles instead of obtuse ones); each triangle is extruded into prisms,
    and each prism is cut into 3 tetrahedra by the lowest-vertex-index rule. That
    rule makes every lateral quadrilateral shared by two prisms get the same
    diagonal from both sides (a surface quadrilateral's diagonal is its own), so
    the mesh is conforming across the patch seams. Cell count = 6 n^2 layers * 6,
    the same as 6 tetrahedra per hexahedron.
    """
    rng = np.random.default_rng(seed)
    # surface lattice points of the cube [0,n]^3
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([I, J, K], axis=-1).reshape(-1, 3)
    on_surf = np.any((lat == 0) | (lat == n), axis=1)
    surf = lat[on_surf]
    ns = surf.shape[0]
    sid = -np.ones((n + 1) ** 3, dtype=np.int64)
    lin = (surf[:, 0] * (n + 1) + surf[:, 1]) * (n + 1) + surf[:, 2]
    sid[lin] = np.arange(ns)

    def S(i, j, k):
        return sid[(i * (n + 1) + j) * (n + 1) + k]

    t = np.tan((surf.astype(np.float64) / n - 0.5) * (math.pi / 2.0))
    unit = t / np.linalg.norm(t, axis=1, keepdims=True)

    # quadrilaterals of the 6 cube faces
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a, b = a.ravel(), b.ravel()
    quads = []
    for axis in range(3):
        for side in (0, n):
            o1, o2 = [x for x in range(3) if x != axis]

            def P(u, v):
                c = [None, None, None]
                c[axis] = np.full_like(u, side)
                c[o1] = u
                c[o2] = v
                return S(c[0], c[1], c[2])
            quads.append(np.stack([P(a, b), P(a + 1, b), P(a + 1, b + 1), P(a, b + 1)], axis=1))
    quads = np.concatenate(quads, axis=0)
    # split each quad along its shorter diagonal (ties: the diagonal through vertex 0)
    d02 = np.linalg.norm(unit[quads[:, 0]] - unit[quads[:, 2]], axis=1)
    d13 = np.linalg.norm(unit[quads[:, 1]] - unit[quads[:, 3]], axis=1)
    m = np.where(d02 <= d13 * (1.0 + 1e-12), 0, 1)
    r = np.arange(quads.shape[0])
    q0 = quads[r, m]
    q1 = quads[r, (m + 1) % 4]
    q2 = quads[r, (m + 2) % 4]
    q3 = quads[r, (m + 3) % 4]
    tris = np.concatenate([np.stack([q0, q1, q2], 1), np.stack([q0, q2, q3], 1)], axis=0)
    tris = np.sort(tris, axis=1)                       # a < b < c (surface indices)

    radii = sphere_radii(layers, r_in, r_out, stretch)
    xyz = (unit[None, :, :] * radii[:, None, None]).reshape(-1, 3)
    L = np.arange(layers)[:, None]
    A = (L * ns + tris[None, :, 0]).ravel()
    B = (L * ns + tris[None, :, 1]).ravel()
    C = (L * ns + tris[None, :, 2]).ravel()
    A2, B2, C2 = A + ns, B + ns, C + ns
    # prism (a,b,c | a',b',c') with a<b<c: the minimum vertex is a, the lateral
    # quad (b,c,c',b') has minimum b, so the diagonals are a-b', a-c', b-c'.
    tet = np.concatenate([np.stack([A, B, C, C2], 1),
                          np.stack([A, B, B2, C2], 1),
                          np.stack([A, A2, B2, C2], 1)], axis=0)
    tet = _orient_positive(xyz, tet)
    if permute:
        tet = tet[rng.permutation(tet.shape[0])]
    inner = tris.astype(np.int64)
    outer = tris.astype(np.int64) + layers * ns
    bface = np.concatenate([inner, outer], axis=0)
    btag = np.concatenate([np.full(inner.shape[0], wall_tag, np.int32),
                           np.full(outer.shape[0], BC_FARFIELD, np.int32)])
    return Mesh(xyz, tet.astype(np.int64), bface, btag, None,
                name=f"sphere{n}x{layers}",
                meta=dict(n=n, layers=layers, r_in=r_in, r_out=r_out, stretch=stretch))


# ----------------------------------------------------------------------------
# states
# ----------------------------------------------------------------------------

def conservative(rho, u, v, w, p, gamma=1.4):
    """(rho, rho U, rho V, rho W, rho E) from primitive variables (Sec. 2)."""
    rho = np.asarray(rho, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack(np.broadcast_arrays(rho, rho * u, rho * v, rho * w, E), axis=-1)


def vertex_mean(mesh) -> np.ndarray:
    """Mean of the vertices of every cell (a sampling point for states)."""
    return mesh.xyz[mesh.cells].mean(axis=1)


def uniform_state(n: int, rho=1.0, u=0.3, v=0.0, w=0.0, p=1.0 / 1.4, gamma=1.4) -> np.ndarray:
    """[n, 5] copies of one conservative state (free stream, Sec. 5.2)."""
    q = conservative(rho, u, v, w, p, gamma)
    return np.tile(q, (n, 1))


def smooth_state(mesh: Mesh, seed: int = BASE_SEED + 7, amp: float = 0.05, gamma=1.4,
                 base=(1.0, 0.3, 0.1, -0.05, 1.0 / 1.4), wavenumber: float = 2.0):
    """Smooth random perturbation of a base state, sampled at vertex means.

    Returns (Q [n,5], G [n,15]) where G holds the exact Cartesian gradients of
    the sampled conservative field (component-major: G[:, 3*c + d] = dQ_c/dx_d),
    a plausible input for the compact scheme's cell-averaged gradients.
    """
    rng = np.random.default_rng(seed)
    x = vertex_mean(mesh)
    k = rng.normal(size=(5, 3)) * wavenumber
    ph = rng.uniform(0, 2 * math.pi, size=5)
    s = np.sin(x @ k.T + ph)                       # [n,5]
    c = np.cos(x @ k.T + ph)
    prim = np.array(base)[None, :] * (1.0 + amp * s)
    dprim = (np.array(base)[None, :, None] * amp * c[:, :, None] * k[None, :, :])
    rho, u, v, w, p = (prim[:, i] for i in range(5))
    Q = conservative(rho, u, v, w, p, gamma)
    drho, du, dv, dw, dp = (dprim[:, i, :] for i in range(5))
    G = np.zeros((x.shape[0], 5, 3))
    G[:, 0] = drho
    G[:, 1] = drho * u[:, None] + rho[:, None] * du
    G[:, 2] = drho * v[:, None] + rho[:, None] * dv
    G[:, 3] = drho * w[:, None] + rho[:, None] * dw
    G[:, 4] = dp / (gamma - 1.0) + 0.5 * drho * (u * u + v * v + w * w)[:, None] \
        + rho[:, None] * (u[:, None] * du + v[:, None] * dv + w[:, None] * dw)
    return Q, G.reshape(-1, 15)


# ----------------------------------------------------------------------------
# flow conditions (Sec. 5.1, 5.2): plain parameter values for a problem
# ----------------------------------------------------------------------------

def cavity_conditions(Mach: float = 0.15, Re: float = 100.0, gamma: float = 1.4, lid_speed: float = 1.0):
    """Lid-driven cavity: rho = 1, lid speed U, sound speed U/Mach, isothermal walls
    at the initial temperature, mu = rho U L / Re with L = 1."""
    p = 1.0 / (gamma * Mach * Mach) * lid_speed ** 2
    return dict(viscous=1, mu=lid_speed / Re, rho_inf=1.0, u_inf=(0.0, 0.0, 0.0), p_inf=p,
                wall_T=p / 1.0, lid_speed=lid_speed, gamma=gamma)


def sphere_conditions(Mach: float = 0.3, Re: float | None = None, aoa_deg: float = 0.0, gamma: float = 1.4):
    """Flow past a unit-diameter sphere: free stream (1, Ma, 0, 0, 1/gamma), rotated by
    the angle of attack in the x-y plane; mu = rho U D / Re (D = 1) when viscous."""
    a = math.radians(aoa_deg)
    u = (Mach * math.cos(a), Mach * math.sin(a), 0.0)
    d = dict(viscous=0 if Re is None else 1, mu=0.0 if Re is None else Mach / Re, rho_inf=1.0,
             u_inf=u, p_inf=1.0 / gamma, wall_T=1.0 / gamma, lid_speed=0.0, gamma=gamma)
    return d


def state_from_conditions(n: int, cond: dict) -> np.ndarray:
    """Uniform initial state of a problem: the free stream (the cavity starts at rest)."""
    u = cond["u_inf"]
    return uniform_state(n, rho=cond["rho_inf"], u=u[0], v=u[1], w=u[2], p=cond["p_inf"],
                         gamma=cond.get("gamma", 1.4))


def sphere_stretch(n_layers: int, r_in: float = 0.5, r_out: float = 10.0, dr1: float | None = None) -> float:
    """Geometric stretching ratio s with dr1 (s^L - 1) / (s - 1) = r_out - r_in; the
    first layer defaults to the tangential size of a patch cell at the wall (pi r_in / (2 n))
    scaled like the C2 grid (dr1 ~ 0.36 of it)."""
    if dr1 is None:
        dr1 = 0.36 * math.pi * r_in / (2 * max(2, n_layers // 2))
    lo, hi = 1.0 + 1e-9, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        tot = dr1 * (mid ** n_layers - 1) / (mid - 1)
        lo, hi = (mid, hi) if tot < r_out - r_in else (lo, mid)
    return 0.5 * (lo + hi)


def batch_problems(n_problems: int = 48, n_min: float = 20e3, n_max: float = 500e3, seed: int = BASE_SEED + 400,
                   viscous_sphere: bool = True):
    """Many independent steady problems of uneven size: kind ~ Bernoulli(1/2)
    cavity / sphere, N ~ log-uniform in [n_min, n_max] tets (cavity n = (N/6)^(1/3),
    sphere patches n = (N/72)^(1/3) with 2n layers), Mach ~ U(0.1, 0.5),
    Re ~ log-uniform in [50, 1000] (the sphere viscous as well when viscous_sphere).
    Returns a list of dicts: kind, n, mesh, cond, n_cells."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_problems):
        kind = "cavity" if rng.random() < 0.5 else "sphere"
        N = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        mach = rng.uniform(0.1, 0.5)
        Re = math.exp(rng.uniform(math.log(50.0), math.log(1000.0)))
        if kind == "cavity":
            n = max(2, int(round((N / 6.0) ** (1.0 / 3.0))))
            mesh = cavity_mesh(n, seed=seed + 1 + k)
            cond = cavity_conditions(mach, Re)
        else:
            n = max(2, int(round((N / 72.0) ** (1.0 / 3.0))))
            mesh = sphere_mesh(n, 2 * n, stretch=sphere_stretch(2 * n),
                               wall_tag=BC_NOSLIP_ADIA if viscous_sphere else BC_SLIP, seed=seed + 1 + k)
            cond = sphere_conditions(mach, Re if viscous_sphere else None)
        out.append(dict(kind=kind, n=n, mesh=mesh, cond=cond, n_cells=mesh.n_tet, mach=mach, Re=Re))
    return out


def serving_requests(n_requests: int = 24, n_min: float = 30e3, n_max: float = 250e3, rate: float = 1.0,
                     seed: int = BASE_SEED + 500, viscous_fraction: float = 0.5, cavity_fraction: float = 0.0):
    """Steady-solve requests with Poisson arrivals (exponential gaps of mean 1/rate s).
    A fraction `cavity_fraction` are lid-driven cavities (Mach ~ U(0.2, 0.5) of the
    lid, Re ~ log-uniform in [50, 1000], n = (N/6)^(1/3) Kuhn-split hexahedra a
    side); the rest are spheres, inviscid (Mach ~ U(0.2, 0.5), angle of attack ~
    U(0, 10) deg) or, a fraction `viscous_fraction` of them, viscous (Mach ~ U(0.2,
    0.5), Re ~ log-uniform in [50, 1000]); N ~ log-uniform in [n_min, n_max] tets
    (sphere patches n = (N/72)^(1/3), 2n layers). With cavity_fraction 0 the draws
    are those of the sphere-only stream. Returns dicts: arrival (s), kind, mesh,
    cond, n_cells."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate)
        N = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        mach = rng.uniform(0.2, 0.5)
        if cavity_fraction > 0.0 and rng.random() < cavity_fraction:
            kind = "cavity"
            cond = cavity_conditions(mach, math.exp(rng.uniform(math.log(50.0), math.log(1000.0))))
            mesh = cavity_mesh(max(2, int(round((N / 6.0) ** (1.0 / 3.0)))), seed=seed + 1 + k)
            out.append(dict(arrival=t, kind=kind, mesh=mesh, cond=cond, n_cells=mesh.n_tet))
            continue
        n = max(2, int(round((N / 72.0) ** (1.0 / 3.0))))
        if rng.random() < 1.0 - viscous_fraction:
            kind = "inviscid sphere"
            cond = sphere_conditions(mach, None, aoa_deg=rng.uniform(0.0, 10.0))
            wall = BC_SLIP
        else:
            kind = "viscous sphere"
            cond = sphere_conditions(mach, math.exp(rng.uniform(math.log(50.0), math.log(1000.0))))
            wall = BC_NOSLIP_ADIA
        mesh = sphere_mesh(n, 2 * n, stretch=sphere_stretch(2 * n), wall_tag=wall, seed=seed + 1 + k)
        out.append(dict(arrival=t, kind=kind, mesh=mesh, cond=cond, n_cells=mesh.n_tet))
    return out
