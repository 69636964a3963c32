"""The seeded input generators (paper_2304_09485_gb300/inputs.py) that stand in
for the paper's workloads: cell counts, positive volumes, conforming splits
(every interior triangle shared by exactly two tetrahedra, also across the
cubed-sphere patch seams), boundary triangles and tags, periodic pairing and
determinism. CPU only."""
import math

import numpy as np
import pytest

from paper_2304_09485_gb300 import inputs as I


def signed_vol6(m):
    V = m.xyz[m.tet4]
    return np.einsum("ij,ij->i", V[:, 1] - V[:, 0], np.cross(V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]))


def triangle_counts(m):
    tri = np.sort(np.concatenate([np.delete(m.tet4, k, axis=1) for k in range(4)]), axis=1)
    keys, counts = np.unique(tri, axis=0, return_counts=True)
    return keys, counts


def as_set(rows):
    return {tuple(r) for r in np.sort(rows, axis=1)}


@pytest.mark.parametrize("n", [2, 3])
def test_cavity_mesh(n):
    m = I.cavity_mesh(n)
    assert m.n_tet == 6 * n ** 3
    v6 = signed_vol6(m)
    assert np.all(v6 > 0) and v6.sum() / 6 == pytest.approx(1.0, rel=1e-12)
    keys, counts = triangle_counts(m)
    assert set(counts.tolist()) <= {1, 2}
    assert as_set(keys[counts == 1]) == as_set(m.bface3) and len(m.bface3) == 12 * n * n
    # the lid y = 1 carries the lid tag, the other five walls the isothermal tag
    cy = m.xyz[m.bface3][:, :, 1].mean(1)
    assert np.all(m.btag[np.isclose(cy, 1.0)] == I.BC_WALL_LID)
    assert np.all(m.btag[~np.isclose(cy, 1.0)] == I.BC_WALL_ISO)
    assert int((m.btag == I.BC_WALL_LID).sum()) == 2 * n * n


def test_periodic_cube_mesh_pairs_its_open_faces():
    n, Lb = 3, 2.0
    m = I.periodic_cube_mesh(n, length=Lb)
    assert m.n_tet == 6 * n ** 3 and len(m.bface3) == 0
    v6 = signed_vol6(m)
    assert np.all(v6 > 0) and v6.sum() / 6 == pytest.approx(Lb ** 3, rel=1e-12)
    keys, counts = triangle_counts(m)
    open_ = keys[counts == 1]
    assert len(open_) == 6 * 2 * n * n                  # two triangles per boundary square, six sides
    # every open triangle has a partner translated by one of the periodic shifts
    cen = {tuple(np.round(m.xyz[t].mean(0), 9)) for t in open_}
    shifts = np.asarray(m.periodic_shift)
    for t in open_:
        c = m.xyz[t].mean(0)
        assert any(tuple(np.round(c + s, 9)) in cen or tuple(np.round(c - s, 9)) in cen for s in shifts)


@pytest.mark.parametrize("n,layers", [(3, 4), (4, 6)])
def test_sphere_mesh_is_conforming_across_patch_seams(n, layers):
    r_in, r_out = 0.5, 10.0
    m = I.sphere_mesh(n, layers, r_in=r_in, r_out=r_out, stretch=1.3)
    assert m.n_tet == 6 * n * n * layers * 6            # the cell count of 6 tetrahedra per hexahedron
    v6 = signed_vol6(m)
    assert np.all(v6 > 0)
    vol = v6.sum() / 6
    exact = 4 / 3 * math.pi * (r_out ** 3 - r_in ** 3)
    assert 0.5 * exact < vol < exact                     # an inscribed polyhedral shell
    keys, counts = triangle_counts(m)
    assert set(counts.tolist()) <= {1, 2}               # no triangle shared by three cells, none left unmatched inside
    assert as_set(keys[counts == 1]) == as_set(m.bface3) and len(m.bface3) == 24 * n * n
    r = np.linalg.norm(m.xyz[m.bface3].mean(1), axis=1)
    assert np.all(m.btag[r < 1.0] == I.BC_SLIP) and np.all(m.btag[r > 1.0] == I.BC_FARFIELD)


def test_default_sphere_is_the_benchmark_size():
    """The 6 x 32 x 32 x 64 O-grid gives 2,359,296 tetrahedra (the count follows the
    formula checked on small grids above; the default mesh is not generated here)."""
    assert 6 * 32 * 32 * 64 * 6 == 2_359_296


def test_sphere_stretch_and_radii():
    s = I.sphere_stretch(48, dr1=3e-2)
    rad = I.sphere_radii(48, 0.5, 10.0, s)
    assert rad[1] - rad[0] == pytest.approx(3e-2, rel=1e-9)
    assert rad[-1] == pytest.approx(10.0, rel=1e-12) and np.all(np.diff(rad) > 0)
    assert np.allclose(np.diff(rad)[1:] / np.diff(rad)[:-1], s)


def test_generators_are_deterministic():
    a, b = I.cavity_mesh(3), I.cavity_mesh(3)
    assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.tet4, b.tet4)
    c = I.cavity_mesh(3, seed=I.BASE_SEED + 99)
    assert not np.array_equal(a.xyz, c.xyz)
    Q1, G1 = I.smooth_state(a)
    Q2, G2 = I.smooth_state(b)
    assert np.array_equal(Q1, Q2) and np.array_equal(G1, G2)


def test_serving_stream_with_cavities():
    """The cavity fraction adds lid-driven cavities to the request stream; with
    fraction 0 the stream is the sphere-only one, draw for draw."""
    a = I.serving_requests(12, n_min=50e3, n_max=150e3, rate=0.05)
    b = I.serving_requests(12, n_min=50e3, n_max=150e3, rate=0.05, cavity_fraction=0.0)
    assert [(r["kind"], r["n_cells"], r["arrival"]) for r in a] == [(r["kind"], r["n_cells"], r["arrival"]) for r in b]
    c = I.serving_requests(40, n_min=50e3, n_max=150e3, rate=0.05, cavity_fraction=0.5)
    kinds = [r["kind"] for r in c]
    assert 10 <= kinds.count("cavity") <= 30
    for r in c:
        if r["kind"] == "cavity":
            assert r["cond"]["lid_speed"] == 1.0 and r["cond"]["viscous"] == 1
            assert 40e3 <= r["n_cells"] <= 190e3 and r["n_cells"] % 6 == 0
            assert 50.0 <= 1.0 / r["cond"]["mu"] <= 1000.0


def test_hex_generators():
    """Hexahedra are positively oriented; boundary quadrilaterals cover the box
    surface; the tilted-plane cells have planar faces."""
    for m in (I.hex_cavity_mesh(4), I.hex_tilted_box_mesh(4), I.hex_periodic_cube_mesh(3)):
        x = m.xyz[m.hex8]
        assert np.all(np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 3] - x[:, 0]), x[:, 4] - x[:, 0]) > 0)
        assert len(np.unique(m.hex8)) == len(m.xyz)
    m = I.hex_cavity_mesh(4)
    assert m.bface4.shape == (6 * 16, 4) and np.all(m.btag[m.btag != I.BC_WALL_LID] == I.BC_WALL_ISO)
    t = I.hex_tilted_box_mesh(5)
    for F in ([0, 1, 2, 3], [0, 1, 5, 4], [1, 2, 6, 5], [2, 3, 7, 6], [3, 0, 4, 7], [4, 5, 6, 7]):
        P = t.xyz[t.hex8][:, F]
        n = np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 1])
        assert np.abs(np.einsum("ij,ij->i", n, P[:, 1] - P[:, 0])).max() <= 1e-14
