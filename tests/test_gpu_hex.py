"""Parity of the CUDA path with the FP64 oracle on hexahedral meshes (Sec. 3.1:
six faces per cell, the eight non-compact sub-stencils of three face
neighbours, one compact sub-stencil per face, 2 x 2 Gauss points per face).

Tolerances are those of the tetrahedral parity tests: residual components
against their flux scale sum_p S_p |F_Euler(Q_i) . n_p|, gradients against
|Q_i| sum_p S_p / |Omega_i|, a step's update in relative L2.
"""
import numpy as np
import pytest

import oracle as O
import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TOL_R = 1e-11
TOL_R_FLUX = 2e-12
MIXED_DQ = 1e-4


def face_sums(om, Q):
    """Per cell: sum over its faces of S |F_Euler(Q_i) . n| (flux scale) and of S."""
    fg = om.face_geometry()
    rho = Q[:, 0]
    u = Q[:, 1:4] / rho[:, None]
    p = (GAMMA - 1) * (Q[:, 4] - 0.5 * rho * np.einsum("ij,ij->i", u, u))
    scale, area = np.zeros_like(Q), np.zeros(len(Q))
    for side in ("left", "right"):
        c = fg[side]
        ok = c >= 0
        ci, n, S = c[ok], fg["normal"][ok], fg["area"][ok]
        un = np.einsum("ij,ij->i", u[ci], n)
        F = np.stack([rho[ci] * un, rho[ci] * u[ci, 0] * un + p[ci] * n[:, 0], rho[ci] * u[ci, 1] * un + p[ci] * n[:, 1],
                      rho[ci] * u[ci, 2] * un + p[ci] * n[:, 2], (Q[ci, 4] + p[ci]) * un], -1)
        np.add.at(scale, ci, S[:, None] * np.abs(F))
        np.add.at(area, ci, S)
    return scale, area / om.vol


MESHES = {
    "hexcav5": lambda: (I.hex_cavity_mesh(5, jitter=0.15), I.cavity_conditions()),
    "hexper4": lambda: (I.hex_periodic_cube_mesh(4, jitter=0.15), I.sphere_conditions(0.3)),
    "hextilt6": lambda: (I.hex_tilted_box_mesh(6), I.sphere_conditions(0.3)),
}
_cache = {}


def setup(name):
    if name not in _cache:
        m, cond = MESHES[name]()
        hm = H.hgks_mesh_create(m, scheme_mask=3)
        assert H.hgks_mesh_info(hm).faces_per_cell == 6
        _cache[name] = (m, cond, O.OracleMesh(m), hm)
    return _cache[name]


def state(m, cond, seed=1):
    base = (cond["rho_inf"], cond["u_inf"][0] + 0.1, cond["u_inf"][1] + 0.05, -0.03, cond["p_inf"])
    return I.smooth_state(m, seed=I.BASE_SEED + seed, amp=0.05, base=base)


CASES = [
    ("hexcav5", dict(scheme=0)), ("hexcav5", dict(scheme=1)),
    ("hexcav5", dict(scheme=1, Pr=0.72)), ("hexcav5", dict(scheme=0, weights=1, Pr=0.72)),
    ("hexper4", dict(scheme=0)), ("hexper4", dict(scheme=1, characteristic=0)),
    ("hextilt6", dict(scheme=0)), ("hextilt6", dict(scheme=1, weights=1)),
    ("hextilt6", dict(scheme=1, flux_dt=1e-3)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[f"{n}-{'-'.join(f'{k}{v}' for k, v in kw.items())}" for n, kw in CASES])
def test_hex_residual_parity(cuda, name, kw):
    import torch
    m, cond, om, hm = setup(name)
    Q, G = state(m, cond)
    po = O.make_params(**{**cond, **kw})
    ph = H.hgks_default_params(**{**cond, **kw})
    out = om.residual(po, Q, G)
    Ro, Go = (out if kw.get("scheme") == 1 else (out, None))
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    Rd, Gn = torch.empty_like(Qd), torch.empty_like(Gd)
    H.hgks_residual(hm, ph, Qd, Gd if kw.get("scheme") == 1 else None, Rd, Gn if kw.get("scheme") == 1 else None)
    torch.cuda.synchronize()
    scale, aov = face_sums(om, Q)
    err = np.abs(hm.to_caller(Rd) - Ro) / scale
    assert err.max() <= TOL_R_FLUX, f"max rel err {err.max():.3e}"
    if kw.get("scheme") == 1:
        gs = np.repeat(np.abs(Q), 3, axis=1) * aov[:, None]
        gerr = np.abs(hm.to_caller(Gn) - Go) / gs
        assert gerr.max() <= TOL_R, f"gradient max rel err {gerr.max():.3e}"


def test_hex_free_stream_on_gpu(cuda):
    """A uniform state on the jittered periodic hexahedra: R = 0 and G_new = 0 to rounding."""
    import torch
    m, cond, om, hm = setup("hexper4")
    Q = I.uniform_state(m.n_cells, rho=1.1, u=0.3, v=-0.2, w=0.1, p=0.9)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(np.zeros((m.n_cells, 15)))
    Rd, Gn = torch.empty_like(Qd), torch.empty_like(Gd)
    H.hgks_residual(hm, H.hgks_default_params(scheme=1), Qd, Gd, Rd, Gn)
    torch.cuda.synchronize()
    assert Rd.abs().max().item() <= 1e-13 and Gn.abs().max().item() <= 1e-12


def test_hex_local_dt_and_jacobian_parity(cuda):
    import torch
    for name, kw in [("hexcav5", dict(scheme=1, Pr=0.72)), ("hextilt6", dict(scheme=0))]:
        m, cond, om, hm = setup(name)
        Q, _ = state(m, cond, seed=5)
        po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(**{**cond, **kw})
        Qd = hm.to_internal(Q)
        dtd = torch.empty(hm.n_cells, dtype=torch.float64, device="cuda")
        H.hgks_local_dt(hm, ph, Qd, dtd)
        dto = om.local_dt(po, Q)
        np.testing.assert_allclose(dtd.cpu().numpy()[hm.inv], dto, rtol=1e-13)
        diag = torch.empty(25, hm.n_cells, dtype=torch.float64, device="cuda")
        off = torch.empty(150, hm.n_cells, dtype=torch.float64, device="cuda")
        H.hgks_assemble(hm, ph, Qd, dtd, diag, off)
        torch.cuda.synchronize()
        Do, Oo = om.jacobian(po, Q, dto)
        Dg = diag.cpu().numpy().T[hm.inv].reshape(-1, 5, 5)
        Og = off.cpu().numpy().T[hm.inv].reshape(-1, 6, 5, 5)
        dscale = np.abs(Do).max(axis=(1, 2))[:, None, None]
        assert (np.abs(Dg - Do) / dscale).max() <= 1e-12
        assert (np.abs(Og - Oo) / dscale[:, None]).max() <= 1e-12
        x = np.random.default_rng(7).normal(size=Q.shape)
        xd = hm.to_internal(x)
        yd, zd = torch.empty_like(xd), torch.empty_like(xd)
        H.hgks_apply_jacobian(hm, xd, yd)
        H.hgks_precondition(hm, 2, xd, zd)
        torch.cuda.synchronize()
        yo = np.einsum("nij,nj->ni", Do, x)
        nb = om.neighbours
        for q in range(6):
            ok = nb[:, q] >= 0
            yo[ok] += np.einsum("nij,nj->ni", Oo[ok, q], x[nb[ok, q]])
        ysc = np.abs(Do).max(axis=(1, 2))[:, None] * np.abs(x).max()
        assert (np.abs(hm.to_caller(yd) - yo) / ysc).max() <= 1e-12
        zo = om.precondition(Do, Oo, 2, x)
        np.testing.assert_allclose(hm.to_caller(zd), zo, rtol=1e-10, atol=1e-12 * np.abs(zo).max())


@pytest.mark.parametrize("name,kw", [("hexcav5", dict(scheme=1, Pr=0.72)), ("hextilt6", dict(scheme=0, krylov_dim=20)),
                                     ("hexcav5", dict(scheme=0, Pr=0.72, jacobi_sweeps=1)),
                                     ("hexcav5", dict(scheme=1, Pr=0.72, grad_relax=0.5))])
def test_hex_gmres_step_parity(cuda, name, kw):
    import torch
    m, cond, om, hm = setup(name)
    Q, G = state(m, cond, seed=9)
    po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(**{**cond, **kw})
    Qo, Go, reso, dQo = om.gmres_step(po, Q, G)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    dQd = torch.empty_like(Qd)
    info = H.hgks_gmres_step(hm, ph, Qd, Gd if kw["scheme"] == 1 else None, dQd)
    assert info.res_l1 == pytest.approx(reso, rel=1e-11)
    rel = np.linalg.norm(hm.to_caller(dQd) - dQo) / np.linalg.norm(dQo)
    assert rel <= 1e-9, rel
    if kw["scheme"] == 1:
        assert np.linalg.norm(hm.to_caller(Gd) - Go) / np.linalg.norm(Go) <= 1e-11
    # the FP32 Krylov part: the same step to the mixed-precision tolerance
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    H.hgks_gmres_step(hm, H.hgks_default_params(**{**cond, **kw, "precision": 1}), Qd,
                      Gd if kw["scheme"] == 1 else None, dQd)
    rel32 = np.linalg.norm(hm.to_caller(dQd) - dQo) / np.linalg.norm(dQo)
    assert rel32 <= MIXED_DQ, rel32


def test_hex_steps_track_oracle(cuda):
    """Five consecutive implicit steps of the lid-driven hexahedral cavity (compact)."""
    m, cond, om, hm = setup("hexcav5")
    kw = dict(scheme=1, Pr=0.72)
    po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(**{**cond, **kw})
    Q = I.state_from_conditions(m.n_cells, cond); G = np.zeros((m.n_cells, 15))
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    for k in range(5):
        Q, G, res, _ = om.gmres_step(po, Q, G)
        info = H.hgks_gmres_step(hm, ph, Qd, Gd)
        # the cavity starts at rest: the first residual is rounding only
        assert info.res_l1 == pytest.approx(res, rel=1e-9, abs=1e-12)
    assert np.linalg.norm(hm.to_caller(Qd) - Q) / np.linalg.norm(Q) <= 1e-9


def test_hex_matrix_free_product(cuda):
    """Eq. (frechet) on hexahedra: the GPU's product against the oracle's."""
    import torch
    m, cond, om, hm = setup("hextilt6")
    kw = dict(scheme=1, jv_mode=1)
    Q, G = state(m, cond, seed=13)
    x = np.random.default_rng(I.BASE_SEED + 82).normal(size=Q.shape) * np.abs(Q).mean(0)
    ph = H.hgks_default_params(**{**cond, **kw}); po = O.make_params(**{**cond, **kw})
    dt = om.local_dt(po, Q)
    Qd, Gd, xd = hm.to_internal(Q), hm.to_internal(G), hm.to_internal(x)
    dtd = hm.to_internal(dt[:, None])[0].contiguous()
    yd = torch.empty_like(Qd)
    H.hgks_apply_jacobian_fd(hm, ph, Qd, Gd, dtd, xd, yd)
    torch.cuda.synchronize()
    yo, so = om.apply_fd(po, Q, G, dt, x)
    scale, _ = face_sums(om, Q)
    err = np.abs(hm.to_caller(yd) - yo) / (scale / so)
    assert err.max() <= 2 * TOL_R, err.max()


def test_hex_noalloc_and_mixed_batches(cuda):
    """The no-allocation residual of a hexahedral mesh equals hgks_residual bit for
    bit; a batch holds one cell kind: hexahedra mixed with tetrahedra are refused
    with HGKS_ERR_ARG before any work."""
    import torch
    m, cond, om, hm = setup("hexcav5")
    ph = H.hgks_default_params(scheme=1, Pr=0.72, **cond)
    Q, G = state(m, cond, seed=23)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    R1, R2 = torch.empty_like(Qd), torch.empty_like(Qd)
    G1, G2 = torch.empty_like(Gd), torch.empty_like(Gd)
    H.hgks_residual(hm, ph, Qd, Gd, R1, G1)
    H.hgks_residual_noalloc(hm, ph, Qd, Gd, R2, G2)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2) and torch.equal(G1, G2)
    ph = H.hgks_default_params(**cond)
    tet = H.hgks_mesh_create(I.cavity_mesh(3), scheme_mask=3)
    with pytest.raises(H.HGKSError) as e:
        H.hgks_batch_create([tet, hm], [ph, ph])
    assert e.value.status == 1
    b = H.hgks_batch_create([tet], [ph])
    with pytest.raises(H.HGKSError) as e:
        H.hgks_batch_add(b, hm, ph)
    assert e.value.status == 1


def _hex_batch(kw, seed):
    """Three hexahedral problems of different size and kind in one batch, and
    the same problems as single meshes (states and handles)."""
    import torch
    probs = [(I.hex_cavity_mesh(4, seed=I.BASE_SEED + seed), I.cavity_conditions(0.15, 100.0)),
             (I.hex_cavity_mesh(5, seed=I.BASE_SEED + seed + 1), I.cavity_conditions(0.2, 100.0)),
             (I.hex_sphere_mesh(4, 6, stretch=I.sphere_stretch(6, dr1=6e-2)), I.sphere_conditions(0.2535, Re=118.0))]
    meshes, params, singles = [], [], []
    for k, (m, cond) in enumerate(probs):
        hm = H.hgks_mesh_create(m, scheme_mask=3)
        p = H.hgks_default_params(Pr=0.72, **cond, **kw)
        Q, G = state(m, cond, seed=seed + k)
        meshes.append(hm); params.append(p); singles.append((hm, p, hm.to_internal(Q), hm.to_internal(G)))
    b = H.hgks_batch_create(meshes, params)
    for k, (hm, p, Qd, Gd) in enumerate(singles):
        H.hgks_batch_set_state(b, k, Qd, Gd)
    torch.cuda.synchronize()
    return b, singles


@pytest.mark.parametrize("precision", [0, 1])
def test_hex_batch_step_equals_single(cuda, precision):
    """One batched implicit step of three hexahedral meshes (compact scheme) equals
    each mesh's step alone: the residual norm to 1e-13, the update to 1e-10 (FP64;
    2e-4 with the FP32 Krylov part, whose sums run in another order); replayed
    from the batch's CUDA graph it equals the eager step bit for bit."""
    import torch
    kw = dict(scheme=1, krylov_dim=8, restarts=2, precision=precision)
    b, singles = _hex_batch(kw, seed=310)
    Q0 = [Qd.clone() for _, _, Qd, _ in singles]
    G0 = [Gd.clone() for _, _, _, Gd in singles]
    infos = H.hgks_batch_gmres_step(b, use_graph=False)
    tol = 1e-10 if precision == 0 else 2e-4
    for k, (hm, p, Qd, Gd) in enumerate(singles):
        si = H.hgks_gmres_step(hm, p, Qd, Gd)
        Qb = torch.empty_like(Qd)
        H.hgks_batch_get_state(b, k, Q=Qb)
        torch.cuda.synchronize()
        assert abs(infos[k].res_l1 - si.res_l1) <= 1e-13 * si.res_l1
        rel = (torch.linalg.norm((Qb - Q0[k]) - (Qd - Q0[k])) / torch.linalg.norm(Qd - Q0[k])).item()
        assert rel <= tol, (k, rel)
    out = {}
    for mode in (False, True):
        for k in range(len(singles)):
            H.hgks_batch_set_state(b, k, Q0[k], G0[k])
        H.hgks_batch_gmres_step(b, use_graph=mode)
        Qs = [torch.empty_like(q) for q in Q0]
        for k in range(len(singles)):
            H.hgks_batch_get_state(b, k, Q=Qs[k])
        torch.cuda.synchronize()
        out[mode] = Qs
    assert all(torch.equal(a, c) for a, c in zip(out[False], out[True]))


def test_hex_batch_solve_converges_like_alone(cuda):
    """Three hexahedral problems solved together to a 1e-5 drop (FP64, compact):
    each converges with the step count, history (1e-9 of its reference) and state
    (1e-9) it has alone."""
    import torch
    kw = dict(scheme=1, krylov_dim=10, restarts=3)
    b, singles = _hex_batch(kw, seed=320)
    starts = [(Qd.clone(), Gd.clone()) for _, _, Qd, Gd in singles]
    infos, hist, ok = H.hgks_batch_solve_steady(b, 1e-5, 2000)
    assert ok
    for k, (hm, p, Qd, Gd) in enumerate(singles):
        Q, G = starts[k][0].clone(), starts[k][1].clone()
        si, hs, conv = H.hgks_solve_steady(hm, p, Q, G, drop_tol=1e-5, max_steps=2000)
        assert conv and infos[k].converged and infos[k].steps == si.steps, (k, infos[k].steps, si.steps)
        np.testing.assert_allclose(hist[k][: si.steps + 1], hs, rtol=0, atol=1e-9 * hs.max())
        Qb, Gb = torch.empty_like(Q), torch.empty_like(G)
        H.hgks_batch_get_state(b, k, Q=Qb, G=Gb)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(Qb - Q) / torch.linalg.norm(Q)).item() <= 1e-9
        assert (torch.linalg.norm(Gb - G) / torch.linalg.norm(G)).item() <= 1e-9


@pytest.mark.parametrize("scheme", [1, 0])
def test_hex_cavity_solve_to_1e8_parity(cuda, scheme):
    """Algorithm 1 to a 1e-8 drop on the 64-hexahedron lid-driven cavity (Ma 0.15,
    Re 100, CFL 10; the oracle converges in 742 (compact) and 754 (non-compact)
    steps): the same step count on the GPU, histories within 1e-8, states within 1e-9."""
    m = I.hex_cavity_mesh(4, jitter=0.1)
    cond = I.cavity_conditions()
    om, hm = O.OracleMesh(m), H.hgks_mesh_create(m, scheme_mask=3)
    kw = dict(scheme=scheme, Pr=0.72)
    Q0 = I.state_from_conditions(m.n_cells, cond)
    G0 = np.zeros((m.n_cells, 15))
    Qo, _, hist_o, conv_o = om.solve_steady(O.make_params(**{**cond, **kw}), Q0, G0 if scheme else None,
                                            drop=1e-8, max_steps=1000)
    Qd, Gd = hm.to_internal(Q0), hm.to_internal(G0)
    info, hist_g, conv_g = H.hgks_solve_steady(hm, H.hgks_default_params(**{**cond, **kw}), Qd,
                                               Gd if scheme else None, drop_tol=1e-8, max_steps=1000)
    assert conv_o and conv_g and info.steps > 500
    assert info.steps == len(hist_o) - 1
    np.testing.assert_allclose(hist_g, hist_o, rtol=1e-8, atol=1e-12 * hist_o.max())
    assert np.linalg.norm(hm.to_caller(Qd) - Qo) / np.linalg.norm(Qo) <= 1e-9


def test_hex_sphere_converged_steady_state_fp64_mixed_and_oracle(cuda):
    """The viscous sphere of Sec. 5.2 (Re 118, Ma 0.2535, linear weights, CFL 20,
    compact HWENO) on a scaled-down hexahedral O-grid of the same construction
    (6 x 4 x 4 patches, 6 layers, 576 cells): Algorithm 1 to a 1e-8 drop in the
    oracle (636 steps), on the GPU in FP64 (the same steps, histories within
    1e-8, state within 1e-9, drag coefficient within 1e-10) and with the FP32
    Krylov part (a converged state is fixed by the FP64 residual: state within
    1e-8, drag within 1e-9)."""
    import math
    m = I.hex_sphere_mesh(4, 6, stretch=I.sphere_stretch(6, dr1=6e-2))
    cond = I.sphere_conditions(0.2535, Re=118.0)
    kw = dict(scheme=1, weights=1, Pr=0.72, cfl=20.0)
    om, hm = O.OracleMesh(m), H.hgks_mesh_create(m, scheme_mask=2)
    Q0, G0 = I.state_from_conditions(m.n_cells, cond), np.zeros((m.n_cells, 15))
    po = O.make_params(**{**cond, **kw})
    Qo, Go, hist_o, conv_o = om.solve_steady(po, Q0, G0, drop=1e-8, max_steps=1500)
    assert conv_o
    qinf = 0.5 * cond["u_inf"][0] ** 2 * math.pi * 0.25
    cd_o = om.wall_force(po, Qo, Go, I.BC_NOSLIP_ADIA)[0] / qinf
    out = {}
    for prec in (0, 1):
        ph = H.hgks_default_params(**{**cond, **kw, "precision": prec})
        Qd, Gd = hm.to_internal(Q0), hm.to_internal(G0)
        info, hist_g, conv_g = H.hgks_solve_steady(hm, ph, Qd, Gd, drop_tol=1e-8, max_steps=1500)
        assert conv_g
        cd_g = H.hgks_wall_force(hm, ph, Qd, Gd, I.BC_NOSLIP_ADIA)[0] / qinf
        out[prec] = (info.steps, hist_g, hm.to_caller(Qd), cd_g)
    steps, hist_g, Qg, cd_g = out[0]
    assert steps == len(hist_o) - 1
    np.testing.assert_allclose(hist_g, hist_o, rtol=1e-8, atol=1e-12 * hist_o.max())
    assert np.linalg.norm(Qg - Qo) / np.linalg.norm(Qo) <= 1e-9
    assert abs(cd_g - cd_o) <= 1e-10 * abs(cd_o)
    _, _, Q32, cd32 = out[1]
    assert np.linalg.norm(Q32 - Qo) / np.linalg.norm(Qo) <= 1e-8
    assert abs(cd32 - cd_o) <= 1e-9 * abs(cd_o)


def test_hex_host_variants_resume_and_wall_force(cuda):
    """The rest of the single-mesh API on hexahedra: the host-buffer residual and
    step equal the device ones bit for bit, a solve resumed from a host snapshot
    equals the uninterrupted one bit for bit, and the wall force matches the
    oracle's (1e-11 of its size)."""
    import torch
    m, cond, om, hm = setup("hexcav5")
    Q, G = state(m, cond, seed=17)
    p = H.hgks_default_params(scheme=1, Pr=0.72, krylov_dim=6, restarts=2, **cond)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    Rd, Gn = torch.empty_like(Qd), torch.empty_like(Gd)
    H.hgks_residual(hm, p, Qd, Gd, Rd, Gn)
    torch.cuda.synchronize()
    Qh, Gh = np.ascontiguousarray(Qd.cpu().numpy()), np.ascontiguousarray(Gd.cpu().numpy())
    Rh, Gnh = np.zeros_like(Qh), np.zeros_like(Gh)
    H.hgks_residual_host(hm, p, Qh, Gh, Rh, Gnh)
    assert np.array_equal(Rh, Rd.cpu().numpy()) and np.array_equal(Gnh, Gn.cpu().numpy())
    info_d = H.hgks_gmres_step(hm, p, Qd, Gd)
    info_h = H.hgks_gmres_step_host(hm, p, Qh, Gh)
    torch.cuda.synchronize()
    assert info_h.res_l1 == info_d.res_l1 and np.array_equal(Qh, Qd.cpu().numpy())
    # checkpoint / resume
    Qa, Ga = hm.to_internal(Q), hm.to_internal(G)
    ia, ha, _ = H.hgks_solve_steady(hm, p, Qa, Ga, drop_tol=1e-12, max_steps=10)
    Qb, Gb = hm.to_internal(Q), hm.to_internal(G)
    i5, h5, _ = H.hgks_solve_steady(hm, p, Qb, Gb, drop_tol=1e-12, max_steps=5)
    Qc, Gc = torch.from_numpy(Qb.cpu().numpy().copy()).cuda(), torch.from_numpy(Gb.cpu().numpy().copy()).cuda()
    ib, hb, _ = H.hgks_solve_resume(hm, p, Qc, Gc, i5, drop_tol=1e-12, max_steps=10)
    torch.cuda.synchronize()
    assert ib.steps == ia.steps == 10 and torch.equal(Qc, Qa) and torch.equal(Gc, Ga)
    np.testing.assert_array_equal(hb[5:], ha[5:])
    # wall force on the lid and on the other walls
    po = O.make_params(scheme=1, Pr=0.72, krylov_dim=6, restarts=2, **cond)
    for tag in (I.BC_WALL_LID, I.BC_WALL_ISO):
        fo = om.wall_force(po, Q, G, tag)
        fg = H.hgks_wall_force(hm, p, hm.to_internal(Q), hm.to_internal(G), tag)
        assert np.abs(fg - fo).max() <= 1e-11 * np.abs(fo).max()


def test_hex_server_results_equal_alone(cuda):
    """A server of hexahedral meshes (hgks_server_create_hex): three requests of
    different size and kind, each served result equals the same solve alone
    (steps, convergence, state within 1e-9); a tetrahedral request to it, and a
    hexahedral one to a tetrahedral server, are refused with HGKS_ERR_ARG."""
    import time
    import torch
    kw = dict(scheme=0, krylov_dim=8, restarts=2, jacobi_sweeps=2)
    probs = [(I.hex_cavity_mesh(4, seed=I.BASE_SEED + 330), I.cavity_conditions(0.2, 100.0)),
             (I.hex_cavity_mesh(5, seed=I.BASE_SEED + 331), I.cavity_conditions(0.3, 200.0)),
             (I.hex_sphere_mesh(4, 6, stretch=I.sphere_stretch(6, dr1=6e-2)), I.sphere_conditions(0.3))]
    srv = H.hgks_server(H.hgks_default_params(**kw), hbm_budget_bytes=int(400e6), max_inflight=4, hexahedra=True)
    ids, reqs = [], []
    for k, (m, cond) in enumerate(probs):
        p = H.hgks_default_params(**{**cond, "Pr": 0.72 if cond["viscous"] else 1.0, **kw})
        Q0, _ = state(m, cond, seed=340 + k)
        ids.append(srv.submit(m, p, Q0, drop_tol=1e-3, max_steps=60))
        reqs.append((m, p, Q0))
    rounds = 0
    while True:
        fin, run, wait = srv.step()
        rounds += 1
        if run == 0 and wait == 0:
            break
        if run == 0:
            time.sleep(0.005)
        assert rounds < 5000
    for rid, (m, p, Q0) in zip(ids, reqs):
        st = srv.status(rid)
        assert st.state == 3
        Qs, _ = srv.collect(rid)
        hm = H.hgks_mesh_create(m, scheme_mask=1)
        Qd = hm.to_internal(Q0)
        info, _, conv = H.hgks_solve_steady(hm, p, Qd, None, drop_tol=1e-3, max_steps=60)
        torch.cuda.synchronize()
        assert st.solve.steps == info.steps and bool(st.solve.converged) == bool(conv)
        Qa = hm.to_caller(Qd)
        assert np.linalg.norm(Qs - Qa) / np.linalg.norm(Qa) <= 1e-9
    tm, tc = I.cavity_mesh(3), I.cavity_conditions()
    tp = H.hgks_default_params(**{**tc, "Pr": 0.72, **kw})
    with pytest.raises(H.HGKSError) as e:
        srv.submit(tm, tp, I.state_from_conditions(tm.n_tet, tc))
    assert e.value.status == 1
    tsrv = H.hgks_server(H.hgks_default_params(**kw), hbm_budget_bytes=int(200e6), max_inflight=2)
    m, p, Q0 = reqs[0]
    with pytest.raises(H.HGKSError) as e:
        tsrv.submit(m, p, Q0)
    assert e.value.status == 1


def test_hex_empty_batch_add_step_equals_single(cuda):
    """An empty hexahedral batch (hgks_batch_create_empty_hex) filled with
    hgks_batch_add: one batched step equals each mesh's step alone (FP64, 1e-10);
    a tetrahedral mesh is refused."""
    import torch
    kw = dict(scheme=0, krylov_dim=8, restarts=2)
    shared = H.hgks_default_params(**kw)
    b = H.hgks_batch_create_empty(20000, 80000, 4, shared, hexahedra=True)
    singles = []
    for k, (m, cond) in enumerate([(I.hex_cavity_mesh(4, seed=I.BASE_SEED + 350), I.cavity_conditions(0.2, 100.0)),
                                   (I.hex_tilted_box_mesh(5), I.sphere_conditions(0.3))]):
        hm = H.hgks_mesh_create(m, scheme_mask=1)
        p = H.hgks_default_params(Pr=0.72 if cond["viscous"] else 1.0, **cond, **kw)
        slot = H.hgks_batch_add(b, hm, p)
        Q, _ = state(m, cond, seed=360 + k)
        Qd = hm.to_internal(Q)
        H.hgks_batch_set_state(b, slot, Qd)
        singles.append((slot, hm, p, Qd))
    infos = H.hgks_batch_gmres_step(b, use_graph=False)
    for slot, hm, p, Qd in singles:
        Q0 = Qd.clone()
        si = H.hgks_gmres_step(hm, p, Qd, None)
        Qb = torch.empty_like(Qd)
        H.hgks_batch_get_state(b, slot, Q=Qb)
        torch.cuda.synchronize()
        assert abs(infos[slot].res_l1 - si.res_l1) <= 1e-13 * si.res_l1
        rel = (torch.linalg.norm((Qb - Q0) - (Qd - Q0)) / torch.linalg.norm(Qd - Q0)).item()
        assert rel <= 1e-10, rel
    tet = H.hgks_mesh_create(I.cavity_mesh(3), scheme_mask=1)
    with pytest.raises(H.HGKSError) as e:
        H.hgks_batch_add(b, tet, H.hgks_default_params(**kw, **I.cavity_conditions()))
    assert e.value.status == 1
