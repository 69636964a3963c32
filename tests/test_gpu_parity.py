"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance for the residual: the paper's method forms R_i as a sum of face
fluxes that cancel (R = 0 for a uniform flow), so each component is compared
against the size of the terms it is summed from,
    |R_gpu - R_oracle|_{i,c} <= 2e-12 * sum_p S_p |F_Euler(Q_i) . n_p|_c,
a relative error of 2e-12 per residual component with respect to its flux
scale (the measured maximum is 4e-13; the contract's 1e-11 bounds the full-size
sampled cells and the gradients). Relative to the residual itself the two
agree to 2e-11 wherever the face fluxes cancel to no less than 1e-2 of their
size; where they cancel further, rounding of the flux terms (1e-16 of the
flux scale in each of two independent FP64 evaluations) bounds what any two
implementations can share. Gradients from Eq. (derivative) are compared against
|Q_i,c| * sum_p S_p / |Omega_i|.
"""
import numpy as np
import pytest

import oracle as O
import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GAMMA = 1.4
TOL_R = 1e-11          # the contract: gradients, full-size sampled cells
TOL_R_FLUX = 2e-12     # residuals of the parity cases (measured maximum 4e-13)
TOL_R_REL = 2e-11      # relative to |R| where |R| >= 1e-2 of the flux scale


def euler_flux_rows(Q, n):
    rho = Q[:, 0]; u = Q[:, 1:4] / rho[:, None]
    p = (GAMMA - 1) * (Q[:, 4] - 0.5 * rho * np.einsum("ij,ij->i", u, u))
    un = np.einsum("ij,ij->i", u, n)
    return np.stack([rho * un, rho * u[:, 0] * un + p * n[:, 0], rho * u[:, 1] * un + p * n[:, 1],
                     rho * u[:, 2] * un + p * n[:, 2], (Q[:, 4] + p) * un], -1)


def flux_scale(om, Q):
    m = om.mesh
    V = m.xyz[m.tet4]
    s = np.zeros_like(Q)
    for f in range(4):
        F3 = V[:, [k for k in range(4) if k != f]]
        nrm = np.cross(F3[:, 1] - F3[:, 0], F3[:, 2] - F3[:, 0])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        s += area[:, None] * np.abs(euler_flux_rows(Q, nrm / (2 * area[:, None])))
    return s


def area_over_volume(om):
    m = om.mesh
    V = m.xyz[m.tet4]
    tot = 0
    for f in range(4):
        F3 = V[:, [k for k in range(4) if k != f]]
        tot = tot + 0.5 * np.linalg.norm(np.cross(F3[:, 1] - F3[:, 0], F3[:, 2] - F3[:, 0]), axis=1)
    return tot / om.vol


MESHES = {
    "cavity5": lambda: (I.cavity_mesh(5), I.cavity_conditions()),
    "cavity8": lambda: (I.cavity_mesh(8), I.cavity_conditions()),
    "periodic5": lambda: (I.periodic_cube_mesh(5), I.sphere_conditions(0.3)),
    "sphere6x6": lambda: (I.sphere_mesh(6, 6, stretch=1.3), I.sphere_conditions(0.3)),
    "sphere6x6_visc": lambda: (I.sphere_mesh(6, 6, stretch=1.3, wall_tag=I.BC_NOSLIP_ADIA),
                               I.sphere_conditions(0.2535, Re=118.0)),
}
_cache = {}


def setup(name):
    if name not in _cache:
        m, cond = MESHES[name]()
        _cache[name] = (m, cond, O.OracleMesh(m), H.hgks_mesh_create(m, scheme_mask=3))
    return _cache[name]


def state(m, cond, seed=1):
    base = (cond["rho_inf"], cond["u_inf"][0] + 0.1, cond["u_inf"][1] + 0.05, -0.03, cond["p_inf"])
    return I.smooth_state(m, seed=I.BASE_SEED + seed, amp=0.05, base=base)


CASES = [
    ("cavity5", dict(scheme=0)), ("cavity5", dict(scheme=1)),
    ("cavity8", dict(scheme=1)), ("cavity8", dict(scheme=0, weights=1)),
    ("periodic5", dict(scheme=0)), ("periodic5", dict(scheme=1, characteristic=0)),
    ("sphere6x6", dict(scheme=0)), ("sphere6x6", dict(scheme=1, weights=1)),
    ("sphere6x6_visc", dict(scheme=1, Pr=0.72)), ("sphere6x6_visc", dict(scheme=0, Pr=0.72, tstar_end=0)),
    ("cavity8", dict(scheme=1, Pr=0.72, flux_dt=1e-3)),
    # walls colder than the cells' T/1.5 at some cells: their images are held at T_w/2
    ("cavity5", dict(scheme=0, wall_T=21.0)),
    # a monatomic gas: K = (5 - 3 gamma) / (gamma - 1) = 0 internal degrees of freedom
    ("sphere6x6", dict(scheme=0, gamma=5.0 / 3.0)), ("cavity5", dict(scheme=1, gamma=5.0 / 3.0)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[f"{n}-{'-'.join(f'{k}{v}' for k, v in kw.items())}" for n, kw in CASES])
def test_residual_parity(cuda, name, kw):
    m, cond, om, hm = setup(name)
    Q, G = state(m, cond)
    po = O.make_params(**{**cond, **kw})
    ph = H.hgks_default_params(**{**cond, **kw})
    out = om.residual(po, Q, G)
    Ro, Go = (out if kw.get("scheme") == 1 else (out, None))
    import torch
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    Rd = torch.empty_like(Qd)
    Gn = torch.empty_like(Gd)
    H.hgks_residual(hm, ph, Qd, Gd if kw.get("scheme") == 1 else None, Rd, Gn if kw.get("scheme") == 1 else None)
    torch.cuda.synchronize()
    Rg = hm.to_caller(Rd)
    scale = flux_scale(om, Q)
    err = np.abs(Rg - Ro) / scale
    assert err.max() <= TOL_R_FLUX, f"max rel err {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"
    big = np.abs(Ro) >= 1e-2 * scale
    assert big.mean() > 0.05
    rel = np.abs(Rg - Ro)[big] / np.abs(Ro)[big]
    assert rel.max() <= TOL_R_REL, f"max error relative to |R| {rel.max():.3e} ({big.mean():.2f} of the components)"
    if kw.get("scheme") == 1:
        Gg = hm.to_caller(Gn)
        gs = np.repeat(np.abs(Q), 3, axis=1) * area_over_volume(om)[:, None]
        gerr = np.abs(Gg - Go) / gs
        assert gerr.max() <= TOL_R, f"gradient max rel err {gerr.max():.3e}"


def test_residual_deterministic_and_host_variant(cuda):
    import torch
    m, cond, om, hm = setup("cavity8")
    Q, G = state(m, cond, seed=3)
    ph = H.hgks_default_params(scheme=1, Pr=0.72, **cond)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    R1, R2 = torch.empty_like(Qd), torch.empty_like(Qd)
    G1, G2 = torch.empty_like(Gd), torch.empty_like(Gd)
    H.hgks_residual(hm, ph, Qd, Gd, R1, G1)
    H.hgks_residual(hm, ph, Qd, Gd, R2, G2)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2) and torch.equal(G1, G2)
    Qh = np.ascontiguousarray(Qd.cpu().numpy()); Gh = np.ascontiguousarray(Gd.cpu().numpy())
    Rh = np.zeros_like(Qh); Gnh = np.zeros_like(Gh)
    H.hgks_residual_host(hm, ph, Qh, Gh, Rh, Gnh)
    assert np.array_equal(Rh, R1.cpu().numpy()) and np.array_equal(Gnh, G1.cpu().numpy())


def test_local_dt_and_jacobian_parity(cuda):
    import torch
    for name, kw in [("cavity8", dict(scheme=1, Pr=0.72)), ("sphere6x6", dict(scheme=0))]:
        m, cond, om, hm = setup(name)
        Q, G = state(m, cond, seed=5)
        po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(**{**cond, **kw})
        Qd = hm.to_internal(Q)
        dtd = torch.empty(hm.n_cells, dtype=torch.float64, device="cuda")
        H.hgks_local_dt(hm, ph, Qd, dtd)
        dto = om.local_dt(po, Q)
        np.testing.assert_allclose(dtd.cpu().numpy()[hm.inv], dto, rtol=1e-13)
        diag = torch.empty(25, hm.n_cells, dtype=torch.float64, device="cuda")
        off = torch.empty(100, hm.n_cells, dtype=torch.float64, device="cuda")
        H.hgks_assemble(hm, ph, Qd, dtd, diag, off)
        torch.cuda.synchronize()
        Do, Oo = om.jacobian(po, Q, dto)
        Dg = diag.cpu().numpy().T[hm.inv].reshape(-1, 5, 5)
        Og = off.cpu().numpy().T[hm.inv].reshape(-1, 4, 5, 5)
        dscale = np.abs(Do).max(axis=(1, 2))[:, None, None]
        assert (np.abs(Dg - Do) / dscale).max() <= 1e-12
        assert (np.abs(Og - Oo) / dscale[:, None]).max() <= 1e-12
        # y = A x and the Jacobi preconditioner
        x = np.random.default_rng(7).normal(size=Q.shape)
        xd = hm.to_internal(x)
        yd = torch.empty_like(xd)
        H.hgks_apply_jacobian(hm, xd, yd)
        zd = torch.empty_like(xd)
        H.hgks_precondition(hm, 2, xd, zd)
        torch.cuda.synchronize()
        yo = np.einsum("nij,nj->ni", Do, x)
        nb = om.neighbours
        for q in range(4):
            ok = nb[:, q] >= 0
            yo[ok] += np.einsum("nij,nj->ni", Oo[ok, q], x[nb[ok, q]])
        ysc = np.abs(Do).max(axis=(1, 2))[:, None] * np.abs(x).max()
        assert (np.abs(hm.to_caller(yd) - yo) / ysc).max() <= 1e-12
        zo = om.precondition(Do, Oo, 2, x)
        np.testing.assert_allclose(hm.to_caller(zd), zo, rtol=1e-10, atol=1e-12 * np.abs(zo).max())


@pytest.mark.parametrize("name,kw", [("cavity8", dict(scheme=1, Pr=0.72)), ("sphere6x6", dict(scheme=0, krylov_dim=20)),
                                     ("sphere6x6_visc", dict(scheme=1, Pr=0.72, cfl=20.0)),
                                     ("sphere6x6_visc", dict(scheme=1, Pr=0.72, cfl=20.0, grad_relax=0.5))])
def test_gmres_step_parity(cuda, name, kw):
    import torch
    m, cond, om, hm = setup(name)
    Q, G = state(m, cond, seed=9)
    po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(**{**cond, **kw})
    Qo, Go, reso, dQo = om.gmres_step(po, Q, G)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    dQd = torch.empty_like(Qd)
    info = H.hgks_gmres_step(hm, ph, Qd, Gd if kw["scheme"] == 1 else None, dQd)
    assert info.res_l1 == pytest.approx(reso, rel=1e-11)
    dQg = hm.to_caller(dQd)
    rel = np.linalg.norm(dQg - dQo) / np.linalg.norm(dQo)
    assert rel <= 1e-9, rel
    if kw["scheme"] == 1:
        Gg = hm.to_caller(Gd)
        assert np.linalg.norm(Gg - Go) / np.linalg.norm(Go) <= 1e-11


@pytest.mark.parametrize("sweeps", [0, 1, 3])
def test_gmres_step_parity_jacobi_sweeps(cuda, sweeps):
    """Other sweep counts of the Jacobi preconditioner (k = 0, odd, 3): the GPU forms
    P^{-1} A v_j in its Neumann form v + E (-E)^k v, whose sign depends on k."""
    import torch
    m, cond, om, hm = setup("sphere6x6")
    Q, G = state(m, cond, seed=12)
    kw = dict(scheme=0, krylov_dim=10, restarts=2, jacobi_sweeps=sweeps)
    po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(**{**cond, **kw})
    _, _, reso, dQo = om.gmres_step(po, Q, G)
    Qd = hm.to_internal(Q)
    dQd = torch.empty_like(Qd)
    info = H.hgks_gmres_step(hm, ph, Qd, None, dQd)
    assert info.res_l1 == pytest.approx(reso, rel=1e-11)
    rel = np.linalg.norm(hm.to_caller(dQd) - dQo) / np.linalg.norm(dQo)
    assert rel <= 1e-9, rel
    # the FP32 Krylov part: the same step to the mixed-precision tolerance
    Qd = hm.to_internal(Q)
    H.hgks_gmres_step(hm, H.hgks_default_params(**{**cond, **kw, "precision": 1}), Qd, None, dQd)
    rel32 = np.linalg.norm(hm.to_caller(dQd) - dQo) / np.linalg.norm(dQo)
    assert rel32 <= MIXED_TOL["dQ_step"], rel32


@pytest.mark.parametrize("relax", [1.0, 0.5])
def test_gmres_steps_track_oracle(cuda, relax):
    """Five consecutive implicit steps on the viscous sphere stay within 1e-9
    (relative L2), with Algorithm 1's gradient update and with it under-relaxed."""
    import torch
    m, cond, om, hm = setup("sphere6x6_visc")
    kw = dict(scheme=1, Pr=0.72, cfl=20.0, grad_relax=relax)
    po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(**{**cond, **kw})
    Q = I.state_from_conditions(m.n_tet, cond); G = np.zeros((m.n_tet, 15))
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    for k in range(5):
        Q, G, res, _ = om.gmres_step(po, Q, G)
        info = H.hgks_gmres_step(hm, ph, Qd, Gd)
        assert info.res_l1 == pytest.approx(res, rel=1e-9, abs=1e-15)
    Qg = hm.to_caller(Qd)
    assert np.linalg.norm(Qg - Q) / np.linalg.norm(Q) <= 1e-9


def test_edge_cases(cuda):
    import ctypes as C
    L = H.lib()
    out = C.c_void_p()
    # empty mesh
    st = L.hgks_mesh_create(None, 0, None, 0, None, None, 0, None, 0, 3, 0, C.byref(out), None)
    assert st == 1
    # a single tetrahedron in the far field: too few cells for the non-compact stencil
    m = I.Mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]), np.array([[0, 1, 2, 3]]),
               np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]), np.full(4, 5, np.int32))
    with pytest.raises(H.HGKSError) as e:
        H.hgks_mesh_create(m, scheme_mask=1)
    assert e.value.status == 2
    # a face that is neither shared nor tagged
    m2 = I.cavity_mesh(2)
    m2.bface3 = m2.bface3[1:]; m2.btag = m2.btag[1:]
    with pytest.raises(H.HGKSError) as e:
        H.hgks_mesh_create(m2)
    assert e.value.status == 2
    # a mesh built for one scheme rejects the other
    hm = H.hgks_mesh_create(I.cavity_mesh(3), scheme_mask=1)
    import torch
    Q = torch.zeros(5, hm.n_cells, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HGKSError):
        H.hgks_residual(hm, H.hgks_default_params(scheme=1), Q, Q, Q, Q)
    with pytest.raises(H.HGKSError):
        H.hgks_gmres_step(hm, H.hgks_default_params(krylov_dim=0), Q)


@pytest.mark.slow
def test_full_size_sphere_sampled(cuda):
    """The 2.36M-cell sphere (32x32 patches, 64 layers), WENO, in the launch configuration
    the benchmark times: residual on sampled cells against the oracle."""
    import torch
    m = I.sphere_mesh(32, 64)
    cond = I.sphere_conditions(0.3)
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    Q, _ = I.smooth_state(m, amp=0.02, base=(1.0, 0.3, 0.0, 0.0, 1 / GAMMA), wavenumber=1.0)
    ph = H.hgks_default_params(scheme=0, krylov_dim=20, **cond)
    Qd = hm.to_internal(Q)
    Rd = torch.empty_like(Qd)
    H.hgks_residual(hm, ph, Qd, None, Rd)
    torch.cuda.synchronize()
    om = O.OracleMesh(m)
    rng = np.random.default_rng(2)
    cells = np.sort(rng.choice(m.n_tet, 400, replace=False))
    Ro = om.residual(O.make_params(scheme=0, krylov_dim=20, **cond), Q, cells=cells)
    Rg = hm.to_caller(Rd)
    scale = flux_scale(om, Q)
    err = np.abs(Rg[cells] - Ro[cells]) / scale[cells]
    assert err.max() <= TOL_R, err.max()


def test_full_size_viscous_sphere_compact_sampled(cuda):
    """The 995,328-cell viscous sphere of the precision workload (6x24x24, 48 layers,
    first layer 3e-2, adiabatic no-slip wall), compact HWENO with Pr 0.72: residual
    and gradient update on sampled cells against the oracle."""
    import torch
    m = I.sphere_mesh(24, 48, stretch=I.sphere_stretch(48, dr1=3e-2), wall_tag=I.BC_NOSLIP_ADIA)
    cond = I.sphere_conditions(0.2535, Re=118.0)
    hm = H.hgks_mesh_create(m, scheme_mask=2)
    Q, G = I.smooth_state(m, amp=0.02, base=(1.0, 0.2535, 0.0, 0.0, 1 / GAMMA), wavenumber=1.0)
    kw = dict(scheme=1, Pr=0.72, cfl=20.0, **cond)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    Rd, Gn = torch.empty_like(Qd), torch.empty_like(Gd)
    H.hgks_residual(hm, H.hgks_default_params(**kw), Qd, Gd, Rd, Gn)
    torch.cuda.synchronize()
    om = O.OracleMesh(m)
    rng = np.random.default_rng(3)
    # sampled cells: random ones and the wall layer (where the viscous terms are largest)
    wall = np.where(np.isin(m.tet4, m.bface3[m.btag == I.BC_NOSLIP_ADIA]).sum(1) >= 3)[0]
    cells = np.unique(np.concatenate([rng.choice(m.n_tet, 300, replace=False), rng.choice(wall, 100, replace=False)]))
    Ro, Go = om.residual(O.make_params(**kw), Q, G, cells=cells)
    Rg, Gg = hm.to_caller(Rd), hm.to_caller(Gn)
    scale = flux_scale(om, Q)
    err = np.abs(Rg[cells] - Ro[cells]) / scale[cells]
    assert err.max() <= TOL_R, err.max()
    # gradients against the cell's largest state component times its area/volume
    # (momentum components of this flow can be zero in a cell)
    gs = (np.abs(Q).max(axis=1) * area_over_volume(om))[cells][:, None]
    gerr = np.abs(Gg[cells] - Go[cells]) / gs
    assert gerr.max() <= TOL_R, gerr.max()


def five_tet_cube():
    """A unit cube split into 5 tetrahedra (odd cell count), far field on all sides."""
    V = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], dtype=np.float64)
    idx = {tuple(v): k for k, v in enumerate(V.astype(int))}
    even = [idx[(0, 0, 0)], idx[(1, 1, 0)], idx[(1, 0, 1)], idx[(0, 1, 1)]]
    tets = [even]
    bf = []
    for odd in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]:
        nb = [idx[tuple(np.array(odd) ^ np.eye(3, dtype=int)[d])] for d in range(3)]
        tets.append([idx[odd]] + nb)
        for d in range(3):
            bf.append([idx[odd]] + [nb[k] for k in range(3) if k != d])
    tet = np.array(tets, dtype=np.int64)
    a = V[tet[:, 0]]
    s = np.einsum("ij,ij->i", V[tet[:, 1]] - a, np.cross(V[tet[:, 2]] - a, V[tet[:, 3]] - a))
    tet[s < 0, 2], tet[s < 0, 3] = tet[s < 0, 3].copy(), tet[s < 0, 2].copy()
    return I.Mesh(V, tet, np.array(bf, dtype=np.int64), np.full(len(bf), I.BC_FARFIELD, np.int32))


@pytest.mark.parametrize("precision", [0, 1])
def test_odd_cell_count(cuda, precision):
    import torch
    m = five_tet_cube()
    cond = I.sphere_conditions(0.3)
    om = O.OracleMesh(m)
    hm = H.hgks_mesh_create(m, scheme_mask=2)
    Q, G = I.smooth_state(m, amp=0.05, base=(1.0, 0.3, 0.05, -0.02, 1 / GAMMA))
    kw = dict(scheme=1, krylov_dim=7, **cond)
    Qo, Go, reso, dQo = om.gmres_step(O.make_params(**kw), Q, G)
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    dQd = torch.empty_like(Qd)
    info = H.hgks_gmres_step(hm, H.hgks_default_params(precision=precision, **kw), Qd, Gd, dQd)
    assert info.res_l1 == pytest.approx(reso, rel=1e-11)
    rel = np.linalg.norm(hm.to_caller(dQd) - dQo) / np.linalg.norm(dQo)
    assert rel <= (1e-9 if precision == 0 else 1e-4), rel


MIXED_TOL = {"dQ_step": 1e-4, "Q_5steps": 1e-6}


@pytest.mark.parametrize("name,kw", [("sphere6x6", dict(scheme=0, krylov_dim=20)),
                                     ("sphere6x6_visc", dict(scheme=1, Pr=0.72, cfl=20.0)),
                                     ("cavity8", dict(scheme=1, Pr=0.72))])
def test_mixed_precision_step_error(cuda, name, kw):
    """FP32 Krylov basis, Arnoldi and Jacobi (FP64 residual, update and least squares):
    the update of one implicit step against the FP64 oracle."""
    import torch
    m, cond, om, hm = setup(name)
    Q, G = state(m, cond, seed=9)
    po = O.make_params(**{**cond, **kw})
    Qo, Go, reso, dQo = om.gmres_step(po, Q, G)
    ph = H.hgks_default_params(precision=1, **{**cond, **kw})
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    dQd = torch.empty_like(Qd)
    info = H.hgks_gmres_step(hm, ph, Qd, Gd if kw["scheme"] == 1 else None, dQd)
    assert info.res_l1 == pytest.approx(reso, rel=1e-11)     # the residual stays FP64
    rel = np.linalg.norm(hm.to_caller(dQd) - dQo) / np.linalg.norm(dQo)
    print(f"mixed precision {name}: relative L2 error of dQ against the FP64 oracle = {rel:.3e}")
    assert rel <= MIXED_TOL["dQ_step"], rel


def test_mixed_precision_trajectory_error(cuda):
    """Five implicit steps on the viscous sphere (compact scheme): mixed precision against
    the FP64 oracle, relative L2 of the state."""
    m, cond, om, hm = setup("sphere6x6_visc")
    kw = dict(scheme=1, Pr=0.72, cfl=20.0)
    po = O.make_params(**{**cond, **kw}); ph = H.hgks_default_params(precision=1, **{**cond, **kw})
    Q = I.state_from_conditions(m.n_tet, cond); G = np.zeros((m.n_tet, 15))
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    for k in range(5):
        Q, G, res, _ = om.gmres_step(po, Q, G)
        H.hgks_gmres_step(hm, ph, Qd, Gd)
    rel = np.linalg.norm(hm.to_caller(Qd) - Q) / np.linalg.norm(Q)
    print(f"mixed precision, 5 steps: relative L2 error of Q against the FP64 oracle = {rel:.3e}")
    assert rel <= MIXED_TOL["Q_5steps"], rel


def test_solve_steady_parity(cuda):
    """Algorithm 1 through hgks_solve_steady on the small inviscid sphere (non-compact
    scheme) against orc_solve_steady: same number of steps to a 5e-2 drop of the density
    residual, and the same state (relative L2 1e-9)."""
    m, cond, om, hm = setup("sphere6x6")
    kw = dict(scheme=0, krylov_dim=10)
    Q0 = I.state_from_conditions(m.n_tet, cond)
    Qo, _, hist_o, conv_o = om.solve_steady(O.make_params(**{**cond, **kw}), Q0, drop=5e-2, max_steps=200)
    Qd = hm.to_internal(Q0)
    info, hist_g, conv_g = H.hgks_solve_steady(hm, H.hgks_default_params(**{**cond, **kw}), Qd, None,
                                               drop_tol=5e-2, max_steps=200)
    assert conv_o and conv_g
    assert info.steps == len(hist_o) - 1
    np.testing.assert_allclose(hist_g, hist_o, rtol=1e-8)
    rel = np.linalg.norm(hm.to_caller(Qd) - Qo) / np.linalg.norm(Qo)
    assert rel <= 1e-9, rel


def test_converged_steady_state_parity(cuda):
    """A long steady solve: the 3,456-tet inviscid sphere (4x4 patches, 6 layers)
    run by Algorithm 1 to a 2e-4 drop of the density residual (about 320 steps)
    on the GPU and in the oracle: the same number of steps, the same residual
    history (relative 1e-8) and the same state (relative L2 1e-9). (The deep
    converged state, a 1e-8 drop, is the lid-driven cavity's:
    tests/test_gpu_steady_cavity.py.)"""
    m = I.sphere_mesh(4, 6, stretch=1.3)
    cond = I.sphere_conditions(0.3)
    om = O.OracleMesh(m)
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    kw = dict(scheme=0, krylov_dim=10)
    Q0 = I.state_from_conditions(m.n_tet, cond)
    Qd = hm.to_internal(Q0)
    info, hist_g, conv_g = H.hgks_solve_steady(hm, H.hgks_default_params(**{**cond, **kw}), Qd, None,
                                               drop_tol=2e-4, max_steps=600)
    Qo, _, hist_o, conv_o = om.solve_steady(O.make_params(**{**cond, **kw}), Q0, drop=2e-4, max_steps=600)
    assert conv_g and conv_o and info.steps > 200
    assert info.steps == len(hist_o) - 1
    np.testing.assert_allclose(hist_g, hist_o, rtol=1e-8)
    rel = np.linalg.norm(hm.to_caller(Qd) - Qo) / np.linalg.norm(Qo)
    assert rel <= 1e-9, rel


def test_solve_resumes_from_a_host_snapshot_bit_for_bit(cuda):
    """Checkpoint/resume: stop a solve at 6 steps, copy (Q, G) to the host and
    back, resume to 12 steps: the iterates equal the uninterrupted 12-step solve."""
    import torch
    m, cond, om, hm = setup("cavity5")
    Q, G = state(m, cond, seed=9)
    p = H.hgks_default_params(scheme=1, Pr=0.72, krylov_dim=6, restarts=2, **cond)
    Qa, Ga = hm.to_internal(Q), hm.to_internal(G)
    ia, ha, _ = H.hgks_solve_steady(hm, p, Qa, Ga, drop_tol=1e-12, max_steps=12)
    Qb, Gb = hm.to_internal(Q), hm.to_internal(G)
    i6, h6, _ = H.hgks_solve_steady(hm, p, Qb, Gb, drop_tol=1e-12, max_steps=6)
    snap_Q, snap_G = Qb.cpu().numpy().copy(), Gb.cpu().numpy().copy()
    Qc, Gc = torch.from_numpy(snap_Q).cuda(), torch.from_numpy(snap_G).cuda()
    ib, hb, _ = H.hgks_solve_resume(hm, p, Qc, Gc, i6, drop_tol=1e-12, max_steps=12)
    torch.cuda.synchronize()
    assert ib.steps == ia.steps == 12 and ib.res_ref == ia.res_ref
    assert torch.equal(Qc, Qa) and torch.equal(Gc, Ga)
    np.testing.assert_array_equal(hb[6:], ha[6:])
    np.testing.assert_array_equal(h6, ha[:7])
