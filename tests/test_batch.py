"""Batches of meshes (hgks_batch_*): every mesh of a batch gives what it gives
alone, through the same C ABI.

A batch runs each phase once for all of its meshes, each mesh with its own
parameters, Krylov space, Hessenberg problem and convergence test. The only
arithmetic that differs from a mesh run alone is the summation order of the
inner products (per-mesh segmented sums instead of one grid-wide sum), so
  - the residual of a mesh in a batch equals its residual alone to rounding
    (compared against the flux scale, as the residual parity tests do), and
    equals the oracle's within the residual tolerance 1e-11;
  - a GMRES step agrees to a relative 1e-10 (FP64) in Q, and the steady states
    of a batch solve agree with the solves alone to the steady-state
    tolerance, a relative L2 of 1e-9, with the same number of steps.
"""
import numpy as np
import pytest

import oracle as O
import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# meshes of uneven size (one smaller than a 256-cell block, none a multiple of
# 256) with different flow conditions: viscous cavities, an inviscid sphere, a
# periodic box
PROBLEMS = [
    ("cavity2", lambda: (I.cavity_mesh(2, seed=I.BASE_SEED + 11), I.cavity_conditions(0.2, 50.0))),
    ("sphere5", lambda: (I.sphere_mesh(5, 4, stretch=1.3), I.sphere_conditions(0.3, aoa_deg=5.0))),
    ("cavity4", lambda: (I.cavity_mesh(4), I.cavity_conditions(0.15, 100.0))),
    ("periodic4", lambda: (I.periodic_cube_mesh(4), I.sphere_conditions(0.4))),
    ("sphere4v", lambda: (I.sphere_mesh(4, 4, stretch=1.3, wall_tag=I.BC_NOSLIP_ADIA), I.sphere_conditions(0.25, Re=118.0))),
]
_cache = {}


def problems():
    if not _cache:
        for name, make in PROBLEMS:
            m, cond = make()
            _cache[name] = (m, cond, H.hgks_mesh_create(m, scheme_mask=3))
    return [(n,) + _cache[n] for n, _ in PROBLEMS]


def perturbed(m, cond, seed):
    u = cond["u_inf"]
    base = (cond["rho_inf"], u[0] + 0.05, u[1] + 0.03, u[2] - 0.02, cond["p_inf"])
    return I.smooth_state(m, seed=I.BASE_SEED + seed, amp=0.03, base=base)


def params_for(cond, **kw):
    return H.hgks_default_params(**{**cond, "Pr": 0.72 if cond["viscous"] else 1.0, **kw})


def make_batch(kw, seed=5):
    """(batch, singles) with the same meshes, parameters and initial states."""
    import torch
    probs = problems()
    params = [params_for(c, **kw) for _, _, c, _ in probs]
    b = H.hgks_batch_create([hm for *_, hm in probs], params)
    singles = []
    for k, (name, m, cond, hm) in enumerate(probs):
        Q, G = perturbed(m, cond, seed + k)
        Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
        H.hgks_batch_set_state(b, k, Qd, Gd if kw.get("scheme") == 1 else None)
        singles.append((name, m, cond, hm, params[k], Qd.clone(), Gd.clone()))
    torch.cuda.synchronize()
    return b, singles


def flux_scale_internal(hm, m, Q):
    """sum over the cell's faces of S |F_Euler(Q_i) . n| (caller order), as [n, 5]."""
    V = m.xyz[m.tet4]
    rho = Q[:, 0]; u = Q[:, 1:4] / rho[:, None]
    p = 0.4 * (Q[:, 4] - 0.5 * rho * np.einsum("ij,ij->i", u, u))
    s = np.zeros_like(Q)
    for f in range(4):
        F3 = V[:, [k for k in range(4) if k != f]]
        nrm = np.cross(F3[:, 1] - F3[:, 0], F3[:, 2] - F3[:, 0])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        n = nrm / (2 * area[:, None])
        un = np.einsum("ij,ij->i", u, n)
        fl = np.stack([rho * un, rho * u[:, 0] * un + p * n[:, 0], rho * u[:, 1] * un + p * n[:, 1],
                       rho * u[:, 2] * un + p * n[:, 2], (Q[:, 4] + p) * un], -1)
        s += area[:, None] * np.abs(fl)
    return s


@pytest.mark.parametrize("scheme", [0, 1], ids=["weno", "hweno"])
def test_batch_residual_equals_single_and_oracle(cuda, scheme):
    import torch
    b, singles = make_batch(dict(scheme=scheme))
    H.hgks_batch_residual(b)
    for k, (name, m, cond, hm, p, Qd, Gd) in enumerate(singles):
        Rb = torch.empty_like(Qd)
        Gb = torch.empty_like(Gd)
        H.hgks_batch_get_state(b, k, R=Rb, G_new=Gb if scheme == 1 else None)
        Rs = torch.empty_like(Qd)
        Gs = torch.empty_like(Gd)
        H.hgks_residual(hm, p, Qd, Gd if scheme == 1 else None, Rs, Gs if scheme == 1 else None)
        torch.cuda.synchronize()
        Q = hm.to_caller(Qd)
        scale = flux_scale_internal(hm, m, Q)
        err = np.abs(hm.to_caller(Rb) - hm.to_caller(Rs)) / scale
        assert err.max() <= 1e-13, f"{name}: batch vs alone {err.max():.3e}"
        if scheme == 1:
            gerr = np.abs((Gb - Gs).cpu().numpy()).max() / max(1e-300, np.abs(Gs.cpu().numpy()).max())
            assert gerr <= 1e-13, f"{name}: gradients batch vs alone {gerr:.3e}"
        if k in (0, 1):      # the oracle on the smallest meshes
            om = O.OracleMesh(m)
            po = O.make_params(**{**cond, "Pr": 0.72 if cond["viscous"] else 1.0, "scheme": scheme})
            out = om.residual(po, Q, hm.to_caller(Gd))
            Ro = out[0] if scheme == 1 else out
            oerr = np.abs(hm.to_caller(Rb) - Ro) / scale
            assert oerr.max() <= 1e-11, f"{name}: batch vs oracle {oerr.max():.3e}"


@pytest.mark.parametrize("precision,sweeps", [(0, 2), (1, 2), (0, 1), (1, 3)],
                         ids=["fp64", "mixed", "fp64-1sweep", "mixed-3sweeps"])
def test_batch_gmres_step_equals_single(cuda, precision, sweeps):
    import torch
    kw = dict(scheme=0, krylov_dim=8, restarts=2, precision=precision, jacobi_sweeps=sweeps)
    b, singles = make_batch(kw, seed=21)
    infos = H.hgks_batch_gmres_step(b)
    tol = 1e-10 if precision == 0 else 2e-4
    for k, (name, m, cond, hm, p, Qd, Gd) in enumerate(singles):
        Q0 = Qd.clone()
        si = H.hgks_gmres_step(hm, p, Qd, None)
        Qb = torch.empty_like(Qd)
        H.hgks_batch_get_state(b, k, Q=Qb)
        torch.cuda.synchronize()
        assert abs(infos[k].res_l1 - si.res_l1) <= 1e-13 * si.res_l1, name
        dQs = (Qd - Q0).cpu().numpy()
        dQb = (Qb - Q0).cpu().numpy()
        rel = np.linalg.norm(dQb - dQs) / np.linalg.norm(dQs)
        assert rel <= tol, f"{name}: step update batch vs alone {rel:.3e}"
        assert abs(infos[k].lin_res[0] - si.lin_res[0]) <= 1e-6 * si.lin_res[0]


def test_batch_solve_equals_single_solves_graph_and_eager(cuda):
    import torch
    kw = dict(scheme=0, krylov_dim=10, restarts=2)
    drop, max_steps = 0.2, 30        # a drop some meshes reach within the limit and some do not
    b, singles = make_batch(kw, seed=31)
    Q0 = [torch.empty_like(s[5]) for s in singles]
    for k in range(len(singles)):
        H.hgks_batch_get_state(b, k, Q=Q0[k])
    infos, hist, _ = H.hgks_batch_solve_steady(b, drop, max_steps, use_graph=True)
    Qg = [torch.empty_like(s[5]) for s in singles]
    for k in range(len(singles)):
        H.hgks_batch_get_state(b, k, Q=Qg[k])
    # the same batch from the same start without the graph: identical launches, identical results
    for k in range(len(singles)):
        H.hgks_batch_set_state(b, k, Q0[k])
    infos_e, hist_e, _ = H.hgks_batch_solve_steady(b, drop, max_steps, use_graph=False)
    for k, (name, m, cond, hm, p, Qd, Gd) in enumerate(singles):
        Qe = torch.empty_like(Qd)
        H.hgks_batch_get_state(b, k, Q=Qe)
        torch.cuda.synchronize()
        assert infos[k].steps == infos_e[k].steps
        assert torch.equal(Qe, Qg[k]), f"{name}: graph and eager replays differ"
        np.testing.assert_array_equal(hist[k], hist_e[k])
        si, hs, conv = H.hgks_solve_steady(hm, p, Qd, None, drop_tol=drop, max_steps=max_steps)
        assert infos[k].steps == si.steps, f"{name}: {infos[k].steps} steps in the batch, {si.steps} alone"
        assert bool(infos[k].converged) == conv
        rel = (torch.linalg.norm(Qg[k] - Qd) / torch.linalg.norm(Qd)).item()
        assert rel <= 1e-9, f"{name}: steady state batch vs alone {rel:.3e}"
        np.testing.assert_allclose(hist[k, : si.steps + 1], hs, rtol=1e-9, atol=0)
    # meshes finish at different steps: the finished ones were skipped while the rest went on
    assert len({i.steps for i in infos}) > 1


def test_zero_steps_only_tests(cuda):
    """max_steps = 0: every mesh evaluates its residual once and stops, state untouched."""
    import torch
    b, singles = make_batch(dict(scheme=0, krylov_dim=6, restarts=1), seed=41)
    infos, hist, conv = H.hgks_batch_solve_steady(b, 1e-8, 0)
    assert not conv
    for k, (name, m, cond, hm, p, Qd, Gd) in enumerate(singles):
        Qb = torch.empty_like(Qd)
        H.hgks_batch_get_state(b, k, Q=Qb)
        si, hs, _ = H.hgks_solve_steady(hm, p, Qd.clone(), None, drop_tol=1e-8, max_steps=0)
        torch.cuda.synchronize()
        assert infos[k].steps == 0 and torch.equal(Qb, Qd)
        assert abs(hist[k, 0] - hs[0]) <= 1e-13 * hs[0]


def test_autotune_keeps_results(cuda):
    import torch
    b, singles = make_batch(dict(scheme=1), seed=51)
    H.hgks_batch_residual(b)
    R0 = [torch.empty_like(s[5]) for s in singles]
    for k in range(len(singles)):
        H.hgks_batch_get_state(b, k, R=R0[k])
    r, f = H.hgks_batch_autotune(b)
    assert r in (64, 128, 256) and f in (64, 128, 256)
    info = H.hgks_batch_info(b)
    assert (info.blk_recon, info.blk_flux) == (r, f)
    assert info.n_meshes == len(singles) and info.n_cells % 256 == 0
    H.hgks_batch_residual(b)
    for k in range(len(singles)):
        R1 = torch.empty_like(R0[k])
        H.hgks_batch_get_state(b, k, R=R1)
        torch.cuda.synchronize()
        assert torch.equal(R1, R0[k])


def test_batch_rejects_disagreeing_shared_parameters(cuda):
    probs = problems()
    p0 = params_for(probs[0][2], scheme=0, krylov_dim=8)
    p1 = params_for(probs[1][2], scheme=0, krylov_dim=10)
    with pytest.raises(H.HGKSError):
        H.hgks_batch_create([probs[0][3], probs[1][3]], [p0, p1])


def test_batch_of_one_mesh_equals_alone(cuda):
    import torch
    name, m, cond, hm = problems()[1]
    p = params_for(cond, scheme=0, krylov_dim=8, restarts=2)
    b = H.hgks_batch_create([hm], [p])
    Q, _ = perturbed(m, cond, 61)
    Qd = hm.to_internal(Q)
    H.hgks_batch_set_state(b, 0, Qd)
    (info,) = H.hgks_batch_gmres_step(b)
    Q0 = Qd.clone()
    si = H.hgks_gmres_step(hm, p, Qd, None)
    Qb = torch.empty_like(Qd)
    H.hgks_batch_get_state(b, 0, Q=Qb)
    torch.cuda.synchronize()
    assert abs(info.res_l1 - si.res_l1) <= 1e-13 * si.res_l1
    rel = (torch.linalg.norm((Qb - Q0) - (Qd - Q0)) / torch.linalg.norm(Qd - Q0)).item()
    assert rel <= 1e-10, rel


def test_batch_step_graph_replay_equals_eager(cuda):
    """hgks_batch_gmres_step replayed from its CUDA graph gives the eager step's
    state and step records bit for bit (twice in a row: the second replay reuses
    the captured graph)."""
    import torch
    kw = dict(scheme=1, krylov_dim=8, restarts=2, precision=1)
    b, singles = make_batch(kw, seed=41)
    n = len(singles)
    Q0 = [torch.empty_like(s[5]) for s in singles]
    G0 = [torch.empty_like(s[6]) for s in singles]
    for k in range(n):
        H.hgks_batch_get_state(b, k, Q=Q0[k], G=G0[k])
    out = {}
    for mode in (False, True):
        for k in range(n):
            H.hgks_batch_set_state(b, k, Q0[k], G0[k])
        infos = [H.hgks_batch_gmres_step(b, use_graph=mode) for _ in range(2)]
        Qs = [torch.empty_like(q) for q in Q0]
        Gs = [torch.empty_like(g) for g in G0]
        for k in range(n):
            H.hgks_batch_get_state(b, k, Q=Qs[k], G=Gs[k])
        torch.cuda.synchronize()
        out[mode] = (infos, Qs, Gs)
    for k in range(n):
        assert torch.equal(out[False][1][k], out[True][1][k]) and torch.equal(out[False][2][k], out[True][2][k])
        for s in range(2):
            assert out[False][0][s][k].res_l1 == out[True][0][s][k].res_l1


def test_batch_of_cavities_converges_like_alone(cuda):
    """Three lid-driven cavities of different size, Mach and Reynolds number
    (compact HWENO, nonlinear weights, CFL 10) solved together to a 1e-5 drop:
    every one converges, with the step count, residual history (1e-9 of its
    reference) and state (relative L2 1e-9) it has when solved alone."""
    import torch
    setups = [(4, 0.15, 100.0), (5, 0.2, 200.0), (4, 0.3, 50.0)]
    meshes, params, states = [], [], []
    for k, (n, ma, re) in enumerate(setups):
        m = I.cavity_mesh(n, seed=I.BASE_SEED + 70 + k)
        cond = I.cavity_conditions(ma, re)
        hm = H.hgks_mesh_create(m, scheme_mask=2)
        meshes.append(hm)
        params.append(H.hgks_default_params(scheme=1, Pr=0.72, **cond))
        Q = hm.to_internal(I.state_from_conditions(m.n_tet, cond))
        states.append((Q, torch.zeros((15, m.n_tet), dtype=torch.float64, device="cuda")))
    b = H.hgks_batch_create(meshes, params)
    for k, (Q, G) in enumerate(states):
        H.hgks_batch_set_state(b, k, Q, G)
    drop, max_steps = 1e-5, 2500
    infos, hist, ok = H.hgks_batch_solve_steady(b, drop, max_steps)
    assert ok
    for k, (hm, p, (Q, G)) in enumerate(zip(meshes, params, states)):
        si, hs, conv = H.hgks_solve_steady(hm, p, Q, G, drop_tol=drop, max_steps=max_steps)
        assert conv and infos[k].converged and infos[k].steps == si.steps, (k, infos[k].steps, si.steps)
        np.testing.assert_allclose(hist[k][: si.steps + 1], hs, rtol=0, atol=1e-9 * hs.max())
        Qb, Gb = torch.empty_like(Q), torch.empty_like(G)
        H.hgks_batch_get_state(b, k, Q=Qb, G=Gb)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(Qb - Q) / torch.linalg.norm(Q)).item() <= 1e-9
        assert (torch.linalg.norm(Gb - G) / torch.linalg.norm(G)).item() <= 1e-9
