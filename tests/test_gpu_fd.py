"""Matrix-free products (jv_mode 1, Eq. (frechet)) on the GPU against the oracle.

y = A x = |Omega|/dt x - (L(Q + sigma x) - L(Q)) / sigma. With the same Q, x and
dt, the GPU and the oracle differ only through their residuals, which agree to
the residual tolerance TOL_R = 1e-11 of the flux scale S (tests of
test_gpu_parity), so |y_gpu - y_oracle| <= 2 TOL_R S / sigma entry by entry:
the bound used below, a consequence of residual parity rather than a new
tolerance. The homogeneity pin of the oracle (x = Q on a periodic inviscid case
with linear weights) is checked on the GPU too.

A GMRES step in this mode solves with an operator that is linear only to
about 1e-5 of its size; the GPU and oracle steps agree to 1e-4 (relative L2 of
dQ; 1e-3 with the FP32 Krylov basis), well below their distance from the
assembled-mode step.
"""
import numpy as np
import pytest

import oracle as O
import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL_R = 1e-11


def flux_scale(om, Q):
    from test_gpu_parity import flux_scale as fs
    return fs(om, Q)


def sigma_of(Q, x):
    return 2.0 ** -26 * (1.0 + np.linalg.norm(Q)) / np.linalg.norm(x)


CASES = [
    ("cavity4-weno", lambda: (I.cavity_mesh(4), I.cavity_conditions(0.2, 100.0)), dict(scheme=0, Pr=0.72)),
    ("cavity4-hweno", lambda: (I.cavity_mesh(4), I.cavity_conditions(0.2, 100.0)), dict(scheme=1, Pr=0.72)),
    ("sphere4-weno", lambda: (I.sphere_mesh(4, 4, stretch=1.3), I.sphere_conditions(0.3, aoa_deg=3.0)), dict(scheme=0)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_fd_product_matches_oracle(cuda, name, make, kw):
    import torch
    m, cond = make()
    om = O.OracleMesh(m)
    hm = H.hgks_mesh_create(m, scheme_mask=3)
    u = cond["u_inf"]
    Q, G = I.smooth_state(m, seed=I.BASE_SEED + 81, amp=0.03,
                          base=(cond["rho_inf"], u[0] + 0.05, u[1] + 0.02, u[2] - 0.01, cond["p_inf"]))
    rng = np.random.default_rng(I.BASE_SEED + 82)
    x = rng.normal(size=Q.shape) * np.abs(Q).mean(0)
    ph = H.hgks_default_params(**{**cond, **kw, "jv_mode": 1})
    po = O.make_params(**{**cond, **kw, "jv_mode": 1})
    dt = om.local_dt(po, Q)
    Qd, Gd, xd = hm.to_internal(Q), hm.to_internal(G), hm.to_internal(x)
    dtd = hm.to_internal(dt[:, None])[0].contiguous()
    yd = torch.empty_like(Qd)
    H.hgks_apply_jacobian_fd(hm, ph, Qd, Gd if kw["scheme"] == 1 else None, dtd, xd, yd)
    torch.cuda.synchronize()
    yg = hm.to_caller(yd)
    yo, so = om.apply_fd(po, Q, G if kw["scheme"] == 1 else None, dt, x)
    assert abs(so - sigma_of(Q, x)) <= 1e-14 * so
    S = flux_scale(om, Q)
    err = np.abs(yg - yo) / (S / so)
    assert err.max() <= 2 * TOL_R, f"{name}: {err.max():.3e} of S/sigma"
    # a product of a zero vector is zero
    z = torch.zeros_like(Qd)
    H.hgks_apply_jacobian_fd(hm, ph, Qd, Gd if kw["scheme"] == 1 else None, dtd, z, yd)
    torch.cuda.synchronize()
    assert torch.count_nonzero(yd).item() == 0


def test_fd_product_homogeneity_on_gpu(cuda):
    import torch
    m = I.periodic_cube_mesh(4)
    om = O.OracleMesh(m)
    cond = I.sphere_conditions(0.3)
    ph = H.hgks_default_params(**cond, weights=1, jv_mode=1)
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    Q, _ = I.smooth_state(m, seed=I.BASE_SEED + 71, amp=0.05)
    Qd = hm.to_internal(Q)
    dtd = torch.empty(m.n_tet, dtype=torch.float64, device="cuda")
    H.hgks_local_dt(hm, ph, Qd, dtd)
    yd, Rd = torch.empty_like(Qd), torch.empty_like(Qd)
    H.hgks_apply_jacobian_fd(hm, ph, Qd, None, dtd, Qd, yd)
    H.hgks_residual(hm, ph, Qd, None, Rd)          # the same dt: L(Q) at its own local step
    torch.cuda.synchronize()
    vol = H.hgks_mesh_volumes(hm)
    expect = (vol / dtd.cpu().numpy())[None, :] * Qd.cpu().numpy() - Rd.cpu().numpy()
    S = hm.to_internal(flux_scale(om, Q)).cpu().numpy()
    sigma = sigma_of(Q, Q)
    err = np.abs(yd.cpu().numpy() - expect) / S
    assert err.max() <= 64 * np.finfo(float).eps / sigma, err.max()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_fd_gmres_step_matches_oracle(cuda, precision):
    import torch
    m, cond = I.cavity_mesh(3, seed=I.BASE_SEED + 83), I.cavity_conditions(0.2, 100.0)
    om = O.OracleMesh(m)
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    Q, _ = I.smooth_state(m, seed=I.BASE_SEED + 84, amp=0.03, base=(1.0, 0.05, 0.02, -0.01, cond["p_inf"]))
    kw = dict(scheme=0, Pr=0.72, krylov_dim=8, restarts=2)
    po = O.make_params(**{**cond, **kw, "jv_mode": 1})
    _, _, res_o, dQo = om.gmres_step(po, Q)
    _, _, _, dQa = om.gmres_step(O.make_params(**{**cond, **kw, "jv_mode": 0}), Q)
    ph = H.hgks_default_params(**{**cond, **kw, "jv_mode": 1, "precision": precision})
    Qd = hm.to_internal(Q)
    dQd = torch.empty_like(Qd)
    info = H.hgks_gmres_step(hm, ph, Qd, None, dQ_out=dQd)
    torch.cuda.synchronize()
    dQg = hm.to_caller(dQd)
    rel = np.linalg.norm(dQg - dQo) / np.linalg.norm(dQo)
    far = np.linalg.norm(dQa - dQo) / np.linalg.norm(dQo)
    tol = 1e-4 if precision == 0 else 1e-3
    assert rel <= tol, f"FD step GPU vs oracle {rel:.3e}"
    assert far >= 30 * 1e-4, f"assembled and matrix-free steps too close ({far:.3e}) for the test to discriminate"
    assert abs(info.res_l1 - res_o) <= 1e-12 * res_o
