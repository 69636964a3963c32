"""Pins of the oracle's matrix-free product (Eq. (frechet)), CPU only.

y = A x = |Omega|/dt x - (L(Q + sigma x) - L(Q)) / sigma, dt and G frozen.
  - Homogeneity: on a periodic mesh with inviscid flow and linear weights every
    step of L (linear reconstruction, characteristic matrices and Maxwellian
    ratios that depend on velocity and temperature only, a density-proportional
    distribution, the collision time of Sec. 5 built from pressure ratios) is
    homogeneous of degree one in Q, so L((1+sigma)Q) = (1+sigma) L(Q) and the
    product with x = Q is |Omega|/dt Q - L(Q) exactly, up to rounding divided by
    sigma. A wrong sign, a missing term or a wrong sigma breaks it.
  - Consistency: with linear weights and no pressure-jump term in the collision
    time L is smooth, so the forward difference agrees with a central difference
    at a larger step to O(sigma + h^2) plus rounding / sigma.
  - GMRES with the matrix-free operator and a full Krylov space reduces
    ||b - A dx|| / ||b|| by orders of magnitude (to the operator's own
    nonlinearity times the condition number, not to rounding).
"""
import numpy as np

import oracle as O
from paper_2304_09485_gb300 import inputs as I


def _flux_scale(om, Q):
    rho = Q[:, 0]; u = Q[:, 1:4] / rho[:, None]
    p = 0.4 * (Q[:, 4] - 0.5 * rho * np.einsum("ij,ij->i", u, u))
    mag = rho * np.abs(u).sum(1) + p + np.abs(Q[:, 4] + p) * np.abs(u).sum(1)
    return (mag * om.vol ** (2.0 / 3.0))[:, None] * np.ones((1, 5))


def test_fd_product_of_Q_is_exact_for_a_homogeneous_residual():
    m = I.periodic_cube_mesh(4)
    om = O.OracleMesh(m)
    cond = I.sphere_conditions(0.3)
    p = O.make_params(**cond, weights=1, jv_mode=1)
    Q, _ = I.smooth_state(m, seed=I.BASE_SEED + 71, amp=0.05)
    dt = om.local_dt(p, Q)
    L = om.residual_dt(p, Q, None, dt)
    y, sigma = om.apply_fd(p, Q, None, dt, Q)
    expect = (om.vol / dt)[:, None] * Q - L
    S = _flux_scale(om, Q)
    err = np.abs(y - expect) / S
    # rounding of L (a few ulps of the face-flux sums) divided by sigma
    tol = 64 * np.finfo(float).eps / sigma
    assert sigma > 0 and err.max() <= tol, (err.max(), tol)
    # the same with nonlinear weights is not homogeneous (epsilon in the weights): the pin discriminates
    pn = O.make_params(**cond, weights=0, weno_eps=1e-2, jv_mode=1)
    yn, _ = om.apply_fd(pn, Q, None, dt, Q)
    Ln = om.residual_dt(pn, Q, None, dt)
    assert (np.abs(yn - ((om.vol / dt)[:, None] * Q - Ln)) / S).max() > 100 * tol


def test_fd_product_agrees_with_a_central_difference():
    m = I.cavity_mesh(3, seed=I.BASE_SEED + 72)
    om = O.OracleMesh(m)
    cond = I.cavity_conditions(0.2, 100.0)
    # linear weights and no pressure-jump term in the collision time: L is smooth
    p = O.make_params(**cond, Pr=0.72, weights=1, tau_C=0.0, jv_mode=1)
    Q, _ = I.smooth_state(m, seed=I.BASE_SEED + 73, amp=0.03, base=(1.0, 0.05, 0.02, -0.01, cond["p_inf"]))
    rng = np.random.default_rng(I.BASE_SEED + 74)
    x = rng.normal(size=Q.shape) * np.abs(Q).mean(0)
    dt = om.local_dt(p, Q)
    y, sigma = om.apply_fd(p, Q, None, dt, x)
    h = 1e2 * sigma
    Lp = om.residual_dt(p, Q + h * x, None, dt)
    Lm = om.residual_dt(p, Q - h * x, None, dt)
    yc = (om.vol / dt)[:, None] * x - (Lp - Lm) / (2 * h)
    rel = np.linalg.norm(y - yc) / np.linalg.norm(yc)
    assert rel <= 1e-5, rel
    # and it is not the first-order assembled operator (the difference is O(1))
    diag, off = om.jacobian(p, Q, dt)
    ya = np.zeros_like(x)
    import ctypes as C
    O.lib().orc_apply_A(C.c_void_p(om.h), O._p(np.ascontiguousarray(diag)), O._p(np.ascontiguousarray(off)),
                        O._p(np.ascontiguousarray(x)), O._p(ya))
    assert np.linalg.norm(ya - yc) / np.linalg.norm(yc) > 1e-3


def test_gmres_with_the_fd_operator_solves_the_system():
    m = I.cavity_mesh(2, seed=I.BASE_SEED + 75)
    om = O.OracleMesh(m)
    cond = I.cavity_conditions(0.2, 100.0)
    n5 = 5 * m.n_tet
    p = O.make_params(**cond, Pr=0.72, weights=1, tau_C=0.0, jv_mode=1, krylov_dim=n5, restarts=1)
    Q, _ = I.smooth_state(m, seed=I.BASE_SEED + 76, amp=0.03, base=(1.0, 0.05, 0.02, -0.01, cond["p_inf"]))
    Q2, _, res, dQ = om.gmres_step(p, Q)
    dt = om.local_dt(p, Q)
    L = om.residual_dt(p, Q, None, dt)
    AdQ, _ = om.apply_fd(p, Q, None, dt, dQ)
    # the difference operator is linear only to O(sigma ||x|| L''/L') (about 5e-5 here)
    # and A is ill conditioned (about 6e6 at CFL 10), so a full Krylov space reduces
    # ||b - A dx|| by orders of magnitude rather than to rounding
    rel = np.linalg.norm(AdQ - L) / np.linalg.norm(L)
    assert rel <= 1e-2, rel
    # the assembled mode gives a different update
    pa = O.make_params(**cond, Pr=0.72, weights=1, tau_C=0.0, jv_mode=0, krylov_dim=n5, restarts=1)
    _, _, _, dQa = om.gmres_step(pa, Q)
    assert np.linalg.norm(dQa - dQ) > 1e-3 * np.linalg.norm(dQ)
