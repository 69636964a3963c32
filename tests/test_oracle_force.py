"""Pins of the oracle's wall force (the drag of the precision workload).

  - A cavity at rest with walls at rest and the fluid's temperature: every
    wall flux is the pressure p n (no slopes, no motion), so the force on the
    lid (y = 1, area 1) is (0, p, 0) and on the five other walls (0, -p, 0).
  - Momentum balance: summed over every boundary tag, the wall forces equal
    minus the summed momentum residual, sum_i R_i = -sum_boundary F S, for any
    state (interior fluxes cancel in pairs).
"""
import numpy as np

import oracle as O
from paper_2304_09485_gb300 import inputs as I


def test_force_of_a_fluid_at_rest_is_the_pressure():
    m = I.cavity_mesh(4)
    om = O.OracleMesh(m)
    cond = I.cavity_conditions(0.2, 100.0)
    p = O.make_params(**{**cond, "lid_speed": 0.0}, Pr=0.72)
    Q = I.state_from_conditions(m.n_tet, cond)
    pr = cond["p_inf"]
    lid = om.wall_force(p, Q, None, I.BC_WALL_LID)
    rest = om.wall_force(p, Q, None, I.BC_WALL_ISO)
    np.testing.assert_allclose(lid, [0.0, pr, 0.0], rtol=0, atol=1e-12 * pr)
    np.testing.assert_allclose(rest, [0.0, -pr, 0.0], rtol=0, atol=1e-12 * pr)


def test_wall_forces_balance_the_momentum_residual():
    m = I.sphere_mesh(4, 4, stretch=1.3, wall_tag=I.BC_NOSLIP_ADIA)
    om = O.OracleMesh(m)
    cond = I.sphere_conditions(0.3, Re=100.0)
    p = O.make_params(**cond, Pr=0.72)
    Q, _ = I.smooth_state(m, seed=I.BASE_SEED + 91, amp=0.03, base=(1.0, 0.32, 0.02, -0.01, cond["p_inf"]))
    R = om.residual(p, Q)
    F = om.wall_force(p, Q, None, I.BC_NOSLIP_ADIA) + om.wall_force(p, Q, None, I.BC_FARFIELD)
    scale = np.abs(om.wall_force(p, Q, None, I.BC_FARFIELD)).max()
    np.testing.assert_allclose(F, -R[:, 1:4].sum(0), rtol=0, atol=1e-11 * scale)
