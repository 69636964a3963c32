"""Wall force (hgks_wall_force) on the GPU: the at-rest pin and the oracle.

The force is a sum of face fluxes that the residual parity tests already bound
(1e-11 of the flux scale per face), so the GPU and oracle forces agree to 1e-11
of the summed flux magnitude.
"""
import numpy as np
import pytest

import oracle as O
import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_force_of_a_fluid_at_rest_on_gpu(cuda):
    m = I.cavity_mesh(4)
    cond = I.cavity_conditions(0.2, 100.0)
    hm = H.hgks_mesh_create(m, scheme_mask=3)
    p = H.hgks_default_params(**{**cond, "lid_speed": 0.0}, Pr=0.72)
    Q = hm.to_internal(I.state_from_conditions(m.n_tet, cond))
    pr = cond["p_inf"]
    np.testing.assert_allclose(H.hgks_wall_force(hm, p, Q, None, I.BC_WALL_LID), [0, pr, 0], rtol=0, atol=1e-12 * pr)
    np.testing.assert_allclose(H.hgks_wall_force(hm, p, Q, None, I.BC_WALL_ISO), [0, -pr, 0], rtol=0, atol=1e-12 * pr)


@pytest.mark.parametrize("scheme", [0, 1], ids=["weno", "hweno"])
def test_wall_force_matches_oracle(cuda, scheme):
    m = I.sphere_mesh(5, 6, stretch=1.3, wall_tag=I.BC_NOSLIP_ADIA)
    cond = I.sphere_conditions(0.2535, Re=118.0)
    om = O.OracleMesh(m)
    hm = H.hgks_mesh_create(m, scheme_mask=3)
    Q, G = I.smooth_state(m, seed=I.BASE_SEED + 92, amp=0.03, base=(1.0, 0.27, 0.01, -0.01, cond["p_inf"]))
    kw = dict(scheme=scheme, Pr=0.72)
    fo = om.wall_force(O.make_params(**cond, **kw), Q, G if scheme else None, I.BC_NOSLIP_ADIA)
    fg = H.hgks_wall_force(hm, H.hgks_default_params(**cond, **kw), hm.to_internal(Q),
                           hm.to_internal(G) if scheme else None, I.BC_NOSLIP_ADIA)
    # scale: the pressure force on one hemisphere, p * pi r^2
    scale = cond["p_inf"] * np.pi * 0.25
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-11 * scale)
    assert np.abs(fo).max() > 1e-3 * scale        # a nonzero force, not a trivial pass
