"""Flow conditions stated as the paper states them (Mach, Re, angle of attack;
Sec. 5.1, 5.2) give exactly the residual of the explicit free stream, wall
temperature and viscosity the test writes out from the same statement, and
every entry point leaves the caller's current device as it found it."""
import math

import numpy as np
import pytest

import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def explicit_sphere(Mach, Re, aoa_deg, gamma=1.4):
    # (rho, U, V, W, p) = (1, Ma cos a, Ma sin a, 0, 1/gamma), mu = rho U D / Re, D = 1
    a = math.radians(aoa_deg)
    return dict(viscous=1 if Re else 0, mu=Mach / Re if Re else 0.0, rho_inf=1.0,
                u_inf=(Mach * math.cos(a), Mach * math.sin(a), 0.0), p_inf=1.0 / gamma, wall_T=1.0 / gamma)


@pytest.mark.parametrize("Mach,Re,aoa", [(0.3, 0.0, 0.0), (0.5, 0.0, 7.5), (0.2535, 118.0, 0.0)])
def test_sphere_conditions_from_mach_re(cuda, Mach, Re, aoa):
    import torch
    m = I.sphere_mesh(4, 4, stretch=1.3, wall_tag=I.BC_NOSLIP_ADIA)
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    base = H.hgks_default_params(scheme=0, Pr=0.72 if Re else 1.0, **explicit_sphere(Mach, Re, aoa))
    stated = H.hgks_default_params(scheme=0, Pr=0.72 if Re else 1.0, Mach=Mach, Re=Re, aoa_deg=aoa,
                                   viscous=0, mu=0.0, rho_inf=0.0, p_inf=0.0, wall_T=0.0, u_inf=(0.0, 0.0, 0.0))
    Q, _ = I.smooth_state(m, amp=0.03, base=(1.0, Mach, 0.01, -0.01, 1.0 / 1.4))
    Qd = hm.to_internal(Q)
    R1, R2 = torch.empty_like(Qd), torch.empty_like(Qd)
    H.hgks_residual(hm, base, Qd, None, R1)
    H.hgks_residual(hm, stated, Qd, None, R2)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2)
    # and through a whole implicit step
    Q1, Q2 = Qd.clone(), Qd.clone()
    i1 = H.hgks_gmres_step(hm, base, Q1, None)
    i2 = H.hgks_gmres_step(hm, stated, Q2, None)
    assert torch.equal(Q1, Q2) and i1.res_l1 == i2.res_l1


def test_cavity_conditions_from_lid_mach(cuda):
    import torch
    m = I.cavity_mesh(4)
    cond = I.cavity_conditions(0.15, 100.0)
    hm = H.hgks_mesh_create(m, scheme_mask=2)
    base = H.hgks_default_params(scheme=1, Pr=0.72, **cond)
    stated = H.hgks_default_params(scheme=1, Pr=0.72, lid_speed=1.0, Mach=0.15, Re=100.0)
    Q, G = I.smooth_state(m, amp=0.03, base=(1.0, 0.05, 0.02, -0.01, cond["p_inf"]))
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    R1, R2, G1, G2 = (torch.empty_like(x) for x in (Qd, Qd, Gd, Gd))
    H.hgks_residual(hm, base, Qd, Gd, R1, G1)
    H.hgks_residual(hm, stated, Qd, Gd, R2, G2)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2) and torch.equal(G1, G2)


def test_stated_conditions_are_checked(cuda):
    import torch
    m = I.cavity_mesh(3)
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    Q = torch.zeros(5, hm.n_cells, dtype=torch.float64, device="cuda")
    for bad in (dict(Mach=-0.1), dict(Mach=0.3, Re=-1.0), dict(Mach=0.3, aoa_deg=float("nan"))):
        with pytest.raises(H.HGKSError) as e:
            H.hgks_residual(hm, H.hgks_default_params(scheme=0, **bad), Q, None, Q)
        assert e.value.status == 1


def test_entry_points_leave_the_current_device(cuda):
    import torch
    m = I.cavity_mesh(3)
    hm = H.hgks_mesh_create(m, scheme_mask=1, device=0)
    before = torch.cuda.current_device()
    Q = hm.to_internal(I.uniform_state(m.n_tet))
    H.hgks_gmres_step(hm, H.hgks_default_params(scheme=0), Q, None)
    assert torch.cuda.current_device() == before
