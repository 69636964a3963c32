"""The precision workload's comparison with the oracle, on a scaled-down sphere of
its construction: viscous flow (Re 118, Ma 0.2535, adiabatic no-slip wall, CFL 20)
with the compact scheme on a 6 x 8 x 8 cubed-sphere grid of 8 layers (18,432
tets), 20 implicit steps from the free stream through the C ABI, in FP64 and with
the FP32 Krylov part, against the oracle's 20 steps: drag coefficient (Eq. (flux)
summed over the wall faces) and state. FP64 agrees with the oracle to the
steady-state tolerance; the FP32 Krylov basis, Arnoldi products and Jacobi sweeps
change each step's update by ~1e-7 of its size, which stays below 1e-6 of the
state and of C_D over the 20 steps."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_precision_sphere_drag_and_state_against_oracle(cuda):
    import torch
    steps = 20
    cond = I.sphere_conditions(0.2535, Re=118.0)
    kw = dict(scheme=1, Pr=0.72, cfl=20.0, krylov_dim=10, restarts=3, jacobi_sweeps=2)
    qinf = 0.5 * cond["rho_inf"] * cond["u_inf"][0] ** 2 * math.pi * 0.25
    m = I.sphere_mesh(8, 8, stretch=I.sphere_stretch(8, dr1=3e-2 * 3), wall_tag=I.BC_NOSLIP_ADIA)
    om = O.OracleMesh(m)
    hm = H.hgks_mesh_create(m, scheme_mask=2)
    Q0 = I.state_from_conditions(m.n_tet, cond)
    G0 = np.zeros((m.n_tet, 15))
    po = O.make_params(**cond, **kw)
    Qr, Gr = Q0.copy(), G0.copy()
    for _ in range(steps):
        Qr, Gr, _, _ = om.gmres_step(po, Qr, Gr)
    cd_o = float(om.wall_force(po, Qr, Gr, I.BC_NOSLIP_ADIA)[0] / qinf)
    for prec, tol_cd, tol_q in ((0, 1e-10, 1e-9), (1, 1e-6, 1e-6)):
        p = H.hgks_default_params(precision=prec, **cond, **kw)
        Q, G = hm.to_internal(Q0), hm.to_internal(G0)
        for _ in range(steps):
            H.hgks_gmres_step(hm, p, Q, G)
        cd = float(H.hgks_wall_force(hm, p, Q, G, I.BC_NOSLIP_ADIA)[0] / qinf)
        Qg = hm.to_caller(Q)
        assert abs(cd - cd_o) <= tol_cd * abs(cd_o), (prec, cd, cd_o)
        assert np.linalg.norm(Qg - Qr) <= tol_q * np.linalg.norm(Qr), prec
