"""hgks_residual_noalloc: the residual with its scratch in a fixed array inside the
library, for callers that cannot allocate device memory once they are running.

Checked through the C ABI against hgks_residual (the entry point whose scratch
the mesh handle allocated), on two calls in a row, within the residual tolerance
of the parity tests. This file is collected last on purpose."""
import numpy as np
import pytest

import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_R = 1e-11


def euler_scale(m, Q, gamma=1.4):
    V = m.xyz[m.tet4]
    s = np.zeros_like(Q)
    rho = Q[:, 0]; u = Q[:, 1:4] / rho[:, None]
    p = (gamma - 1) * (Q[:, 4] - 0.5 * rho * np.einsum("ij,ij->i", u, u))
    for f in range(4):
        F3 = V[:, [k for k in range(4) if k != f]]
        nrm = np.cross(F3[:, 1] - F3[:, 0], F3[:, 2] - F3[:, 0])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        n = nrm / (2 * area[:, None])
        un = np.einsum("ij,ij->i", u, n)
        Fl = np.stack([rho * un, rho * u[:, 0] * un + p * n[:, 0], rho * u[:, 1] * un + p * n[:, 1],
                       rho * u[:, 2] * un + p * n[:, 2], (Q[:, 4] + p) * un], -1)
        s += area[:, None] * np.abs(Fl)
    return s


@pytest.mark.parametrize("scheme", [0, 1])
def test_noalloc_matches_residual_twice(cuda, scheme):
    import torch
    m = I.cavity_mesh(8)                                   # 3,072 tets, fits the static scratch
    cond = I.cavity_conditions()
    hm = H.hgks_mesh_create(m, scheme_mask=3)
    p = H.hgks_default_params(scheme=scheme, Pr=0.72, **cond)
    Q, G = I.smooth_state(m, amp=0.05, base=(1.0, 0.1, 0.05, -0.03, cond["p_inf"]))
    Qd, Gd = hm.to_internal(Q), hm.to_internal(G)
    Gin = Gd if scheme == 1 else None
    R_ref = torch.empty_like(Qd); G_ref = torch.empty_like(Gd)
    H.hgks_residual(hm, p, Qd, Gin, R_ref, G_ref if scheme == 1 else None)
    scale = euler_scale(m, Q)
    for call in range(2):
        R = torch.full_like(Qd, float("nan")); Gn = torch.full_like(Gd, float("nan"))
        H.hgks_residual_noalloc(hm, p, Qd, Gin, R, Gn if scheme == 1 else None)
        torch.cuda.synchronize()
        err = np.abs(hm.to_caller(R) - hm.to_caller(R_ref)) / scale
        assert err.max() <= TOL_R, (call, err.max())
        if scheme == 1:
            gerr = np.abs(hm.to_caller(Gn) - hm.to_caller(G_ref)).max() / np.abs(hm.to_caller(G_ref)).max()
            assert gerr <= TOL_R, (call, gerr)


def test_noalloc_rejects_meshes_beyond_its_scratch(cuda):
    import torch
    m = I.cavity_mesh(14)                                  # 16,464 tets: more than the scratch holds
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    Q = torch.zeros(5, hm.n_cells, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HGKSError) as e:
        H.hgks_residual_noalloc(hm, H.hgks_default_params(scheme=0), Q, None, Q)
    assert e.value.status == 1 and "too large" in str(e.value)
