"""hgks_residual_noalloc: the residual with its scratch in a fixed array inside the
library, for callers that cannot allocate device memory once they are running
(device memory handed to another runtime at start-up, or a service that must not
enter the CUDA allocator while it answers requests).

Checked through the C ABI against hgks_residual (the entry point whose scratch
the mesh handle allocated), on two calls in a row. Both run the same kernels in
the same order on the same data, so the results must agree bit for bit (well
inside the 1e-11 residual tolerance of the parity tests). The handle given to
the no-allocation call has never run hgks_residual itself, the reference comes
from a second handle of the same mesh, and free device memory must not change
across a call once the static array is in place. This file is collected last on
purpose."""
import numpy as np
import pytest

import paper_2304_09485_gb300 as H
from paper_2304_09485_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme", [0, 1])
def test_noalloc_matches_residual_twice(cuda, scheme):
    import torch
    m = I.cavity_mesh(8)                                   # 3,072 tets, fits the static scratch
    cond = I.cavity_conditions()
    p = H.hgks_default_params(scheme=scheme, Pr=0.72, **cond)
    Q, G = I.smooth_state(m, amp=0.05, base=(1.0, 0.1, 0.05, -0.03, cond["p_inf"]))
    fresh = H.hgks_mesh_create(m, scheme_mask=3)           # only ever used by the no-allocation call
    ref = H.hgks_mesh_create(m, scheme_mask=3)
    assert np.array_equal(fresh.perm, ref.perm)
    Qd, Gd = fresh.to_internal(Q), fresh.to_internal(G)
    Gin = Gd if scheme == 1 else None
    R_ref = torch.empty_like(Qd); G_ref = torch.empty_like(Gd)
    H.hgks_residual(ref, p, Qd, Gin, R_ref, G_ref if scheme == 1 else None)
    torch.cuda.synchronize()
    dev_before = torch.cuda.current_device()
    for call in range(2):
        R = torch.full_like(Qd, float("nan")); Gn = torch.full_like(Gd, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        H.hgks_residual_noalloc(fresh, p, Qd, Gin, R, Gn if scheme == 1 else None)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert torch.equal(R, R_ref), (call, (R - R_ref).abs().max().item())
        if scheme == 1:
            assert torch.equal(Gn, G_ref), (call, (Gn - G_ref).abs().max().item())
        if call == 1:
            # the static array was loaded by the first call: nothing is allocated now
            assert free1 == free0, (free0, free1)
    assert torch.cuda.current_device() == dev_before


def test_noalloc_rejects_meshes_beyond_its_scratch(cuda):
    import torch
    m = I.cavity_mesh(14)                                  # 16,464 tets: more than the scratch holds
    hm = H.hgks_mesh_create(m, scheme_mask=1)
    Q = torch.zeros(5, hm.n_cells, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HGKSError) as e:
        H.hgks_residual_noalloc(hm, H.hgks_default_params(scheme=0), Q, None, Q)
    assert e.value.status == 1 and "too large" in str(e.value)
