"""The Python binding refuses array arguments that the C entry points would
read or write out of bounds (a host array where a device pointer is due,
another dtype, a strided view, a buffer shorter than the mesh needs, an empty
batch slot) with HGKS_ERR_ARG before any pointer reaches the library. CPU only:
a tensor subclass that reports itself as a CUDA tensor stands in for device
memory, and no entry point is called."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2304_09485_gb300 as H


class FakeCuda(torch.Tensor):
    """A CPU tensor that claims to live on the GPU (only the checks look at it)."""

    @property
    def is_cuda(self):
        return True


def fake(*shape, dtype=torch.float64):
    return torch.zeros(*shape, dtype=dtype).as_subclass(FakeCuda)


def refused(fn, *args, word):
    with pytest.raises(H.HGKSError) as e:
        fn(*args)
    assert e.value.status == H.HGKS_ERR_ARG and word in str(e.value), str(e.value)


def test_device_arrays_are_checked():
    n = 10
    ok = fake(5, n)
    assert H._dev(ok, 5, n, "Q") == ok.data_ptr()
    assert H._dev(fake(15 * n), 15, n, "G") is not None      # the layout is the caller's: only the size counts
    assert H._dev(None, 5, n, "Q") is None
    refused(H._dev, torch.zeros(5, n, dtype=torch.float64), 5, n, "Q", word="Q")          # host tensor
    refused(H._dev, np.zeros((5, n)), 5, n, "Q", word="ndarray")                          # numpy array
    refused(H._dev, fake(5, n, dtype=torch.float32), 5, n, "Q", word="float32")           # dtype
    refused(H._dev, fake(n, 5).T, 5, n, "Q", word="contiguous")                           # strided view
    refused(H._dev, fake(5, n - 1), 5, n, "R", word="5 x 10")                             # short buffer


def test_host_arrays_are_checked():
    n = 7
    a = np.zeros((5, n))
    assert H._host(a, 5, n, "Q_host") == a.ctypes.data
    t = torch.zeros(5, n, dtype=torch.float64)
    assert H._host(t, 5, n, "Q_host") == t.data_ptr()
    refused(H._host, np.zeros((5, n), dtype=np.float32), 5, n, "Q_host", word="float32")
    refused(H._host, np.zeros((n, 5)).T, 5, n, "Q_host", word="Q_host")
    refused(H._host, np.zeros((5, n - 1)), 5, n, "Q_host", word="5 x 7")
    refused(H._host, fake(5, n), 5, n, "Q_host", word="Q_host")


def test_single_mesh_calls_check_before_calling_the_library():
    """A mesh object with a NULL handle: every refusal happens in the binding
    (the library would answer HGKS_ERR_ARG for the NULL handle with another message)."""
    m = H.hgks_mesh(0, np.arange(10), 10, faces_per_cell=6)
    p = H.hgks_params()
    Q, G, dt = fake(5, 10), fake(15, 10), fake(10)
    refused(H.hgks_residual, m, p, Q, G, fake(5, 9), word="R")
    refused(H.hgks_residual, m, p, Q, fake(5, 10), fake(5, 10), fake(15, 10), word="G")
    refused(H.hgks_residual_noalloc, m, p, torch.zeros(5, 10, dtype=torch.float64), None, Q, word="Q")
    refused(H.hgks_local_dt, m, p, Q, fake(9), word="dt")
    refused(H.hgks_assemble, m, p, Q, dt, fake(25, 10), fake(100, 10), word="off_out")   # six faces per cell
    refused(H.hgks_apply_jacobian, m, fake(5, 10, dtype=torch.float32), Q, word="x")
    refused(H.hgks_apply_jacobian_fd, m, p, Q, None, dt, Q, fake(4, 10), word="y")
    refused(H.hgks_precondition, m, 2, Q, np.zeros((5, 10)), word="x")
    refused(H.hgks_gmres_step, m, p, Q, G, fake(5, 3), word="dQ_out")
    refused(H.hgks_solve_steady, m, p, fake(10, 5).T, word="Q")
    refused(H.hgks_residual_host, m, p, np.zeros((5, 10)), None, np.zeros((5, 9)), None, word="R_host")
    refused(H.hgks_gmres_step_host, m, p, Q, word="Q_host")


def test_batch_slots_are_checked():
    b = H.hgks_batch(0, [H.hgks_mesh(0, np.arange(8), 8), None], [H.hgks_params(), None])
    refused(H.hgks_batch_set_state, b, 0, fake(5, 7), word="Q")
    refused(H.hgks_batch_get_state, b, 0, None, fake(14, 8), word="G")
    refused(H.hgks_batch_set_state, b, 1, fake(5, 8), word="slot 1")
    refused(H.hgks_batch_get_state, b, 2, fake(5, 8), word="slot 2")


def test_server_submit_checks_the_initial_state():
    from paper_2304_09485_gb300 import inputs as I
    s = object.__new__(H.hgks_server)
    s.handle, s.n_cells = C.c_void_p(0), {}
    m = I.cavity_mesh(2)
    refused(s.submit, m, H.hgks_params(), np.zeros((m.n_tet - 1, 5)), word="need")
    refused(s.submit, m, H.hgks_params(), np.zeros((m.n_tet, 5)), np.zeros((m.n_tet, 5)), word="need")
