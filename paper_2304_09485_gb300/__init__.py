"""GB300-native implicit high-order gas-kinetic scheme (HGKS) hot path.

Python binding of libhgks (include/hgks.h): the same entry points, argument
marshalling only. Every step of the residual and of the GMRES step runs in the
library's CUDA kernels; PyTorch provides device memory and streams. If the
library is missing or no CUDA device is present the calls raise; nothing
falls back to a CPU path.

Device state arrays are torch tensors in the library's internal cell order and
component-major layout: Q [5, N], G [15, N] (row 3*c + d), R [5, N].
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native

HGKS_OK = 0
HGKS_ERR_ARG = 1
HGKS_ERR_NONPHYSICAL = 5
HGKS_ERR_NOT_CONVERGED = 7
HGKS_ERR_CANCELLED = 9
HGKS_WENO, HGKS_HWENO = 0, 1
HGKS_NONLINEAR, HGKS_LINEAR = 0, 1
HGKS_FP64, HGKS_MIXED = 0, 1


class hgks_params(C.Structure):
    _fields_ = [("scheme", C.c_int32), ("weights", C.c_int32), ("viscous", C.c_int32),
                ("characteristic", C.c_int32), ("precision", C.c_int32), ("jv_mode", C.c_int32),
                ("krylov_dim", C.c_int32), ("restarts", C.c_int32), ("jacobi_sweeps", C.c_int32),
                ("tstar_end", C.c_int32),
                ("gamma", C.c_double), ("Pr", C.c_double), ("mu", C.c_double), ("cfl", C.c_double),
                ("flux_cfl", C.c_double), ("tau_eps", C.c_double), ("tau_C", C.c_double),
                ("lin_weight", C.c_double), ("weno_eps", C.c_double), ("flux_dt", C.c_double),
                ("rho_inf", C.c_double), ("u_inf", C.c_double * 3), ("p_inf", C.c_double),
                ("wall_T", C.c_double), ("lid_speed", C.c_double),
                ("Mach", C.c_double), ("Re", C.c_double), ("aoa_deg", C.c_double), ("grad_relax", C.c_double)]


class hgks_mesh_info_t(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_faces", C.c_int64), ("n_boundary_faces", C.c_int64),
                ("device_bytes", C.c_int64), ("device", C.c_int32), ("schemes", C.c_int32),
                ("faces_per_cell", C.c_int32), ("reserved", C.c_int32)]


class hgks_step_info(C.Structure):
    _fields_ = [("res_l1", C.c_double), ("lin_res", C.c_double * 2), ("krylov_iters", C.c_int32),
                ("nonphysical", C.c_int32)]


class hgks_solve_info(C.Structure):
    _fields_ = [("steps", C.c_int32), ("converged", C.c_int32), ("res_ref", C.c_double),
                ("res_final", C.c_double)]


class hgks_batch_info_t(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_faces", C.c_int64), ("device_bytes", C.c_int64),
                ("n_meshes", C.c_int32), ("blk_recon", C.c_int32), ("blk_flux", C.c_int32)]


class hgks_request_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("n_cells", C.c_int64), ("solve", hgks_solve_info),
                ("t_submit", C.c_double), ("t_built", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class HGKSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hgks status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = _native.load()
        vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.c_void_p
        P = C.POINTER(hgks_params)
        sig = {
            "hgks_default_params": [P],
            "hgks_mesh_create": [dp, i64, dp, i64, dp, dp, i64, dp, i32, i32, i32, C.POINTER(vp), dp],
            "hgks_mesh_create_hex": [dp, i64, dp, i64, dp, dp, i64, dp, i32, i32, i32, C.POINTER(vp), dp],
            "hgks_mesh_destroy": [vp],
            "hgks_mesh_info": [vp, C.POINTER(hgks_mesh_info_t)],
            "hgks_mesh_volumes": [vp, dp],
            "hgks_residual": [vp, P, dp, dp, dp, dp, vp],
            "hgks_local_dt": [vp, P, dp, dp, vp],
            "hgks_assemble": [vp, P, dp, dp, dp, dp, vp],
            "hgks_apply_jacobian": [vp, dp, dp, vp],
            "hgks_apply_jacobian_fd": [vp, P, dp, dp, dp, dp, dp, vp],
            "hgks_wall_force": [vp, P, dp, dp, i32, dp, vp],
            "hgks_precondition": [vp, i32, dp, dp, vp],
            "hgks_gmres_step": [vp, P, dp, dp, dp, C.POINTER(hgks_step_info), vp],
            "hgks_solve_steady": [vp, P, dp, dp, C.c_double, i32, dp, C.POINTER(hgks_solve_info), vp],
            "hgks_solve_resume": [vp, P, dp, dp, C.c_double, i32, C.POINTER(hgks_solve_info), dp,
                                  C.POINTER(hgks_solve_info), vp],
            "hgks_residual_host": [vp, P, dp, dp, dp, dp, vp],
            "hgks_gmres_step_host": [vp, P, dp, dp, C.POINTER(hgks_step_info), vp],
            "hgks_sync": [vp],
            "hgks_residual_noalloc": [vp, P, dp, dp, dp, dp, vp],
            "hgks_batch_create": [dp, P, i32, C.POINTER(vp)],
            "hgks_batch_destroy": [vp],
            "hgks_batch_create_empty": [i32, i64, i64, i32, P, C.POINTER(vp)],
            "hgks_batch_create_empty_hex": [i32, i64, i64, i32, P, C.POINTER(vp)],
            "hgks_batch_add": [vp, vp, P, C.POINTER(C.c_int32)],
            "hgks_batch_remove": [vp, i32],
            "hgks_server_create": [i32, i64, i32, P, i32, C.POINTER(vp)],
            "hgks_server_create_hex": [i32, i64, i32, P, i32, C.POINTER(vp)],
            "hgks_server_destroy": [vp],
            "hgks_server_submit": [vp, dp, i64, dp, i64, dp, dp, i64, dp, i32, P, dp, dp, C.c_double, i32,
                                   C.POINTER(C.c_int64)],
            "hgks_server_submit_hex": [vp, dp, i64, dp, i64, dp, dp, i64, dp, i32, P, dp, dp, C.c_double, i32,
                                       C.POINTER(C.c_int64)],
            "hgks_server_step": [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
            "hgks_server_status": [vp, i64, C.POINTER(hgks_request_info)],
            "hgks_server_collect": [vp, i64, dp, dp],
            "hgks_server_cancel": [vp, i64],
            "hgks_server_info": [vp, C.POINTER(hgks_batch_info_t)],
            "hgks_batch_info": [vp, C.POINTER(hgks_batch_info_t)],
            "hgks_batch_set_state": [vp, i32, dp, dp, vp],
            "hgks_batch_get_state": [vp, i32, dp, dp, dp, dp, vp],
            "hgks_batch_residual": [vp, vp],
            "hgks_batch_gmres_step": [vp, dp, i32, vp],
            "hgks_batch_solve_steady": [vp, C.c_double, i32, i32, dp, dp, vp],
            "hgks_batch_autotune": [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), vp],
            "hgks_profile_begin": [],
            "hgks_fp64_peak": [i32, C.c_double, C.POINTER(C.c_double)],
            "hgks_profile_end": [i32, dp, dp, dp, C.POINTER(C.c_int32)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.hgks_last_error.restype = C.c_char_p
        L.hgks_launch_count.restype = C.c_int64
        L.hgks_launch_count.argtypes = [i32]
        _lib = L
    return _lib


def _check(st, allow=()):
    if st != HGKS_OK and st not in allow:
        raise HGKSError(st, lib().hgks_last_error().decode())
    return st


def _ptr(t):
    """Device (torch) or host (numpy) data pointer, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _dev(t, rows, n, name):
    """Data pointer of a device-array argument, or None for NULL. The C entry
    points take raw double pointers and their kernels touch rows x n values, so
    anything but a contiguous float64 CUDA tensor of at least that many values (a
    host array, another dtype, a strided view, a short buffer) is refused here
    with HGKS_ERR_ARG instead of being read or written out of bounds on the GPU."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and t.numel() >= rows * n):
        raise HGKSError(HGKS_ERR_ARG, f"{name}: expected a contiguous float64 CUDA tensor of at least "
                                      f"{rows} x {n} values, got {_describe(t)}")
    return t.data_ptr()


def _host(a, rows, n, name):
    """Data pointer of a host-array argument (a C-contiguous float64 numpy array
    or CPU tensor of at least rows x n values), or None; otherwise HGKS_ERR_ARG."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype == np.float64 and a.flags.c_contiguous and a.size >= rows * n:
            return a.ctypes.data
    else:
        import torch
        if (isinstance(a, torch.Tensor) and not a.is_cuda and a.device.type == "cpu" and a.dtype == torch.float64
                and a.is_contiguous() and a.numel() >= rows * n):
            return a.data_ptr()
    raise HGKSError(HGKS_ERR_ARG, f"{name}: expected a C-contiguous float64 host array of at least "
                                  f"{rows} x {n} values, got {_describe(a)}")


def _describe(t):
    what = f"{type(t).__name__} {getattr(t, 'dtype', '')} {tuple(getattr(t, 'shape', ()))}"
    dev = getattr(t, "device", None)
    return what + (f" on {dev}" if dev is not None else "")


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def hgks_default_params(**overrides) -> hgks_params:
    p = hgks_params()
    _check(lib().hgks_default_params(C.byref(p)))
    for k, v in overrides.items():
        if k == "u_inf":
            p.u_inf[:] = list(v)
        else:
            setattr(p, k, v)
    return p


class hgks_mesh:
    """A mesh handle; .perm[internal] = caller cell index."""

    def __init__(self, handle, perm, n_cells, faces_per_cell=4):
        self.handle = C.c_void_p(handle)
        self.faces_per_cell = faces_per_cell
        self.perm = perm
        self.inv = np.empty_like(perm)
        self.inv[perm] = np.arange(len(perm))
        self.n_cells = n_cells

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            try:
                lib().hgks_mesh_destroy(self.handle)
            except Exception:
                pass
            self.handle = C.c_void_p(0)

    # marshalling between caller order [n, k] and internal component-major [k, n]
    def to_internal(self, A, device="cuda"):
        import torch
        a = np.ascontiguousarray(np.asarray(A, dtype=np.float64)[self.perm].T)
        return torch.from_numpy(a).to(device)

    def to_caller(self, T):
        a = T.detach().cpu().numpy() if hasattr(T, "detach") else np.asarray(T)
        return np.ascontiguousarray(a.T[self.inv])


def hgks_mesh_create(mesh, scheme_mask=3, device=0) -> hgks_mesh:
    """Build a library mesh from an inputs.Mesh (tetrahedra: hgks_mesh_create) or
    an inputs.HexMesh (hexahedra: hgks_mesh_create_hex); host arrays, caller order."""
    hexa = hasattr(mesh, "hex8")
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    cells = np.ascontiguousarray(mesh.hex8 if hexa else mesh.tet4, dtype=np.int64)
    nfv = 4 if hexa else 3
    bf = np.ascontiguousarray(mesh.bface4 if hexa else mesh.bface3, dtype=np.int64).reshape(-1, nfv)
    bt = np.ascontiguousarray(mesh.btag, dtype=np.int32)
    ps = mesh.periodic_shift
    psa = np.ascontiguousarray(ps if ps is not None else np.zeros((0, 3)), dtype=np.float64)
    perm = np.zeros(max(1, cells.shape[0]), dtype=np.int64)
    h = C.c_void_p()
    fn = lib().hgks_mesh_create_hex if hexa else lib().hgks_mesh_create
    _check(fn(_ptr(xyz), xyz.shape[0], _ptr(cells), cells.shape[0], _ptr(bf) if len(bf) else None,
              _ptr(bt) if len(bt) else None, bf.shape[0], _ptr(psa) if len(psa) else None,
              psa.shape[0], scheme_mask, device, C.byref(h), _ptr(perm)))
    return hgks_mesh(h.value, perm[: cells.shape[0]], cells.shape[0], 6 if hexa else 4)


def hgks_mesh_info(mesh: hgks_mesh) -> hgks_mesh_info_t:
    info = hgks_mesh_info_t()
    _check(lib().hgks_mesh_info(mesh.handle, C.byref(info)))
    return info


def hgks_mesh_volumes(mesh: hgks_mesh) -> np.ndarray:
    v = np.zeros(mesh.n_cells)
    _check(lib().hgks_mesh_volumes(mesh.handle, _ptr(v)))
    return v


def hgks_residual(mesh, params, Q, G, R, G_new=None, stream=None):
    n = mesh.n_cells
    _check(lib().hgks_residual(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"),
                               _dev(R, 5, n, "R"), _dev(G_new, 15, n, "G_new"), _stream(stream)))


def hgks_residual_noalloc(mesh, params, Q, G, R, G_new=None, stream=None):
    """hgks_residual with its scratch in the library's fixed static array (no allocation)."""
    n = mesh.n_cells
    _check(lib().hgks_residual_noalloc(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"),
                                       _dev(R, 5, n, "R"), _dev(G_new, 15, n, "G_new"), _stream(stream)))


def hgks_local_dt(mesh, params, Q, dt, stream=None):
    n = mesh.n_cells
    _check(lib().hgks_local_dt(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(dt, 1, n, "dt"),
                               _stream(stream)))


def hgks_assemble(mesh, params, Q, dt, diag_out=None, off_out=None, stream=None):
    n = mesh.n_cells
    _check(lib().hgks_assemble(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(dt, 1, n, "dt"),
                               _dev(diag_out, 25, n, "diag_out"),
                               _dev(off_out, 25 * mesh.faces_per_cell, n, "off_out"), _stream(stream)))


def hgks_apply_jacobian(mesh, x, y, stream=None):
    n = mesh.n_cells
    _check(lib().hgks_apply_jacobian(mesh.handle, _dev(x, 5, n, "x"), _dev(y, 5, n, "y"), _stream(stream)))


def hgks_apply_jacobian_fd(mesh, params, Q, G, dt, x, y, stream=None):
    n = mesh.n_cells
    _check(lib().hgks_apply_jacobian_fd(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"),
                                        _dev(dt, 1, n, "dt"), _dev(x, 5, n, "x"), _dev(y, 5, n, "y"),
                                        _stream(stream)))


def hgks_wall_force(mesh, params, Q, G, tag, stream=None) -> np.ndarray:
    f = np.zeros(3)
    n = mesh.n_cells
    _check(lib().hgks_wall_force(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"), tag,
                                 _ptr(f), _stream(stream)))
    return f


def hgks_precondition(mesh, sweeps, b, x, stream=None):
    n = mesh.n_cells
    _check(lib().hgks_precondition(mesh.handle, sweeps, _dev(b, 5, n, "b"), _dev(x, 5, n, "x"), _stream(stream)))


def hgks_gmres_step(mesh, params, Q, G=None, dQ_out=None, stream=None) -> hgks_step_info:
    info = hgks_step_info()
    n = mesh.n_cells
    _check(lib().hgks_gmres_step(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"),
                                 _dev(dQ_out, 5, n, "dQ_out"), C.byref(info), _stream(stream)))
    return info


def hgks_solve_steady(mesh, params, Q, G=None, drop_tol=1e-8, max_steps=1000, stream=None):
    hist = np.zeros(max_steps + 1)
    info = hgks_solve_info()
    n = mesh.n_cells
    st = _check(lib().hgks_solve_steady(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"),
                                        drop_tol, max_steps,
                                        _ptr(hist), C.byref(info), _stream(stream)), allow=(HGKS_ERR_NOT_CONVERGED,))
    return info, hist[: info.steps + 1], st == HGKS_OK


def hgks_solve_resume(mesh, params, Q, G, frm, drop_tol=1e-8, max_steps=1000, stream=None):
    """Continue a solve from its state and hgks_solve_info: (info, hist [absolute steps], converged)."""
    hist = np.zeros(max_steps + 1)
    info = hgks_solve_info()
    n = mesh.n_cells
    st = _check(lib().hgks_solve_resume(mesh.handle, C.byref(params), _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"),
                                        drop_tol, max_steps,
                                        C.byref(frm), _ptr(hist), C.byref(info), _stream(stream)),
                allow=(HGKS_ERR_NOT_CONVERGED,))
    return info, hist[: info.steps + 1], st == HGKS_OK


def hgks_residual_host(mesh, params, Q_host, G_host, R_host, G_new_host, stream=None):
    n = mesh.n_cells
    _check(lib().hgks_residual_host(mesh.handle, C.byref(params), _host(Q_host, 5, n, "Q_host"),
                                    _host(G_host, 15, n, "G_host"), _host(R_host, 5, n, "R_host"),
                                    _host(G_new_host, 15, n, "G_new_host"), _stream(stream)))


def hgks_gmres_step_host(mesh, params, Q_host, G_host=None, stream=None) -> hgks_step_info:
    info = hgks_step_info()
    n = mesh.n_cells
    _check(lib().hgks_gmres_step_host(mesh.handle, C.byref(params), _host(Q_host, 5, n, "Q_host"),
                                      _host(G_host, 15, n, "G_host"), C.byref(info), _stream(stream)))
    return info


class hgks_batch:
    """A batch handle over several meshes (hgks_batch_create); keeps the meshes' order."""

    def __init__(self, handle, meshes, params):
        self.handle = C.c_void_p(handle)
        self.meshes = list(meshes)
        self.params = list(params)

    def __len__(self):
        return len(self.meshes)

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            try:
                lib().hgks_batch_destroy(self.handle)
            except Exception:
                pass
            self.handle = C.c_void_p(0)


def hgks_batch_create(meshes, params) -> hgks_batch:
    n = len(meshes)
    hs = (C.c_void_p * n)(*[m.handle.value for m in meshes])
    ps = (hgks_params * n)(*params)
    h = C.c_void_p()
    _check(lib().hgks_batch_create(C.addressof(hs), ps, n, C.byref(h)))
    return hgks_batch(h.value, meshes, params)


def hgks_batch_create_empty(cell_capacity, face_capacity, max_meshes, shared, device=0, hexahedra=False) -> hgks_batch:
    h = C.c_void_p()
    fn = lib().hgks_batch_create_empty_hex if hexahedra else lib().hgks_batch_create_empty
    _check(fn(device, cell_capacity, face_capacity, max_meshes, C.byref(shared), C.byref(h)))
    b = hgks_batch(h.value, [None] * max_meshes, [None] * max_meshes)
    return b


def hgks_batch_add(batch, mesh, params) -> int:
    k = C.c_int32(-1)
    _check(lib().hgks_batch_add(batch.handle, mesh.handle, C.byref(params), C.byref(k)))
    batch.meshes[k.value] = mesh
    batch.params[k.value] = params
    return k.value


def hgks_batch_remove(batch, k):
    _check(lib().hgks_batch_remove(batch.handle, k))
    batch.meshes[k] = None
    batch.params[k] = None


def hgks_batch_info(batch) -> hgks_batch_info_t:
    info = hgks_batch_info_t()
    _check(lib().hgks_batch_info(batch.handle, C.byref(info)))
    return info


def _slot_cells(batch, k):
    """Cells of the mesh in slot k (HGKS_ERR_ARG for a slot out of range or empty)."""
    if not (0 <= k < len(batch.meshes)) or batch.meshes[k] is None:
        raise HGKSError(HGKS_ERR_ARG, f"batch slot {k} holds no mesh")
    return batch.meshes[k].n_cells


def hgks_batch_set_state(batch, k, Q, G=None, stream=None):
    n = _slot_cells(batch, k)
    _check(lib().hgks_batch_set_state(batch.handle, k, _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"), _stream(stream)))


def hgks_batch_get_state(batch, k, Q=None, G=None, R=None, G_new=None, stream=None):
    n = _slot_cells(batch, k)
    _check(lib().hgks_batch_get_state(batch.handle, k, _dev(Q, 5, n, "Q"), _dev(G, 15, n, "G"), _dev(R, 5, n, "R"),
                                      _dev(G_new, 15, n, "G_new"), _stream(stream)))


def hgks_batch_residual(batch, stream=None):
    _check(lib().hgks_batch_residual(batch.handle, _stream(stream)))


def hgks_batch_gmres_step(batch, use_graph=True, stream=None):
    info = (hgks_step_info * len(batch))()
    _check(lib().hgks_batch_gmres_step(batch.handle, info, 1 if use_graph else 0, _stream(stream)))
    return list(info)


def hgks_batch_solve_steady(batch, drop_tol=1e-8, max_steps=1000, use_graph=True, stream=None, raise_nonfinite=True):
    """(infos, hist [n, max_steps+1], all_converged) of Algorithm 1 run on every mesh of the batch.
    With raise_nonfinite=False a mesh whose residual went non-finite does not raise: its
    record shows it (res_final not finite) and all_converged is False."""
    n = len(batch)
    hist = np.zeros((n, max_steps + 1))
    info = (hgks_solve_info * n)()
    allow = (HGKS_ERR_NOT_CONVERGED,) if raise_nonfinite else (HGKS_ERR_NOT_CONVERGED, HGKS_ERR_NONPHYSICAL)
    st = _check(lib().hgks_batch_solve_steady(batch.handle, drop_tol, max_steps, 1 if use_graph else 0, _ptr(hist),
                                              info, _stream(stream)), allow=allow)
    return list(info), hist, st == HGKS_OK


def hgks_batch_autotune(batch, stream=None):
    r, f = C.c_int32(0), C.c_int32(0)
    _check(lib().hgks_batch_autotune(batch.handle, C.byref(r), C.byref(f), _stream(stream)))
    return r.value, f.value


class hgks_server:
    """Continuous-batching request server (hgks_server_*); hexahedra=True makes a
    server of hexahedral meshes (hgks_server_create_hex)."""

    def __init__(self, shared, hbm_budget_bytes, max_inflight=64, use_graph=True, device=0, hexahedra=False):
        h = C.c_void_p()
        fn = lib().hgks_server_create_hex if hexahedra else lib().hgks_server_create
        _check(fn(device, int(hbm_budget_bytes), max_inflight, C.byref(shared), 1 if use_graph else 0, C.byref(h)))
        self.handle = h
        self.n_cells = {}

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value:
            try:
                lib().hgks_server_destroy(self.handle)
            except Exception:
                pass
            self.handle = C.c_void_p(0)

    def submit(self, mesh, params, Q0, G0=None, drop_tol=1e-8, max_steps=1000) -> int:
        """Queue a solve of an inputs.Mesh (or inputs.HexMesh) from Q0 (caller order
        [n, 5]); returns its id."""
        hexa = hasattr(mesh, "hex8")
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        tet = np.ascontiguousarray(mesh.hex8 if hexa else mesh.tet4, dtype=np.int64)
        bf = np.ascontiguousarray(mesh.bface4 if hexa else mesh.bface3, dtype=np.int64).reshape(-1, 4 if hexa else 3)
        bt = np.ascontiguousarray(mesh.btag, dtype=np.int32)
        ps = mesh.periodic_shift
        psa = np.ascontiguousarray(ps if ps is not None else np.zeros((0, 3)), dtype=np.float64)
        q = np.ascontiguousarray(Q0, dtype=np.float64)
        g = None if G0 is None else np.ascontiguousarray(G0, dtype=np.float64)
        n = tet.shape[0]
        if q.size < 5 * n or (g is not None and g.size < 15 * n):
            raise HGKSError(HGKS_ERR_ARG, f"Q0 / G0 hold {q.size} / {0 if g is None else g.size} values, "
                                          f"the mesh's {n} cells need {5 * n} / {15 * n}")
        rid = C.c_int64(0)
        fn = lib().hgks_server_submit_hex if hexa else lib().hgks_server_submit
        _check(fn(self.handle, _ptr(xyz), xyz.shape[0], _ptr(tet), tet.shape[0],
                  _ptr(bf) if len(bf) else None, _ptr(bt) if len(bt) else None, bf.shape[0],
                  _ptr(psa) if len(psa) else None, psa.shape[0], C.byref(params), _ptr(q),
                  _ptr(g), drop_tol, max_steps, C.byref(rid)))
        self.n_cells[rid.value] = tet.shape[0]
        return rid.value

    def step(self):
        """One scheduling round: (finished in this round, running, waiting)."""
        f, r, w = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        _check(lib().hgks_server_step(self.handle, C.byref(f), C.byref(r), C.byref(w)))
        return f.value, r.value, w.value

    def status(self, rid) -> hgks_request_info:
        info = hgks_request_info()
        _check(lib().hgks_server_status(self.handle, rid, C.byref(info)))
        return info

    def cancel(self, rid):
        _check(lib().hgks_server_cancel(self.handle, rid))

    def collect(self, rid, with_gradients=False):
        n = self.n_cells.pop(rid)
        Q = np.zeros((n, 5))
        G = np.zeros((n, 15)) if with_gradients else None
        _check(lib().hgks_server_collect(self.handle, rid, _ptr(Q), _ptr(G)))
        return Q, G

    def info(self) -> hgks_batch_info_t:
        info = hgks_batch_info_t()
        _check(lib().hgks_server_info(self.handle, C.byref(info)))
        return info


def hgks_sync(stream=None):
    _check(lib().hgks_sync(_stream(stream)))


def hgks_profile_begin():
    _check(lib().hgks_profile_begin())


def hgks_profile_end(max_kernels=32):
    """{kernel name: (total ms, launches)} of the kernels timed since hgks_profile_begin()."""
    names = C.create_string_buffer(32 * max_kernels)
    ms = np.zeros(max_kernels)
    cnt = np.zeros(max_kernels, dtype=np.int64)
    n = C.c_int32(0)
    _check(lib().hgks_profile_end(max_kernels, C.addressof(names), _ptr(ms), _ptr(cnt), C.byref(n)))
    out = {}
    for k in range(min(n.value, max_kernels)):
        nm = names.raw[32 * k:32 * k + 32].split(b"\0")[0].decode()
        out[nm] = (float(ms[k]), int(cnt[k]))
    return out


def hgks_launch_count(reset=False) -> int:
    return int(lib().hgks_launch_count(1 if reset else 0))


def hgks_fp64_peak(device=0, seconds=2.0) -> float:
    """Measured FP64 FMA rate of the device in GFLOP/s (the FP64 roofline)."""
    g = C.c_double(0)
    _check(lib().hgks_fp64_peak(int(device), float(seconds), C.byref(g)))
    return g.value
