"""Oracle: a plain FP64 CPU restatement of the implicit HGKS method.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference arm may import this package. It shares no code with
the CUDA library (paper_2304_09485_gb300) and neither imports the other; the
only common module is the seeded input generator
paper_2304_09485_gb300.inputs, which holds none of the method's arithmetic.

The C sources (orc_*.c) restate the paper step by step; this file loads them
through ctypes and converts between numpy arrays and C pointers. Arrays are in
the caller's cell order: Q [n,5], G [n,15] (component-major: 3*c + d).

Parity unpinned: the local time step beyond its scaling invariants (the paper
gives no formula) and the boundary states beyond their involution, rest-state,
wall-symmetry and mass properties and the uniform flows they leave steady;
every other routine has pins in tests/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_linalg.c", "orc_mesh.c", "orc_gks.c", "orc_recon.c", "orc_solver.c"]
LIBNAME = os.path.join(HERE, "_build", "liboracle.so")


# A test that plants a mistake in the oracle builds a modified copy of the
# sources elsewhere (compile_library) and points this variable at it; lib()
# then loads that copy instead of building the oracle.
PLANTED_ENV = "HGKS_ORACLE_LIB"


def compile_library(src_dir: str, out_path: str) -> str:
    """gcc (-O2, OpenMP, no FP contraction) of the oracle sources in src_dir."""
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp] + [os.path.join(src_dir, s) for s in SOURCES] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile the oracle in place (oracle/_build/liboracle.so)."""
    os.makedirs(os.path.dirname(LIBNAME), exist_ok=True)
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "orc.h")]
    if not force and os.path.exists(LIBNAME):
        t = os.path.getmtime(LIBNAME)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIBNAME
    return compile_library(HERE, LIBNAME)


class Params(C.Structure):
    _fields_ = [("scheme", C.c_int32), ("weights", C.c_int32), ("viscous", C.c_int32),
                ("characteristic", C.c_int32), ("krylov_dim", C.c_int32), ("restarts", C.c_int32),
                ("jacobi_sweeps", C.c_int32), ("tstar_end", C.c_int32), ("jv_mode", C.c_int32),
                ("gamma", C.c_double), ("Pr", C.c_double), ("mu", C.c_double), ("cfl", C.c_double), ("flux_cfl", C.c_double),
                ("tau_eps", C.c_double), ("tau_C", C.c_double), ("lin_weight", C.c_double),
                ("weno_eps", C.c_double), ("flux_dt", C.c_double),
                ("rho_inf", C.c_double), ("u_inf", C.c_double * 3), ("p_inf", C.c_double),
                ("wall_T", C.c_double), ("lid_speed", C.c_double), ("grad_relax", C.c_double)]


def make_params(**kw) -> Params:
    """Parameters with the paper's defaults (Sec. 3.4, Sec. 4, Sec. 5)."""
    d = dict(scheme=0, weights=0, viscous=0, characteristic=1, krylov_dim=10, restarts=3,
             jacobi_sweeps=2, tstar_end=1, jv_mode=0, gamma=1.4, Pr=1.0, mu=0.0, cfl=10.0, flux_cfl=1.0, tau_eps=0.1,
             tau_C=1.0, lin_weight=0.025, weno_eps=1e-6, flux_dt=0.0, rho_inf=1.0,
             u_inf=(0.3, 0.0, 0.0), p_inf=1.0 / 1.4, wall_T=1.0 / 1.4, lid_speed=0.0,
             grad_relax=1.0)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        if k == "u_inf":
            p.u_inf[:] = list(v)
        else:
            setattr(p, k, v)
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get(PLANTED_ENV) or build()
        L = C.CDLL(path)
        vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
        L.orc_mesh_create_cells.restype = vp
        L.orc_mesh_create_cells.argtypes = [dp, i64, C.POINTER(C.c_int64), C.c_int32, i64, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int32), i64, dp, i32, C.c_char_p, C.c_int]
        L.orc_mesh_destroy.argtypes = [vp]
        for name in ["orc_residual", "orc_residual_dt", "orc_apply_fd", "orc_wall_force", "orc_local_dt", "orc_jacobian",
                     "orc_precondition", "orc_gmres",
                     "orc_gmres_step", "orc_solve_steady", "orc_recon_side", "orc_fit_cell", "orc_slope",
                     "orc_lu_solve", "orc_inverse", "orc_stencil"]:
            getattr(L, name).restype = C.c_int
        L.orc_set_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_monomial_moment.restype = C.c_double
        L.orc_monomial_moment.argtypes = [dp, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pi(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


# mesh struct field offsets are read through a mirror of the C struct
class _MeshC(C.Structure):
    _fields_ = [("nv", C.c_int64), ("nc", C.c_int64), ("nf", C.c_int64),
                ("xyz", C.POINTER(C.c_double)), ("cv", C.POINTER(C.c_int64)),
                ("vol", C.POINTER(C.c_double)), ("cen", C.POINTER(C.c_double)), ("h", C.POINTER(C.c_double)),
                ("cface", C.POINTER(C.c_int64)), ("cnb", C.POINTER(C.c_int64)), ("cshift", C.POINTER(C.c_double)),
                ("cside", C.POINTER(C.c_int32)), ("fl", C.POINTER(C.c_int64)), ("fr", C.POINTER(C.c_int64)),
                ("flp", C.POINTER(C.c_int32)), ("frp", C.POINTER(C.c_int32)), ("ftag", C.POINTER(C.c_int32)),
                ("farea", C.POINTER(C.c_double)), ("fnrm", C.POINTER(C.c_double)), ("fgp", C.POINTER(C.c_double)),
                ("fshift", C.POINTER(C.c_double)), ("fcen", C.POINTER(C.c_double)), ("fit", C.c_void_p),
                ("nvc", C.c_int32), ("nfc", C.c_int32), ("ngp", C.c_int32), ("pad", C.c_int32),
                ("fgw", C.POINTER(C.c_double))]


class OracleMesh:
    """An oracle mesh built from an inputs.Mesh or inputs.HexMesh (caller order)."""

    def __init__(self, mesh):
        L = lib()
        self.mesh = mesh
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        cells = np.ascontiguousarray(mesh.cells, dtype=np.int64)
        nvc = cells.shape[1]
        bf = np.ascontiguousarray(mesh.bface4 if nvc == 8 else mesh.bface3, dtype=np.int64).reshape(-1, 4 if nvc == 8 else 3)
        bt = np.ascontiguousarray(mesh.btag, dtype=np.int32)
        ps = mesh.periodic_shift
        psa = np.ascontiguousarray(ps if ps is not None else np.zeros((0, 3)), dtype=np.float64)
        err = C.create_string_buffer(256)
        self.h = L.orc_mesh_create_cells(_p(xyz), xyz.shape[0], _pi(cells), nvc, cells.shape[0], _pi(bf),
                                         bt.ctypes.data_as(C.POINTER(C.c_int32)), bf.shape[0], _p(psa),
                                         psa.shape[0], err, 256)
        if not self.h:
            raise ValueError("oracle mesh: " + err.value.decode())
        self.s = C.cast(self.h, C.POINTER(_MeshC)).contents
        self.nc, self.nf = int(self.s.nc), int(self.s.nf)
        self.nfc, self.ngp = int(self.s.nfc), int(self.s.ngp)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_mesh_destroy(self.h)
            self.h = None

    def arr(self, name, shape, dtype=np.float64):
        ptr = getattr(self.s, name)
        n = int(np.prod(shape))
        return np.ctypeslib.as_array(ptr, shape=(n,)).reshape(shape).astype(dtype).copy()

    @property
    def vol(self):
        return self.arr("vol", (self.nc,))

    @property
    def centroid(self):
        return self.arr("cen", (self.nc, 3))

    @property
    def neighbours(self):
        return self.arr("cnb", (self.nc, self.nfc), np.int64)

    # -- residual ---------------------------------------------------------
    def residual(self, params, Q, G=None, cells=None):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        R = np.zeros_like(Q)
        Gn = np.zeros((self.nc, 15)) if params.scheme == 1 else None
        Ga = np.ascontiguousarray(G, dtype=np.float64) if G is not None else None
        ca = np.ascontiguousarray(cells, dtype=np.int64) if cells is not None else None
        rc = lib().orc_residual(C.c_void_p(self.h), C.byref(params), _p(Q), _p(Ga) if Ga is not None else None,
                                _p(R), _p(Gn) if Gn is not None else None,
                                _pi(ca) if ca is not None else None, 0 if ca is None else len(ca))
        if rc:
            raise RuntimeError(f"orc_residual failed ({rc})")
        return (R, Gn) if Gn is not None else R

    def local_dt(self, params, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        dt = np.zeros(self.nc)
        lib().orc_local_dt(C.c_void_p(self.h), C.byref(params), _p(Q), _p(dt))
        return dt

    def jacobian(self, params, Q, dt=None):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        if dt is None:
            dt = self.local_dt(params, Q)
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        diag = np.zeros((self.nc, 5, 5))
        off = np.zeros((self.nc, self.nfc, 5, 5))
        lib().orc_jacobian(C.c_void_p(self.h), C.byref(params), _p(Q), _p(dt), _p(diag), _p(off))
        return diag, off

    def precondition(self, diag, off, sweeps, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        rc = lib().orc_precondition(C.c_void_p(self.h), _p(np.ascontiguousarray(diag)),
                                    _p(np.ascontiguousarray(off)), int(sweeps), _p(b), _p(x))
        if rc:
            raise RuntimeError("singular diagonal block")
        return x

    def gmres(self, params, diag, off, rhs):
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        dx = np.zeros_like(rhs)
        hist = np.zeros(max(1, params.restarts))
        rc = lib().orc_gmres(C.c_void_p(self.h), _p(np.ascontiguousarray(diag)), _p(np.ascontiguousarray(off)),
                             C.byref(params), _p(rhs), _p(dx), _p(hist))
        if rc:
            raise RuntimeError("orc_gmres failed")
        return dx, hist

    def residual_dt(self, params, Q, G, dt):
        """R = L(Q) with the given local time step (caller order [n, 5])."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        Ga = np.ascontiguousarray(G, dtype=np.float64) if G is not None else None
        R = np.zeros_like(Q)
        rc = lib().orc_residual_dt(C.c_void_p(self.h), C.byref(params), _p(Q), _p(Ga) if Ga is not None else None,
                                   _p(np.ascontiguousarray(dt, dtype=np.float64)), _p(R), None, None, C.c_int64(0))
        if rc:
            raise RuntimeError(f"orc_residual_dt failed ({rc})")
        return R

    def wall_force(self, params, Q, G, tag):
        """Force [3] of the flow on the boundary faces with the given tag."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        Ga = np.ascontiguousarray(G, dtype=np.float64) if G is not None else None
        f = np.zeros(3)
        rc = lib().orc_wall_force(C.c_void_p(self.h), C.byref(params), _p(Q), _p(Ga) if Ga is not None else None,
                                  int(tag), _p(f))
        if rc:
            raise RuntimeError("orc_wall_force failed")
        return f

    def apply_fd(self, params, Q, G, dt, x):
        """(y, sigma): y = |Omega|/dt x - (L(Q + sigma x) - L(Q)) / sigma, Eq. (frechet)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        Ga = np.ascontiguousarray(G, dtype=np.float64) if G is not None else None
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        LQ = self.residual_dt(params, Q, G, dt)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        sig = C.c_double(0)
        rc = lib().orc_apply_fd(C.c_void_p(self.h), C.byref(params), _p(Q), _p(Ga) if Ga is not None else None,
                                _p(dt), _p(LQ), _p(x), _p(y), C.byref(sig))
        if rc:
            raise RuntimeError("orc_apply_fd failed")
        return y, sig.value

    def gmres_step(self, params, Q, G=None):
        Q = np.array(Q, dtype=np.float64, copy=True)
        G = np.array(G, dtype=np.float64, copy=True) if G is not None else None
        res = C.c_double(0)
        dQ = np.zeros_like(Q)
        rc = lib().orc_gmres_step(C.c_void_p(self.h), C.byref(params), _p(Q), _p(G) if G is not None else None,
                                  C.byref(res), _p(dQ))
        if rc:
            raise RuntimeError("orc_gmres_step failed")
        return Q, G, res.value, dQ

    def solve_steady(self, params, Q, G=None, drop=1e-8, max_steps=1000):
        Q = np.array(Q, dtype=np.float64, copy=True)
        G = np.array(G, dtype=np.float64, copy=True) if G is not None else None
        hist = np.zeros(max_steps + 2)
        steps = C.c_int(0)
        rc = lib().orc_solve_steady(C.c_void_p(self.h), C.byref(params), _p(Q), _p(G) if G is not None else None,
                                    C.c_double(drop), int(max_steps), _p(hist), C.byref(steps))
        if rc < 0:
            raise RuntimeError("orc_solve_steady failed")
        return Q, G, hist[: steps.value + 1], rc == 0

    def recon_side(self, params, Q, G, cell, slot):
        """Values/gradients at the ngp Gauss points of face `slot` of `cell`.

        Returns (Wloc [ngp,5], dWloc [ngp,3,5] along (n,t1,t2), Wglob [ngp,5], gradglob [ngp,5,3])."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        Ga = np.ascontiguousarray(G, dtype=np.float64) if G is not None else None
        g = self.ngp
        Wl = np.zeros((g, 5)); dWl = np.zeros((g, 3, 5)); Wg = np.zeros((g, 5)); gg = np.zeros((g, 5, 3))
        rc = lib().orc_recon_side(C.c_void_p(self.h), C.byref(params), _p(Q), _p(Ga) if Ga is not None else None,
                                  C.c_int64(cell), C.c_int(slot), _p(Wl), _p(dWl), _p(Wg), _p(gg))
        if rc:
            raise RuntimeError("orc_recon_side failed")
        return Wl, dWl, Wg, gg

    def stencil(self, cell, which=-1):
        """(cells, valid) of the non-compact big stencil (which = -1) or of
        sub-stencil `which` of `cell`."""
        out = np.zeros(64, dtype=np.int64)
        v = C.c_int(0)
        n = lib().orc_stencil(C.c_void_p(self.h), C.c_int64(cell), int(which), _pi(out), C.byref(v))
        if n < 0:
            raise RuntimeError("orc_stencil failed")
        return out[:n].copy(), bool(v.value)

    def face_geometry(self):
        """Per face: area, unit normal (left to right), Gauss points [ngp, 3]
        (left cell's frame) and Gauss weights [ngp]; left/right cells."""
        return dict(area=self.arr("farea", (self.nf,)), normal=self.arr("fnrm", (self.nf, 3)),
                    gp=self.arr("fgp", (self.nf, self.ngp, 3)), gw=self.arr("fgw", (self.nf, self.ngp)),
                    left=self.arr("fl", (self.nf,), np.int64), right=self.arr("fr", (self.nf,), np.int64),
                    shift=self.arr("fshift", (self.nf, 3)))

    def face_gauss_points(self, cell, slot):
        f = int(self.arr("cface", (self.nc, self.nfc), np.int64)[cell, slot])
        side = int(self.arr("cside", (self.nc, self.nfc), np.int32)[cell, slot])
        gp = self.arr("fgp", (self.nf, self.ngp, 3))[f]
        if side == 1:
            gp = gp - self.arr("fshift", (self.nf, 3))[f][None, :]
        return gp


# -- point-wise pieces, for the tests that pin the oracle ---------------------

def gks_flux(params, Wl, dWl, Wr, dWr, dt):
    """Time-averaged flux and point value at one Gauss point (face frame)."""
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (Wl, dWl, Wr, dWr)]
    F = np.zeros(5); Qp = np.zeros(5)
    lib().orc_gks_flux(C.byref(params), _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), C.c_double(dt), _p(F), _p(Qp))
    return F, Qp


def boundary_state(params, tag, T3, Wl, dWl):
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (T3, Wl, dWl)]
    Wr = np.zeros(5); dWr = np.zeros((3, 5))
    lib().orc_boundary_state(C.byref(params), C.c_int(tag), _p(a[0]), _p(a[1]), _p(a[2]), _p(Wr), _p(dWr))
    return Wr, dWr


def monomial_moment(prim, K, rng, iu, iv, iw, ixi):
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    return lib().orc_monomial_moment(_p(prim), K, rng, iu, iv, iw, ixi)


def slope(prim, K, dQ):
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    dQ = np.ascontiguousarray(dQ, dtype=np.float64)
    a = np.zeros(5)
    if lib().orc_slope(_p(prim), C.c_double(K), _p(dQ), _p(a)):
        raise RuntimeError("singular moment matrix")
    return a


def lu_solve(A, b):
    """x with A x = b by the oracle's elimination (the primitive its steps call)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(len(b))
    if lib().orc_lu_solve(int(len(b)), _p(A), _p(b), _p(x)):
        raise RuntimeError("singular matrix")
    return x


def lsq_pinv(A):
    """X (cols x rows) with X b the least-squares solution of A x = b (Householder QR)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    X = np.zeros((A.shape[1], A.shape[0]))
    if lib().orc_lsq_pinv(int(A.shape[0]), int(A.shape[1]), _p(A), _p(X)):
        raise RuntimeError("rank-deficient or short matrix")
    return X


def euler_jacobian(Q, n, gamma=1.4):
    J = np.zeros((5, 5))
    lib().orc_euler_jacobian(_p(np.ascontiguousarray(Q, dtype=np.float64)),
                             _p(np.ascontiguousarray(n, dtype=np.float64)), C.c_double(gamma), _p(J))
    return J


def char_eigen(Qloc, gamma=1.4):
    R = np.zeros((5, 5)); L = np.zeros((5, 5))
    lib().orc_char_eigen(_p(np.ascontiguousarray(Qloc, dtype=np.float64)), C.c_double(gamma), _p(R), _p(L))
    return R, L


def face_frame(n):
    T = np.zeros((3, 3))
    lib().orc_face_frame(_p(np.ascontiguousarray(n, dtype=np.float64)), _p(T))
    return T


def primitive(Q, gamma=1.4):
    pr = np.zeros(5)
    lib().orc_primitive(_p(np.ascontiguousarray(Q, dtype=np.float64)), C.c_double(gamma), _p(pr))
    return pr


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's loops (n > 0; n = 0 leaves them); returns the previous maximum."""
    return int(lib().orc_set_threads(int(n)))
