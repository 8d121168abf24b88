"""FP64 CPU oracle for the hyperbolic (Euler) step of arXiv:2106.02159.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may build, load or call this package. The
CUDA library never imports it and shares no code with it.

``build()`` compiles ``euler_oracle.c`` with gcc (IEEE FP64, no contraction,
no fast-math, OpenMP over rows) into ``oracle/_build/``. The Python side only
marshals numpy arrays into the C structs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "euler_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libeuler_oracle.so")

BC_SLIP, BC_DIRICHLET, BC_DO_NOTHING, BC_CHARACTERISTIC, BC_GODUNOV = 1, 2, 3, 4, 5

_lib = None


_FMA_LIB_PATH = os.path.join(_BUILD, "libeuler_oracle_fma.so")


def fma_flags():
    """Flags of the contracted build: a*b+c fused wherever the compiler likes
    (the rounding a GPU compiler applies by default)."""
    import platform
    flags = ["-ffp-contract=fast"]
    if platform.machine() in ("x86_64", "AMD64"):
        flags.insert(0, "-mfma")
    return flags


def build(force: bool = False, src: str | None = None, out: str | None = None, extra=(), variant: str = "ieee") -> str:
    """Compile the oracle (or, for mutation tests, another copy of its source).

    variant "ieee": no contraction (the reference build). variant "fma": the
    same source with fused multiply-adds, used only to measure how much the
    method's result moves under a different valid rounding."""
    src = src or _SRC
    if variant == "fma" and out is None:
        out = _FMA_LIB_PATH
        extra = tuple(extra) + tuple(fma_flags())
    out = out or _LIB_PATH
    if (not force and out in (_LIB_PATH, _FMA_LIB_PATH) and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
           *extra, src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n", ctypes.c_int), ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("cij", ctypes.c_void_p),
        ("mij", ctypes.c_void_p), ("mi", ctypes.c_void_p),
        ("n_bnd", ctypes.c_int), ("bnd_node", ctypes.c_void_p), ("bnd_kind", ctypes.c_void_p),
        ("bnd_normal", ctypes.c_void_p), ("bnd_state", ctypes.c_void_p),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("limiter_passes", ctypes.c_int),
        ("bound_relaxation", ctypes.c_int),
    ]


class _Parabolic(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_void_p), ("G", ctypes.c_void_p), ("n_cells", ctypes.c_int), ("nv", ctypes.c_int),
        ("nq", ctypes.c_int), ("cells", ctypes.c_void_p), ("qw", ctypes.c_void_p), ("qphi", ctypes.c_void_p),
        ("qgrad", ctypes.c_void_p), ("n_wall", ctypes.c_int), ("wall", ctypes.c_void_p), ("mu", ctypes.c_double),
        ("lam", ctypes.c_double), ("kappa_cv", ctypes.c_double), ("cg_tol", ctypes.c_double),
        ("cg_max_iter", ctypes.c_int),
    ]


class _ParabolicInfo(ctypes.Structure):
    _fields_ = [("cg_iter_velocity", ctypes.c_int), ("cg_iter_energy", ctypes.c_int), ("cg_iter_low", ctypes.c_int),
                ("limited", ctypes.c_int), ("min_e", ctypes.c_double)]


class _Trace(ctypes.Structure):
    _fields_ = [
        ("dij", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("UL", ctypes.c_void_p),
        ("FH", ctypes.c_void_p), ("bounds", ctypes.c_void_p), ("P", ctypes.c_void_p),
        ("lij", ctypes.c_void_p), ("Upass", ctypes.c_void_p), ("tau_bound", ctypes.c_double),
    ]


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_create.restype = ctypes.c_void_p
    lib.oracle_create.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(ctypes.c_int)]
    lib.oracle_destroy.argtypes = [ctypes.c_void_p]
    lib.oracle_lambda_max.restype = ctypes.c_double
    lib.oracle_lambda_max.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_double]
    lib.oracle_lambda_max_batch.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int, ctypes.c_double, dp]
    lib.oracle_entropy_gradient.argtypes = [dp, ctypes.c_int, ctypes.c_double, dp]
    lib.oracle_entropy_eta.restype = ctypes.c_double
    lib.oracle_entropy_eta.argtypes = [dp, ctypes.c_int, ctypes.c_double]
    lib.oracle_line_search.restype = ctypes.c_double
    lib.oracle_line_search.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_double]
    lib.oracle_bc_characteristic.restype = None
    lib.oracle_bc_characteristic.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_double]
    lib.oracle_bc_godunov.restype = None
    lib.oracle_bc_godunov.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_double]
    lib.oracle_set_threads.restype = ctypes.c_int
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_count_not_admissible.restype = ctypes.c_int64
    lib.oracle_count_not_admissible.argtypes = [ctypes.c_void_p, dp]
    lib.oracle_cfl_dt.restype = ctypes.c_double
    lib.oracle_cfl_dt.argtypes = [ctypes.c_void_p, dp]
    lib.oracle_forward_euler.restype = ctypes.c_int
    lib.oracle_forward_euler.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, dp, dp, ctypes.POINTER(_Trace)]
    lib.oracle_apply_bc.argtypes = [ctypes.c_void_p, dp]
    lib.oracle_ssprk3_step.restype = ctypes.c_int
    lib.oracle_ssprk3_step.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, dp, dp]
    lib.oracle_ssprk3_step_adaptive.restype = ctypes.c_int
    lib.oracle_ssprk3_step_adaptive.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, dp, dp,
                                                ctypes.POINTER(ctypes.c_int)]
    lib.oracle_parabolic_step.restype = ctypes.c_int
    lib.oracle_parabolic_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Parabolic), dp, ctypes.c_double,
                                          ctypes.POINTER(_ParabolicInfo)]
    lib.oracle_ns_step.restype = ctypes.c_int
    lib.oracle_ns_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Parabolic), dp, ctypes.c_double, dp,
                                   ctypes.POINTER(_ParabolicInfo)]
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_run.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, ctypes.c_double, dp]
    lib.oracle_run_to.restype = ctypes.c_int
    lib.oracle_run_to.argtypes = [ctypes.c_void_p, dp, ctypes.c_double, ctypes.c_int, dp,
                                  ctypes.POINTER(ctypes.c_int)]
    return lib


_fma_lib = None


def load_fma():
    """The contracted build of the same oracle source (see build())."""
    global _fma_lib
    if _fma_lib is None:
        _fma_lib = _bind(ctypes.CDLL(build(variant="fma")))
    return _fma_lib


def load(path: str | None = None):
    """Load the oracle library (building it first if needed)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int = 0, lib=None) -> int:
    return (lib or load()).oracle_set_threads(n)


def lambda_max(ul, ur, n, gamma=1.4, lib=None) -> float:
    lib = lib or load()
    ul = np.ascontiguousarray(ul, dtype=np.float64)
    ur = np.ascontiguousarray(ur, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    return lib.oracle_lambda_max(_dptr(ul), _dptr(ur), _dptr(n), n.size, gamma)


def lambda_max_batch(ul, ur, n, gamma=1.4, lib=None):
    """ul, ur: [m, dim+2], n: [m, dim] -> [m]."""
    lib = lib or load()
    ul = np.ascontiguousarray(ul, dtype=np.float64)
    ur = np.ascontiguousarray(ur, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.empty(ul.shape[0])
    lib.oracle_lambda_max_batch(ul.shape[0], _dptr(ul), _dptr(ur), _dptr(n), n.shape[1], gamma, _dptr(out))
    return out


def entropy_gradient(u, gamma=1.4, lib=None):
    lib = lib or load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    lib.oracle_entropy_gradient(_dptr(u), u.size - 2, gamma, _dptr(out))
    return out


def entropy_eta(u, gamma=1.4, lib=None) -> float:
    lib = lib or load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib.oracle_entropy_eta(_dptr(u), u.size - 2, gamma)


def line_search(ub, P, rho_min, rho_max, phi_min, gamma=1.4, lib=None) -> float:
    lib = lib or load()
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    return lib.oracle_line_search(_dptr(ub), _dptr(P), rho_min, rho_max, phi_min, ub.size - 2, gamma)


def bc_characteristic(u, normal, ud, gamma=1.4, lib=None) -> np.ndarray:
    """Characteristic non-reflecting post-processing of one state (Sec. 4.2.2)."""
    lib = lib or load()
    out = np.array(u, dtype=np.float64, copy=True)
    nrm = np.ascontiguousarray(normal, dtype=np.float64)
    ud = np.ascontiguousarray(ud, dtype=np.float64)
    lib.oracle_bc_characteristic(_dptr(out), _dptr(nrm), _dptr(ud), out.size - 2, gamma)
    return out


def bc_godunov(u, normal, ud, gamma=1.4, lib=None) -> np.ndarray:
    """Godunov non-reflecting post-processing of one state (Sec. 4.2.1)."""
    lib = lib or load()
    out = np.array(u, dtype=np.float64, copy=True)
    nrm = np.ascontiguousarray(normal, dtype=np.float64)
    ud = np.ascontiguousarray(ud, dtype=np.float64)
    lib.oracle_bc_godunov(_dptr(out), _dptr(nrm), _dptr(ud), out.size - 2, gamma)
    return out


class OracleError(RuntimeError):
    pass


class Oracle:
    """One oracle context bound to a mesh (arrays are kept alive here)."""

    def __init__(self, mesh, gamma=1.4, cfl=0.5, limiter_passes=2, bnd_state=None, bound_relaxation=False,
                 lib=None):
        self.lib = lib or load()
        self.mesh = mesh
        self.dim = mesh.dim
        self.S = mesh.dim + 2
        self.n = mesh.n
        self.nnz = mesh.nnz
        self.limiter_passes = limiter_passes
        self._keep = dict(
            row_ptr=np.ascontiguousarray(mesh.row_ptr, dtype=np.int64),
            col=np.ascontiguousarray(mesh.col, dtype=np.int32),
            cij=np.ascontiguousarray(mesh.cij, dtype=np.float64),
            mij=np.ascontiguousarray(mesh.mij, dtype=np.float64),
            mi=np.ascontiguousarray(mesh.mi, dtype=np.float64),
            bnd_node=np.ascontiguousarray(mesh.bnd_node, dtype=np.int32),
            bnd_kind=np.ascontiguousarray(mesh.bnd_kind, dtype=np.int32),
            bnd_normal=np.ascontiguousarray(mesh.bnd_normal, dtype=np.float64),
            bnd_state=None if bnd_state is None else np.ascontiguousarray(bnd_state, dtype=np.float64),
        )
        k = self._keep
        self._prob = _Problem(
            dim=mesh.dim, n=mesh.n, nnz=mesh.nnz, row_ptr=_ptr(k["row_ptr"]), col=_ptr(k["col"]),
            cij=_ptr(k["cij"]), mij=_ptr(k["mij"]), mi=_ptr(k["mi"]), n_bnd=mesh.n_bnd,
            bnd_node=_ptr(k["bnd_node"]), bnd_kind=_ptr(k["bnd_kind"]), bnd_normal=_ptr(k["bnd_normal"]),
            bnd_state=_ptr(k["bnd_state"]), gamma=gamma, cfl=cfl, limiter_passes=limiter_passes,
            bound_relaxation=int(bool(bound_relaxation)))
        st = ctypes.c_int(0)
        self._ctx = self.lib.oracle_create(ctypes.byref(self._prob), ctypes.byref(st))
        if not self._ctx:
            raise OracleError(f"oracle_create failed with status {st.value}")

    def close(self):
        if getattr(self, "_ctx", None):
            self.lib.oracle_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        self.close()

    def _state(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (self.S, self.n), U.shape
        return U

    def count_not_admissible(self, U) -> int:
        U = self._state(U)
        return int(self.lib.oracle_count_not_admissible(self._ctx, _dptr(U)))

    def cfl_dt(self, U) -> float:
        U = self._state(U)
        return float(self.lib.oracle_cfl_dt(self._ctx, _dptr(U)))

    def forward_euler(self, U, tau=0.0, trace=False):
        """One forward-Euler stage (no boundary post-processing).

        Returns (U_new, tau_used, trace_dict or None)."""
        U = self._state(U)
        out = np.empty_like(U)
        tau_used = ctypes.c_double(0.0)
        tr = None
        arrays = None
        if trace:
            L = self.limiter_passes
            arrays = dict(dij=np.empty(self.nnz), alpha=np.empty(self.n), UL=np.empty((self.S, self.n)),
                          FH=np.empty((self.S, self.n)), bounds=np.empty((3, self.n)),
                          P=np.empty((self.S, self.nnz)), lij=np.empty((L, self.nnz)),
                          Upass=np.empty((L, self.S, self.n)))
            tr = _Trace(**{k: _ptr(v) for k, v in arrays.items()}, tau_bound=0.0)
        st = self.lib.oracle_forward_euler(self._ctx, _dptr(U), float(tau), _dptr(out), ctypes.byref(tau_used),
                                           ctypes.byref(tr) if tr is not None else None)
        if st:
            raise OracleError(f"oracle_forward_euler failed with status {st}")
        if arrays is not None:
            arrays["tau_bound"] = tr.tau_bound
        return out, tau_used.value, arrays

    def apply_bc(self, U):
        U = np.array(U, dtype=np.float64, order="C", copy=True)
        self.lib.oracle_apply_bc(self._ctx, _dptr(U))
        return U

    def ssprk3_step(self, U, dt=0.0):
        """One SSPRK(3,3) step; returns (U_new, dt_used, stage_tau_bounds[3])."""
        U = np.array(self._state(U), copy=True)
        used = ctypes.c_double(0.0)
        bounds = np.zeros(3)
        st = self.lib.oracle_ssprk3_step(self._ctx, _dptr(U), float(dt), ctypes.byref(used), _dptr(bounds))
        if st:
            raise OracleError(f"oracle_ssprk3_step failed with status {st}")
        return U, used.value, bounds

    def ssprk3_step_adaptive(self, U, cfl_max):
        """One SSPRK(3,3) step with the CFL number adapted above 1 (restart with
        half the CFL number while a low-order state leaves the admissible set);
        returns (U_new, dt_used, cfl_used, restarts)."""
        U = np.array(self._state(U), copy=True)
        dt, cfl, r = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int(0)
        st = self.lib.oracle_ssprk3_step_adaptive(self._ctx, _dptr(U), float(cfl_max), ctypes.byref(dt),
                                                  ctypes.byref(cfl), ctypes.byref(r))
        if st:
            raise OracleError(f"oracle_ssprk3_step_adaptive failed with status {st}")
        return U, dt.value, cfl.value, r.value

    def set_viscosity(self, pdata, mu, lam=0.0, kappa_cv=0.0, wall=None, cg_tol=1e-13, cg_max_iter=2000):
        """The finite-element data of meshes.parabolic_data and the constants of
        the parabolic sub-step (Sec. 5); wall: no-slip node ids."""
        keep = dict(L=np.ascontiguousarray(pdata["L"], dtype=np.float64),
                    G=np.ascontiguousarray(pdata["G"], dtype=np.float64),
                    cells=np.ascontiguousarray(pdata["cells"], dtype=np.int32),
                    qw=np.ascontiguousarray(pdata["qw"], dtype=np.float64),
                    qphi=np.ascontiguousarray(pdata["qphi"], dtype=np.float64),
                    qgrad=np.ascontiguousarray(pdata["qgrad"], dtype=np.float64),
                    wall=np.ascontiguousarray(np.zeros(0) if wall is None else wall, dtype=np.int32))
        nc, nq, nv = keep["qphi"].shape
        self._par_keep = keep
        self._par = _Parabolic(L=_ptr(keep["L"]), G=_ptr(keep["G"]), n_cells=nc, nv=nv, nq=nq,
                               cells=_ptr(keep["cells"]), qw=_ptr(keep["qw"]), qphi=_ptr(keep["qphi"]),
                               qgrad=_ptr(keep["qgrad"]), n_wall=int(keep["wall"].size), wall=_ptr(keep["wall"]),
                               mu=float(mu), lam=float(lam), kappa_cv=float(kappa_cv), cg_tol=float(cg_tol),
                               cg_max_iter=int(cg_max_iter))

    def parabolic_step(self, U, dt):
        """U <- S_P(dt) U (Sec. 5); returns (U_new, info dict)."""
        U = np.array(self._state(U), copy=True)
        info = _ParabolicInfo()
        st = self.lib.oracle_parabolic_step(self._ctx, ctypes.byref(self._par), _dptr(U), float(dt), ctypes.byref(info))
        if st:
            raise OracleError(f"oracle_parabolic_step failed with status {st}")
        return U, {f: getattr(info, f) for f, _ in _ParabolicInfo._fields_}

    def ns_step(self, U, dt=0.0):
        """Strang step H(tau) P(2 tau) H(tau); returns (U_new, tau, info dict)."""
        U = np.array(self._state(U), copy=True)
        info = _ParabolicInfo()
        tau = ctypes.c_double(0.0)
        st = self.lib.oracle_ns_step(self._ctx, ctypes.byref(self._par), _dptr(U), float(dt), ctypes.byref(tau),
                                     ctypes.byref(info))
        if st:
            raise OracleError(f"oracle_ns_step failed with status {st}")
        return U, tau.value, {f: getattr(info, f) for f, _ in _ParabolicInfo._fields_}

    def run(self, U, nsteps, dt=0.0):
        U = np.array(self._state(U), copy=True)
        t = ctypes.c_double(0.0)
        st = self.lib.oracle_run(self._ctx, _dptr(U), int(nsteps), float(dt), ctypes.byref(t))
        if st:
            raise OracleError(f"oracle_run failed with status {st}")
        return U, t.value

    def run_to(self, U, t_final, max_steps=10 ** 7):
        U = np.array(self._state(U), copy=True)
        t = ctypes.c_double(0.0)
        steps = ctypes.c_int(0)
        st = self.lib.oracle_run_to(self._ctx, _dptr(U), float(t_final), int(max_steps), ctypes.byref(t),
                                    ctypes.byref(steps))
        if st:
            raise OracleError(f"oracle_run_to failed with status {st}")
        return U, t.value, steps.value
