"""ctypes binding of the C ABI in ``include/euler_hyp.h``.

Argument marshalling only: every step of the hyperbolic solver runs in the
CUDA library ``libeuler_hyp.so`` built from ``csrc/`` for sm_103a. There is
no CPU fallback: if the library is missing or no GPU is present, the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
CSRC = os.path.join(_HERE, "csrc")
BUILD_DIR = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libeuler_hyp.so")
SOURCES = ("kernels.cu", "capi.cu", "noalloc.cu", "parabolic.cu", "batch.cu")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]

EH_OK, EH_ERR_INVALID_ARG, EH_ERR_OOM, EH_ERR_BAD_MESH = 0, 1, 2, 3
EH_ERR_NOT_ADMISSIBLE, EH_ERR_CFL, EH_ERR_CUDA, EH_ERR_STATE = 4, 5, 6, 7
EH_BC_SLIP, EH_BC_DIRICHLET, EH_BC_DO_NOTHING, EH_BC_CHARACTERISTIC, EH_BC_GODUNOV = 1, 2, 3, 4, 5
EH_PRECISION_FP64, EH_PRECISION_MIXED = 0, 1
EH_BATCH_MERGED, EH_BATCH_PER_REQUEST_STREAMS = 0, 1
(EH_TRACE_D_IJ, EH_TRACE_ALPHA, EH_TRACE_U_LOW, EH_TRACE_F_HIGH, EH_TRACE_BOUNDS, EH_TRACE_L_PASS1,
 EH_TRACE_U_PASS1, EH_TRACE_TAU, EH_TRACE_TAU_BOUND, EH_TRACE_P_PASS1, EH_TRACE_L_LAST) = range(11)

# every symbol the header declares
EXPORTS = ("eh_config_default", "eh_create", "eh_upload_mesh", "eh_set_state", "eh_get_state",
           "eh_apply_boundary_conditions", "eh_cfl_dt", "eh_stage", "eh_step", "eh_run", "eh_synchronize",
           "eh_get_diagnostics", "eh_trace", "eh_get_mesh_index", "eh_profile_enable", "eh_profile_read", "eh_launches_per_step",
           "eh_last_error", "eh_status_string", "eh_destroy", "eh_cfl_dt_noalloc", "eh_set_instances",
           "eh_get_instances", "eh_autotune", "eh_get_block_sizes", "eh_get_rows_per_sm", "eh_set_launch_shape",
           "eh_step_adaptive", "eh_set_viscosity", "eh_parabolic_step", "eh_step_ns",
           "eh_estimate_device_bytes", "eh_batch_create", "eh_batch_admit", "eh_batch_advance", "eh_batch_poll",
           "eh_batch_active", "eh_batch_last_error", "eh_batch_destroy", "eh_batch_set_mode", "eh_batch_repacks",
           "eh_get_instance_steps", "eh_estimate_request_bytes")
CFL_NOALLOC_MAX_ROWS = 1 << 23
KERNEL_NAMES = ("prep", "visc", "low", "tau", "lim1", "pass", "final", "lsearch")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libeuler_hyp.so for sm_103a (nvcc; no GPU needed)."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, "kernels.cuh"), os.path.join(_ROOT, "include", "euler_hyp.h")]
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(d) for d in deps):
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + ".tmp"
    cmd = ["nvcc", *NVCC_FLAGS, "-o", tmp, *srcs]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("limiter_passes", ctypes.c_int), ("bound_relaxation", ctypes.c_int), ("precision", ctypes.c_int),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p)]


class Diagnostics(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("steps", ctypes.c_int64), ("last_dt", ctypes.c_double),
                ("last_stage_bound", ctypes.c_double * 3), ("cfl_violations", ctypes.c_int64),
                ("not_admissible", ctypes.c_int64), ("line_searches_deferred", ctypes.c_int64),
                ("line_searches_iterated", ctypes.c_int64), ("low_order_not_admissible", ctypes.c_int64),
                ("rho_min", ctypes.c_double), ("e_min", ctypes.c_double), ("total", ctypes.c_double * 5)]


class ParabolicInfo(ctypes.Structure):
    _fields_ = [("cg_iter_velocity", ctypes.c_int32), ("cg_iter_energy", ctypes.c_int32),
                ("cg_iter_low", ctypes.c_int32), ("limited", ctypes.c_int32), ("min_e", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load the library (built in-tree). Raises OSError if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: run paper_2106_02159_gb300.binding.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    vp, dp, i32, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int64
    lib.eh_config_default.argtypes = [ctypes.POINTER(Config)]
    lib.eh_config_default.restype = None
    lib.eh_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    lib.eh_upload_mesh.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
    lib.eh_set_state.argtypes = [vp, vp, ctypes.c_int]
    lib.eh_get_state.argtypes = [vp, vp, ctypes.c_int]
    lib.eh_apply_boundary_conditions.argtypes = [vp]
    lib.eh_cfl_dt.argtypes = [vp, dp]
    lib.eh_stage.argtypes = [vp, ctypes.c_double, dp]
    lib.eh_step.argtypes = [vp, ctypes.c_double, dp]
    lib.eh_run.argtypes = [vp, i32, ctypes.c_double]
    lib.eh_synchronize.argtypes = [vp]
    lib.eh_get_diagnostics.argtypes = [vp, ctypes.POINTER(Diagnostics)]
    lib.eh_trace.argtypes = [vp, ctypes.c_int, dp, i64]
    lib.eh_get_mesh_index.argtypes = [vp, vp, vp, vp]
    lib.eh_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.eh_profile_read.argtypes = [vp, ctypes.c_int, dp, ctypes.POINTER(i64)]
    lib.eh_launches_per_step.argtypes = [vp]
    lib.eh_launches_per_step.restype = i32
    lib.eh_last_error.argtypes = [vp]
    lib.eh_last_error.restype = ctypes.c_char_p
    lib.eh_status_string.argtypes = [ctypes.c_int]
    lib.eh_status_string.restype = ctypes.c_char_p
    lib.eh_destroy.argtypes = [vp]
    lib.eh_destroy.restype = None
    lib.eh_set_instances.argtypes = [vp, i32, vp, vp]
    lib.eh_get_instances.argtypes = [vp, vp, vp, vp]
    lib.eh_autotune.argtypes = [vp, i32, vp]
    lib.eh_get_block_sizes.argtypes = [vp, vp]
    lib.eh_get_rows_per_sm.argtypes = [vp, vp]
    lib.eh_set_launch_shape.argtypes = [vp, i32, i32, i32]
    lib.eh_step_adaptive.argtypes = [vp, ctypes.c_double, dp, dp, ctypes.POINTER(i32)]
    lib.eh_set_viscosity.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, vp, i32, i32, i32,
                                     vp, vp, vp, vp, i32, vp, ctypes.c_double, i32]
    lib.eh_parabolic_step.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ParabolicInfo)]
    lib.eh_step_ns.argtypes = [vp, ctypes.c_double, dp, ctypes.POINTER(ParabolicInfo)]
    lib.eh_cfl_dt_noalloc.argtypes = [i32, ctypes.c_double, ctypes.c_double, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    u64 = ctypes.c_uint64
    lib.eh_estimate_device_bytes.argtypes = [i32, i32, i32, i64, ctypes.POINTER(u64)]
    lib.eh_batch_create.argtypes = [ctypes.POINTER(Config), u64, ctypes.POINTER(vp)]
    lib.eh_batch_admit.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, ctypes.c_double,
                                   ctypes.POINTER(i64)]
    lib.eh_batch_advance.argtypes = [vp, i32, ctypes.POINTER(i32)]
    lib.eh_batch_poll.argtypes = [vp, i64, ctypes.POINTER(i32), vp, dp, ctypes.POINTER(i64)]
    lib.eh_batch_active.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(u64)]
    lib.eh_batch_last_error.argtypes = [vp]
    lib.eh_batch_last_error.restype = ctypes.c_char_p
    lib.eh_batch_destroy.argtypes = [vp]
    lib.eh_batch_set_mode.argtypes = [vp, i32]
    lib.eh_estimate_request_bytes.argtypes = [i32, i32, i32, i32, i64, i32, ctypes.POINTER(u64)]
    lib.eh_batch_repacks.argtypes = [vp, ctypes.POINTER(i64)]
    lib.eh_get_instance_steps.argtypes = [vp, vp]
    lib.eh_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("eh_config_default", "eh_destroy", "eh_launches_per_step", "eh_last_error",
                        "eh_status_string", "eh_batch_last_error", "eh_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    if path == LIB_PATH:
        _lib = lib
    return lib


def cfl_dt_noalloc(dim, gamma, cfl, row_ptr, col, cij, mi, is_boundary, U, dt_out, stream=None, lib=None):
    """eh_cfl_dt_noalloc on CUDA tensors (device pointers; nothing is allocated
    by the library). dt_out: a one-element float64 CUDA tensor. Queues the
    work on ``stream`` (a torch.cuda.Stream or None) without synchronising."""
    lib = lib or load()
    n = int(mi.shape[0])
    if n > CFL_NOALLOC_MAX_ROWS:
        raise ValueError(f"eh_cfl_dt_noalloc handles at most {CFL_NOALLOC_MAX_ROWS} rows, got {n}")
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = lib.eh_cfl_dt_noalloc(dim, gamma, cfl, n, int(col.shape[0]), ptr(row_ptr), ptr(col), ptr(cij), ptr(mi),
                               ptr(is_boundary), ptr(U), ptr(dt_out),
                               None if stream is None else ctypes.c_void_p(stream.cuda_stream))
    if st != EH_OK:
        raise EulerError(st, f"eh_cfl_dt_noalloc: {lib.eh_status_string(st).decode()}")


class EulerError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def estimate_device_bytes(dim, precision, n, nnz, lib=None) -> int:
    """Device bytes a context needs for a mesh (eh_estimate_device_bytes)."""
    lib = lib or load()
    out = ctypes.c_uint64(0)
    st = lib.eh_estimate_device_bytes(int(dim), int(precision), int(n), int(nnz), ctypes.byref(out))
    if st != EH_OK:
        raise EulerError(st, "eh_estimate_device_bytes: invalid arguments")
    return int(out.value)


def estimate_request_bytes(dim, precision, mode, n, nnz, n_bnd, lib=None) -> int:
    """Device bytes a batch in ``mode`` counts for a request (eh_estimate_request_bytes)."""
    lib = lib or load()
    out = ctypes.c_uint64(0)
    st = lib.eh_estimate_request_bytes(int(dim), int(precision), int(mode), int(n), int(nnz), int(n_bnd),
                                       ctypes.byref(out))
    if st != EH_OK:
        raise EulerError(st, "eh_estimate_request_bytes: invalid arguments")
    return int(out.value)


class Batch:
    """A served stream of independent solves (eh_batch_create ... eh_batch_destroy)."""

    def __init__(self, hbm_budget_bytes, dim=2, gamma=1.4, cfl=0.5, limiter_passes=2, bound_relaxation=False,
                 device=0, precision=EH_PRECISION_FP64, mode=EH_BATCH_MERGED, lib=None):
        self.lib = lib or load()
        cfg = Config()
        self.lib.eh_config_default(ctypes.byref(cfg))
        cfg.dim, cfg.gamma, cfg.cfl, cfg.limiter_passes = dim, gamma, cfl, limiter_passes
        cfg.bound_relaxation, cfg.precision, cfg.device = int(bool(bound_relaxation)), precision, device
        cfg.stream = None
        self.dim, self.S = dim, dim + 2
        b = ctypes.c_void_p()
        st = self.lib.eh_batch_create(ctypes.byref(cfg), int(hbm_budget_bytes), ctypes.byref(b))
        if st != EH_OK:
            raise EulerError(st, f"eh_batch_create failed: {self.lib.eh_status_string(st).decode()}")
        self.b = b
        self.n_of = {}
        self._check(self.lib.eh_batch_set_mode(self.b, int(mode)), "eh_batch_set_mode")

    def repacks(self) -> int:
        """Times a merged batch rebuilt its context."""
        r = ctypes.c_int64(0)
        self._check(self.lib.eh_batch_repacks(self.b, ctypes.byref(r)), "eh_batch_repacks")
        return int(r.value)

    def _check(self, st, what):
        if st != EH_OK:
            raise EulerError(st, f"{what}: {self.lib.eh_batch_last_error(self.b).decode()}")

    def admit(self, mesh, U0, t_final, bnd_state=None):
        """Admits a request; returns its ticket, or None when it does not fit
        the budget now (EH_ERR_OOM)."""
        k = dict(row_ptr=_arr(mesh.row_ptr, np.int64), col=_arr(mesh.col, np.int32), cij=_arr(mesh.cij, np.float64),
                 mij=_arr(mesh.mij, np.float64), mi=_arr(mesh.mi, np.float64), bnd_node=_arr(mesh.bnd_node, np.int32),
                 bnd_kind=_arr(mesh.bnd_kind, np.int32), bnd_normal=_arr(mesh.bnd_normal, np.float64),
                 bnd_state=None if bnd_state is None else _arr(bnd_state, np.float64), U0=_arr(U0, np.float64))
        assert k["U0"].shape == (self.S, mesh.n), k["U0"].shape
        ticket = ctypes.c_int64(0)
        st = self.lib.eh_batch_admit(self.b, mesh.n, mesh.nnz, _p(k["row_ptr"]), _p(k["col"]), _p(k["cij"]),
                                     _p(k["mij"]), _p(k["mi"]), mesh.n_bnd, _p(k["bnd_node"]), _p(k["bnd_kind"]),
                                     _p(k["bnd_normal"]), _p(k["bnd_state"]), _p(k["U0"]), float(t_final),
                                     ctypes.byref(ticket))
        if st == EH_ERR_OOM:
            return None
        self._check(st, "eh_batch_admit")
        self.n_of[ticket.value] = mesh.n
        return ticket.value

    def advance(self, steps=1) -> int:
        """steps SSPRK(3,3) steps of every running request; returns the
        number of finished requests not yet polled."""
        fin = ctypes.c_int32(0)
        self._check(self.lib.eh_batch_advance(self.b, int(steps), ctypes.byref(fin)), "eh_batch_advance")
        return int(fin.value)

    def poll(self, ticket):
        """None while the request runs; else (U [S, n], t, steps) and the
        request is retired."""
        done, t, steps = ctypes.c_int32(0), ctypes.c_double(0.0), ctypes.c_int64(0)
        n = self.n_of.get(ticket)
        U = None if n is None else np.empty((self.S, n))
        st = self.lib.eh_batch_poll(self.b, int(ticket), ctypes.byref(done), _p(U), ctypes.byref(t),
                                    ctypes.byref(steps))
        if done.value:
            del self.n_of[ticket]
        self._check(st, "eh_batch_poll")
        return (U, t.value, steps.value) if done.value else None

    def active(self):
        """(requests admitted and not yet polled, device bytes they hold)."""
        n, used = ctypes.c_int32(0), ctypes.c_uint64(0)
        self._check(self.lib.eh_batch_active(self.b, ctypes.byref(n), ctypes.byref(used)), "eh_batch_active")
        return int(n.value), int(used.value)

    def close(self):
        if getattr(self, "b", None):
            self.lib.eh_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        self.close()


class Solver:
    """One context of the C library (eh_create ... eh_destroy)."""

    def __init__(self, dim=2, gamma=1.4, cfl=0.5, limiter_passes=2, bound_relaxation=False, device=0, stream=None,
                 precision=EH_PRECISION_FP64, lib=None):
        self.lib = lib or load()
        cfg = Config()
        self.lib.eh_config_default(ctypes.byref(cfg))
        cfg.dim, cfg.gamma, cfg.cfl, cfg.limiter_passes = dim, gamma, cfl, limiter_passes
        cfg.bound_relaxation, cfg.precision, cfg.device = int(bool(bound_relaxation)), precision, device
        cfg.stream = stream
        self.cfg = cfg
        self.dim, self.S = dim, dim + 2
        ctx = ctypes.c_void_p()
        st = self.lib.eh_create(ctypes.byref(cfg), ctypes.byref(ctx))
        if st != EH_OK:
            raise EulerError(st, f"eh_create failed: {self.lib.eh_status_string(st).decode()}")
        self.ctx = ctx
        self.n = self.nnz = 0

    def _check(self, st, what):
        if st != EH_OK:
            raise EulerError(st, f"{what}: {self.lib.eh_last_error(self.ctx).decode()}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.eh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def upload_mesh(self, mesh, bnd_state=None):
        self._mesh_keep = k = dict(
            row_ptr=_arr(mesh.row_ptr, np.int64), col=_arr(mesh.col, np.int32), cij=_arr(mesh.cij, np.float64),
            mij=_arr(mesh.mij, np.float64), mi=_arr(mesh.mi, np.float64), bnd_node=_arr(mesh.bnd_node, np.int32),
            bnd_kind=_arr(mesh.bnd_kind, np.int32), bnd_normal=_arr(mesh.bnd_normal, np.float64),
            bnd_state=None if bnd_state is None else _arr(bnd_state, np.float64))
        st = self.lib.eh_upload_mesh(self.ctx, mesh.n, mesh.nnz, _p(k["row_ptr"]), _p(k["col"]), _p(k["cij"]),
                                     _p(k["mij"]), _p(k["mi"]), mesh.n_bnd, _p(k["bnd_node"]), _p(k["bnd_kind"]),
                                     _p(k["bnd_normal"]), _p(k["bnd_state"]))
        self._check(st, "eh_upload_mesh")
        self.n, self.nnz = mesh.n, mesh.nnz
        del self._mesh_keep

    def set_state(self, U):
        """U: numpy [S, n] (host) or a CUDA tensor of that shape (device)."""
        if hasattr(U, "is_cuda") and U.is_cuda:
            assert U.is_contiguous() and tuple(U.shape) == (self.S, self.n)
            self._check(self.lib.eh_set_state(self.ctx, ctypes.c_void_p(U.data_ptr()), 1), "eh_set_state")
        else:
            U = _arr(U, np.float64)
            assert U.shape == (self.S, self.n), U.shape
            self._check(self.lib.eh_set_state(self.ctx, _p(U), 0), "eh_set_state")

    def get_state(self, out=None):
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            self._check(self.lib.eh_get_state(self.ctx, ctypes.c_void_p(out.data_ptr()), 1), "eh_get_state")
            return out
        U = np.empty((self.S, self.n)) if out is None else out
        self._check(self.lib.eh_get_state(self.ctx, _p(U), 0), "eh_get_state")
        return U

    def apply_boundary_conditions(self):
        self._check(self.lib.eh_apply_boundary_conditions(self.ctx), "eh_apply_boundary_conditions")

    def cfl_dt(self) -> float:
        dt = ctypes.c_double(0.0)
        self._check(self.lib.eh_cfl_dt(self.ctx, ctypes.byref(dt)), "eh_cfl_dt")
        return dt.value

    def stage(self, tau=0.0, sync=True):
        used = ctypes.c_double(0.0)
        self._check(self.lib.eh_stage(self.ctx, float(tau), ctypes.byref(used) if sync else None), "eh_stage")
        return used.value if sync else None

    def step(self, dt=0.0, sync=True):
        used = ctypes.c_double(0.0)
        self._check(self.lib.eh_step(self.ctx, float(dt), ctypes.byref(used) if sync else None), "eh_step")
        return used.value if sync else None

    def run(self, nsteps, dt=0.0):
        self._check(self.lib.eh_run(self.ctx, int(nsteps), float(dt)), "eh_run")

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
        self._check(self.lib.eh_set_viscosity(self.ctx, float(mu), float(lam), float(kappa_cv), _p(keep["L"]),
                                              _p(keep["G"]), nc, nv, nq, _p(keep["cells"]), _p(keep["qw"]),
                                              _p(keep["qphi"]), _p(keep["qgrad"]), int(keep["wall"].size),
                                              _p(keep["wall"]), float(cg_tol), int(cg_max_iter)),
                    "eh_set_viscosity")

    def parabolic_step(self, dt):
        info = ParabolicInfo()
        self._check(self.lib.eh_parabolic_step(self.ctx, float(dt), ctypes.byref(info)), "eh_parabolic_step")
        return {f: getattr(info, f) for f, _ in ParabolicInfo._fields_}

    def step_ns(self, dt=0.0):
        """One Strang-split Navier-Stokes step; returns (tau, info)."""
        info = ParabolicInfo()
        tau = ctypes.c_double(0.0)
        self._check(self.lib.eh_step_ns(self.ctx, float(dt), ctypes.byref(tau), ctypes.byref(info)), "eh_step_ns")
        return tau.value, {f: getattr(info, f) for f, _ in ParabolicInfo._fields_}

    def step_adaptive(self, cfl_max):
        """One step with the CFL number adapted above 1; returns (dt, cfl, restarts)."""
        dt, cfl, r = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int32(0)
        self._check(self.lib.eh_step_adaptive(self.ctx, float(cfl_max), ctypes.byref(dt), ctypes.byref(cfl),
                                              ctypes.byref(r)), "eh_step_adaptive")
        return dt.value, cfl.value, r.value

    def synchronize(self):
        self._check(self.lib.eh_synchronize(self.ctx), "eh_synchronize")

    def diagnostics(self) -> dict:
        d = Diagnostics()
        self._check(self.lib.eh_get_diagnostics(self.ctx, ctypes.byref(d)), "eh_get_diagnostics")
        return dict(t=d.t, steps=d.steps, last_dt=d.last_dt, last_stage_bound=list(d.last_stage_bound),
                    cfl_violations=d.cfl_violations, not_admissible=d.not_admissible,
                    line_searches_deferred=d.line_searches_deferred,
                    line_searches_iterated=d.line_searches_iterated,
                    low_order_not_admissible=d.low_order_not_admissible,
                    rho_min=d.rho_min, e_min=d.e_min, total=list(d.total)[:self.S])

    def trace(self, what):
        sizes = {EH_TRACE_D_IJ: self.nnz, EH_TRACE_ALPHA: self.n, EH_TRACE_U_LOW: self.S * self.n,
                 EH_TRACE_F_HIGH: self.S * self.n, EH_TRACE_BOUNDS: 3 * self.n, EH_TRACE_L_PASS1: self.nnz,
                 EH_TRACE_U_PASS1: self.S * self.n, EH_TRACE_TAU: 1, EH_TRACE_TAU_BOUND: 1,
                 EH_TRACE_P_PASS1: self.S * self.nnz, EH_TRACE_L_LAST: self.nnz}
        count = sizes[what]
        out = np.empty(count)
        self._check(self.lib.eh_trace(self.ctx, what, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), count),
                    "eh_trace")
        if what in (EH_TRACE_U_LOW, EH_TRACE_F_HIGH, EH_TRACE_U_PASS1):
            return out.reshape(self.S, self.n)
        if what == EH_TRACE_BOUNDS:
            return out.reshape(3, self.n)
        if what == EH_TRACE_P_PASS1:
            return out.reshape(self.S, self.nnz)
        if what in (EH_TRACE_TAU, EH_TRACE_TAU_BOUND):
            return float(out[0])
        return out

    def mesh_index(self):
        """(row_ptr, col, transpose) as the device holds them (eh_get_mesh_index)."""
        row_ptr = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(self.nnz, dtype=np.int32)
        tr = np.empty(self.nnz, dtype=np.int32)
        self._check(self.lib.eh_get_mesh_index(self.ctx, row_ptr.ctypes.data_as(ctypes.c_void_p),
                                               col.ctypes.data_as(ctypes.c_void_p),
                                               tr.ctypes.data_as(ctypes.c_void_p)), "eh_get_mesh_index")
        return row_ptr, col, tr

    def profile(self, enable: bool):
        self._check(self.lib.eh_profile_enable(self.ctx, int(bool(enable))), "eh_profile_enable")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since profiling was enabled."""
        out = {}
        for k, name in enumerate(KERNEL_NAMES):
            ms, cnt = ctypes.c_double(0.0), ctypes.c_int64(0)
            self._check(self.lib.eh_profile_read(self.ctx, k, ctypes.byref(ms), ctypes.byref(cnt)), "eh_profile_read")
            out[name] = (ms.value, cnt.value)
        return out

    def set_instances(self, row_offset, t_final=None):
        """Declare the uploaded (block-diagonal) mesh as independent instances."""
        off = _arr(row_offset, np.int64)
        tf = None if t_final is None else _arr(t_final, np.float64)
        self._check(self.lib.eh_set_instances(self.ctx, off.size - 1, _p(off), _p(tf)), "eh_set_instances")
        self.ninst = off.size - 1

    def instances(self) -> dict:
        k = getattr(self, "ninst", 1)
        t, dt, b = np.empty(k), np.empty(k), np.empty((3, k))
        self._check(self.lib.eh_get_instances(self.ctx, _p(t), _p(dt), _p(b)), "eh_get_instances")
        steps = np.empty(k, dtype=np.int64)
        self._check(self.lib.eh_get_instance_steps(self.ctx, _p(steps)), "eh_get_instance_steps")
        return dict(t=t, last_dt=dt, stage_bound=b, steps=steps)

    def autotune(self, steps_per_candidate=2) -> dict:
        chosen = np.zeros(len(KERNEL_NAMES), dtype=np.int32)
        self._check(self.lib.eh_autotune(self.ctx, int(steps_per_candidate), _p(chosen)), "eh_autotune")
        return dict(zip(KERNEL_NAMES, chosen.tolist()))

    def block_sizes(self) -> dict:
        out = np.zeros(len(KERNEL_NAMES), dtype=np.int32)
        self._check(self.lib.eh_get_block_sizes(self.ctx, _p(out)), "eh_get_block_sizes")
        return dict(zip(KERNEL_NAMES, out.tolist()))

    def rows_per_sm(self) -> dict:
        out = np.zeros(len(KERNEL_NAMES), dtype=np.int32)
        self._check(self.lib.eh_get_rows_per_sm(self.ctx, _p(out)), "eh_get_rows_per_sm")
        return dict(zip(KERNEL_NAMES, out.tolist()))

    def set_launch_shape(self, kernel: str, threads_per_block: int, rows_per_sm: int = 0):
        self._check(self.lib.eh_set_launch_shape(self.ctx, KERNEL_NAMES.index(kernel), int(threads_per_block),
                                                 int(rows_per_sm)), "eh_set_launch_shape")

    def launches_per_step(self) -> int:
        return int(self.lib.eh_launches_per_step(self.ctx))
