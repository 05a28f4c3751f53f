"""Thin ctypes binding of libafc (include/afc.h).

Argument marshalling only: every numerical step runs in the CUDA library.  The
functions keep the C names; ``Problem`` wraps a handle for convenience.  Arrays
are numpy float64 (host) or torch CUDA tensors (device, where a call accepts
device pointers).  Importing this module without a built libafc.so raises
ImportError: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "afc.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libafc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = C.CDLL(LIB_PATH)

# ---- enums (mirror include/afc.h) ----
AFC_OK, AFC_NOT_CONVERGED = 0, 1
AFC_E_INVALID, AFC_E_OOM, AFC_E_CUDA, AFC_E_NAN, AFC_E_TIMEOUT, AFC_E_STATE = -1, -2, -3, -4, -5, -6
AFC_P1, AFC_Q1 = 0, 1
AFC_FAMILY_FCT, AFC_FAMILY_MC = 0, 1
AFC_SSP2, AFC_SSP3, AFC_CN_NONLINEAR, AFC_CN_LINEAR = 0, 1, 2, 3
AFC_LIM_NONE, AFC_LIM_GALERKIN, AFC_LIM_ZALESAK, AFC_LIM_MC, AFC_LIM_MU = 0, 1, 2, 3, 4
AFC_KSP_BICGSTAB, AFC_KSP_GMRES = 0, 1
AFC_FP64, AFC_MIXED = 0, 1
AFC_MAT_MC, AFC_MAT_A, AFC_MAT_D, AFC_MAT_LOW, AFC_MAT_K, AFC_MAT_S = 0, 1, 2, 3, 4, 5
AFC_BATCH_AUTO, AFC_BATCH_PER_PASS, AFC_BATCH_PER_STAGE, AFC_BATCH_PER_STEP = 0, 1, 2, 3
AFC_REQ_TRANSIENT, AFC_REQ_STATIONARY = 0, 1
AFC_SERVE_BATCHED, AFC_SERVE_SERIAL = 0, 1
AFC_REQ_PENDING, AFC_REQ_RUNNING, AFC_REQ_DONE, AFC_REQ_FAILED, AFC_REQ_CANCELLED = 0, 1, 2, 3, 4

ELEM = {"p1": AFC_P1, "q1": AFC_Q1}


class afc_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("nnz", C.c_int64), ("n_edges", C.c_int64), ("n_offsets", C.c_int32),
                ("max_offset", C.c_int32), ("device_bytes", C.c_int64), ("assembled", C.c_int32),
                ("family", C.c_int32)]


class afc_opts(C.Structure):
    _fields_ = [("scheme", C.c_int32), ("limiter", C.c_int32), ("dt", C.c_double), ("fp_tol", C.c_double),
                ("fp_maxit", C.c_int32), ("fp_fixed_its", C.c_int32), ("omega", C.c_double), ("ksp", C.c_int32),
                ("ksp_maxit", C.c_int32), ("ksp_atol", C.c_double), ("ksp_rtol", C.c_double),
                ("gmres_restart", C.c_int32), ("precision", C.c_int32), ("prelimit", C.c_int32),
                ("graph", C.c_int32)]


class afc_stats(C.Structure):
    _fields_ = [("outer_its", C.c_int32), ("inner_its", C.c_int32), ("stages", C.c_int32), ("status", C.c_int32),
                ("res0", C.c_double), ("res_final", C.c_double), ("umin", C.c_double), ("umax", C.c_double),
                ("dmp_violation", C.c_double), ("t_ms", C.c_double)]


class afc_batch_tuning(C.Structure):
    _fields_ = [("mode", C.c_int32), ("block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("ms_per_step", C.c_double)]


class afc_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("elem", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("eps", C.c_double), ("c", C.c_double),
                ("b", C.POINTER(C.c_double)), ("f", C.POINTER(C.c_double)), ("dir_mask", C.POINTER(C.c_uint8)),
                ("u_dir", C.POINTER(C.c_double)), ("u0", C.POINTER(C.c_double)), ("family", C.c_int32),
                ("steps", C.c_int32), ("cfl", C.c_double), ("opts", afc_opts)]


class afc_result(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("stats", afc_stats), ("n_nodes", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("message", C.c_char * 160)]


class afc_serve_config(C.Structure):
    _fields_ = [("mode", C.c_int32), ("max_active", C.c_int32), ("hbm_budget", C.c_int64),
                ("stationary_workers", C.c_int32), ("max_chunk", C.c_int32), ("builders", C.c_int32)]


class afc_serve_info(C.Structure):
    _fields_ = [("pending", C.c_int64), ("active", C.c_int64), ("bytes_in_use", C.c_int64),
                ("completed", C.c_int64), ("failed", C.c_int64), ("chunks", C.c_int64),
                ("batched_steps", C.c_int64), ("max_batch", C.c_int64), ("instance_steps", C.c_int64),
                ("clock", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_U8 = C.POINTER(C.c_uint8)

_SIGS = {
    "afc_create_structured": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _D, _D, C.c_int, _P, C.POINTER(_P)]),
    "afc_create_from_elements": (C.c_int, [C.c_int, C.c_int64, _D, C.c_int64, _I32, C.c_int, _P, C.POINTER(_P)]),
    "afc_destroy": (C.c_int, [_P]),
    "afc_set_coefficients": (C.c_int, [_P, C.c_double, _D, _D, _D, C.c_double, _D]),
    "afc_set_dirichlet": (C.c_int, [_P, _U8, _D]),
    "afc_assemble": (C.c_int, [_P, C.c_int, C.c_int]),
    "afc_get_info": (C.c_int, [_P, C.POINTER(afc_info)]),
    "afc_export_csr": (C.c_int, [_P, C.c_int, _I32, _I32, _D]),
    "afc_export_lumped_mass": (C.c_int, [_P, _D]),
    "afc_set_solution": (C.c_int, [_P, _P, C.c_int]),
    "afc_get_solution": (C.c_int, [_P, _P, C.c_int]),
    "afc_cfl_timestep": (C.c_int, [_P, C.c_double, _D]),
    "afc_default_opts": (None, [C.POINTER(afc_opts)]),
    "afc_step": (C.c_int, [_P, C.POINTER(afc_opts), C.POINTER(afc_stats)]),
    "afc_solve_stationary": (C.c_int, [_P, C.POINTER(afc_opts), C.POINTER(afc_stats)]),
    "afc_fe_stage": (C.c_int, [_P, C.c_double, C.c_int, _D, _D, _D, _D, _D]),
    "afc_cn_limited_sum": (C.c_int, [_P, C.c_double, C.c_int, C.c_int, _D, _D, _D, _D, _D, _D]),
    "afc_mc_limited_sum": (C.c_int, [_P, C.c_int, _D, _D, _D, _D]),
    "afc_mc_limited_sum_noalloc": (C.c_int, [_P, C.c_int, _P, _P]),
    "afc_mc_residual_sweep": (C.c_int, [_P, C.c_int]),
    "afc_get_residual": (C.c_int, [_P, _D]),
    "afc_apply": (C.c_int, [_P, C.c_int, _D, _D]),
    "afc_linear_solve": (C.c_int, [_P, C.c_int, C.c_double, C.POINTER(afc_opts), _D, _D, _I32, _D]),
    "afc_profile": (C.c_int, [_P, C.c_int]),
    "afc_profile_read": (C.c_int, [_P, C.c_int, C.c_char_p, _D, C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int64)]),
    "afc_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P)]),
    "afc_batch_destroy": (C.c_int, [_P]),
    "afc_batch_step": (C.c_int, [_P, C.POINTER(afc_opts), _D, C.c_int, C.POINTER(afc_stats)]),
    "afc_batch_set_tuning": (C.c_int, [_P, C.POINTER(afc_batch_tuning)]),
    "afc_batch_get_tuning": (C.c_int, [_P, C.POINTER(afc_batch_tuning)]),
    "afc_batch_tune": (C.c_int, [_P, C.POINTER(afc_opts), _D, C.POINTER(afc_batch_tuning)]),
    "afc_batch_info": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "afc_serve_default_config": (None, [C.POINTER(afc_serve_config)]),
    "afc_serve_estimate_bytes": (C.c_int64, [C.POINTER(afc_request)]),
    "afc_serve_create": (C.c_int, [C.c_int, C.POINTER(afc_serve_config), C.POINTER(_P)]),
    "afc_serve_submit": (C.c_int, [_P, C.POINTER(afc_request), C.POINTER(C.c_int64)]),
    "afc_serve_poll": (C.c_int, [_P, C.c_int64, C.POINTER(afc_result), _D]),
    "afc_serve_wait": (C.c_int, [_P, C.c_int64, C.c_double, C.POINTER(afc_result), _D]),
    "afc_serve_cancel": (C.c_int, [_P, C.c_int64]),
    "afc_serve_release": (C.c_int, [_P, C.c_int64]),
    "afc_serve_get_info": (C.c_int, [_P, C.POINTER(afc_serve_info)]),
    "afc_serve_destroy": (C.c_int, [_P]),
    "afc_selftest_grid_wait": (C.c_int, [C.c_int, C.c_double, C.POINTER(C.c_int), _D]),
    "afc_selftest_split": (C.c_int, [C.c_int, _D, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_float), _D]),
    "afc_set_grid_wait_limit": (C.c_int, [_P, C.c_double]),
    "afc_status_str": (C.c_char_p, [C.c_int]),
    "afc_last_error": (C.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class AfcError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str | None = None):
        msg = _lib.afc_status_str(status).decode()
        if detail is None:
            detail = _lib.afc_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}): {detail}")
        self.status = status


def check_device_vector(t, n: int, device: int, name: str, where: str):
    """Reject, before any library call, a tensor that a device-pointer entry point
    cannot take: it must be a contiguous CUDA float64 tensor of exactly n elements
    on `device`.  Raises AfcError(AFC_E_INVALID)."""
    def bad(why):
        raise AfcError(AFC_E_INVALID, where, f"{name} {why}")
    if not (hasattr(t, "data_ptr") and hasattr(t, "is_cuda")):
        bad("is not a tensor")
    if not t.is_cuda:
        bad("is not on a CUDA device")
    if str(t.dtype) != "torch.float64":
        bad(f"has dtype {t.dtype}, not torch.float64")
    if not t.is_contiguous():
        bad("is not contiguous")
    if t.numel() != n:
        bad(f"has {t.numel()} elements, not {n}")
    if t.device.index is not None and t.device.index != device:
        bad(f"is on cuda:{t.device.index}, the problem on cuda:{device}")


def _check(st: int, where: str, allow_not_converged=False) -> int:
    if st == AFC_OK or (allow_not_converged and st == AFC_NOT_CONVERGED):
        return st
    raise AfcError(st, where)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def selftest_split(x, device: int = 0):
    """Run afc_selftest_split: the device's float pairs (hi, lo) of the doubles x and hi
    widened back to double."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    n = a.size
    hi = np.zeros(n, np.float32)
    lo = np.zeros(n, np.float32)
    back = np.zeros(n, np.float64)
    fp = C.POINTER(C.c_float)
    _check(_lib.afc_selftest_split(int(device), _dp(a), n, hi.ctypes.data_as(fp), lo.ctypes.data_as(fp), _dp(back)),
           "afc_selftest_split")
    return hi, lo, back


def selftest_grid_wait(limit_ms: float = 50.0, device: int = 0) -> tuple[int, float]:
    """Run afc_selftest_grid_wait: (status the expired barrier reports, launch ms)."""
    obs = C.c_int(-1)
    ms = C.c_double(0.0)
    _check(_lib.afc_selftest_grid_wait(int(device), float(limit_ms), C.byref(obs), C.byref(ms)),
           "afc_selftest_grid_wait")
    return obs.value, ms.value


def default_opts(**kw) -> afc_opts:
    o = afc_opts()
    _lib.afc_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def stats_dict(s: afc_stats) -> dict:
    return {name: getattr(s, name) for name, _ in afc_stats._fields_}


def current_stream_handle():
    """The current torch CUDA stream as a cudaStream_t, or None (legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch absent
        pass
    return None


class Problem:
    """Owner of one afc_problem handle."""

    def __init__(self, handle: C.c_void_p, n_nodes: int, device: int = 0):
        self.h = handle
        self.N = int(n_nodes)
        self.device = int(device)

    @classmethod
    def structured(cls, elem, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), device=0, stream=None):
        if np.isscalar(n):
            n = (int(n),) * 3
        h = C.c_void_p()
        lo_a, hi_a = _f64(lo, 3), _f64(hi, 3)
        st = _lib.afc_create_structured(ELEM.get(elem, elem), int(n[0]), int(n[1]), int(n[2]), _dp(lo_a), _dp(hi_a),
                                        device, stream if stream is not None else current_stream_handle(),
                                        C.byref(h))
        _check(st, "afc_create_structured")
        return cls(h, int(np.prod(n)), device)

    @classmethod
    def from_elements(cls, elem, xyz, conn, device=0, stream=None):
        xyz = _f64(xyz)
        conn = np.ascontiguousarray(np.asarray(conn, dtype=np.int32))
        nl = 4 if ELEM.get(elem, elem) == AFC_P1 else 8
        h = C.c_void_p()
        st = _lib.afc_create_from_elements(ELEM.get(elem, elem), xyz.size // 3, _dp(xyz), conn.size // nl,
                                           conn.ctypes.data_as(_I32), device,
                                           stream if stream is not None else current_stream_handle(), C.byref(h))
        _check(st, "afc_create_from_elements")
        return cls(h, xyz.size // 3, device)

    def close(self):
        if self.h:
            _lib.afc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- data ----
    def set_coefficients(self, eps, b, c=0.0, f=None):
        """b: nodal velocity (N, 3), or one 3-vector for a constant field; c: a constant
        reaction or nodal values (N,); f: nodal source (N,) or None."""
        ba = np.asarray(b, dtype=np.float64)
        bn, bc = (None, _f64(ba, 3)) if ba.shape == (3,) else \
            (_f64(np.broadcast_to(ba, (self.N, 3)), 3 * self.N), None)
        ca = np.asarray(c, dtype=np.float64)
        cn, cc = (None, float(ca)) if ca.ndim == 0 else (_f64(np.broadcast_to(ca, (self.N,)), self.N), 0.0)
        fa = None if f is None else _f64(np.broadcast_to(np.asarray(f, dtype=np.float64), (self.N,)), self.N)
        _check(_lib.afc_set_coefficients(self.h, float(eps), None if bn is None else _dp(bn),
                                         None if bc is None else _dp(bc), None if cn is None else _dp(cn), cc,
                                         None if fa is None else _dp(fa)), "afc_set_coefficients")

    def set_dirichlet(self, mask, values):
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        v = _f64(np.broadcast_to(np.asarray(values, dtype=np.float64), (self.N,)), self.N)
        _check(_lib.afc_set_dirichlet(self.h, m.ctypes.data_as(_U8), _dp(v)), "afc_set_dirichlet")

    def assemble(self, family=AFC_FAMILY_FCT, precision=AFC_FP64):
        _check(_lib.afc_assemble(self.h, family, precision), "afc_assemble")

    def info(self) -> dict:
        i = afc_info()
        _check(_lib.afc_get_info(self.h, C.byref(i)), "afc_get_info")
        return {name: getattr(i, name) for name, _ in afc_info._fields_}

    def export_csr(self, which):
        inf = self.info()
        rowptr = np.zeros(self.N + 1, np.int32)
        col = np.zeros(inf["nnz"], np.int32)
        val = np.zeros(inf["nnz"], np.float64)
        _check(_lib.afc_export_csr(self.h, which, rowptr.ctypes.data_as(_I32), col.ctypes.data_as(_I32), _dp(val)),
               "afc_export_csr")
        return rowptr, col, val

    def lumped_mass(self):
        out = np.zeros(self.N)
        _check(_lib.afc_export_lumped_mass(self.h, _dp(out)), "afc_export_lumped_mass")
        return out

    def set_solution(self, u):
        if hasattr(u, "is_cuda") and u.is_cuda:
            t = u.contiguous().to(dtype=__import__("torch").float64)
            _check(_lib.afc_set_solution(self.h, C.c_void_p(t.data_ptr()), 1), "afc_set_solution")
            return
        a = _f64(u, self.N)
        _check(_lib.afc_set_solution(self.h, a.ctypes.data_as(C.c_void_p), 0), "afc_set_solution")

    def get_solution(self, out=None):
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            _check(_lib.afc_get_solution(self.h, C.c_void_p(out.data_ptr()), 1), "afc_get_solution")
            return out
        a = np.zeros(self.N)
        _check(_lib.afc_get_solution(self.h, a.ctypes.data_as(C.c_void_p), 0), "afc_get_solution")
        return a

    def cfl_timestep(self, cfl) -> float:
        dt = C.c_double()
        _check(_lib.afc_cfl_timestep(self.h, float(cfl), C.byref(dt)), "afc_cfl_timestep")
        return dt.value

    # ---- hot path ----
    def step(self, opts: afc_opts) -> dict:
        s = afc_stats()
        st = _lib.afc_step(self.h, C.byref(opts), C.byref(s))
        _check(st, "afc_step", allow_not_converged=True)
        return stats_dict(s)

    def solve_stationary(self, opts: afc_opts) -> dict:
        s = afc_stats()
        st = _lib.afc_solve_stationary(self.h, C.byref(opts), C.byref(s))
        _check(st, "afc_solve_stationary", allow_not_converged=True)
        return stats_dict(s)

    # ---- single passes ----
    def fe_stage(self, dt, limiter=AFC_LIM_ZALESAK) -> dict:
        out = {k: np.zeros(self.N) for k in ("u_tilde", "Rp", "Rm", "Fstar", "u_new")}
        _check(_lib.afc_fe_stage(self.h, float(dt), limiter, *(_dp(out[k]) for k in
                                 ("u_tilde", "Rp", "Rm", "Fstar", "u_new"))), "afc_fe_stage")
        return out

    def cn_limited_sum(self, dt, u_new, u_old, limiter=AFC_LIM_ZALESAK, prelimit=1) -> dict:
        un, uo = _f64(u_new, self.N), _f64(u_old, self.N)
        out = {k: np.zeros(self.N) for k in ("u_tilde", "Rp", "Rm", "Fstar")}
        _check(_lib.afc_cn_limited_sum(self.h, float(dt), limiter, prelimit, _dp(un), _dp(uo),
                                       *(_dp(out[k]) for k in ("u_tilde", "Rp", "Rm", "Fstar"))),
               "afc_cn_limited_sum")
        return out

    def mc_limited_sum(self, u, limiter=AFC_LIM_MC) -> dict:
        ua = _f64(u, self.N)
        out = {k: np.zeros(self.N) for k in ("umax", "umin", "Fstar")}
        _check(_lib.afc_mc_limited_sum(self.h, limiter, _dp(ua), *(_dp(out[k]) for k in ("umax", "umin", "Fstar"))),
               "afc_mc_limited_sum")
        return out

    def mc_limited_sum_noalloc(self, u, Fstar, limiter=AFC_LIM_MC):
        """Device-pointer variant that allocates nothing (u, Fstar: contiguous CUDA
        float64 tensors of N elements on the problem's device, checked here)."""
        check_device_vector(u, self.N, self.device, "u", "afc_mc_limited_sum_noalloc")
        check_device_vector(Fstar, self.N, self.device, "Fstar", "afc_mc_limited_sum_noalloc")
        _check(_lib.afc_mc_limited_sum_noalloc(self.h, limiter, C.c_void_p(u.data_ptr()),
                                               C.c_void_p(Fstar.data_ptr())), "afc_mc_limited_sum_noalloc")
        return Fstar

    def get_residual(self) -> np.ndarray:
        """The residual f + F*(u) - AA u that the last mc_residual_sweep left (host copy)."""
        r = np.zeros(self.N)
        _check(_lib.afc_get_residual(self.h, _dp(r)), "afc_get_residual")
        return r

    def set_grid_wait_limit(self, limit_ms: float):
        """Bounded-wait limit (ms) of the grid barriers of this problem's persistent solver launches."""
        _check(_lib.afc_set_grid_wait_limit(self.h, float(limit_ms)), "afc_set_grid_wait_limit")

    def mc_residual_sweep(self, limiter=AFC_LIM_MC):
        """Enqueue one MC limiter + residual sweep on the stored solution (no sync)."""
        _check(_lib.afc_mc_residual_sweep(self.h, limiter), "afc_mc_residual_sweep")

    def apply(self, which, x):
        xa = _f64(x, self.N)
        y = np.zeros(self.N)
        _check(_lib.afc_apply(self.h, which, _dp(xa), _dp(y)), "afc_apply")
        return y

    def profile(self, on: bool):
        _check(_lib.afc_profile(self.h, 1 if on else 0), "afc_profile")

    def profile_read(self) -> tuple[dict, int]:
        """({kernel name: (total_ms, launches)}, launches issued since creation)."""
        cap = 256
        names = C.create_string_buffer(48 * cap)
        tot = np.zeros(cap)
        cnt = np.zeros(cap, np.int64)
        n = C.c_int()
        allc = C.c_int64()
        _check(_lib.afc_profile_read(self.h, cap, names, _dp(tot), cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                                     C.byref(n), C.byref(allc)), "afc_profile_read")
        raw = names.raw
        out = {}
        for k in range(n.value):
            nm = raw[48 * k:48 * k + 48].split(b"\0", 1)[0].decode()
            out[nm] = (float(tot[k]), int(cnt[k]))
        return out, allc.value

    def launches(self) -> int:
        allc = C.c_int64()
        _check(_lib.afc_profile_read(self.h, 0, None, None, None, None, C.byref(allc)), "afc_profile_read")
        return allc.value

    def linear_solve(self, system, rhs, opts: afc_opts, dt=0.0):
        r = _f64(rhs, self.N)
        x = np.zeros(self.N)
        its = C.c_int32()
        res = C.c_double()
        st = _lib.afc_linear_solve(self.h, system, float(dt), C.byref(opts), _dp(r), _dp(x), C.byref(its),
                                   C.byref(res))
        _check(st, "afc_linear_solve", allow_not_converged=True)
        return x, its.value, res.value


def tuning_dict(t: afc_batch_tuning) -> dict:
    return {name: getattr(t, name) for name, _ in afc_batch_tuning._fields_}


class Batch:
    """Owner of one afc_batch handle over a list of assembled Problems (kept alive here)."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.h for p in self.problems])
        h = C.c_void_p()
        _check(_lib.afc_batch_create(arr, len(self.problems), C.byref(h)), "afc_batch_create")
        self.h = h

    def close(self):
        if self.h:
            _lib.afc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, opts: afc_opts, dt=None, nsteps=1) -> list:
        n = len(self.problems)
        dta = None if dt is None else _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)), n)
        stats = (afc_stats * n)()
        _check(_lib.afc_batch_step(self.h, C.byref(opts), None if dta is None else _dp(dta), int(nsteps), stats),
               "afc_batch_step")
        return [stats_dict(s) for s in stats]

    def set_tuning(self, mode, block=256, blocks_per_sm=0):
        t = afc_batch_tuning(mode, block, blocks_per_sm, 0.0)
        _check(_lib.afc_batch_set_tuning(self.h, C.byref(t)), "afc_batch_set_tuning")

    def get_tuning(self) -> dict:
        t = afc_batch_tuning()
        _check(_lib.afc_batch_get_tuning(self.h, C.byref(t)), "afc_batch_get_tuning")
        return tuning_dict(t)

    def tune(self, opts: afc_opts, dt=None) -> dict:
        n = len(self.problems)
        dta = None if dt is None else _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)), n)
        t = afc_batch_tuning()
        _check(_lib.afc_batch_tune(self.h, C.byref(opts), None if dta is None else _dp(dta), C.byref(t)),
               "afc_batch_tune")
        return tuning_dict(t)

    def info(self) -> tuple[int, int]:
        """(total nodes, kernel launches issued by the batch's calls)."""
        tn, nl = C.c_int64(), C.c_int64()
        _check(_lib.afc_batch_info(self.h, C.byref(tn), C.byref(nl)), "afc_batch_info")
        return tn.value, nl.value


def _struct_dict(x) -> dict:
    out = {}
    for name, _ in x._fields_:
        v = getattr(x, name)
        if isinstance(v, afc_stats):
            v = stats_dict(v)
        elif isinstance(v, bytes):
            v = v.decode(errors="replace")
        out[name] = v
    return out


def serve_config(**kw) -> afc_serve_config:
    c = afc_serve_config()
    _lib.afc_serve_default_config(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


class Request:
    """An afc_request plus the arrays it points to (kept alive until submission)."""

    def __init__(self, kind, elem, n, eps, c, b, u0, dir_mask, u_dir, f=None, opts=None, steps=0, cfl=0.5,
                 family=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        if np.isscalar(n):
            n = (int(n),) * 3
        N = int(np.prod(n))
        self.N = N
        self._b = _f64(np.broadcast_to(np.asarray(b, dtype=np.float64), (N, 3)), 3 * N)
        self._u0 = _f64(u0, N)
        self._m = np.ascontiguousarray(np.asarray(dir_mask, dtype=np.uint8))
        self._ud = _f64(np.broadcast_to(np.asarray(u_dir, dtype=np.float64), (N,)), N)
        self._f = None if f is None else _f64(np.broadcast_to(np.asarray(f, dtype=np.float64), (N,)), N)
        r = afc_request()
        r.kind = kind
        r.elem = ELEM.get(elem, elem)
        r.n[:] = [int(v) for v in n]
        r.lo[:] = [float(v) for v in lo]
        r.hi[:] = [float(v) for v in hi]
        r.eps, r.c = float(eps), float(c)
        r.b, r.u0, r.u_dir = _dp(self._b), _dp(self._u0), _dp(self._ud)
        r.dir_mask = self._m.ctypes.data_as(_U8)
        r.f = _dp(self._f) if self._f is not None else None
        if family is None:
            family = AFC_FAMILY_MC if kind == AFC_REQ_STATIONARY else AFC_FAMILY_FCT
        r.family = family
        r.steps = int(steps)
        r.cfl = float(cfl)
        r.opts = opts if opts is not None else default_opts()
        self.c = r

    def estimate_bytes(self) -> int:
        return int(_lib.afc_serve_estimate_bytes(C.byref(self.c)))


class Server:
    """Owner of one afc_server handle."""

    def __init__(self, device=0, **cfg):
        c = serve_config(**cfg)
        h = C.c_void_p()
        _check(_lib.afc_serve_create(int(device), C.byref(c), C.byref(h)), "afc_serve_create")
        self.h = h
        self.sizes = {}

    def close(self):
        if self.h:
            _lib.afc_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, req: Request) -> int:
        rid = C.c_int64()
        _check(_lib.afc_serve_submit(self.h, C.byref(req.c), C.byref(rid)), "afc_serve_submit")
        self.sizes[rid.value] = req.N
        return rid.value

    def poll(self, rid, want_u=False):
        res = afc_result()
        u = np.zeros(self.sizes[rid]) if want_u else None
        _check(_lib.afc_serve_poll(self.h, int(rid), C.byref(res), _dp(u) if u is not None else None),
               "afc_serve_poll")
        return _struct_dict(res), u

    def wait(self, rid, timeout=-1.0, want_u=True):
        res = afc_result()
        u = np.zeros(self.sizes[rid]) if want_u else None
        _check(_lib.afc_serve_wait(self.h, int(rid), float(timeout), C.byref(res),
                                   _dp(u) if u is not None else None), "afc_serve_wait")
        return _struct_dict(res), u

    def cancel(self, rid):
        _check(_lib.afc_serve_cancel(self.h, int(rid)), "afc_serve_cancel")

    def release(self, rid):
        _check(_lib.afc_serve_release(self.h, int(rid)), "afc_serve_release")
        self.sizes.pop(rid, None)

    def info(self) -> dict:
        i = afc_serve_info()
        _check(_lib.afc_serve_get_info(self.h, C.byref(i)), "afc_serve_get_info")
        return _struct_dict(i)
