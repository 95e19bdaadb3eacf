"""Python binding of libba (include/ba.h): argument marshalling only.

Every step of the bundle-adjustment path runs in the CUDA kernels of
``csrc/``; this module converts numpy arrays to pointers, calls the C ABI and
turns non-zero statuses into ``BAError``.  There is no fallback: if the
compiled library is missing, loading fails loudly.

The functions carry the C names (``ba_problem_create``, ``ba_linearize``,
``ba_form_rcs``, ``ba_solve_rcs``, ``ba_back_substitute``, ``ba_lm_step``, the
getters and ``ba_problem_destroy``); ``Problem`` wraps a handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

BA_OK = 0
BA_ERR_INVALID_ARG = 1
BA_ERR_OOM = 2
BA_ERR_CUDA = 3
BA_ERR_NONFINITE = 4
BA_ERR_NOT_SPD = 5
BA_ERR_NO_CONVERGENCE = 6
BA_ERR_TIMEOUT = 7
BA_ERR_STATE = 8
BA_ERR_INTERNAL = 9
BA_FP64 = 0
BA_FP32 = 1
BA_PCG_AUTO, BA_PCG_STANDARD, BA_PCG_SPLIT, BA_PCG_IMPLICIT = 0, 1, 2, 3
BA_FMT_BSMC, BA_FMT_BSR_FULL, BA_FMT_CSR, BA_FMT_IMPLICIT, BA_FMT_BSMC_ONCE = 0, 1, 2, 3, 4
BA_LOSS_PLAIN = 0
BA_LOSS_HUBER = 1
BA_PC_BLOCK_JACOBI = 0

STATUS_NAMES = {0: "BA_OK", 1: "BA_ERR_INVALID_ARG", 2: "BA_ERR_OOM", 3: "BA_ERR_CUDA", 4: "BA_ERR_NONFINITE",
                5: "BA_ERR_NOT_SPD", 6: "BA_ERR_NO_CONVERGENCE", 7: "BA_ERR_TIMEOUT", 8: "BA_ERR_STATE",
                9: "BA_ERR_INTERNAL"}


class BAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ba_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("robust", ctypes.c_int32),
                ("huber_delta", ctypes.c_double), ("lambda0", ctypes.c_double), ("pcg_rel_tol", ctypes.c_double),
                ("pcg_max_iters", ctypes.c_int32), ("inner_rel_tol", ctypes.c_double),
                ("refine_max", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("device_mem_cap", ctypes.c_size_t),
                ("group_max_obs", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("solve_precision", ctypes.c_int32),
                ("pcg_variant", ctypes.c_int32)]


class ba_step_info(ctypes.Structure):
    _fields_ = [("cost_before", ctypes.c_double), ("cost_after", ctypes.c_double),
                ("cost_trial", ctypes.c_double), ("predicted", ctypes.c_double), ("rho", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("accepted", ctypes.c_int32), ("pcg_iters", ctypes.c_int32),
                ("refine_steps", ctypes.c_int32), ("used_fallback", ctypes.c_int32),
                ("rcs_rel_resid", ctypes.c_double), ("n_cheirality", ctypes.c_int64),
                ("n_v_fp64", ctypes.c_int64), ("ms", ctypes.c_float * 8)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "ms"}
        d["lambda"] = d.pop("lambda_")
        d["ms"] = list(self.ms)
        return d


class ba_stats(ctypes.Structure):
    _fields_ = [("n_cams", ctypes.c_int32), ("n_pts", ctypes.c_int64), ("n_obs", ctypes.c_int64),
                ("nnzb", ctypes.c_int64), ("n_groups", ctypes.c_int64), ("n_partials", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("pcg_phase_us", ctypes.c_double * 3),
                ("rcs_phase_us", ctypes.c_double * 3), ("pcg_work_imbalance", ctypes.c_double),
                ("n_v_fp64", ctypes.c_int64)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_S = ctypes.c_int  # ba_status

# (name, restype, argtypes) of every C entry point in include/*.h
SIGNATURES = [
    ("ba_options_default", None, [ctypes.POINTER(ba_options)]),
    ("ba_problem_create", _S, [ctypes.POINTER(ba_options), ctypes.c_int32, _D, ctypes.c_int64, _D,
                               ctypes.c_int64, _I32, _I64, _D, ctypes.POINTER(_P)]),
    ("ba_problem_create_rcs", _S, [ctypes.POINTER(ba_options), ctypes.c_int32, ctypes.c_int64, _I32, _I32, _D, _D,
                                   ctypes.POINTER(_P)]),
    ("ba_linearize", _S, [_P, _D]),
    ("ba_form_rcs", _S, [_P, ctypes.c_double]),
    ("ba_solve_rcs", _S, [_P, ctypes.POINTER(ba_step_info)]),
    ("ba_back_substitute", _S, [_P]),
    ("ba_lm_step", _S, [_P, ctypes.POINTER(ba_step_info)]),
    ("ba_get_cameras", _S, [_P, _D]),
    ("ba_get_points", _S, [_P, _D]),
    ("ba_get_rcs", _S, [_P, _I64, _I32, _I32, _D, _D]),
    ("ba_get_step", _S, [_P, _D, _D]),
    ("ba_rcs_spmv", _S, [_P, ctypes.c_int32, _P, _P, _I64]),
    ("ba_triangulate", _S, [_P, ctypes.c_int32, _I64, _D]),
    ("ba_get_linearization", _S, [_P, _D, _D, _D]),
    ("ba_set_state", _S, [_P, _D, _D, ctypes.c_double, ctypes.c_double]),
    ("ba_get_lm_state", _S, [_P, _D, _D, _D]),
    ("ba_get_stats", _S, [_P, ctypes.POINTER(ba_stats)]),
    ("ba_get_kernel_time", _S, [_P, ctypes.c_int32, _I64, _D]),
    ("ba_reset_kernel_times", _S, [_P]),
    ("ba_set_profile", _S, [_P, ctypes.c_int32]),
    ("ba_debug_arm_wait_timeout", _S, [_P, ctypes.c_int64]),
    ("ba_kernel_name", ctypes.c_char_p, [ctypes.c_int32]),
    ("ba_problem_destroy", None, [_P]),
    ("ba_last_error", ctypes.c_char_p, []),
    ("ba_symbolic_pattern", _S, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _I32, _I64, _I32, _I32, _I64]),
    ("ba_pcg_solve_static", _S, [ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_double,
                                 ctypes.c_int32, _P, _I32, _D]),
    ("ba_precond_net_num_params", ctypes.c_int32, []),
    ("ba_precond_net_create", _S, [ctypes.POINTER(ctypes.c_float), ctypes.c_uint64, _P, ctypes.POINTER(_P)]),
    ("ba_precond_net_destroy", None, [_P]),
    ("ba_precond_net_get_params", _S, [_P, ctypes.POINTER(ctypes.c_float)]),
    ("ba_precond_net_set_params", _S, [_P, ctypes.POINTER(ctypes.c_float)]),
    ("ba_set_precond_net", _S, [_P, _P]),
    ("ba_precond_net_forward", _S, [_P, _P, ctypes.POINTER(ctypes.c_float), _D]),
    ("ba_precond_net_train_step", _S, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), ctypes.c_uint64,
                                       ctypes.c_double, _D, ctypes.POINTER(ctypes.c_float)]),
    ("ba_vbsmc_create", _S, [ctypes.POINTER(ba_options), ctypes.c_int32, _I32, ctypes.c_int64, _I32, _I32, _D, _D,
                             ctypes.POINTER(_P)]),
    ("ba_vbsmc_create_interiors", _S, [ctypes.POINTER(ba_options), ctypes.c_int32, _D, _D, _I32, ctypes.c_int64, _D,
                                       ctypes.c_int64, _I32, _I64, _D, ctypes.c_double, ctypes.POINTER(_P)]),
    ("ba_vbsmc_create_shared", _S, [ctypes.POINTER(ba_options), ctypes.c_int32, _D, ctypes.c_int32, _D, _I32,
                                    ctypes.c_int64, _D, ctypes.c_int64, _I32, _I64, _D, ctypes.c_double,
                                    ctypes.POINTER(_P)]),
    ("ba_vbi_problem_create", _S, [ctypes.POINTER(ba_options), ctypes.c_int32, _D, _D, _I32, ctypes.c_int64, _D,
                                   ctypes.c_int64, _I32, _I64, _D, ctypes.POINTER(_P)]),
    ("ba_vbi_lm_step", _S, [_P, ctypes.POINTER(ba_step_info)]),
    ("ba_vbi_get_state", _S, [_P, _D, _D, _D]),
    ("ba_vbi_set_state", _S, [_P, _D, _D, _D, ctypes.c_double, ctypes.c_double]),
    ("ba_vbi_get_lm_state", _S, [_P, _D, _D, _D]),
    ("ba_vbi_get_step", _S, [_P, _D, _D]),
    ("ba_vbi_system", _P, [_P]),
    ("ba_vbi_info", _S, [_P, _I64, _I64, _I64]),
    ("ba_vbi_problem_destroy", None, [_P]),
    ("ba_vbsmc_get_system", _S, [_P, _I32, _I32, _D, _D]),
    ("ba_vbsmc_spmv", _S, [_P, _P, _P]),
    ("ba_vbsmc_solve", _S, [_P, ctypes.c_double, ctypes.c_int32, _D, _I32, _D, _D]),
    ("ba_vbsmc_info", _S, [_P, _I64, _I64, _I64]),
    ("ba_vbsmc_destroy", None, [_P]),
    ("ba_tc_gemm", _S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_int64, _P,
                        ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _P, _P]),
]

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libba.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"libba.so not found at {LIB}; build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _err() -> str:
    m = lib().ba_last_error()
    return m.decode() if m else ""


def _check(status: int, allow=()):
    if status != BA_OK and status not in allow:
        raise BAError(status, _err())
    return status


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def ba_options_default(**kw) -> ba_options:
    o = ba_options()
    lib().ba_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"ba_options has no field {k}")
        setattr(o, k, v)
    return o


def ba_problem_create(opts: ba_options, cams, pts, obs_cam, obs_pt, obs_uv):
    cams = np.ascontiguousarray(cams, dtype=np.float64).reshape(-1, 6)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    obs_cam = np.ascontiguousarray(obs_cam, dtype=np.int32)
    obs_pt = np.ascontiguousarray(obs_pt, dtype=np.int64)
    obs_uv = np.ascontiguousarray(obs_uv, dtype=np.float64).reshape(-1, 2)
    if not (len(obs_cam) == len(obs_pt) == len(obs_uv)):
        raise ValueError("observation arrays differ in length")
    h = _P()
    _check(lib().ba_problem_create(ctypes.byref(opts), len(cams), _dp(cams), len(pts), _dp(pts), len(obs_cam),
                                   obs_cam.ctypes.data_as(_I32), obs_pt.ctypes.data_as(_I64), _dp(obs_uv),
                                   ctypes.byref(h)))
    return h


def ba_linearize(h) -> float:
    c = ctypes.c_double()
    _check(lib().ba_linearize(h, ctypes.byref(c)))
    return c.value


def ba_form_rcs(h, lam: float) -> None:
    _check(lib().ba_form_rcs(h, float(lam)))


def ba_solve_rcs(h):
    """Returns (info dict, converged)."""
    info = ba_step_info()
    s = _check(lib().ba_solve_rcs(h, ctypes.byref(info)), allow=(BA_ERR_NO_CONVERGENCE,))
    return info.as_dict(), s == BA_OK


def ba_back_substitute(h) -> None:
    _check(lib().ba_back_substitute(h))


def ba_lm_step(h) -> dict:
    info = ba_step_info()
    _check(lib().ba_lm_step(h, ctypes.byref(info)))
    return info.as_dict()


def ba_get_stats(h) -> dict:
    s = ba_stats()
    _check(lib().ba_get_stats(h, ctypes.byref(s)))
    out = {f: getattr(s, f) for f, _ in s._fields_}
    out["pcg_phase_us"] = list(out["pcg_phase_us"])
    out["rcs_phase_us"] = list(out["rcs_phase_us"])
    return out


def ba_get_cameras(h, n, out=None):
    out = np.empty((n, 6)) if out is None else out
    _check(lib().ba_get_cameras(h, _dp(out)))
    return out


def ba_get_points(h, P, out=None):
    out = np.empty((P, 3)) if out is None else out
    _check(lib().ba_get_points(h, _dp(out)))
    return out


def ba_get_rcs(h, n):
    nnzb = ctypes.c_int64()
    _check(lib().ba_get_rcs(h, ctypes.byref(nnzb), None, None, None, None))
    row_ptr = np.empty(n + 1, np.int32)
    col = np.empty(nnzb.value, np.int32)
    val = np.empty((nnzb.value, 6, 6))
    b = np.empty((n, 6))
    _check(lib().ba_get_rcs(h, ctypes.byref(nnzb), row_ptr.ctypes.data_as(_I32), col.ctypes.data_as(_I32),
                            _dp(val), _dp(b)))
    return row_ptr, col, val, b


def ba_rcs_spmv(h, fmt, x_ptr, y_ptr):
    """y = S x with the RCS in format fmt (BA_FMT_*); x_ptr, y_ptr are device
    addresses (ints) of 6n values in the problem's precision; queued on the
    problem's stream.  Returns the format's array bytes."""
    nb = ctypes.c_int64()
    _check(lib().ba_rcs_spmv(h, int(fmt), ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), ctypes.byref(nb)))
    return nb.value


def ba_triangulate(h, gn_iters=3):
    """Re-triangulates every point from the current cameras; returns
    (points left unchanged, cost at the new state)."""
    nf = ctypes.c_int64()
    cost = ctypes.c_double()
    _check(lib().ba_triangulate(h, int(gn_iters), ctypes.byref(nf), ctypes.byref(cost)))
    return nf.value, cost.value


def ba_get_step(h, n, P):
    dxc = np.empty((n, 6))
    dxp = np.empty((P, 3))
    _check(lib().ba_get_step(h, _dp(dxc), _dp(dxp)))
    return dxc, dxp


def ba_get_linearization(h, m):
    e = np.empty((m, 2))
    Jc = np.empty((m, 2, 6))
    Jp = np.empty((m, 2, 3))
    _check(lib().ba_get_linearization(h, _dp(e), _dp(Jc), _dp(Jp)))
    return e, Jc, Jp


def ba_set_state(h, cams, pts, lam, nu=2.0):
    c = None if cams is None else np.ascontiguousarray(cams, dtype=np.float64)
    p = None if pts is None else np.ascontiguousarray(pts, dtype=np.float64)
    _check(lib().ba_set_state(h, _dp(c), _dp(p), float(lam), float(nu)))


def ba_get_lm_state(h):
    lam, nu, cost = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().ba_get_lm_state(h, ctypes.byref(lam), ctypes.byref(nu), ctypes.byref(cost)))
    return lam.value, nu.value, cost.value


def ba_kernel_names():
    out = []
    k = 0
    while True:
        n = lib().ba_kernel_name(k)
        if n is None:
            return out
        out.append(n.decode())
        k += 1


def ba_get_kernel_time(h, k: int):
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(lib().ba_get_kernel_time(h, int(k), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def ba_reset_kernel_times(h):
    _check(lib().ba_reset_kernel_times(h))


def ba_set_profile(h, level):
    _check(lib().ba_set_profile(h, int(level)))


def ba_problem_destroy(h):
    if h:
        lib().ba_problem_destroy(h)


def ba_symbolic_pattern(n_cams, n_pts, obs_cam, obs_pt):
    obs_cam = np.ascontiguousarray(obs_cam, dtype=np.int32)
    obs_pt = np.ascontiguousarray(obs_pt, dtype=np.int64)
    nnzb = ctypes.c_int64()
    row_ptr = np.empty(n_cams + 1, np.int32)
    _check(lib().ba_symbolic_pattern(n_cams, n_pts, len(obs_cam), obs_cam.ctypes.data_as(_I32),
                                     obs_pt.ctypes.data_as(_I64), row_ptr.ctypes.data_as(_I32), None,
                                     ctypes.byref(nnzb)))
    col = np.empty(nnzb.value, np.int32)
    _check(lib().ba_symbolic_pattern(n_cams, n_pts, len(obs_cam), obs_cam.ctypes.data_as(_I32),
                                     obs_pt.ctypes.data_as(_I64), row_ptr.ctypes.data_as(_I32),
                                     col.ctypes.data_as(_I32), ctypes.byref(nnzb)))
    return row_ptr, col


def ba_problem_create_rcs(opts, row_ptr, col, val, b):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64).reshape(-1, 36)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1, 6)
    n = len(row_ptr) - 1
    if len(b) != n or len(val) != len(col):
        raise ValueError("inconsistent BSMC arrays")
    h = _P()
    _check(lib().ba_problem_create_rcs(ctypes.byref(opts), n, len(col), row_ptr.ctypes.data_as(_I32),
                                       col.ctypes.data_as(_I32), _dp(val), _dp(b), ctypes.byref(h)))
    return h


class Problem:
    """A libba problem handle with numpy in / out."""

    def __init__(self, cams, pts, obs_cam, obs_pt, obs_uv, stream="current", **opts):
        if stream == "current":
            stream = _default_stream()
        self.opts = ba_options_default(cuda_stream=stream, **opts)
        self.n = len(cams)
        self.P = len(pts)
        self.m = len(obs_cam)
        self.h = ba_problem_create(self.opts, cams, pts, obs_cam, obs_pt, obs_uv)

    @classmethod
    def from_rcs(cls, row_ptr, col, val, b, stream="current", **opts):
        """A problem holding only a reduced camera system (see ba_problem_create_rcs)."""
        self = cls.__new__(cls)
        if stream == "current":
            stream = _default_stream()
        self.opts = ba_options_default(cuda_stream=stream, **opts)
        self.n = len(row_ptr) - 1
        self.P = 0
        self.m = 0
        self.h = ba_problem_create_rcs(self.opts, row_ptr, col, val, b)
        return self

    def close(self):
        if getattr(self, "h", None):
            ba_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def linearize(self):
        return ba_linearize(self.h)

    def form_rcs(self, lam):
        ba_form_rcs(self.h, lam)

    def solve_rcs(self):
        return ba_solve_rcs(self.h)

    def back_substitute(self):
        ba_back_substitute(self.h)

    def lm_step(self):
        return ba_lm_step(self.h)

    def cameras(self):
        return ba_get_cameras(self.h, self.n)

    def points(self):
        return ba_get_points(self.h, self.P)

    def rcs(self):
        return ba_get_rcs(self.h, self.n)

    def triangulate(self, gn_iters=3):
        """Points re-triangulated from the current cameras (linear, then
        Gauss-Newton); returns (points left unchanged, new cost)."""
        return ba_triangulate(self.h, gn_iters)

    def rcs_spmv(self, fmt, x, y):
        """y = S x (torch CUDA tensors of 6n values, float64 for FP64
        problems, float32 for FP32) with the RCS in format fmt; returns the
        format's array bytes."""
        return ba_rcs_spmv(self.h, fmt, x.data_ptr(), y.data_ptr())

    def step(self):
        return ba_get_step(self.h, self.n, self.P)

    def linearization(self):
        return ba_get_linearization(self.h, self.m)

    def set_state(self, cams, pts, lam, nu=2.0):
        ba_set_state(self.h, cams, pts, lam, nu)

    def lm_state(self):
        return ba_get_lm_state(self.h)

    def stats(self):
        return ba_get_stats(self.h)

    def kernel_times(self):
        return {name: ba_get_kernel_time(self.h, k) for k, name in enumerate(ba_kernel_names())}

    def reset_kernel_times(self):
        ba_reset_kernel_times(self.h)

    def set_profile(self, level):
        """0: no kernel timing, 1: kernel times, 2: also the PCG and RCS phase timers."""
        ba_set_profile(self.h, level)

    def arm_wait_timeout(self, limit_cycles):
        """Test hook: the next PCG launch misses one arrival at its first
        all-reduce and gives up after limit_cycles SM cycles (include/ba.h)."""
        _check(lib().ba_debug_arm_wait_timeout(self.h, int(limit_cycles)))


def ba_pcg_solve_static(n, nnzb, row_ptr, col, val, b, x, rel_tol, max_iters=0, stream=None):
    """Allocation-free FP32 PCG on a BSMC system held in caller-owned device
    buffers (addresses as ints, e.g. torch ``data_ptr()``); see include/ba.h.
    Returns (status, iterations, final relative residual); raises BAError on
    every status except BA_OK and BA_ERR_NO_CONVERGENCE."""
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    s = _check(lib().ba_pcg_solve_static(int(n), int(nnzb), row_ptr, col, val, b, x, float(rel_tol),
                                         int(max_iters), stream, ctypes.byref(it), ctypes.byref(rel)),
               allow=(BA_ERR_NO_CONVERGENCE,))
    return s, it.value, rel.value


def ba_tc_gemm(M, N, K, A, a_rs, a_cs, B, b_rs, b_cs, C, c_rs, c_cs, accumulate=False, err=None, stream=None):
    """C = A @ B (or C += A @ B) on the tensor cores; addresses are device
    pointers (ints), strides in elements; see include/ba.h."""
    _check(lib().ba_tc_gemm(int(M), int(N), int(K), A, a_rs, a_cs, B, b_rs, b_cs, C, c_rs, c_cs,
                            1 if accumulate else 0, err, stream))


_F = ctypes.POINTER(ctypes.c_float)


def _fp(a):
    return a.ctypes.data_as(_F) if a is not None else None


class PrecondNet:
    """The learned block-Jacobi correction (see include/ba.h)."""

    def __init__(self, params=None, seed=0, stream="current"):
        if stream == "current":
            stream = _default_stream()
        self.nparams = lib().ba_precond_net_num_params()
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        if p is not None and p.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters")
        h = _P()
        _check(lib().ba_precond_net_create(_fp(p), int(seed), stream, ctypes.byref(h)))
        self.h = h

    @classmethod
    def load(cls, path=None, stream="current"):
        """A net with the weights stored by the training module (default: the
        packaged weights trained on aerial-shaped systems)."""
        path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                    "precond_net_aerial.npz")
        with np.load(path, allow_pickle=False) as d:
            return cls(params=d["params"], stream=stream)

    def close(self):
        if getattr(self, "h", None):
            lib().ba_precond_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.nparams, np.float32)
        _check(lib().ba_precond_net_get_params(self.h, _fp(out)))
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().ba_precond_net_set_params(self.h, _fp(p)))

    def forward(self, problem):
        o = np.empty((problem.n, 21), np.float32)
        minv = np.empty((problem.n, 6, 6))
        _check(lib().ba_precond_net_forward(self.h, problem.h, _fp(o), _dp(minv)))
        return o, minv

    def train_step(self, problem, kp=4, probes=None, seed=0, lr=0.0, want_grads=False):
        pr = None if probes is None else np.ascontiguousarray(probes, dtype=np.float32)
        loss = ctypes.c_double()
        g = np.empty(self.nparams, np.float32) if want_grads else None
        _check(lib().ba_precond_net_train_step(self.h, problem.h, int(kp), _fp(pr), int(seed), float(lr),
                                               ctypes.byref(loss), _fp(g)))
        return (loss.value, g) if want_grads else loss.value


def ba_set_precond_net(problem, net):
    _check(lib().ba_set_precond_net(problem.h, None if net is None else net.h))


def unpack_params(p):
    """Packed parameters -> dict of the oracle's layout (W1, b1, W2, b2, Wo, bo)."""
    p = np.asarray(p, dtype=np.float64)
    out, off = {}, 0
    for name, shape in (("W1", (48, 64)), ("b1", (64,)), ("W2", (128, 64)), ("b2", (64,)), ("Wo", (64, 21)),
                        ("bo", (21,))):
        cnt = int(np.prod(shape))
        out[name] = p[off:off + cnt].reshape(shape)
        off += cnt
    return out


def pack_params(d):
    return np.concatenate([np.asarray(d[k], dtype=np.float32).reshape(-1) for k in ("W1", "b1", "W2", "b2", "Wo",
                                                                                      "bo")])


BA_VB_CMAX = 16


class VBSMC:
    """A variable-size BSMC system (include/ba_vbsmc.h): cameras with c_i
    unknowns each (6 exterior, 11 with five interiors), the upper blocks
    packed row by row (block (i, j) row-major c_i x c_j), b of sum c_i."""

    def __init__(self, cdim, row_ptr, col, val, b, stream="current", **opts):
        if stream == "current":
            stream = _default_stream()
        self.opts = ba_options_default(cuda_stream=stream, **opts)
        self.cdim = np.ascontiguousarray(cdim, dtype=np.int32)
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64).reshape(-1)
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        n = len(self.cdim)
        if len(row_ptr) != n + 1:
            raise BAError(BA_ERR_INVALID_ARG, "row_ptr must have n + 1 entries")
        if len(b) != int(self.cdim.sum()):
            raise BAError(BA_ERR_INVALID_ARG, "b must have sum(cdim) entries")
        if len(row_ptr) and row_ptr[-1] == len(col) and len(col):
            rows = np.repeat(np.arange(n), np.diff(row_ptr))
            if rows.size == len(col) and np.all((col >= 0) & (col < n)):
                need = int((self.cdim[rows].astype(np.int64) * self.cdim[col]).sum())
                if len(val) != need:
                    raise BAError(BA_ERR_INVALID_ARG, f"val must have {need} entries")
        h = _P()
        _check(lib().ba_vbsmc_create(ctypes.byref(self.opts), n, self.cdim.ctypes.data_as(_I32), len(col),
                                     row_ptr.ctypes.data_as(_I32), col.ctypes.data_as(_I32), _dp(val), _dp(b),
                                     ctypes.byref(h)))
        self.h = h
        self.n = n

    @classmethod
    def from_scene(cls, cams, intr, cdim, pts, obs_cam, obs_pt, obs_uv, lam, stream="current", **opts):
        """The RCS of a scene whose cameras carry interiors [f, cx, cy, k1, k2]
        (c_i = 6: held fixed, 11: estimated), formed on the device at damping
        lam (ba_vbsmc_create_interiors)."""
        if stream == "current":
            stream = _default_stream()
        self = cls.__new__(cls)
        self.opts = ba_options_default(cuda_stream=stream, **opts)
        n = len(cams)
        self.cdim = np.ascontiguousarray(cdim, dtype=np.int32)
        cams = _f64(cams, (n, 6))
        intr = _f64(intr, (n, 5))
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        P = len(pts)
        pts = _f64(pts, (P, 3))
        obs_cam = np.ascontiguousarray(obs_cam, dtype=np.int32)
        obs_pt = np.ascontiguousarray(obs_pt, dtype=np.int64)
        m = len(obs_cam)
        obs_uv = _f64(obs_uv, (m, 2))
        if len(self.cdim) != n or len(obs_pt) != m:
            raise BAError(BA_ERR_INVALID_ARG, "array lengths disagree")
        h = _P()
        _check(lib().ba_vbsmc_create_interiors(ctypes.byref(self.opts), n, _dp(cams), _dp(intr),
                                               self.cdim.ctypes.data_as(_I32), P, _dp(pts), m,
                                               obs_cam.ctypes.data_as(_I32), obs_pt.ctypes.data_as(_I64),
                                               _dp(obs_uv), float(lam), ctypes.byref(h)))
        self.h = h
        self.n = n
        return self

    @classmethod
    def from_shared(cls, cams, intr_phys, phys, pts, obs_cam, obs_pt, obs_uv, lam, stream="current", **opts):
        """The RCS when the images of each physical camera share its interiors
        [f, cx, cy, k1, k2]: n image blocks of six unknowns, then one block of
        five per physical camera (ba_vbsmc_create_shared)."""
        if stream == "current":
            stream = _default_stream()
        self = cls.__new__(cls)
        self.opts = ba_options_default(cuda_stream=stream, **opts)
        n = len(cams)
        K = len(intr_phys)
        cams = _f64(cams, (n, 6))
        intr_phys = _f64(intr_phys, (K, 5))
        phys = np.ascontiguousarray(phys, dtype=np.int32)
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        P = len(pts)
        pts = _f64(pts, (P, 3))
        obs_cam = np.ascontiguousarray(obs_cam, dtype=np.int32)
        obs_pt = np.ascontiguousarray(obs_pt, dtype=np.int64)
        m = len(obs_cam)
        obs_uv = _f64(obs_uv, (m, 2))
        if len(phys) != n or len(obs_pt) != m:
            raise BAError(BA_ERR_INVALID_ARG, "array lengths disagree")
        self.cdim = np.array([6] * n + [5] * K, dtype=np.int32)
        h = _P()
        _check(lib().ba_vbsmc_create_shared(ctypes.byref(self.opts), n, _dp(cams), K, _dp(intr_phys),
                                            phys.ctypes.data_as(_I32), P, _dp(pts), m, obs_cam.ctypes.data_as(_I32),
                                            obs_pt.ctypes.data_as(_I64), _dp(obs_uv), float(lam), ctypes.byref(h)))
        self.h = h
        self.n = n + K
        return self

    @classmethod
    def borrowed(cls, h, cdim):
        """A view of a system owned by another object (not destroyed here)."""
        self = cls.__new__(cls)
        self.h = h
        self.cdim = np.ascontiguousarray(cdim, dtype=np.int32)
        self.n = len(self.cdim)
        self._borrowed = True
        return self

    def system(self):
        """(row_ptr, col, packed block values, b) as host arrays (float64)."""
        N = ctypes.c_int64()
        nb = ctypes.c_int64()
        _check(lib().ba_vbsmc_info(self.h, ctypes.byref(N), None, ctypes.byref(nb)))
        row_ptr = np.empty(self.n + 1, dtype=np.int32)
        col = np.empty(nb.value, dtype=np.int32)
        _check(lib().ba_vbsmc_get_system(self.h, row_ptr.ctypes.data_as(_I32), col.ctypes.data_as(_I32), None, None))
        rows = np.repeat(np.arange(self.n), np.diff(row_ptr))
        nval = int((self.cdim[rows].astype(np.int64) * self.cdim[col]).sum())
        val = np.empty(nval)
        b = np.empty(N.value)
        _check(lib().ba_vbsmc_get_system(self.h, None, None, _dp(val), _dp(b)))
        return row_ptr, col, val, b

    def spmv(self, x, y):
        """y = S x for torch device tensors of sum c_i values in the system's
        precision; queued on the system's stream."""
        _check(lib().ba_vbsmc_spmv(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())))

    def solve(self, tol, max_iters=0, allow=()):
        """Block-Jacobi PCG from 0: returns (x, iterations, ||r|| / ||r0||,
        device ms, status)."""
        N, _ = self.info()
        x = np.empty(N)
        it = ctypes.c_int32()
        rel = ctypes.c_double()
        ms = ctypes.c_double()
        st = _check(lib().ba_vbsmc_solve(self.h, float(tol), int(max_iters), _dp(x), ctypes.byref(it),
                                         ctypes.byref(rel), ctypes.byref(ms)), allow)
        return x, it.value, rel.value, ms.value, st

    def info(self):
        """(unknowns, bytes of the stored format)."""
        N = ctypes.c_int64()
        nb = ctypes.c_int64()
        _check(lib().ba_vbsmc_info(self.h, ctypes.byref(N), ctypes.byref(nb), None))
        return N.value, nb.value

    def close(self):
        if getattr(self, "h", None):
            if not getattr(self, "_borrowed", False):
                lib().ba_vbsmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VBIProblem:
    """An LM problem whose cameras carry interiors [f, cx, cy, k1, k2]
    (cdim 11: estimated, 6: held fixed), on the device (include/ba_vbsmc.h,
    ba_vbi_*).  States are in the caller's order."""

    def __init__(self, cams, intr, cdim, pts, obs_cam, obs_pt, obs_uv, stream="current", **opts):
        if stream == "current":
            stream = _default_stream()
        self.opts = ba_options_default(cuda_stream=stream, **opts)
        n = len(cams)
        self.cdim = np.ascontiguousarray(cdim, dtype=np.int32)
        cams = _f64(cams, (n, 6))
        intr = _f64(intr, (n, 5))
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        P = len(pts)
        pts = _f64(pts, (P, 3))
        obs_cam = np.ascontiguousarray(obs_cam, dtype=np.int32)
        obs_pt = np.ascontiguousarray(obs_pt, dtype=np.int64)
        m = len(obs_cam)
        obs_uv = _f64(obs_uv, (m, 2))
        if len(self.cdim) != n or len(obs_pt) != m:
            raise BAError(BA_ERR_INVALID_ARG, "array lengths disagree")
        h = _P()
        _check(lib().ba_vbi_problem_create(ctypes.byref(self.opts), n, _dp(cams), _dp(intr),
                                           self.cdim.ctypes.data_as(_I32), P, _dp(pts), m,
                                           obs_cam.ctypes.data_as(_I32), obs_pt.ctypes.data_as(_I64), _dp(obs_uv),
                                           ctypes.byref(h)))
        self.h, self.n, self.P = h, n, P

    def lm_step(self):
        info = ba_step_info()
        _check(lib().ba_vbi_lm_step(self.h, ctypes.byref(info)))
        return info.as_dict()

    def state(self):
        """(cams n x 6, intr n x 5, pts P x 3)."""
        c = np.empty((self.n, 6))
        k = np.empty((self.n, 5))
        x = np.empty((self.P, 3))
        _check(lib().ba_vbi_get_state(self.h, _dp(c), _dp(k), _dp(x)))
        return c, k, x

    def set_state(self, cams, intr, pts, lam, nu):
        _check(lib().ba_vbi_set_state(self.h, _dp(_f64(cams, (self.n, 6))), _dp(_f64(intr, (self.n, 5))),
                                      _dp(_f64(pts, (self.P, 3))), float(lam), float(nu)))

    def lm_state(self):
        lam, nu, F = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().ba_vbi_get_lm_state(self.h, ctypes.byref(lam), ctypes.byref(nu), ctypes.byref(F)))
        return lam.value, nu.value, F.value

    def step(self):
        """(dx_c as one vector of sum c_i values, dx_p P x 3) of the last step."""
        dxc = np.empty(int(self.cdim.sum()))
        dxp = np.empty((self.P, 3))
        _check(lib().ba_vbi_get_step(self.h, _dp(dxc), _dp(dxp)))
        return dxc, dxp

    def system(self):
        """The variable-size RCS of the last formation, as a borrowed VBSMC."""
        return VBSMC.borrowed(lib().ba_vbi_system(self.h), self.cdim)

    def info(self):
        N, nb, by = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ba_vbi_info(self.h, ctypes.byref(N), ctypes.byref(nb), ctypes.byref(by)))
        return {"unknowns": N.value, "blocks": nb.value, "device_bytes": by.value}

    def close(self):
        if getattr(self, "h", None):
            lib().ba_vbi_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
