"""Python binding of libtlqr (include/tlqr.h): argument marshalling only.

Every function keeps the C name.  Arrays are float64 and C-contiguous:
numpy arrays are passed as host memory (TLQR_MEM_HOST), CUDA torch tensors as
device memory (TLQR_MEM_DEVICE).  All arithmetic happens in the CUDA library;
if it cannot be loaded the import-time call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtlqr.so")

TLQR_OK = 0
TLQR_ERR_ARG = 1
TLQR_ERR_TIMEOUT = 7
TLQR_ERR_NO_CONVERGENCE = 8
TLQR_MEM_DEVICE, TLQR_MEM_HOST = 0, 1
TLQR_PREC_FP64, TLQR_PREC_MIXED = 0, 1
TLQR_OP_ROOT, TLQR_OP_RAKE, TLQR_OP_COMPRESS = 0, 1, 2
TLQR_MAX_DIM = 64
TLQR_BATCHED_GENERIC = 0x100
STATUS_NAMES = {0: "TLQR_OK", 1: "TLQR_ERR_ARG", 2: "TLQR_ERR_TOPOLOGY", 3: "TLQR_ERR_NOT_PD",
                4: "TLQR_ERR_SINGULAR", 5: "TLQR_ERR_NONFINITE", 6: "TLQR_ERR_OOM",
                7: "TLQR_ERR_TIMEOUT", 8: "TLQR_ERR_NO_CONVERGENCE", 9: "TLQR_ERR_CUDA",
                10: "TLQR_ERR_STATE"}

_i32 = ctypes.c_int32
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p


class TLQRError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({tlqr_status_string(code)})")


class tlqr_options(ctypes.Structure):
    _fields_ = [("n", _i32), ("m", _i32), ("precision", _i32), ("has_M", _i32), ("has_delta", _i32),
                ("max_refine", _i32), ("refine_tol", ctypes.c_double), ("use_graphs", _i32),
                ("generic_kernels", _i32), ("async_ops", _i32), ("spin_limit", _i32), ("test_withhold", _i32),
                ("tail_ops", _i32), ("async_solve", _i32), ("residual", _i32),
                ("fp64_resolve", _i32), ("pdl", _i32)]


class tlqr_problem(ctypes.Structure):
    _fields_ = [("mem", _i32), ("Q", _dp), ("q", _dp), ("M", _dp), ("R", _dp), ("r", _dp),
                ("A", _dp), ("B", _dp), ("c", _dp), ("Delta", _dp)]


class tlqr_solution(ctypes.Structure):
    _fields_ = [("mem", _i32), ("x", _dp), ("u", _dp), ("y", _dp), ("P", _dp), ("K", _dp)]


class tlqr_ipm_options(ctypes.Structure):
    _fields_ = [("max_iter", _i32), ("mu0", ctypes.c_double), ("sigma", ctypes.c_double), ("tau", ctypes.c_double),
                ("tol", ctypes.c_double), ("no_fp64_fallback", _i32)]


class tlqr_ipm_info(ctypes.Structure):
    _fields_ = [("iterations", _i32), ("mu", ctypes.c_double), ("mean_gap", ctypes.c_double),
                ("last_alpha", ctypes.c_double), ("last_eta", ctypes.c_double), ("fp64_solves", _i32)]


class tlqr_autotune_entry(ctypes.Structure):
    _fields_ = [("async_ops", _i32), ("async_solve", _i32), ("tail_ops", _i32), ("residual", _i32),
                ("status", _i32), ("ms", ctypes.c_double)]


class tlqr_plan_stats_t(ctypes.Structure):
    _fields_ = [(k, _i32) for k in ("N", "root", "rounds", "n_rake", "n_compress", "n_combine",
                                    "n_absorb", "levels", "height", "max_degree", "n_trees")]


class tlqr_kernel_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("units", ctypes.c_int64), ("timed", ctypes.c_int64),
                ("ms", ctypes.c_double)]


class tlqr_info(ctypes.Structure):
    _fields_ = [("refine_steps", _i32), ("eta", ctypes.c_double), ("abs_residual", ctypes.c_double),
                ("fp64_resolves", _i32)]


_lib = None
EXPORTS = ["tlqr_plan_create", "tlqr_plan_create_forest", "tlqr_plan_destroy", "tlqr_plan_stats", "tlqr_plan_schedule",
           "tlqr_factor_create", "tlqr_factor_destroy", "tlqr_factor", "tlqr_solve_rhs", "tlqr_solve",
           "tlqr_get_PK", "tlqr_kkt_residual", "tlqr_last_info", "tlqr_status_string",
           "tlqr_batched_tau", "tlqr_batched_compose", "tlqr_batched_condense", "tlqr_batched_expand",
           "tlqr_batched_local_factor", "tlqr_batched_compose_T",
           "tlqr_lift_node_controls", "tlqr_project_lifted", "tlqr_profile_mask", "tlqr_profile_read",
           "tlqr_kkt_residual_noalloc", "tlqr_profile_launches", "tlqr_tree_residuals",
           "tlqr_factor_workspace_bytes", "tlqr_factor_bytes", "tlqr_async_schedule", "tlqr_solve_adjoint",
           "tlqr_lift_node_controls_device", "tlqr_project_lifted_device", "tlqr_factor_dims", "tlqr_ipm_box",
           "tlqr_pipe_peak", "tlqr_solve_rhs_panel",
           "tlqr_factor_options", "tlqr_autotune", "tlqr_update_solve"]

KERNEL_KINDS = ["condense", "rake", "absorb", "compress", "expand", "local_factor", "compose_T", "aff_init",
                "aff_rake", "aff_absorb", "aff_compress", "aff_expand", "local_solve", "state_compress",
                "state_expand", "recover", "residual", "export", "aff_tail", "state_tail", "factor_tail"]


def lib():
    """Load libtlqr.so (building it first if it is missing or older than its sources)."""
    global _lib
    if _lib is None:
        from . import build as _build
        try:
            _build.build()
        except (OSError, FileNotFoundError) as e:   # no nvcc: use what is there, or fail below
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"libtlqr.so is missing and cannot be built: {e}") from e
        L = ctypes.CDLL(_LIB_PATH)
        L.tlqr_status_string.restype = ctypes.c_char_p
        L.tlqr_status_string.argtypes = [ctypes.c_int]
        L.tlqr_plan_create.argtypes = [_ip, _i32, ctypes.POINTER(_vp)]
        L.tlqr_plan_create_forest.argtypes = [_ip, _i32, ctypes.POINTER(_vp)]
        L.tlqr_plan_destroy.argtypes = [_vp]
        L.tlqr_plan_destroy.restype = None
        L.tlqr_plan_stats.argtypes = [_vp, ctypes.POINTER(tlqr_plan_stats_t)]
        L.tlqr_plan_schedule.argtypes = [_vp, _ip, _ip]
        L.tlqr_factor_create.argtypes = [_vp, ctypes.POINTER(tlqr_options), ctypes.POINTER(_vp)]
        L.tlqr_factor_destroy.argtypes = [_vp]
        L.tlqr_factor_destroy.restype = None
        L.tlqr_factor.argtypes = [_vp, ctypes.POINTER(tlqr_problem), _vp]
        L.tlqr_solve_rhs.argtypes = [_vp, _i32, _dp, _dp, _dp, _dp, _dp, _dp, _vp]
        L.tlqr_solve.argtypes = [_vp, ctypes.POINTER(tlqr_problem), ctypes.POINTER(tlqr_solution), _vp]
        L.tlqr_get_PK.argtypes = [_vp, _i32, _dp, _dp, _vp]
        L.tlqr_kkt_residual.argtypes = [_vp, ctypes.POINTER(tlqr_problem), _i32, _dp, _dp, _dp, _dp, _vp]
        L.tlqr_last_info.argtypes = [_vp, ctypes.POINTER(tlqr_info)]
        L.tlqr_batched_tau.argtypes = [_i32, _i32] + [_dp] * 5 + [_i32, _vp]
        L.tlqr_batched_compose.argtypes = [_i32, _i32] + [_dp] * 11 + [_i32, _vp]
        L.tlqr_batched_condense.argtypes = [_i32, _i32, _i32] + [_dp] * 8 + [_i32, _vp]
        L.tlqr_lift_node_controls_device.argtypes = ([_ip, _i32, _i32, _i32] + [_dp] * 9 + [_ip, _ip] + [_dp] * 9
                                                     + [_ip, _vp])
        L.tlqr_project_lifted_device.argtypes = [_i32, _i32, _i32, _ip] + [_dp] * 6 + [_vp]
        L.tlqr_factor_dims.argtypes = [_vp, _ip]
        L.tlqr_autotune.argtypes = [_vp, ctypes.POINTER(tlqr_options), ctypes.POINTER(tlqr_problem), _i32,
                                    ctypes.POINTER(tlqr_options), ctypes.POINTER(tlqr_autotune_entry), _i32, _ip,
                                    _vp]
        L.tlqr_factor_options.argtypes = [_vp, ctypes.POINTER(tlqr_options)]
        L.tlqr_solve_rhs_panel.argtypes = [_vp, _i32] + [_dp] * 6 + [_vp]
        L.tlqr_pipe_peak.argtypes = [_i32, _dp, _vp]
        L.tlqr_ipm_box.argtypes = ([_vp, _vp, ctypes.POINTER(tlqr_problem), _dp, _dp, ctypes.POINTER(tlqr_ipm_options)]
                                   + [_dp] * 5 + [ctypes.POINTER(tlqr_ipm_info), _vp])
        L.tlqr_solve_adjoint.argtypes = [_vp, _i32] + [_dp] * 6 + [_vp]
        L.tlqr_update_solve.argtypes = [_vp, _i32] + [_dp] * 5 + [ctypes.POINTER(tlqr_solution), _vp]
        L.tlqr_async_schedule.argtypes = [_vp, _i32, _i32, _i32] + [_ip] * 7
        L.tlqr_batched_expand.argtypes = [_i32, _i32] + [_dp] * 5 + [_i32, _vp]
        L.tlqr_batched_local_factor.argtypes = [_i32, _i32, _i32] + [_dp] * 8 + [_i32, _vp]
        L.tlqr_batched_compose_T.argtypes = [_i32, _i32] + [_dp] * 3 + [_i32, _vp]
        L.tlqr_lift_node_controls.argtypes = [_ip, _i32, _i32, _i32] + [_dp] * 9 + [_ip, _ip] + [_dp] * 9 + [_ip]
        L.tlqr_project_lifted.argtypes = [_i32, _i32, _i32, _ip] + [_dp] * 6
        L.tlqr_profile_mask.argtypes = [_vp, ctypes.c_uint32]
        L.tlqr_profile_read.argtypes = [_vp, ctypes.POINTER(tlqr_kernel_profile)]
        L.tlqr_factor_workspace_bytes.argtypes = [_vp, ctypes.POINTER(tlqr_options), ctypes.POINTER(ctypes.c_size_t)]
        L.tlqr_factor_bytes.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
        L.tlqr_tree_residuals.argtypes = [_vp, _dp, _dp, _i32]
        L.tlqr_profile_launches.argtypes = [_vp, _ip, ctypes.POINTER(ctypes.c_int64), _dp, _i32, _ip]
        L.tlqr_kkt_residual_noalloc.argtypes = [_vp, _i32, _i32, ctypes.POINTER(tlqr_problem), _dp, _dp, _dp, _dp, _vp]
        _lib = L
    return _lib


def tlqr_status_string(code: int) -> str:
    return lib().tlqr_status_string(int(code)).decode()


def _check(rc: int, where: str):
    if rc != TLQR_OK:
        raise TLQRError(rc, where)


# ------------------------------------------------------------------ pointers

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _mem_of(a) -> int:
    if a is None:
        return -1
    if _is_torch(a):
        return TLQR_MEM_DEVICE if a.is_cuda else TLQR_MEM_HOST
    return TLQR_MEM_HOST


def _ptr(a):
    """float64 contiguous array -> double*; None -> NULL."""
    if a is None:
        return _dp()
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be float64 and contiguous")
        return ctypes.cast(ctypes.c_void_p(a.data_ptr()), _dp)
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("arrays must be float64 and C-contiguous")
    return a.ctypes.data_as(_dp)


def _iptr(a):
    if a is None:
        return _ip()
    if a.dtype != np.int32 or not a.flags.c_contiguous:
        raise TypeError("index arrays must be int32 and C-contiguous")
    return a.ctypes.data_as(_ip)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _mem_all(arrays) -> int:
    mems = {_mem_of(a) for a in arrays if a is not None}
    if len(mems) != 1:
        raise ValueError("all arrays of one call must be host arrays or all CUDA tensors")
    return mems.pop()


# ------------------------------------------------------------------ plan

def tlqr_plan_create(parent) -> ctypes.c_void_p:
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    h = _vp()
    _check(lib().tlqr_plan_create(_iptr(parent), len(parent), ctypes.byref(h)), "tlqr_plan_create")
    return h


def tlqr_plan_create_forest(parent) -> ctypes.c_void_p:
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    h = _vp()
    _check(lib().tlqr_plan_create_forest(_iptr(parent), len(parent), ctypes.byref(h)), "tlqr_plan_create_forest")
    return h


def tlqr_plan_destroy(plan) -> None:
    lib().tlqr_plan_destroy(plan)


def tlqr_plan_stats(plan) -> dict:
    s = tlqr_plan_stats_t()
    _check(lib().tlqr_plan_stats(plan, ctypes.byref(s)), "tlqr_plan_stats")
    return {k: getattr(s, k) for k, _ in tlqr_plan_stats_t._fields_}


def tlqr_plan_schedule(plan, N: int):
    rnd = np.zeros(N, dtype=np.int32)
    op = np.zeros(N, dtype=np.int32)
    _check(lib().tlqr_plan_schedule(plan, _iptr(rnd), _iptr(op)), "tlqr_plan_schedule")
    return rnd, op


# ------------------------------------------------------------------ factor / solve

def make_options(n, m, precision=TLQR_PREC_FP64, has_M=False, has_delta=False, max_refine=10,
                 refine_tol=1e-8, use_graphs=True, generic_kernels=False, async_ops=0, spin_limit=0,
                 test_withhold=False, tail_ops=0, async_solve=0, residual=0, fp64_resolve=0,
                 pdl=0) -> tlqr_options:
    o = tlqr_options()
    o.tail_ops, o.async_solve, o.residual = int(tail_ops), int(async_solve), int(residual)
    o.fp64_resolve, o.pdl = int(fp64_resolve), int(pdl)
    o.generic_kernels = int(bool(generic_kernels))
    o.async_ops, o.spin_limit, o.test_withhold = int(async_ops), int(spin_limit), int(test_withhold)
    o.n, o.m, o.precision = int(n), int(m), int(precision)
    o.has_M, o.has_delta = int(bool(has_M)), int(bool(has_delta))
    o.max_refine, o.refine_tol, o.use_graphs = int(max_refine), float(refine_tol), int(bool(use_graphs))
    return o


def tlqr_factor_create(plan, opts: tlqr_options) -> ctypes.c_void_p:
    h = _vp()
    _check(lib().tlqr_factor_create(plan, ctypes.byref(opts), ctypes.byref(h)), "tlqr_factor_create")
    return h


def tlqr_factor_workspace_bytes(plan, opts: tlqr_options) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().tlqr_factor_workspace_bytes(plan, ctypes.byref(opts), ctypes.byref(b)), "tlqr_factor_workspace_bytes")
    return int(b.value)


def tlqr_factor_bytes(f) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().tlqr_factor_bytes(f, ctypes.byref(b)), "tlqr_factor_bytes")
    return int(b.value)


def tlqr_factor_destroy(f) -> None:
    lib().tlqr_factor_destroy(f)


def make_problem(data: dict) -> tlqr_problem:
    keys = ("Q", "q", "M", "R", "r", "A", "B", "c", "Delta")
    p = tlqr_problem()
    p.mem = _mem_all([data.get(k) for k in keys])
    for k in keys:
        setattr(p, k, _ptr(data.get(k)))
    return p


def make_solution(x, u, y, P=None, K=None) -> tlqr_solution:
    s = tlqr_solution()
    s.mem = _mem_all([x, u, y, P, K])
    s.x, s.u, s.y, s.P, s.K = _ptr(x), _ptr(u), _ptr(y), _ptr(P), _ptr(K)
    return s


def tlqr_factor(f, data: dict, stream=None) -> None:
    p = make_problem(data)
    _check(lib().tlqr_factor(f, ctypes.byref(p), _stream(stream)), "tlqr_factor")


def tlqr_solve(f, data: dict, x, u, y, P=None, K=None, stream=None) -> None:
    p = make_problem(data)
    s = make_solution(x, u, y, P, K)
    _check(lib().tlqr_solve(f, ctypes.byref(p), ctypes.byref(s), _stream(stream)), "tlqr_solve")


def tlqr_update_solve(f, x, u, y, dq=None, dr=None, q=None, r=None, c=None, P=None, K=None, stream=None) -> None:
    """Add diag(dq_i) to Q_i and diag(dr_i) to R_i of the resident problem, replace
    q, r, c (None: unchanged), then factor and solve it into x, u, y."""
    inputs = [a for a in (dq, dr, q, r, c) if a is not None]
    mem = _mem_all(inputs) if inputs else TLQR_MEM_DEVICE
    s = make_solution(x, u, y, P, K)
    _check(lib().tlqr_update_solve(f, mem, *[_ptr(a) for a in (dq, dr, q, r, c)], ctypes.byref(s), _stream(stream)),
           "tlqr_update_solve")


def tlqr_solve_rhs(f, q, r, c, x, u, y, stream=None) -> None:
    mem = _mem_all([q, r, c, x, u, y])
    _check(lib().tlqr_solve_rhs(f, mem, _ptr(q), _ptr(r), _ptr(c), _ptr(x), _ptr(u), _ptr(y),
                                _stream(stream)), "tlqr_solve_rhs")


def tlqr_solve_rhs_panel(f, q, r, c, x, u, y, stream=None) -> None:
    """nrhs right-hand sides at once: q, c, x, y [nrhs, N, n]; r, u [nrhs, N, m] (CUDA tensors)."""
    _check(lib().tlqr_solve_rhs_panel(f, int(q.shape[0]), *[_ptr(a) for a in (q, r, c, x, u, y)], _stream(stream)),
           "tlqr_solve_rhs_panel")


def tlqr_solve_adjoint(f, xbar, ubar, ybar, qbar, rbar, cbar, stream=None) -> None:
    """Gradient of a loss with respect to (q, r, c) from its gradient with respect to (x, u, y)."""
    mem = _mem_all([xbar, ubar, ybar, qbar, rbar, cbar])
    _check(lib().tlqr_solve_adjoint(f, mem, *[_ptr(a) for a in (xbar, ubar, ybar, qbar, rbar, cbar)],
                                    _stream(stream)), "tlqr_solve_adjoint")


def tlqr_pipe_peak(precision, stream=None) -> float:
    """Measured FP32 (TLQR_PREC_MIXED) or FP64 FMA throughput of the device, TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(lib().tlqr_pipe_peak(int(precision), ctypes.byref(v), _stream(stream)), "tlqr_pipe_peak")
    return v.value


def tlqr_autotune(plan, opts: tlqr_options, data: dict, trials: int = 5, stream=None):
    """Time the candidate execution shapes; returns (best options, table rows)."""
    p = make_problem(data)
    best = tlqr_options()
    table = (tlqr_autotune_entry * 32)()
    cnt = np.zeros(1, dtype=np.int32)
    _check(lib().tlqr_autotune(plan, ctypes.byref(opts), ctypes.byref(p), int(trials), ctypes.byref(best), table,
                               32, _iptr(cnt), _stream(stream)), "tlqr_autotune")
    rows = [dict(async_ops=t.async_ops, async_solve=t.async_solve, tail_ops=t.tail_ops, residual=t.residual,
                 status=t.status, ms=t.ms) for t in table[:int(cnt[0])]]
    return best, rows


def tlqr_factor_dims(f):
    d = np.zeros(3, dtype=np.int32)
    _check(lib().tlqr_factor_dims(f, _iptr(d)), "tlqr_factor_dims")
    return int(d[0]), int(d[1]), int(d[2])


def tlqr_ipm_box(plan, f, data: dict, u_lo, u_hi, x, u, y, lam_lo, lam_hi, max_iter=0, mu0=0.0, sigma=0.0, tau=0.0,
                 tol=0.0, no_fp64_fallback=False, stream=None) -> dict:
    """Box-constrained tree LQR by the primal-dual interior-point driver (device arrays)."""
    p = make_problem(data)
    o = tlqr_ipm_options(int(max_iter), float(mu0), float(sigma), float(tau), float(tol), int(bool(no_fp64_fallback)))
    info = tlqr_ipm_info()
    _check(lib().tlqr_ipm_box(plan, f, ctypes.byref(p), _ptr(u_lo), _ptr(u_hi), ctypes.byref(o), _ptr(x), _ptr(u),
                              _ptr(y), _ptr(lam_lo), _ptr(lam_hi), ctypes.byref(info), _stream(stream)),
           "tlqr_ipm_box")
    return dict(iterations=info.iterations, mu=info.mu, mean_gap=info.mean_gap, last_alpha=info.last_alpha,
                last_eta=info.last_eta, fp64_solves=info.fp64_solves)


def tlqr_get_PK(f, P, K, stream=None) -> None:
    mem = _mem_all([P, K])
    _check(lib().tlqr_get_PK(f, mem, _ptr(P), _ptr(K), _stream(stream)), "tlqr_get_PK")


def tlqr_kkt_residual(f, data: dict, x, u, y, stream=None):
    p = make_problem(data)
    mem = _mem_all([x, u, y])
    st = np.zeros(2)
    _check(lib().tlqr_kkt_residual(f, ctypes.byref(p), mem, _ptr(x), _ptr(u), _ptr(y), _ptr(st),
                                   _stream(stream)), "tlqr_kkt_residual")
    return dict(abs=float(st[0]), eta=float(st[1]))


def tlqr_kkt_residual_noalloc(plan, n: int, m: int, data: dict, x, u, y, stream=None):
    """FP64 KKT residual from a plan alone, with no device allocation (device arrays only:
    host arrays raise TLQRError with TLQR_ERR_ARG)."""
    p = make_problem(data)
    if p.mem != TLQR_MEM_DEVICE or _mem_all([x, u, y]) != TLQR_MEM_DEVICE:
        raise TLQRError(TLQR_ERR_ARG, "tlqr_kkt_residual_noalloc")
    st = np.zeros(2)
    _check(lib().tlqr_kkt_residual_noalloc(plan, int(n), int(m), ctypes.byref(p), _ptr(x), _ptr(u), _ptr(y),
                                           _ptr(st), _stream(stream)), "tlqr_kkt_residual_noalloc")
    return dict(abs=float(st[0]), eta=float(st[1]))


def tlqr_last_info(f) -> dict:
    i = tlqr_info()
    _check(lib().tlqr_last_info(f, ctypes.byref(i)), "tlqr_last_info")
    return dict(refine_steps=i.refine_steps, eta=i.eta, abs_residual=i.abs_residual, fp64_resolves=i.fp64_resolves)


def tlqr_tree_residuals(f, n_trees: int):
    """Per-tree (||K z - b||, eta) of the last residual evaluation, as two arrays."""
    a = np.zeros(max(1, n_trees))
    e = np.zeros(max(1, n_trees))
    _check(lib().tlqr_tree_residuals(f, _ptr(a), _ptr(e), n_trees), "tlqr_tree_residuals")
    return a[:n_trees], e[:n_trees]


def tlqr_profile_mask(f, kinds) -> None:
    """Time the launches of the named kernel kinds with CUDA events (empty = off)."""
    mask = 0
    for k in kinds:
        mask |= 1 << KERNEL_KINDS.index(k)
    _check(lib().tlqr_profile_mask(f, mask), "tlqr_profile_mask")


def tlqr_profile_launches(f, max_records: int = 1 << 16):
    """Timed launches since the last read, in launch order: list of (kind, units, ms)."""
    kind = np.zeros(max_records, dtype=np.int32)
    units = np.zeros(max_records, dtype=np.int64)
    ms = np.zeros(max_records)
    cnt = _i32(0)
    _check(lib().tlqr_profile_launches(f, _iptr(kind), units.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       _ptr(ms), max_records, ctypes.byref(cnt)), "tlqr_profile_launches")
    k = min(cnt.value, max_records)
    return [(KERNEL_KINDS[kind[t]], int(units[t]), float(ms[t])) for t in range(k)]


def tlqr_profile_read(f) -> dict:
    arr = (tlqr_kernel_profile * len(KERNEL_KINDS))()
    _check(lib().tlqr_profile_read(f, arr), "tlqr_profile_read")
    return {k: dict(launches=a.launches, units=a.units, timed=a.timed, ms=a.ms)
            for k, a in zip(KERNEL_KINDS, arr)}


# ------------------------------------------------------------------ batched primitives (device)

def tlqr_batched_tau(A, C, P, U, out, precision=TLQR_PREC_FP64, stream=None) -> None:
    count, n = A.shape[0], A.shape[1]
    _check(lib().tlqr_batched_tau(count, n, _ptr(A), _ptr(C), _ptr(P), _ptr(U), _ptr(out), precision,
                                  _stream(stream)), "tlqr_batched_tau")


def tlqr_batched_compose(Al, Cl, Pl, Ar, Cr, Pr, U, An, Cn, Pn, Pt, precision=TLQR_PREC_FP64,
                         stream=None) -> None:
    count, n = Al.shape[0], Al.shape[1]
    _check(lib().tlqr_batched_compose(count, n, *[_ptr(a) for a in (Al, Cl, Pl, Ar, Cr, Pr, U, An, Cn, Pn, Pt)],
                                      precision, _stream(stream)), "tlqr_batched_compose")


def tlqr_batched_condense(A, B, R, M, Delta, Abar, Cbar, Pbar, precision=TLQR_PREC_FP64, stream=None) -> None:
    count, n, m = B.shape
    _check(lib().tlqr_batched_condense(count, n, m, *[_ptr(a) for a in (A, B, R, M, Delta, Abar, Cbar, Pbar)],
                                       precision, _stream(stream)), "tlqr_batched_condense")


def tlqr_batched_expand(Ar, Cr, Pt, Pk, Pj, precision=TLQR_PREC_FP64, stream=None) -> None:
    count, n = Ar.shape[0], Ar.shape[1]
    _check(lib().tlqr_batched_expand(count, n, *[_ptr(a) for a in (Ar, Cr, Pt, Pk, Pj)], precision,
                                     _stream(stream)), "tlqr_batched_expand")


def tlqr_batched_local_factor(P, A, B, R, M, Delta, K, T, precision=TLQR_PREC_FP64, stream=None) -> None:
    count, n, m = B.shape
    _check(lib().tlqr_batched_local_factor(count, n, m, *[_ptr(a) for a in (P, A, B, R, M, Delta, K, T)],
                                           precision, _stream(stream)), "tlqr_batched_local_factor")


def tlqr_batched_compose_T(Tk, Tj, out, precision=TLQR_PREC_FP64, stream=None) -> None:
    count, n = Tk.shape[0], Tk.shape[1]
    _check(lib().tlqr_batched_compose_T(count, n, _ptr(Tk), _ptr(Tj), _ptr(out), precision, _stream(stream)),
           "tlqr_batched_compose_T")


def tlqr_async_schedule(plan, n: int, async_ops: int = 0, which: int = 0) -> dict:
    """Operation list of a level-asynchronous launch (host only): which = 0 the
    factorisation tail, 1 the affine pass, 2 the state pass."""
    counts = np.zeros(4, dtype=np.int32)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(_i32))
    L = lib()
    nul = ctypes.POINTER(_i32)()
    _check(L.tlqr_async_schedule(plan, int(n), int(which), int(async_ops), ip(counts), nul, nul, nul, nul, nul, nul),
           "tlqr_async_schedule")
    P = int(counts[1])
    out = dict(r0=int(counts[0]), n_ops=P, n_flags=int(counts[2]), levels=int(counts[3]))
    arr = {k: np.zeros(max(1, P) * (3 if k.startswith("dep") else 1), dtype=np.int32)
           for k in ("kind", "node", "round", "dep_flag", "dep_target", "signal")}
    _check(L.tlqr_async_schedule(plan, int(n), int(which), int(async_ops), ip(counts), *[ip(arr[k]) for k in
                                 ("kind", "node", "round", "dep_flag", "dep_target", "signal")]),
           "tlqr_async_schedule")
    for k, v in arr.items():
        out[k] = v[:P * 3].reshape(P, 3) if k.startswith("dep") else v[:P]
    return out


# ------------------------------------------------------------------ lifting (host)

def tlqr_lift_node_controls(parent, n: int, m: int, nd: dict) -> dict:
    """Prop. 2 lifting; nd holds Q, q, Mv, Rv, rv, Av, Bv, c, Delta (numpy, node-indexed)."""
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    N = len(parent)
    Nl = _i32(0)
    L = lib()
    args = [_ptr(np.ascontiguousarray(nd[k], dtype=np.float64)) if nd.get(k) is not None else _dp()
            for k in ("Q", "q", "Mv", "Rv", "rv", "Av", "Bv", "c", "Delta")]
    _check(L.tlqr_lift_node_controls(_iptr(parent), N, n, m, *args, ctypes.byref(Nl), _ip(),
                                     *([_dp()] * 9), _ip()), "tlqr_lift_node_controls")
    Nl = Nl.value
    s = n + m
    out = dict(parent=np.zeros(Nl, dtype=np.int32), Q=np.zeros((Nl, s, s)), q=np.zeros((Nl, s)),
               M=np.zeros((Nl, s, m)), R=np.zeros((Nl, m, m)), r=np.zeros((Nl, m)),
               A=np.zeros((Nl, s, s)), B=np.zeros((Nl, s, m)), c=np.zeros((Nl, s)),
               Delta=np.zeros((Nl, s, s)), map=np.zeros(2 * N, dtype=np.int32))
    nl = _i32(0)
    _check(L.tlqr_lift_node_controls(_iptr(parent), N, n, m, *args, ctypes.byref(nl), _iptr(out["parent"]),
                                     *[_ptr(out[k]) for k in ("Q", "q", "M", "R", "r", "A", "B", "c", "Delta")],
                                     _iptr(out["map"])), "tlqr_lift_node_controls")
    return out


def tlqr_project_lifted(N: int, n: int, m: int, lmap, lx, lu, ly):
    x = np.zeros((N, n)); v = np.zeros((N, m)); y = np.zeros((N, n))
    _check(lib().tlqr_project_lifted(N, n, m, _iptr(np.ascontiguousarray(lmap, dtype=np.int32)),
                                     _ptr(np.ascontiguousarray(lx)), _ptr(np.ascontiguousarray(lu)),
                                     _ptr(np.ascontiguousarray(ly)), _ptr(x), _ptr(v), _ptr(y)),
           "tlqr_project_lifted")
    return x, v, y


def tlqr_lift_node_controls_device(parent, n: int, m: int, nd: dict, stream=None) -> dict:
    """Prop. 2 lifting of node-form data held in CUDA tensors; lifted blocks are
    written on the device (torch tensors out), topology arrays are numpy."""
    import torch
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    N = len(parent)
    L = lib()
    args = [_ptr(nd.get(k)) for k in ("Q", "q", "Mv", "Rv", "rv", "Av", "Bv", "c", "Delta")]
    Nl = _i32(0)
    _check(L.tlqr_lift_node_controls_device(_iptr(parent), N, n, m, *args, ctypes.byref(Nl), _ip(),
                                            *([_dp()] * 9), _ip(), _stream(stream)),
           "tlqr_lift_node_controls_device")
    Nl = Nl.value
    s = n + m
    dev = nd["Q"].device
    z = lambda *sh: torch.empty(sh, dtype=torch.float64, device=dev)
    out = dict(parent=np.zeros(Nl, dtype=np.int32), Q=z(Nl, s, s), q=z(Nl, s), M=z(Nl, s, m), R=z(Nl, m, m),
               r=z(Nl, m), A=z(Nl, s, s), B=z(Nl, s, m), c=z(Nl, s), Delta=z(Nl, s, s),
               map=np.zeros(2 * N, dtype=np.int32))
    nl = _i32(0)
    _check(L.tlqr_lift_node_controls_device(_iptr(parent), N, n, m, *args, ctypes.byref(nl), _iptr(out["parent"]),
                                            *[_ptr(out[k]) for k in ("Q", "q", "M", "R", "r", "A", "B", "c",
                                                                     "Delta")],
                                            _iptr(out["map"]), _stream(stream)), "tlqr_lift_node_controls_device")
    return out


def tlqr_project_lifted_device(N: int, n: int, m: int, lmap, lx, lu, ly, stream=None):
    import torch
    dev = lx.device
    x = torch.empty((N, n), dtype=torch.float64, device=dev)
    v = torch.empty((N, m), dtype=torch.float64, device=dev)
    y = torch.empty((N, n), dtype=torch.float64, device=dev)
    _check(lib().tlqr_project_lifted_device(N, n, m, _iptr(np.ascontiguousarray(lmap, dtype=np.int32)),
                                            _ptr(lx), _ptr(lu), _ptr(ly), _ptr(x), _ptr(v), _ptr(y),
                                            _stream(stream)), "tlqr_project_lifted_device")
    return x, v, y


# ------------------------------------------------------------------ ownership helper

class TreeLQR:
    """Owns one plan and one factor object; every method is a direct C call."""

    def __init__(self, parent, n, m, precision=TLQR_PREC_FP64, has_M=False, has_delta=False, forest=False, **kw):
        self.parent = np.ascontiguousarray(parent, dtype=np.int32)
        self.N, self.n, self.m = len(self.parent), int(n), int(m)
        self.plan = tlqr_plan_create_forest(self.parent) if forest else tlqr_plan_create(self.parent)
        self.opts = make_options(n, m, precision, has_M, has_delta, **kw)
        try:
            self.f = tlqr_factor_create(self.plan, self.opts)
        except Exception:
            tlqr_plan_destroy(self.plan)
            raise

    def stats(self):
        return tlqr_plan_stats(self.plan)

    def close(self):
        if getattr(self, "f", None):
            tlqr_factor_destroy(self.f)
            self.f = None
        if getattr(self, "plan", None):
            tlqr_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
