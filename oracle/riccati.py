"""ORACLE -- test infrastructure only.

ctypes wrapper around ``tlqr_oracle.c``: the sequential FP64 tree Riccati
recursion (Sec. XI-A "CPU seq."; recursion of Sec. V-C and Sec. VI) and the KKT
residual of eq. (kkt) with the normwise backward error

    eta = ||K z - b||_inf / (||K||_inf ||z||_inf + ||b||_inf).

The shared library is compiled from source with gcc on first use (or by the
repository's build step) into ``oracle/liboracle_tlqr.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tlqr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_tlqr.so")
_lib = None

ORACLE_ERRORS = {1: "bad topology", 2: "G not positive definite", 3: "singular F", 4: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the C oracle (portable -O2, no host-specific ISA flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i32 = ctypes.c_int32
        lib.oracle_tree_riccati.restype = ctypes.c_int
        lib.oracle_tree_riccati.argtypes = [i32, i32, i32, ip] + [dp] * 9 + [dp] * 6
        lib.oracle_kkt_residual.restype = ctypes.c_int
        lib.oracle_kkt_residual.argtypes = [i32, i32, i32, ip] + [dp] * 9 + [dp] * 3 + [dp] * 4
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(data: dict):
    out = {}
    for k in ("Q", "q", "M", "R", "r", "A", "B", "c", "Delta"):
        v = data.get(k)
        out[k] = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    return out


def tree_riccati(parent, n: int, m: int, data: dict) -> dict:
    """Solve the KKT system eq. (kkt) by the sequential tree Riccati recursion.

    Returns dict(x (N,n), u (N,m), y (N,n), P (N,n,n), K (N,m,n), p (N,n)).
    Edge-indexed outputs use the child slot; the root slot of u and K is zero.
    """
    lib = _load()
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    N = len(parent)
    d = _prep(data)
    x = np.zeros((N, n)); u = np.zeros((N, m)); y = np.zeros((N, n))
    P = np.zeros((N, n, n)); K = np.zeros((N, m, n)); p = np.zeros((N, n))
    rc = lib.oracle_tree_riccati(N, n, m, parent.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 _dp(d["Q"]), _dp(d["q"]), _dp(d["M"]), _dp(d["R"]), _dp(d["r"]),
                                 _dp(d["A"]), _dp(d["B"]), _dp(d["c"]), _dp(d["Delta"]),
                                 _dp(x), _dp(u), _dp(y), _dp(P), _dp(K), _dp(p))
    if rc:
        raise RuntimeError(f"oracle_tree_riccati failed: {ORACLE_ERRORS.get(rc, rc)}")
    return dict(x=x, u=u, y=y, P=P, K=K, p=p)


def kkt_residual(parent, n: int, m: int, data: dict, x, u, y) -> dict:
    """Residual blocks of eq. (kkt) and eta (normwise backward error)."""
    lib = _load()
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    N = len(parent)
    d = _prep(data)
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    rx = np.zeros((N, n)); ru = np.zeros((N, m)); rc_ = np.zeros((N, n)); st = np.zeros(5)
    rc = lib.oracle_kkt_residual(N, n, m, parent.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 _dp(d["Q"]), _dp(d["q"]), _dp(d["M"]), _dp(d["R"]), _dp(d["r"]),
                                 _dp(d["A"]), _dp(d["B"]), _dp(d["c"]), _dp(d["Delta"]),
                                 _dp(x), _dp(u), _dp(y), _dp(rx), _dp(ru), _dp(rc_), _dp(st))
    if rc:
        raise RuntimeError(f"oracle_kkt_residual failed: {ORACLE_ERRORS.get(rc, rc)}")
    return dict(res_x=rx, res_u=ru, res_c=rc_, abs=st[0], eta=st[1], normK=st[2], normz=st[3], normb=st[4])


def forward_error(sol: dict, ref: dict, parent) -> float:
    """max |z - z_ref| / max |z_ref| over (x, u, y), root control slot excluded."""
    nonroot = np.asarray(parent) >= 0
    num = max(np.abs(sol["x"] - ref["x"]).max(), np.abs(sol["y"] - ref["y"]).max(),
              np.abs(sol["u"][nonroot] - ref["u"][nonroot]).max() if nonroot.any() else 0.0)
    den = max(np.abs(ref["x"]).max(), np.abs(ref["y"]).max(),
              np.abs(ref["u"][nonroot]).max() if nonroot.any() else 0.0)
    return float(num / den) if den > 0 else float(num)
