"""CPU oracle for the three structured solves (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  The product library never does, and this package
imports nothing from the product.

``oracle.c`` holds the plain FP64 recurrences; this module compiles it with gcc
(``-O2 -ffp-contract=off``, so no fused multiply-adds change the rounding) and
calls it through ctypes.  ctypes releases the GIL during the foreign call, so a
thread pool over instances runs the oracle on several host cores.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it; returns the path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            llp = ctypes.POINTER(ctypes.c_longlong)
            c_int = ctypes.c_int
            L.oracle_potrf_upper.argtypes = [c_int, dp, c_int, dp, c_int]
            L.oracle_trsyl_lu.argtypes = [c_int, dp, c_int, dp, c_int, dp, c_int, dp, c_int]
            L.oracle_trlyap_l.argtypes = [c_int, dp, c_int, dp, c_int, dp, c_int]
            for f in (L.oracle_potrf_upper, L.oracle_trsyl_lu, L.oracle_trlyap_l):
                f.restype = c_int
            L.oracle_potrf_upper_batch.argtypes = [c_int, ip, llp, dp, dp, ip]
            L.oracle_trsyl_lu_batch.argtypes = [c_int, ip, llp, dp, dp, dp, dp, ip]
            L.oracle_trlyap_l_batch.argtypes = [c_int, ip, llp, dp, dp, dp, ip]
            L.oracle_trsyl_rect.argtypes = [c_int, c_int, dp, c_int, dp, c_int, dp, c_int, dp, c_int]
            L.oracle_trsyl_rect.restype = c_int
            L.oracle_trsyl_rect_batch.argtypes = [c_int, ip, ip, llp, llp, llp, dp, dp, dp, dp, ip]
            L.oracle_posv_upper.argtypes = [c_int, c_int, dp, c_int, dp, c_int, dp, c_int, dp, c_int]
            L.oracle_posv_upper.restype = c_int
            L.oracle_posv_upper_batch.argtypes = [c_int, ip, ip, llp, llp, dp, dp, dp, dp, ip]
            for f in (L.oracle_potrf_upper_batch, L.oracle_trsyl_lu_batch,
                      L.oracle_trlyap_l_batch, L.oracle_trsyl_rect_batch, L.oracle_posv_upper_batch):
                f.restype = None
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(m):
    return np.asfortranarray(np.asarray(m, dtype=np.float64))


# ---- single instances (column-major numpy matrices in, new matrices out) ----

def potrf_upper(a):
    """Upper Cholesky factor X of A (X^T X = A); returns (X, info).

    Only the upper triangle of X is written; its strict lower part is zero."""
    a = _f64(a)
    n = a.shape[0]
    x = np.zeros((n, n), dtype=np.float64, order="F")
    info = lib().oracle_potrf_upper(n, _dp(a), n, _dp(x), n)
    return x, int(info)


def trsyl_lu(l, u, c):
    """X with L X + X U = C (L lower, U upper triangular); returns (X, info)."""
    l, u, c = _f64(l), _f64(u), _f64(c)
    n = c.shape[0]
    x = np.zeros((n, n), dtype=np.float64, order="F")
    info = lib().oracle_trsyl_lu(n, _dp(l), n, _dp(u), n, _dp(c), n, _dp(x), n)
    return x, int(info)


def trsyl_rect(l, u, c):
    """X (m x n) with L X + X U = C, L (m x m) lower, U (n x n) upper
    triangular; returns (X, info)."""
    l, u, c = _f64(l), _f64(u), _f64(c)
    m, n = c.shape
    x = np.zeros((m, n), dtype=np.float64, order="F")
    info = lib().oracle_trsyl_rect(m, n, _dp(l), max(m, 1), _dp(u), max(n, 1), _dp(c), max(m, 1),
                                   _dp(x), max(m, 1))
    return x, int(info)


def posv_upper(a, b):
    """X with A X = B (A SPD, upper triangle read) through the upper Cholesky
    factor; returns (X, R, info)."""
    a, b = _f64(a), _f64(b)
    n, k = b.shape
    r = np.zeros((n, n), dtype=np.float64, order="F")
    x = np.zeros((n, k), dtype=np.float64, order="F")
    ld = max(n, 1)
    info = lib().oracle_posv_upper(n, k, _dp(a), ld, _dp(r), ld, _dp(b), ld, _dp(x), ld)
    return x, r, int(info)


def trlyap_l(l, s):
    """Lower triangle of the symmetric X with L X + X L^T = S; returns (X, info).

    The strict upper part of the returned X is zero."""
    l, s = _f64(l), _f64(s)
    n = s.shape[0]
    x = np.zeros((n, n), dtype=np.float64, order="F")
    info = lib().oracle_trlyap_l(n, _dp(l), n, _dp(s), n, _dp(x), n)
    return x, int(info)


# ---- packed batches (the layout of paper_1906_08613_gb300.inputs.Packed) ----

def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _llp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))


def solve_packed(op: str, n, off, ops: dict, out=None, lo: int = 0, hi=None):
    """Solve instances lo..hi-1 of a packed batch in place into ``out``.

    ``op`` is "potrf", "trsyl" or "trlyap"; ``ops`` maps operand names (A; L, U,
    C; L, S) to flat float64 buffers.  Returns (out, info[lo:hi])."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    hi = len(n) if hi is None else hi
    if out is None:
        out = np.zeros_like(next(iter(ops.values())))
    cnt = hi - lo
    info = np.zeros(max(cnt, 1), dtype=np.int32)
    nn = n[lo:hi]
    oo = off[lo:hi]
    L = lib()
    if cnt <= 0:
        return out, info[:0]
    if op == "potrf":
        L.oracle_potrf_upper_batch(cnt, _ip(nn), _llp(oo), _dp(ops["A"]), _dp(out), _ip(info))
    elif op == "trsyl":
        L.oracle_trsyl_lu_batch(cnt, _ip(nn), _llp(oo), _dp(ops["L"]), _dp(ops["U"]),
                                _dp(ops["C"]), _dp(out), _ip(info))
    elif op == "trlyap":
        L.oracle_trlyap_l_batch(cnt, _ip(nn), _llp(oo), _dp(ops["L"]), _dp(ops["S"]),
                                _dp(out), _ip(info))
    else:
        raise ValueError(op)
    return out, info[:cnt]


def solve_packed_parallel(op: str, n, off, ops: dict, threads: int, out=None,
                          indices=None):
    """Solve the instances listed in ``indices`` (default: all) on ``threads``
    host threads, one instance per task.  Returns (out, info)."""
    from concurrent.futures import ThreadPoolExecutor
    n = np.ascontiguousarray(n, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    if out is None:
        out = np.zeros_like(next(iter(ops.values())))
    idx = np.arange(len(n)) if indices is None else np.asarray(indices)
    info = np.zeros(len(n), dtype=np.int32)

    def one(b):
        _, inf = solve_packed(op, n, off, ops, out=out, lo=int(b), hi=int(b) + 1)
        info[b] = inf[0]

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        list(ex.map(one, idx))
    return out, info


def solve_rect_packed(pk, out=None, lo: int = 0, hi=None):
    """Rectangular Sylvester on instances lo..hi-1 of a RectPacked batch
    (paper_1906_08613_gb300.inputs.RectPacked), written into ``out`` (laid out
    like C).  Returns (out, info[lo:hi])."""
    hi = pk.batch if hi is None else hi
    if out is None:
        out = np.zeros_like(pk.ops["C"])
    cnt = hi - lo
    info = np.zeros(max(cnt, 1), dtype=np.int32)
    if cnt <= 0:
        return out, info[:0]
    a = lambda v: np.ascontiguousarray(v[lo:hi])
    m, n = a(pk.m).astype(np.int32), a(pk.n).astype(np.int32)
    oL, oU, oC = a(pk.offL).astype(np.int64), a(pk.offU).astype(np.int64), a(pk.offC).astype(np.int64)
    lib().oracle_trsyl_rect_batch(cnt, _ip(m), _ip(n), _llp(oL), _llp(oU), _llp(oC),
                                  _dp(pk.ops["L"]), _dp(pk.ops["U"]), _dp(pk.ops["C"]), _dp(out), _ip(info))
    return out, info[:cnt]


def solve_posv_packed(pk, lo: int = 0, hi=None, out_x=None, out_r=None):
    """SPD solves of instances lo..hi-1 of a PosvPacked batch
    (paper_1906_08613_gb300.inputs.PosvPacked).  Returns (X, R, info[lo:hi])."""
    hi = pk.batch if hi is None else hi
    out_x = np.zeros_like(pk.ops["B"]) if out_x is None else out_x
    out_r = np.zeros_like(pk.ops["A"]) if out_r is None else out_r
    cnt = hi - lo
    info = np.zeros(max(cnt, 1), dtype=np.int32)
    if cnt <= 0:
        return out_x, out_r, info[:0]
    a = lambda v: np.ascontiguousarray(v[lo:hi])
    n, k = a(pk.n).astype(np.int32), a(pk.k).astype(np.int32)
    oA, oB = a(pk.offA).astype(np.int64), a(pk.offB).astype(np.int64)
    lib().oracle_posv_upper_batch(cnt, _ip(n), _ip(k), _llp(oA), _llp(oB), _dp(pk.ops["A"]), _dp(out_r),
                                  _dp(pk.ops["B"]), _dp(out_x), _ip(info))
    return out_x, out_r, info[:cnt]
