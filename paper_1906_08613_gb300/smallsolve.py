"""Python binding of the C ABI in include/smallsolve.h (ctypes, marshalling only).

Every function here converts its arguments and calls the entry point of the
same name in libsmallsolve.so; all arithmetic runs in the library's CUDA
kernels.  The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1906_08613_gb300.build``); if it is missing, loading fails
with an error rather than falling back to anything else.

Device pointers are passed as Python ints (e.g. ``tensor.data_ptr()``) and
streams as the integer handle of a ``cudaStream_t`` (``torch.cuda.Stream
.cuda_stream``; 0 is the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsmallsolve.so")

OP_POTRF, OP_TRSYL, OP_TRLYAP = 0, 1, 2
OPS = {"potrf": OP_POTRF, "trsyl": OP_TRSYL, "trlyap": OP_TRLYAP}

MODE_FP64 = 0
MODE_FP32_REFINED = 1
MODE_TF32_REFINED = 2
MODE_BF16_REFINED = 3
MODE_FP32_RAW = 4
MODE_TF32_RAW = 5
MODE_BF16_RAW = 6
MODE_DF = 8
MODES = {"fp64": 0, "fp32_refined": 1, "tf32_refined": 2, "bf16_refined": 3,
         "fp32_raw": 4, "tf32_raw": 5, "bf16_raw": 6, "df": MODE_DF}

MODE_AUTO = 7
REFINED_MODES = (MODE_FP32_REFINED, MODE_TF32_REFINED, MODE_BF16_REFINED)

CFG_DEFAULT = -1
CFG_TABLE = -2

ERR_CUDA = -100
ERR_SCRATCH_LIMIT = -101
ERR_IO = -102
ERR_NO_SELECTOR = -103
SELECTOR_PER_BIN = 0
SELECTOR_CALL = 1
SELECTOR_MODES = (MODE_FP64, MODE_FP32_REFINED, MODE_TF32_REFINED, MODE_BF16_REFINED, MODE_DF)
SELECTOR_MAX_ROWS = 13 * 5
INFO_BAD_SIZE = -1
INFO_ALIASED = -3
INFO_RANGE = -4
INFO_TIMEOUT = -5
INFO_NO_WORK = -2
MAX_N = 4096
MLP_IN, MLP_HIDDEN, MLP_OUT = 10, 64, 8
MLP_PARAMS = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + \
    MLP_OUT * MLP_HIDDEN + MLP_OUT
NUM_BINS = 13
REFINE_TOL = 1e-13
REFINE_MAXIT = 10

_lock = threading.Lock()
_lib = None


class SmallSolveError(RuntimeError):
    pass


def lib():
    """Load libsmallsolve.so (once)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise SmallSolveError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            i, vp, sz = ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
            L.potrf_upper.argtypes = [i, i, vp, vp, vp, vp, vp, vp, i, i, vp, sz, vp]
            L.trsyl_lu.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i, i, vp, sz, vp]
            L.trlyap_l.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp, vp, i, i, vp, sz, vp]
            L.trsyl_rect.argtypes = [i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i, i, vp, sz, vp]
            L.posv_upper.argtypes = [i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i, i, vp, sz, vp]
            for f in (L.potrf_upper, L.trsyl_lu, L.trlyap_l, L.trsyl_rect, L.posv_upper):
                f.restype = i
            L.trsyl_lu_noalloc.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.trsyl_lu_noalloc.restype = i
            L.ss_workspace_size.argtypes = [i, i, i, i, ctypes.POINTER(sz)]
            L.ss_workspace_size.restype = i
            L.ss_config_count.argtypes = [i, i]
            L.ss_config_count.restype = i
            ip = ctypes.POINTER(i)
            L.ss_config_describe.argtypes = [i, i, i, ip, ip, ip]
            L.ss_config_describe.restype = i
            L.ss_set_config_table.argtypes = [i, i, i, ip]
            L.ss_set_config_table.restype = i
            L.ss_set_auto_table.argtypes = [i, i, ip, ip]
            L.ss_set_auto_table.restype = i
            fl = ctypes.c_float
            L.ss_mlp_workspace_size.argtypes = [i, ctypes.POINTER(sz)]
            L.ss_mlp_workspace_size.restype = i
            L.ss_mlp_forward.argtypes = [vp, i, vp, vp, vp]
            L.ss_mlp_forward.restype = i
            L.ss_mlp_grad.argtypes = [vp, i, vp, vp, vp, fl, vp, vp, vp, sz, vp]
            L.ss_mlp_grad.restype = i
            L.ss_mlp_adam.argtypes = [vp, vp, vp, vp, i, fl, fl, fl, fl, vp]
            L.ss_mlp_adam.restype = i
            L.ss_version.argtypes = []
            L.ss_version.restype = i
            L.ss_umma_selftest.argtypes = [i, i, i, vp, vp, vp, vp, i, vp, vp]
            L.ss_umma_selftest.restype = i
            L.ss_launch_count.argtypes = []
            L.ss_launch_count.restype = ctypes.c_longlong
            L.ss_profile_enable.argtypes = [i]
            L.ss_profile_enable.restype = i
            L.ss_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i)]
            L.ss_profile_read.restype = i
            fp = ctypes.POINTER(fl)
            dp = ctypes.POINTER(ctypes.c_double)
            L.ss_autotune.argtypes = [i, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, i, fp, ip, ip, vp]
            L.ss_selector_set.argtypes = [fp, ip, ip]
            L.ss_selector_get.argtypes = [fp, ip, ip]
            L.ss_selector_clear.argtypes = []
            L.ss_selector_save.argtypes = [ctypes.c_char_p]
            L.ss_selector_load.argtypes = [ctypes.c_char_p]
            L.ss_selector_train.argtypes = [fp, fp, fp, i, fp, i, fl, fp, vp]
            L.ss_selector_queries.argtypes = [i, i, ip, fp, ip]
            L.ss_selector_decide.argtypes = [i, i, ip, i, fp, ip, ip, dp]
            L.ss_selector_predict.argtypes = [i, i, ip, i, ip, ip, dp, vp]
            L.ss_selector_install.argtypes = [i, i, ip, i, vp]
            for f in (L.ss_autotune, L.ss_selector_set, L.ss_selector_get, L.ss_selector_clear, L.ss_selector_save,
                      L.ss_selector_load, L.ss_selector_train, L.ss_selector_queries, L.ss_selector_decide,
                      L.ss_selector_predict, L.ss_selector_install):
                f.restype = i
            _lib = L
    return _lib


def _check(rc: int, name: str) -> int:
    if rc != 0:
        raise SmallSolveError(f"{name} returned {rc}")
    return rc


def potrf_upper(batch, max_n, d_n, d_A, d_lda, d_X, d_ldx, d_info, mode=MODE_FP64,
                cfg=CFG_DEFAULT, d_work=0, work_bytes=0, stream=0, check=True):
    rc = lib().potrf_upper(batch, max_n, d_n, d_A, d_lda, d_X, d_ldx, d_info, mode, cfg,
                           d_work or None, work_bytes, stream or None)
    return _check(rc, "potrf_upper") if check else rc


def trsyl_lu(batch, max_n, d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx, d_info,
             mode=MODE_FP64, cfg=CFG_DEFAULT, d_work=0, work_bytes=0, stream=0, check=True):
    rc = lib().trsyl_lu(batch, max_n, d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx,
                        d_info, mode, cfg, d_work or None, work_bytes, stream or None)
    return _check(rc, "trsyl_lu") if check else rc


def trsyl_rect(batch, max_m, max_n, d_m, d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx, d_info,
               mode=MODE_FP64, cfg=CFG_DEFAULT, d_work=0, work_bytes=0, stream=0, check=True):
    """Rectangular Sylvester L X + X U = C (L m x m, U n x n, X m x n)."""
    rc = lib().trsyl_rect(batch, max_m, max_n, d_m, d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx,
                          d_info, mode, cfg, d_work, work_bytes, stream)
    return _check(rc, "trsyl_rect") if check else rc


def posv_upper(batch, max_n, max_k, d_n, d_k, d_A, d_lda, d_R, d_ldr, d_B, d_ldb, d_X, d_ldx, d_info,
               mode=MODE_FP64, cfg=CFG_DEFAULT, d_work=0, work_bytes=0, stream=0, check=True):
    """SPD solve A X = B through the upper Cholesky factor R (written to d_R)."""
    rc = lib().posv_upper(batch, max_n, max_k, d_n, d_k, d_A, d_lda, d_R, d_ldr, d_B, d_ldb, d_X, d_ldx,
                          d_info, mode, cfg, d_work, work_bytes, stream)
    return _check(rc, "posv_upper") if check else rc


def trsyl_lu_noalloc(batch, max_n, d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx, d_info,
                     stream=0, check=True):
    """trsyl_lu (FP64, default configuration) using the library's fixed scratch
    area instead of a caller-provided workspace; allocates nothing."""
    rc = lib().trsyl_lu_noalloc(batch, max_n, d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X,
                                d_ldx, d_info, stream or None)
    return _check(rc, "trsyl_lu_noalloc") if check else rc


def trlyap_l(batch, max_n, d_n, d_L, d_ldl, d_S, d_lds, d_X, d_ldx, d_info, mode=MODE_FP64,
             cfg=CFG_DEFAULT, d_work=0, work_bytes=0, stream=0, check=True):
    rc = lib().trlyap_l(batch, max_n, d_n, d_L, d_ldl, d_S, d_lds, d_X, d_ldx, d_info, mode,
                        cfg, d_work or None, work_bytes, stream or None)
    return _check(rc, "trlyap_l") if check else rc


def ss_workspace_size(op, batch, max_n, mode) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().ss_workspace_size(op, batch, max_n, mode, ctypes.byref(out)), "ss_workspace_size")
    return int(out.value)


def ss_config_count(op, mode) -> int:
    return int(lib().ss_config_count(op, mode))


def ss_config_describe(op, mode, cfg):
    b, t, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().ss_config_describe(op, mode, cfg, ctypes.byref(b), ctypes.byref(t),
                                    ctypes.byref(v)), "ss_config_describe")
    return int(b.value), int(t.value), int(v.value)


def ss_set_config_table(op, mode, cfg_by_bin) -> None:
    arr = (ctypes.c_int * max(1, len(cfg_by_bin)))(*[int(c) for c in cfg_by_bin])
    _check(lib().ss_set_config_table(op, mode, len(cfg_by_bin), arr), "ss_set_config_table")


def ss_set_auto_table(op, mode_by_bin, cfg_by_bin) -> None:
    """Per-size-bin (mode, cfg) choices for MODE_AUTO (empty lists clear)."""
    nb = len(mode_by_bin)
    assert len(cfg_by_bin) == nb
    ma = (ctypes.c_int * max(1, nb))(*[int(m) for m in mode_by_bin])
    ca = (ctypes.c_int * max(1, nb))(*[int(c) for c in cfg_by_bin])
    _check(lib().ss_set_auto_table(op, nb, ma, ca), "ss_set_auto_table")


def ss_mlp_workspace_size(nrows) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().ss_mlp_workspace_size(nrows, ctypes.byref(out)), "ss_mlp_workspace_size")
    return int(out.value)


def ss_mlp_forward(d_params, nrows, d_x, d_y, stream=0):
    return _check(lib().ss_mlp_forward(d_params, nrows, d_x, d_y, stream or None), "ss_mlp_forward")


def ss_mlp_grad(d_params, nrows, d_x, d_t, d_mask, mask_total, d_grad, d_loss, d_work, work_bytes,
                stream=0):
    return _check(lib().ss_mlp_grad(d_params, nrows, d_x, d_t, d_mask, float(mask_total), d_grad,
                                    d_loss, d_work, work_bytes, stream or None), "ss_mlp_grad")


UMMA_TF32, UMMA_BF16 = 0, 1


def ss_umma_selftest(kind, n, k, d_a, d_b, d_c, d_d, flags, d_status, stream=0, check=True):
    rc = lib().ss_umma_selftest(kind, n, k, d_a, d_b, d_c or None, d_d, flags, d_status, stream or None)
    return _check(rc, "ss_umma_selftest") if check else rc


def ss_mlp_adam(d_params, d_grad, d_m, d_v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    return _check(lib().ss_mlp_adam(d_params, d_grad, d_m, d_v, step, lr, beta1, beta2, eps,
                                    stream or None), "ss_mlp_adam")


def ss_version() -> int:
    return int(lib().ss_version())


def ss_launch_count() -> int:
    return int(lib().ss_launch_count())


def ss_profile_enable(on: bool) -> None:
    _check(lib().ss_profile_enable(1 if on else 0), "ss_profile_enable")


def ss_profile_read():
    """(total milliseconds, number of calls) of the solve kernels recorded
    since the last read."""
    t = ctypes.c_double(0.0)
    c = ctypes.c_int(0)
    _check(lib().ss_profile_read(ctypes.byref(t), ctypes.byref(c)), "ss_profile_read")
    return float(t.value), int(c.value)


def size_bin(n: int) -> int:
    """bin(n) = ceil(log2(max(n, 1))), the index of the per-size config table."""
    k = 0
    while (1 << k) < n:
        k += 1
    return k


# ---------------------------------------------------------------- autotuner

def ss_autotune(op, mode, batch, max_n, d_n, d_A, d_lda, d_B, d_ldb, d_C, d_ldc, d_X, d_ldx, d_info,
                d_work, work_bytes, reps=3, stream=0):
    """Times every configuration of `mode` on the given batch (see the header);
    returns (ms per configuration, bad instances per configuration, best cfg)."""
    cnt = ss_config_count(op, mode)
    ms = (ctypes.c_float * max(cnt, 1))()
    bad = (ctypes.c_int * max(cnt, 1))()
    best = ctypes.c_int(-1)
    _check(lib().ss_autotune(op, mode, batch, max_n, d_n, d_A, d_lda, d_B or None, d_ldb or None, d_C or None,
                             d_ldc or None, d_X, d_ldx, d_info, d_work, work_bytes, reps, ms, bad,
                             ctypes.byref(best), stream or None), "ss_autotune")
    return [float(v) for v in ms[:cnt]], [int(v) for v in bad[:cnt]], int(best.value)


# ------------------------------------------------------------------ selector

def _int_array(vals):
    return (ctypes.c_int * max(1, len(vals)))(*[int(v) for v in vals])


def _float_ptr(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def ss_selector_set(params, cfg_count=None, batch_max=None) -> None:
    """params: SS_MLP_PARAMS floats; cfg_count: 15 ints (op * 5 + selector
    mode) or None; batch_max: 3 * 13 * 5 ints or None."""
    keep, pp = _float_ptr(params)
    assert keep.size == MLP_PARAMS
    cc = _int_array(cfg_count) if cfg_count is not None else None
    bm = _int_array(batch_max) if batch_max is not None else None
    _check(lib().ss_selector_set(pp, cc, bm), "ss_selector_set")


def ss_selector_get():
    """(params, cfg_count, batch_max) of the library's model."""
    import numpy as np
    p = np.zeros(MLP_PARAMS, dtype=np.float32)
    cc = (ctypes.c_int * 15)()
    bm = (ctypes.c_int * (3 * NUM_BINS * 5))()
    _check(lib().ss_selector_get(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), cc, bm), "ss_selector_get")
    return p, list(cc), list(bm)


def ss_selector_clear() -> None:
    _check(lib().ss_selector_clear(), "ss_selector_clear")


def ss_selector_save(path: str) -> None:
    _check(lib().ss_selector_save(os.fsencode(path)), "ss_selector_save")


def ss_selector_load(path: str) -> None:
    _check(lib().ss_selector_load(os.fsencode(path)), "ss_selector_load")


def ss_selector_train(X, T, M, steps, lr, init=None, stream=0):
    """Trains the library's model on the GPU; returns the loss before each step."""
    import numpy as np
    kx, px = _float_ptr(X)
    kt, pt = _float_ptr(T)
    km, pm = _float_ptr(M)
    ki, pi = _float_ptr(init) if init is not None else (None, None)
    loss = np.zeros(max(int(steps), 1), dtype=np.float32)
    _check(lib().ss_selector_train(px, pt, pm, int(kx.shape[0]), pi, int(steps), float(lr),
                                   loss.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), stream or None),
           "ss_selector_train")
    return loss[:steps]


def ss_selector_queries(op, count_by_bin):
    """Feature rows [nrows x SS_MLP_IN] the selector evaluates for a call."""
    import numpy as np
    x = np.zeros((SELECTOR_MAX_ROWS, MLP_IN), dtype=np.float32)
    nr = ctypes.c_int(0)
    _check(lib().ss_selector_queries(op, len(count_by_bin), _int_array(count_by_bin),
                                     x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(nr)),
           "ss_selector_queries")
    return x[:nr.value].copy()


def ss_selector_decide(op, count_by_bin, policy, y):
    """(modes, cfgs, predicted ms) from network outputs y for those rows."""
    nb = len(count_by_bin)
    ky, py = _float_ptr(y)
    m = (ctypes.c_int * max(nb, 1))()
    c = (ctypes.c_int * max(nb, 1))()
    ms = ctypes.c_double(0.0)
    _check(lib().ss_selector_decide(op, nb, _int_array(count_by_bin), policy, py, m, c, ctypes.byref(ms)),
           "ss_selector_decide")
    return list(m[:nb]), list(c[:nb]), float(ms.value)


def ss_selector_predict(op, count_by_bin, policy, stream=0):
    """(modes, cfgs, predicted ms) by the CUDA forward of the library's model."""
    nb = len(count_by_bin)
    m = (ctypes.c_int * max(nb, 1))()
    c = (ctypes.c_int * max(nb, 1))()
    ms = ctypes.c_double(0.0)
    _check(lib().ss_selector_predict(op, nb, _int_array(count_by_bin), policy, m, c, ctypes.byref(ms),
                                     stream or None), "ss_selector_predict")
    return list(m[:nb]), list(c[:nb]), float(ms.value)


def ss_selector_install(op, count_by_bin, policy, stream=0) -> None:
    _check(lib().ss_selector_install(op, len(count_by_bin), _int_array(count_by_bin), policy, stream or None),
           "ss_selector_install")
