"""The C-ABI library loads and exports every entry point that
include/smallsolve.h declares; host-side argument checks and configuration
queries work without a GPU (no kernel is launched here)."""
import os
import re

import pytest

from paper_1906_08613_gb300 import build as libbuild
from paper_1906_08613_gb300 import smallsolve as ss

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "smallsolve.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|size_t|void|long long)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ss.lib()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("potrf_upper", "trsyl_lu", "trlyap_l", "ss_workspace_size"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in smallsolve.h but not exported"


def test_info_codes_match_header():
    import re
    text = open(HEADER).read()
    codes = dict(re.findall(r"#define SS_(INFO_[A-Z_]+)\s+\((-?\d+)\)", text))
    assert codes and all(getattr(ss, k) == int(v) for k, v in codes.items())


def test_host_side_queries(lib):
    assert ss.ss_version() >= 1
    for op in (ss.OP_POTRF, ss.OP_TRSYL, ss.OP_TRLYAP):
        cnt = ss.ss_config_count(op, ss.MODE_FP64)
        assert cnt >= 1
        for c in range(cnt):
            b, t, v = ss.ss_config_describe(op, ss.MODE_FP64, c)
            assert b in (8, 16, 32, 64) and t % 32 == 0 and t >= b
        assert ss.ss_workspace_size(op, 1000, 128, ss.MODE_FP64) >= 4 * 1000
    assert lib.ss_config_count(7, 0) < 0
    assert lib.ss_workspace_size(0, -1, 4, 0, None) < 0


def test_argument_errors_before_launch(lib):
    # Each returns before any CUDA call: negative batch, size bound, null
    # pointer arrays, invalid mode / cfg, missing or short workspace.
    assert ss.potrf_upper(-1, 4, 1, 1, 1, 1, 1, 1, check=False) == -1
    assert ss.potrf_upper(1, ss.MAX_N + 1, 1, 1, 1, 1, 1, 1, check=False) == -2
    assert ss.potrf_upper(1, 4, 0, 1, 1, 1, 1, 1, check=False) == -3
    assert ss.trsyl_lu(1, 4, 1, 1, 1, 1, 1, 0, 1, 1, 1, 1, check=False) == -8
    assert ss.trlyap_l(1, 4, 1, 1, 1, 1, 1, 1, 1, 0, check=False) == -10
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, mode=99, check=False) == -9
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, cfg=999, check=False) == -10
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, d_work=0, check=False) == -11
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, d_work=1, work_bytes=1, check=False) == -12
    assert ss.trsyl_lu(0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0) == 0


def test_rect_argument_errors_before_launch(lib):
    r = lambda *a, **k: ss.trsyl_rect(*a, check=False, **k)
    ptr = [1] * 11                       # d_m, d_n, d_L, d_ldl, ..., d_info: arguments 4..14
    assert r(-1, 4, 4, *ptr) == -1
    assert r(1, ss.MAX_N + 1, 4, *ptr) == -2
    assert r(1, 4, -1, *ptr) == -3
    for k in range(11):
        p = list(ptr)
        p[k] = 0
        assert r(1, 4, 4, *p) == -(4 + k)
    assert r(1, 4, 4, *ptr, mode=ss.MODE_FP32_REFINED) == -15
    assert r(1, 4, 4, *ptr, mode=ss.MODE_AUTO) == -15
    assert r(1, 4, 4, *ptr, cfg=999) == -16
    assert r(1, 4, 4, *ptr, d_work=0) == -17
    assert r(1, 4, 4, *ptr, d_work=1, work_bytes=1) == -18
    assert ss.trsyl_rect(0, 0, 0, *([0] * 11)) == 0


def test_posv_argument_errors_before_launch(lib):
    r = lambda *a, **k: ss.posv_upper(*a, check=False, **k)
    ptr = [1] * 11                       # d_n, d_k, d_A, d_lda, ..., d_info: arguments 4..14
    assert r(-1, 4, 4, *ptr) == -1
    assert r(1, ss.MAX_N + 1, 4, *ptr) == -2
    assert r(1, 4, -1, *ptr) == -3
    for k in range(11):
        p = list(ptr)
        p[k] = 0
        assert r(1, 4, 4, *p) == -(4 + k)
    assert r(1, 4, 4, *ptr, mode=ss.MODE_TF32_REFINED) == -15
    assert r(1, 4, 4, *ptr, cfg=999) == -16
    assert r(1, 4, 4, *ptr, d_work=0) == -17
    assert r(1, 4, 4, *ptr, d_work=1, work_bytes=1) == -18
    assert ss.posv_upper(0, 0, 0, *([0] * 11)) == 0


def test_df_mode_host_side(lib):
    import re
    text = open(HEADER).read()
    assert int(re.search(r"#define SS_MODE_DF\s+(\d+)", text).group(1)) == ss.MODE_DF
    assert ss.MODES["df"] == ss.MODE_DF
    for op, want in ((ss.OP_POTRF, 3), (ss.OP_TRSYL, 6), (ss.OP_TRLYAP, 6)):
        cnt = ss.ss_config_count(op, ss.MODE_DF)
        assert cnt == want
        # variant 4: the double-float pipeline; bit 3 (Sylvester / Lyapunov):
        # its form for one or two CTAs per SM
        assert all(ss.ss_config_describe(op, ss.MODE_DF, c)[2] & ~8 == 4 for c in range(cnt))
        assert sum(ss.ss_config_describe(op, ss.MODE_DF, c)[2] == 12 for c in range(cnt)) == (3 if op != ss.OP_POTRF else 1)
        # FP64's workspace plus 24 bytes per instance (the scale pre-pass's
        # exponents and diagonal maximum, the flag that hands an instance to
        # the rescaled pass), 256-byte aligned; for Sylvester / Lyapunov also
        # the pre-split double-float copies of L, U and X (scratch offsets, and
        # 3 pairs = 24 bytes per max_n^2 per instance).
        al = lambda x: (x + 255) // 256 * 256
        extra = ss.ss_workspace_size(op, 1000, 128, ss.MODE_DF) - ss.ss_workspace_size(op, 1000, 128, ss.MODE_FP64)
        # (Cholesky: X as pairs, 8 bytes per max_n^2 per instance).
        want = al(1000 * 24) + al(1000 * 8) + al(1000 * 128 * 128 * (8 if op == ss.OP_POTRF else 24))
        assert extra == want
    # Argument checks of the DF forms run before any launch.
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, mode=ss.MODE_DF, cfg=3, check=False) == -10
    assert ss.posv_upper(1, 4, 4, *([1] * 11), mode=ss.MODE_DF, cfg=3, check=False) == -16
    assert ss.posv_upper(1, 4, 4, *([1] * 11), mode=ss.MODE_FP32_REFINED, check=False) == -15
    ss.ss_set_auto_table(ss.OP_TRSYL, [ss.MODE_DF, ss.MODE_FP64], [2, 0])
    ss.ss_set_auto_table(ss.OP_POTRF, [ss.MODE_DF], [1])
    ss.ss_set_auto_table(ss.OP_TRSYL, [], [])
    ss.ss_set_auto_table(ss.OP_POTRF, [], [])
    with pytest.raises(ss.SmallSolveError):
        ss.ss_set_auto_table(ss.OP_POTRF, [ss.MODE_DF], [3])
    with pytest.raises(ss.SmallSolveError):
        ss.ss_set_config_table(ss.OP_TRLYAP, ss.MODE_DF, [6])


def test_config_table_validation(lib):
    with pytest.raises(ss.SmallSolveError):
        ss.ss_set_config_table(ss.OP_TRSYL, ss.MODE_FP64, [999])
    ss.ss_set_config_table(ss.OP_TRSYL, ss.MODE_FP64, [0, 1, -1])
    ss.ss_set_config_table(ss.OP_TRSYL, ss.MODE_FP64, [])
