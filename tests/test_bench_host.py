"""Host-side arithmetic of bench.py: the flop and byte counts behind the
roofline fraction, the two peaks it divides by, and the mode names in the JSON
line (no GPU needed)."""
import math

import pytest

import bench
from paper_1906_08613_gb300 import selector as sel
from paper_1906_08613_gb300 import smallsolve as ss


def test_flop_counts():
    # The paper's counts (Fig. 2 caption) and the algorithmic ones.
    assert bench.flops_paper("potrf", [3]) == pytest.approx(9.0)
    assert bench.flops_paper("trsyl", [2]) == pytest.approx(16.0)
    assert bench.flops_paper("trlyap", [2]) == pytest.approx(16.0)
    assert bench.flops_algorithmic("potrf", [3, 3]) == pytest.approx(18.0)
    assert bench.flops_algorithmic("trsyl", [2]) == pytest.approx(16.0)
    assert bench.flops_algorithmic("trlyap", [2]) == pytest.approx(8.0)     # symmetric X: n^3


def test_algorithmic_bytes():
    # n = 2: a stored triangle holds 3 values, a full 2 x 2 operand 4.
    assert bench.bytes_algorithmic("potrf", [2]) == pytest.approx(8 * (3 + 3))
    assert bench.bytes_algorithmic("trsyl", [2]) == pytest.approx(8 * (3 + 3 + 4 + 4))
    assert bench.bytes_algorithmic("trlyap", [2]) == pytest.approx(8 * (3 + 3 + 3))


def test_peaks():
    assert bench.FP64_PEAK_GFLOPS == pytest.approx(152 * 2 * 2 * 2.07)
    # FP32 instruction rate over 13 instructions per double-float
    # multiply-add, counted as the 2 flops of the FP64 operation.
    assert bench.DF_OPS_PER_TERM == 13
    assert bench.DF_PEAK_GFLOPS == pytest.approx(152 * 128 * 2.07 / 13 * 2)
    assert math.isclose(bench.DF_PEAK_GFLOPS / bench.FP64_PEAK_GFLOPS, 128 / (2 * 13), rel_tol=1e-12)


def test_mode_names_in_the_json_line():
    for mode in sel.MODE_ORDER:                 # every mode the selector may put in a table
        assert mode in bench.DTYPE_OF_MODE
        assert bench.inv_mode(ss.MODES[mode]) == mode
    assert bench.inv_mode(ss.MODE_DF) == "df"
