"""Parity of the tensor-memory (tcgen05) configurations of the refined modes
with the FP64 oracle: the low-precision solve keeps its trailing matrix in
TMEM as the tensor cores' FP32 accumulator and applies the trailing updates
as 128-row TF32 / BF16 MMA tiles; refinement brings every instance to the
1e-11 gate.  Sizes cover one and two TMEM tiles, ragged tails, pivot
failures inside and after the first tile, and the blocked fallback above
n = 256."""
import numpy as np
import pytest

from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import assert_parity, oracle_batch, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENT = -3.5
TC_MODES = ["tf32_refined", "bf16_refined"]
SIZES = [1, 2, 7, 16, 31, 32, 33, 48, 63, 64, 65, 96, 100, 127, 128, 129, 144, 160, 161, 200, 224, 255, 256, 257, 300]


def tc_cfg(op, mode):
    """The tensor-memory configuration: variant bit 2."""
    o, m = ss.OPS[op], ss.MODES[mode]
    for c in range(ss.ss_config_count(o, m)):
        if ss.ss_config_describe(o, m, c)[2] & 4:
            return c
    pytest.skip(f"no tensor-memory configuration for {op} {mode}")


def run(op, pk, mode, cfg, **kw):
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op, x_fill=SENT, **kw)
    db.solve(mode=ss.MODES[mode], cfg=cfg)
    torch.cuda.synchronize()
    return db.x_host(), db.info_host()


@pytest.mark.parametrize("mode", TC_MODES)
def test_cholesky_tensor_memory_sizes(mode):
    n = np.array(SIZES, dtype=np.int32)
    pk = inputs.cholesky_batch(n, seed=51)
    ref, rinfo = oracle_batch("potrf", pk)
    x, info = run("potrf", pk, mode, tc_cfg("potrf", mode))
    assert np.array_equal(info, rinfo) and np.all(info == 0)
    assert_parity("potrf", pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("mode", ["tf32_raw", "bf16_raw"])
def test_cholesky_tensor_memory_raw_error_is_the_low_precision(mode):
    n = np.array([40, 130, 256], dtype=np.int32)
    pk = inputs.cholesky_batch(n, seed=52)
    ref, _ = oracle_batch("potrf", pk)
    x, info = run("potrf", pk, mode, tc_cfg("potrf", mode.replace("raw", "refined")))
    assert np.all(info == 0)
    errs = rel_errors("potrf", pk, x, ref)
    assert np.all(errs < (2e-2 if mode == "tf32_raw" else 1e-1)), errs
    assert np.all(errs > 1e-7)   # genuinely TF32 / BF16, not an FP32 factor


@pytest.mark.parametrize("mode", TC_MODES)
def test_cholesky_tensor_memory_pivot_failures(mode):
    n = np.array([40, 200, 200, 60, 300], dtype=np.int32)
    pk = inputs.cholesky_batch(n, seed=53)
    pk.view("A", 0)[12, 12] = -100.0     # minor 13, first block
    pk.view("A", 1)[40, 40] = -1e4       # minor 41, second block of the first tile
    pk.view("A", 2)[150, 150] = -1e6     # minor 151, second TMEM tile
    pk.view("A", 3)[np.tril_indices(60, -1)] = np.nan   # never read
    pk.view("A", 4)[280, 280] = -1e6     # n > 256: blocked fallback
    ref, rinfo = oracle_batch("potrf", pk)
    x, info = run("potrf", pk, mode, tc_cfg("potrf", mode))
    assert list(info) == list(rinfo) == [13, 41, 151, 0, 281]
    nb, o = 60, int(pk.off[3])
    g = x[o:o + nb * nb].reshape(nb, nb, order="F")
    r = ref[o:o + nb * nb].reshape(nb, nb, order="F")
    assert np.linalg.norm(np.triu(g - r)) <= 1e-11 * np.linalg.norm(np.triu(r))
    assert np.all(g[np.tril_indices(nb, -1)] == SENT)


@pytest.mark.parametrize("mode", TC_MODES)
def test_cholesky_tensor_memory_scaled_instances(mode):
    n = np.array([50, 140, 256, 90, 180, 33], dtype=np.int32)
    pk = inputs.cholesky_batch(n, seed=54)
    inputs.scale_instances(pk, "potrf", inputs.range_shifts(len(n), "potrf", seed=5))
    ref, rinfo = oracle_batch("potrf", pk)
    x, info = run("potrf", pk, mode, tc_cfg("potrf", mode))
    assert np.array_equal(info, rinfo)
    assert_parity("potrf", pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("mode", TC_MODES)
def test_cholesky_tensor_memory_full_workload(mode):
    pk = inputs.make_workload("potrf_8192xLU8-256", seed=1234)
    x, info = run("potrf", pk, mode, tc_cfg("potrf", mode))
    ref, rinfo = oracle_batch("potrf", pk, threads=16)
    assert np.all(info == 0) and np.all(rinfo == 0)
    assert_parity("potrf", pk, x, ref, sentinel=SENT)


SYL_SIZES = [1, 2, 7, 16, 31, 32, 33, 48, 63, 64, 65, 96, 100, 127, 128, 129, 160]


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
@pytest.mark.parametrize("mode", TC_MODES)
def test_sylvester_lyapunov_tensor_memory_sizes(op, mode):
    n = np.array(SYL_SIZES, dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=61)
    ref, rinfo = oracle_batch(op, pk)
    x, info = run(op, pk, mode, tc_cfg(op, mode))
    assert np.array_equal(info, rinfo) and np.all(info == 0)
    assert_parity(op, pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
@pytest.mark.parametrize("mode", ["tf32_raw", "bf16_raw"])
def test_sylvester_lyapunov_tensor_memory_raw_error_is_the_low_precision(op, mode):
    n = np.array([40, 96, 128], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=62)
    ref, _ = oracle_batch(op, pk)
    x, info = run(op, pk, mode, tc_cfg(op, mode.replace("raw", "refined")))
    assert np.all(info == 0)
    errs = rel_errors(op, pk, x, ref)
    assert np.all(errs < (2e-2 if mode == "tf32_raw" else 1e-1)), errs
    assert np.all(errs > 1e-7)


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
@pytest.mark.parametrize("mode", TC_MODES)
def test_sylvester_lyapunov_tensor_memory_scaled_and_flagged(op, mode):
    n = np.array([50, 128, 90, 33, 70, 100, 10, 128], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=63)
    inputs.scale_instances(pk, op, inputs.range_shifts(len(n), op, seed=6))
    # instance 6: a tiny divisor l_ii + u_jj (info 1)
    l = pk.view("L", 6)
    if op == "trsyl":
        pk.view("U", 6)[2, 2] = -l[6, 6]
    else:
        l[3, 3] = 0.0
    ref, rinfo = oracle_batch(op, pk)
    x, info = run(op, pk, mode, tc_cfg(op, mode))
    assert info[6] == 1 and rinfo[6] == 1
    ok = np.flatnonzero(rinfo == 0)
    assert np.array_equal(info[ok], rinfo[ok])
    errs = rel_errors(op, pk, x, ref)
    assert np.all(errs[ok] <= 1e-11), errs


@pytest.mark.parametrize("name", ["trlyap_2048x128", "trsyl_4096xU4-128"])
@pytest.mark.parametrize("mode", TC_MODES)
def test_sylvester_lyapunov_tensor_memory_full_workload(name, mode):
    op = inputs.WORKLOADS[name]["op"]
    pk = inputs.make_workload(name, seed=1234)
    x, info = run(op, pk, mode, tc_cfg(op, mode))
    ref, rinfo = oracle_batch(op, pk, threads=16)
    assert np.all(info == 0) and np.all(rinfo == 0)
    assert_parity(op, pk, x, ref, sentinel=SENT)
