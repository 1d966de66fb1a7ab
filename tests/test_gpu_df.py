"""Parity of SS_MODE_DF (the warp-specialised pipelines with double-float
block updates on the FP32 pipe: Sylvester / Lyapunov with double-float
diagonal blocks and FP64 divisions, Cholesky with an FP64 diagonal warp) with
the CPU oracle, through the C ABI.

Gate: ||X - X_oracle||_F / ||X_oracle||_F <= 1e-11 per instance, as for FP64;
the mode's own bound, DF_TOL, is tighter (the split keeps about 48 bits of each
operand: an error of a few 2^-47 relative per term, far below the gate).
Info codes are compared exactly; the triangle of X that Lyapunov must not
write is checked against a sentinel."""
import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import TOL, assert_parity, oracle_batch, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EDGE_SIZES = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 47, 63, 64, 65, 100, 127, 128, 129]
SENT = -7.25
DF_TOL = 1e-12
DF = ss.MODE_DF


def run(op, pk, cfg=ss.CFG_DEFAULT, mode=DF, **kw):
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op, x_fill=SENT, **kw)
    db.solve(mode=mode, cfg=cfg)
    torch.cuda.synchronize()
    return db.x_host(), db.info_host()


def test_df_configs_are_warp_specialised():
    for op in (ss.OP_POTRF, ss.OP_TRSYL, ss.OP_TRLYAP):
        cnt = ss.ss_config_count(op, DF)
        assert cnt >= 1
        for c in range(cnt):
            # 4: the double-float pipeline; 12: its form for few CTAs per SM
            assert ss.ss_config_describe(op, DF, c)[2] in (4, 12)


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
@pytest.mark.parametrize("cfg", [0, 1, 2, 3, 4, 5])
def test_df_every_config_edge_sizes(op, cfg):
    n = np.array(EDGE_SIZES, dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=110 + cfg)
    x, info = run(op, pk, cfg=cfg)
    ref, rinfo = oracle_batch(op, pk)
    assert np.array_equal(info, rinfo)
    errs = assert_parity(op, pk, x, ref, sentinel=SENT)
    assert errs.max() <= DF_TOL, f"max rel err {errs.max():.3e}"


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
@pytest.mark.parametrize("cfg", [0, 1, 2, 3, 4, 5])
def test_df_queue_and_in_place(op, cfg):
    # More instances than resident CTAs, sizes from one block to many with
    # ragged edges; then a sub-batch in place (X == C / S).
    n = inputs.sizes_uniform(1100, 1, 160, seed=177)
    pk = inputs.make_batch(op, n, seed=178)
    ref, rinfo = oracle_batch(op, pk)
    x, info = run(op, pk, cfg=cfg)
    assert np.array_equal(info, rinfo)
    errs = assert_parity(op, pk, x, ref, sentinel=SENT)
    assert errs.max() <= DF_TOL
    from paper_1906_08613_gb300.device import DeviceBatch
    sub = inputs.make_batch(op, n[:64], seed=179)
    ref2, _ = oracle_batch(op, sub)
    db = DeviceBatch(sub.n, sub.off, sub.ops, op, alias_rhs=True)
    db.solve(mode=DF, cfg=cfg)
    torch.cuda.synchronize()
    assert np.all(db.info_host() == 0)
    assert_parity(op, sub, db.x_host(), ref2)


@pytest.mark.parametrize("name", ["trsyl_4096xU4-128", "trlyap_2048x128"])
def test_df_full_workloads(name):
    """The measured workloads at full size in the default DF configuration,
    every instance checked; the error the bench reports for this mode."""
    op = inputs.WORKLOADS[name]["op"]
    pk = inputs.make_workload(name, seed=1234)
    x, info = run(op, pk)
    ref, rinfo = oracle_batch(op, pk, threads=16)
    assert np.all(info == 0) and np.all(rinfo == 0)
    errs = assert_parity(op, pk, x, ref, sentinel=SENT)
    assert errs.max() <= DF_TOL, f"max rel err {errs.max():.3e}"


def test_df_large_orders():
    # Orders above the tuned range (many blocks per instance, long queues of
    # block products per block).
    for op in ("trsyl", "trlyap"):
        n = np.array([200, 257, 384], dtype=np.int32)
        pk = inputs.make_batch(op, n, seed=181)
        ref, rinfo = oracle_batch(op, pk)
        for cfg in (ss.CFG_DEFAULT, 3, 4, 5):     # 3..5: the few-CTAs-per-SM forms
            x, info = run(op, pk, cfg=cfg)
            assert np.array_equal(info, rinfo)
            errs = assert_parity(op, pk, x, ref, sentinel=SENT)
            assert errs.max() <= DF_TOL


def test_df_singular_divisor_and_bad_sizes():
    pk = inputs.sylvester_batch(np.array([3, 20], dtype=np.int32), seed=2)
    l = pk.view("L", 1)
    u = pk.view("U", 1)
    u[5, 5] = -l[9, 9]                    # l_99 + u_55 = 0
    _, info = run("trsyl", pk)
    assert list(info) == [0, 1]
    from paper_1906_08613_gb300.device import DeviceBatch
    pk = inputs.sylvester_batch(np.array([4, 6, 0, 5], dtype=np.int32), seed=3)
    db = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl", max_n=5)
    db.solve(mode=DF)
    torch.cuda.synchronize()
    assert list(db.info_host()) == [0, ss.INFO_BAD_SIZE, 0, 0]


def test_df_rect_edge_sizes():
    from paper_1906_08613_gb300.device import DeviceRectBatch
    rng = np.random.default_rng(405)
    sizes = [1, 2, 3, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 129]
    pairs = [(a, b) for a in (1, 16, 17, 129) for b in (1, 3, 33, 100)]
    pairs += [(int(a), int(b)) for a, b in zip(rng.choice(sizes, 24), rng.choice(sizes, 24))]
    m, n = zip(*pairs)
    pk = inputs.sylvester_rect_batch(m, n, seed=406)
    ref, rinfo = oracle.solve_rect_packed(pk)
    for cfg in range(ss.ss_config_count(ss.OP_TRSYL, DF)):
        db = DeviceRectBatch(pk, x_fill=SENT)
        db.solve(mode=DF, cfg=cfg)
        torch.cuda.synchronize()
        x, info = db.x_host(), db.info_host()
        assert np.array_equal(info, rinfo)
        for b in range(pk.batch):
            o, k = int(pk.offC[b]), int(pk.m[b]) * int(pk.n[b])
            r = ref[o:o + k]
            err = np.linalg.norm(x[o:o + k] - r) / max(np.linalg.norm(r), 1e-300)
            assert err <= DF_TOL, (cfg, b, pk.m[b], pk.n[b], err)


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
def test_df_in_auto_table_beside_fp64(op):
    # SS_MODE_AUTO with DF and FP64 bins alternating: two kinds of launch
    # group in one call.
    n = inputs.sizes_uniform(400, 1, 200, seed=190)
    pk = inputs.make_batch(op, n, seed=191)
    ref, rinfo = oracle_batch(op, pk)
    o = ss.OPS[op]
    modes = [DF if k % 2 else ss.MODE_FP64 for k in range(ss.NUM_BINS)]
    cfgs = [k % 3 if k % 2 else -1 for k in range(ss.NUM_BINS)]
    ss.ss_set_auto_table(o, modes, cfgs)
    try:
        x, info = run(op, pk, mode=ss.MODE_AUTO)
    finally:
        ss.ss_set_auto_table(o, [], [])
    assert np.array_equal(info, rinfo)
    assert_parity(op, pk, x, ref, sentinel=SENT)


def test_df_error_against_fp64_on_the_same_batch():
    # Both forms on one batch: FP64 near rounding level, DF within its bound.
    n = inputs.sizes_uniform(200, 4, 128, seed=192)
    pk = inputs.make_batch("trsyl", n, seed=193)
    ref, _ = oracle_batch("trsyl", pk)
    x64, _ = run("trsyl", pk, mode=ss.MODE_FP64)
    xdf, _ = run("trsyl", pk)
    e64 = rel_errors("trsyl", pk, x64, ref)
    edf = rel_errors("trsyl", pk, xdf, ref)
    assert e64.max() <= 1e-13
    assert edf.max() <= DF_TOL
    assert edf.max() <= TOL


# ------------------------------------------------------------------ Cholesky

@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_df_potrf_every_config_edge_sizes(cfg):
    n = np.array(EDGE_SIZES, dtype=np.int32)
    pk = inputs.make_batch("potrf", n, seed=120 + cfg)
    x, info = run("potrf", pk, cfg=cfg)
    ref, rinfo = oracle_batch("potrf", pk)
    assert np.array_equal(info, rinfo)
    errs = assert_parity("potrf", pk, x, ref, sentinel=SENT)
    assert errs.max() <= DF_TOL, f"max rel err {errs.max():.3e}"


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_df_potrf_queue_in_place_and_failures(cfg):
    n = inputs.sizes_uniform(1100, 1, 160, seed=121)
    pk = inputs.make_batch("potrf", n, seed=122)
    ref, rinfo = oracle_batch("potrf", pk)
    x, info = run("potrf", pk, cfg=cfg)
    assert np.array_equal(info, rinfo)
    errs = assert_parity("potrf", pk, x, ref, sentinel=SENT)
    assert errs.max() <= DF_TOL
    from paper_1906_08613_gb300.device import DeviceBatch
    sub = inputs.make_batch("potrf", n[:64], seed=123)
    ref2, _ = oracle_batch("potrf", sub)
    db = DeviceBatch(sub.n, sub.off, sub.ops, "potrf", alias_rhs=True)
    db.solve(mode=DF, cfg=cfg)
    torch.cuda.synchronize()
    assert np.all(db.info_host() == 0)
    assert_parity("potrf", sub, db.x_host(), ref2)
    # Leading minors that are not positive: info = their order, the columns
    # before the failing pivot as the oracle's.
    m = np.array([12, 40, 70, 9], dtype=np.int32)
    pk = inputs.make_batch("potrf", m, seed=124 + cfg)
    fails = {0: 5, 1: 30, 2: 66}
    for b, k in fails.items():
        pk.view("A", b)[k, k] = -1.0
    ref, rinfo = oracle_batch("potrf", pk)
    x, info = run("potrf", pk, cfg=cfg)
    assert np.array_equal(info, rinfo)
    for b in range(pk.batch):
        nb, o = int(m[b]), int(pk.off[b])
        g = x[o:o + nb * nb].reshape(nb, nb, order="F")
        r = ref[o:o + nb * nb].reshape(nb, nb, order="F")
        good = fails.get(b, nb)
        gu, ru = np.triu(g[:, :good]), np.triu(r[:, :good])
        assert np.linalg.norm(gu - ru) <= DF_TOL * max(np.linalg.norm(ru), 1e-300)


@pytest.mark.parametrize("name", ["potrf_1024x64", "potrf_8192xLU8-256"])
def test_df_potrf_full_workloads(name):
    pk = inputs.make_workload(name, seed=1234)
    x, info = run("potrf", pk)
    ref, rinfo = oracle_batch("potrf", pk, threads=16)
    assert np.all(info == 0) and np.all(rinfo == 0)
    errs = assert_parity("potrf", pk, x, ref, sentinel=SENT)
    assert errs.max() <= DF_TOL, f"max rel err {errs.max():.3e}"


@pytest.mark.parametrize("kmax", [16, 40])
def test_df_posv_factor_and_solves(kmax):
    # k <= 16 and k up to 40 take the 16- and 32-column chunk kernels.
    from paper_1906_08613_gb300.device import DevicePosvBatch
    n = inputs.sizes_uniform(300, 1, 140, seed=125 + kmax)
    k = inputs.sizes_uniform(300, 1, kmax, seed=126)
    pk = inputs.posv_batch(n, k, seed=127)
    xr, rr, rinfo = oracle.solve_posv_packed(pk)
    for cfg in range(ss.ss_config_count(ss.OP_POTRF, DF)):
        db = DevicePosvBatch(pk, x_fill=SENT)
        db.solve(mode=DF, cfg=cfg)
        torch.cuda.synchronize()
        assert np.array_equal(db.info_host(), rinfo)
        x = db.x_host()
        for b in range(pk.batch):
            o, c = int(pk.offB[b]), int(pk.n[b]) * int(pk.k[b])
            r = xr[o:o + c]
            err = np.linalg.norm(x[o:o + c] - r) / max(np.linalg.norm(r), 1e-300)
            assert err <= DF_TOL, (cfg, b, err)
