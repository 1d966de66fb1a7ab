"""Parity of the plain FP64 CUDA path with the CPU oracle, through the C ABI.

Gate: ||X - X_oracle||_F / ||X_oracle||_F <= 1e-11 per instance, on the same
seeded inputs; the triangle of X that an operation must not write is checked
against a sentinel; info codes are compared exactly."""
import numpy as np
import pytest

from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import assert_parity, oracle_batch, RHS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EDGE_SIZES = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 47, 63, 64, 65, 100, 127, 128, 129]
SENT = -7.25


def run(op, pk, mode=ss.MODE_FP64, cfg=ss.CFG_DEFAULT, **kw):
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op, x_fill=SENT, **kw)
    db.solve(mode=mode, cfg=cfg)
    torch.cuda.synchronize()
    return db.x_host(), db.info_host()


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
@pytest.mark.parametrize("cfg", list(range(8)))
def test_fp64_every_config_edge_sizes(op, cfg):
    if cfg >= ss.ss_config_count(ss.OPS[op], ss.MODE_FP64):
        pytest.skip("no such configuration for this operation")
    n = np.array(EDGE_SIZES, dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=10 + cfg)
    x, info = run(op, pk, cfg=cfg)
    ref, rinfo = oracle_batch(op, pk)
    assert np.array_equal(info, rinfo)
    assert_parity(op, pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
def test_fp64_mixed_sizes_default_and_table(op):
    n = inputs.sizes_uniform(300, 1, 200, seed=5)
    pk = inputs.make_batch(op, n, seed=5)
    ref, rinfo = oracle_batch(op, pk)
    x, info = run(op, pk)
    assert np.array_equal(info, rinfo)
    assert_parity(op, pk, x, ref, sentinel=SENT)
    # Per-size table: a different configuration in every bin.
    o = ss.OPS[op]
    ss.ss_set_config_table(o, ss.MODE_FP64, [k % 5 for k in range(ss.NUM_BINS)])
    try:
        x, info = run(op, pk, cfg=ss.CFG_TABLE)
    finally:
        ss.ss_set_config_table(o, ss.MODE_FP64, [])
    assert np.array_equal(info, rinfo)
    assert_parity(op, pk, x, ref, sentinel=SENT)


WS_CFGS = [c for c in range(8) if c < ss.ss_config_count(ss.OP_TRSYL, ss.MODE_FP64)
           and ss.ss_config_describe(ss.OP_TRSYL, ss.MODE_FP64, c)[2] == 2]


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
@pytest.mark.parametrize("cfg", WS_CFGS)
def test_fp64_warp_specialised_queue_and_in_place(op, cfg):
    # More instances than resident CTAs (the queue's dynamic phase), sizes
    # from one block to many with ragged edges, then the same batch in place.
    n = inputs.sizes_uniform(1100, 1, 160, seed=77)
    pk = inputs.make_batch(op, n, seed=78)
    ref, rinfo = oracle_batch(op, pk)
    x, info = run(op, pk, cfg=cfg)
    assert np.array_equal(info, rinfo)
    assert_parity(op, pk, x, ref, sentinel=SENT)
    from paper_1906_08613_gb300.device import DeviceBatch
    sub = inputs.make_batch(op, n[:64], seed=79)
    ref2, _ = oracle_batch(op, sub)
    db = DeviceBatch(sub.n, sub.off, sub.ops, op, alias_rhs=True)
    db.solve(cfg=cfg)
    torch.cuda.synchronize()
    assert np.all(db.info_host() == 0)
    assert_parity(op, sub, db.x_host(), ref2)


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
def test_fp64_in_place(op):
    n = np.array([5, 33, 70, 128], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=21)
    ref, _ = oracle_batch(op, pk)
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op, alias_rhs=True)
    db.solve()
    torch.cuda.synchronize()
    assert np.all(db.info_host() == 0)
    assert_parity(op, pk, db.x_host(), ref)


def test_cholesky_integer_exact_on_gpu():
    n = np.array([1, 3, 8, 16, 40], dtype=np.int32)
    pk = inputs.cholesky_batch(n, seed=3, exact=True)
    x, info = run("potrf", pk, cfg=3)
    assert np.all(info == 0)
    for b in range(pk.batch):
        nb, o = int(n[b]), int(pk.off[b])
        got = np.triu(x[o:o + nb * nb].reshape(nb, nb, order="F"))
        assert np.allclose(got, pk.view("X0", b), rtol=0, atol=1e-12)


def test_failure_codes_and_bad_sizes():
    # Non-SPD pivots at known positions; a singular Sylvester operator.
    n = np.array([4, 40, 6], dtype=np.int32)
    pk = inputs.cholesky_batch(n, seed=1)
    a1 = pk.view("A", 1)
    a1[37, 37] = -1e6                     # leading minor 38 fails
    a2 = pk.view("A", 2)
    a2[0, 0] = np.nan
    x, info = run("potrf", pk)
    assert list(info) == [0, 38, 1]

    pk = inputs.sylvester_batch(np.array([3, 20], dtype=np.int32), seed=2)
    l = pk.view("L", 1)
    u = pk.view("U", 1)
    u[5, 5] = -l[9, 9]                    # l_99 + u_55 = 0
    _, info = run("trsyl", pk)
    assert list(info) == [0, 1]

    # Device-side sizes above max_n or negative are skipped with info = -1.
    from paper_1906_08613_gb300.device import DeviceBatch
    pk = inputs.sylvester_batch(np.array([4, 6, 5], dtype=np.int32), seed=3)
    db = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl", max_n=5)
    db.solve()
    torch.cuda.synchronize()
    assert list(db.info_host()) == [0, ss.INFO_BAD_SIZE, 0]


def test_empty_and_zero_sized():
    from paper_1906_08613_gb300.device import DeviceBatch
    pk = inputs.sylvester_batch(np.array([0, 3, 0], dtype=np.int32), seed=4)
    db = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl")
    db.solve()
    torch.cuda.synchronize()
    assert list(db.info_host()) == [0, 0, 0]
    # batch = 0 returns immediately.
    assert ss.trsyl_lu(0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0) == 0


def test_argument_errors():
    assert ss.trsyl_lu(-1, 4, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, check=False) == -1
    assert ss.potrf_upper(1, 99999, 1, 1, 1, 1, 1, 1, check=False) == -2
    assert ss.potrf_upper(1, 4, 0, 1, 1, 1, 1, 1, check=False) == -3
    # mode out of range, cfg out of range, missing workspace
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, mode=99, check=False) == -9
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, cfg=999, check=False) == -10
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, d_work=0, check=False) == -11
    assert ss.potrf_upper(1, 4, 1, 1, 1, 1, 1, 1, d_work=1, work_bytes=1, check=False) == -12


@pytest.mark.parametrize("name", ["potrf_1024x64", "trsyl_4096xU4-128", "trlyap_2048x128",
                                  "potrf_8192xLU8-256"])
def test_fp64_full_workloads(name):
    """The measured workloads at full size, every instance checked."""
    op = inputs.WORKLOADS[name]["op"]
    pk = inputs.make_workload(name, seed=1234)
    x, info = run(op, pk)
    ref, rinfo = oracle_batch(op, pk, threads=16)
    assert np.all(info == 0) and np.all(rinfo == 0)
    assert_parity(op, pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("cfg", list(range(8)))
def test_potrf_failure_every_config(cfg):
    # A leading minor that is not positive: info = its order, the columns
    # before the failing pivot equal the oracle's, the strict lower triangle
    # of X stays untouched.
    n = np.array([12, 40, 70, 9], dtype=np.int32)
    pk = inputs.make_batch("potrf", n, seed=70 + cfg)
    fails = {0: 5, 1: 30, 2: 66}
    for b, k in fails.items():
        a = pk.view("A", b)
        a[k, k] = -1.0
    ref, rinfo = oracle_batch("potrf", pk)
    assert [int(rinfo[b]) for b in fails] == [k + 1 for k in fails.values()]
    x, info = run("potrf", pk, cfg=cfg)
    assert np.array_equal(info, rinfo)
    for b in range(pk.batch):
        nb, o = int(n[b]), int(pk.off[b])
        g = x[o:o + nb * nb].reshape(nb, nb, order="F")
        r = ref[o:o + nb * nb].reshape(nb, nb, order="F")
        good = fails.get(b, nb)
        gu, ru = np.triu(g[:, :good]), np.triu(r[:, :good])
        assert np.linalg.norm(gu - ru) <= 1e-11 * max(np.linalg.norm(ru), 1e-300)
        assert np.all(g[np.tril_indices(nb, -1)] == SENT)
