"""Parity of the rectangular FP64 Sylvester solve (trsyl_rect: L m x m, U n x n,
X m x n) with the CPU oracle, through the C ABI: every Sylvester
configuration on ragged edge sizes, a batch larger than the resident CTAs,
empty and out-of-range sizes, in-place X == C, a singular divisor, and
sampled instances of the full-size workload.  Gate: relative Frobenius error
<= 1e-11 per instance; info codes equal."""
import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENT = -7.25
EDGE = [1, 2, 3, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 129]


def edge_pairs():
    rng = np.random.default_rng(404)
    pairs = [(a, b) for a in (1, 16, 17, 129) for b in (1, 3, 33, 100)]
    pairs += [(int(a), int(b)) for a, b in zip(rng.choice(EDGE, 24), rng.choice(EDGE, 24))]
    return pairs


def run(pk, cfg=ss.CFG_DEFAULT, **kw):
    from paper_1906_08613_gb300.device import DeviceRectBatch
    db = DeviceRectBatch(pk, x_fill=SENT, **kw)
    db.solve(cfg=cfg)
    torch.cuda.synchronize()
    return db, db.x_host(), db.info_host()


def rel_errs(pk, x, ref, idx=None):
    out = []
    for b in (range(pk.batch) if idx is None else idx):
        o, k = int(pk.offC[b]), int(pk.m[b]) * int(pk.n[b])
        r = ref[o:o + k]
        out.append(np.linalg.norm(x[o:o + k] - r) / max(np.linalg.norm(r), 1e-300) if k else 0.0)
    return np.array(out)


SYL_CFGS = list(range(8))


@pytest.mark.parametrize("cfg", SYL_CFGS)
def test_rect_every_config_edge_sizes(cfg):
    if cfg >= ss.ss_config_count(ss.OP_TRSYL, ss.MODE_FP64):
        pytest.skip("no such configuration")
    m, n = zip(*edge_pairs())
    pk = inputs.sylvester_rect_batch(m, n, seed=30 + cfg)
    ref, rinfo = oracle.solve_rect_packed(pk)
    _, x, info = run(pk, cfg=cfg)
    assert np.array_equal(info, rinfo)
    errs = rel_errs(pk, x, ref)
    assert np.all(errs <= TOL), f"max rel err {errs.max():.3e} at {int(np.argmax(errs))}"


@pytest.mark.parametrize("cfg", [ss.CFG_DEFAULT, 2, 5, 6])
def test_rect_queue_beyond_resident_ctas(cfg):
    m = inputs.sizes_uniform(1300, 1, 160, seed=91)
    n = inputs.sizes_uniform(1300, 1, 160, seed=92)
    pk = inputs.sylvester_rect_batch(m, n, seed=93)
    ref, rinfo = oracle.solve_rect_packed(pk)
    _, x, info = run(pk, cfg=cfg)
    assert np.array_equal(info, rinfo)
    assert np.all(rel_errs(pk, x, ref) <= TOL)


def test_rect_empty_bad_sizes_and_in_place():
    m = np.array([0, 5, 7, 40, 3, 20], dtype=np.int32)
    n = np.array([6, 0, 9, 20, 50, 30], dtype=np.int32)
    pk = inputs.sylvester_rect_batch(m, n, seed=94)
    ref, _ = oracle.solve_rect_packed(pk)
    # device bounds below two instances' sizes: m = 40 > 39 (index 3), n = 50 > 49 (index 4)
    db, x, info = run(pk, max_m=39, max_n=49)
    assert list(info) == [0, 0, 0, ss.INFO_BAD_SIZE, ss.INFO_BAD_SIZE, 0]
    for b in (3, 4):
        o, k = int(pk.offC[b]), int(m[b]) * int(n[b])
        assert np.all(x[o:o + k] == SENT)
    assert np.all(rel_errs(pk, x, ref, idx=[2, 5]) <= TOL)
    from paper_1906_08613_gb300.device import DeviceRectBatch
    db = DeviceRectBatch(pk, alias_rhs=True)
    db.solve()
    torch.cuda.synchronize()
    assert np.all(db.info_host() == 0)
    assert np.all(rel_errs(pk, db.x_host(), ref, idx=[2, 3, 4, 5]) <= TOL)


def test_rect_singular_divisor_info():
    pk = inputs.sylvester_rect_batch([6, 6], [4, 4], seed=95)
    L = pk.view("L", 1)
    U = pk.view("U", 1)
    L[2, 2] = -U[3, 3]              # divisor l_22 + u_33 = 0 exactly
    ref, rinfo = oracle.solve_rect_packed(pk)
    assert list(rinfo) == [0, 1]
    _, x, info = run(pk)
    assert list(info) == [0, 1]
    assert rel_errs(pk, x, ref, idx=[0])[0] <= TOL


@pytest.mark.parametrize("cfg", [ss.CFG_DEFAULT, 6])
def test_rect_full_workload_sampled(cfg):
    pk = inputs.make_rect_workload("trsyl_rect_4096xU4-128xU4-128", seed=1234)
    _, x, info = run(pk, cfg=cfg)
    assert np.all(info == 0)
    rng = np.random.default_rng(96)
    idx = sorted(set(rng.choice(pk.batch, 96, replace=False).tolist()) | {int(np.argmax(pk.m * pk.n))})
    ref = np.zeros_like(x)
    for b in idx:
        oracle.solve_rect_packed(pk, out=ref, lo=b, hi=b + 1)
    assert np.all(rel_errs(pk, x, ref, idx=idx) <= TOL)
