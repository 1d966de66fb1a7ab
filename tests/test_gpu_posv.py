"""Parity of the batched SPD solve (posv_upper: Cholesky factor, then
R^T Y = B and R X = Y) with the CPU oracle, through the C ABI: every Cholesky
configuration for the factor stage on ragged edge sizes and right-hand-side
counts around the 32-column chunk, a batch larger than the resident CTAs, a
non-SPD instance, out-of-range n and k, in-place R == A and X == B, and
sampled instances of the full-size workload.  Gate: relative Frobenius error
<= 1e-11 per instance for X and for the upper triangle of R; info codes equal."""
import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENT = -7.25


def run(pk, cfg=ss.CFG_DEFAULT, **kw):
    from paper_1906_08613_gb300.device import DevicePosvBatch
    db = DevicePosvBatch(pk, x_fill=SENT, **kw)
    db.solve(cfg=cfg)
    torch.cuda.synchronize()
    return db


def errs_x(pk, x, ref, idx=None):
    out = []
    for b in (range(pk.batch) if idx is None else idx):
        o, c = int(pk.offB[b]), int(pk.n[b]) * int(pk.k[b])
        r = ref[o:o + c]
        out.append(np.linalg.norm(x[o:o + c] - r) / max(np.linalg.norm(r), 1e-300) if c else 0.0)
    return np.array(out)


def errs_r(pk, r, ref, idx=None):
    out = []
    for b in (range(pk.batch) if idx is None else idx):
        nb, o = int(pk.n[b]), int(pk.offA[b])
        if nb == 0:
            out.append(0.0)
            continue
        g = np.triu(r[o:o + nb * nb].reshape(nb, nb, order="F"))
        q = np.triu(ref[o:o + nb * nb].reshape(nb, nb, order="F"))
        out.append(np.linalg.norm(g - q) / np.linalg.norm(q))
    return np.array(out)


def edge_batch(seed):
    n = [1, 2, 5, 15, 16, 17, 31, 32, 33, 64, 65, 100, 129, 16, 40, 70]
    k = [1, 3, 1, 16, 31, 32, 33, 70, 1, 16, 2, 5, 9, 64, 32, 33]
    return inputs.posv_batch(n, k, seed=seed)


@pytest.mark.parametrize("cfg", list(range(8)))
def test_posv_every_factor_config_edge_sizes(cfg):
    if cfg >= ss.ss_config_count(ss.OP_POTRF, ss.MODE_FP64):
        pytest.skip("no such configuration")
    pk = edge_batch(50 + cfg)
    xr, rr, rinfo = oracle.solve_posv_packed(pk)
    db = run(pk, cfg=cfg)
    assert np.array_equal(db.info_host(), rinfo)
    assert np.all(errs_x(pk, db.x_host(), xr) <= TOL)
    assert np.all(errs_r(pk, db.r_host(), rr) <= TOL)


@pytest.mark.parametrize("cfg", [ss.CFG_DEFAULT, 5])
def test_posv_queue_beyond_resident_ctas(cfg):
    n = inputs.sizes_uniform(1200, 1, 160, seed=61)
    k = inputs.sizes_uniform(1200, 1, 40, seed=62)
    pk = inputs.posv_batch(n, k, seed=63)
    xr, _, rinfo = oracle.solve_posv_packed(pk)
    db = run(pk, cfg=cfg)
    assert np.array_equal(db.info_host(), rinfo)
    assert np.all(errs_x(pk, db.x_host(), xr) <= TOL)


def test_posv_failures_bad_sizes_and_in_place():
    pk = inputs.posv_batch([6, 6, 8, 20, 9, 0], [2, 2, 3, 5, 70, 4], seed=64)
    a1 = pk.view("A", 1)
    a1[3, 3] = -50.0                       # not positive definite: pivot 4 fails
    xr, rr, rinfo = oracle.solve_posv_packed(pk)
    assert rinfo[1] == 4
    # device bounds: n = 20 > 19 (instance 3), k = 70 > 64 (instance 4)
    db = run(pk, max_n=19, max_k=64)
    info = db.info_host()
    assert list(info) == [0, 4, 0, ss.INFO_BAD_SIZE, ss.INFO_BAD_SIZE, 0]
    x = db.x_host()
    for b in (1, 3, 4):
        o, c = int(pk.offB[b]), int(pk.n[b]) * int(pk.k[b])
        assert np.all(x[o:o + c] == SENT)
    assert np.all(errs_x(pk, x, xr, idx=[0, 2]) <= TOL)
    from paper_1906_08613_gb300.device import DevicePosvBatch
    db = DevicePosvBatch(pk, alias=True)
    db.solve()
    torch.cuda.synchronize()
    assert list(db.info_host()) == [0, 4, 0, 0, 0, 0]
    assert np.all(errs_x(pk, db.x_host(), xr, idx=[0, 2, 3, 4]) <= TOL)
    assert np.all(errs_r(pk, db.r_host(), rr, idx=[0, 2, 3, 4]) <= TOL)


def test_posv_full_workload_sampled():
    pk = inputs.make_posv_workload("posv_4096xU8-128xk16", seed=1234)
    db = run(pk)
    assert np.all(db.info_host() == 0)
    x = db.x_host()
    rng = np.random.default_rng(65)
    idx = sorted(set(rng.choice(pk.batch, 96, replace=False).tolist()) | {int(np.argmax(pk.n))})
    xr = np.zeros_like(x)
    rr = np.zeros_like(pk.ops["A"])
    for b in idx:
        oracle.solve_posv_packed(pk, lo=b, hi=b + 1, out_x=xr, out_r=rr)
    assert np.all(errs_x(pk, x, xr, idx=idx) <= TOL)
