"""Large instances next to small ones, and the largest size bound: one
persistent CTA then works through hundreds of blocks of one instance (the
blocked paths stream L, U and X through L2), while the scheduler starts it
first.  Orders ~1000 keep the oracle at a few seconds; max_n = SS_MAX_N
exercises the binning pass at its largest histogram."""
import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import assert_parity, oracle_batch, TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op,big", [("trsyl", 1000), ("trlyap", 700), ("potrf", 1500)])
@pytest.mark.parametrize("mode", [ss.MODE_FP64, ss.MODE_FP32_REFINED])
def test_large_instance_among_small(op, big, mode):
    from paper_1906_08613_gb300.device import DeviceBatch
    n = np.array([big, 3, 40, 129, 17], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=81)
    ref, rinfo = oracle_batch(op, pk)
    db = DeviceBatch(pk.n, pk.off, pk.ops, op)
    db.solve(mode=mode)
    torch.cuda.synchronize()
    assert np.array_equal(db.info_host(), rinfo)
    assert_parity(op, pk, db.x_host(), ref)


def test_max_size_bound_with_small_instances():
    from paper_1906_08613_gb300.device import DeviceBatch
    n = inputs.sizes_uniform(300, 1, 64, seed=82)
    pk = inputs.make_batch("trsyl", n, seed=83)
    ref, rinfo = oracle_batch("trsyl", pk)
    db = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl", max_n=ss.MAX_N)
    db.solve()
    torch.cuda.synchronize()
    assert np.array_equal(db.info_host(), rinfo)
    assert_parity("trsyl", pk, db.x_host(), ref)


def test_large_rect_and_posv():
    from paper_1906_08613_gb300.device import DevicePosvBatch, DeviceRectBatch
    rk = inputs.sylvester_rect_batch([1000, 40, 5], [40, 900, 5], seed=84)
    xr, ri = oracle.solve_rect_packed(rk)
    dr = DeviceRectBatch(rk)
    dr.solve()
    pv = inputs.posv_batch([1000, 33], [100, 3], seed=85)
    xp, _, pi = oracle.solve_posv_packed(pv)
    dp = DevicePosvBatch(pv)
    dp.solve()
    torch.cuda.synchronize()
    assert np.array_equal(dr.info_host(), ri) and np.array_equal(dp.info_host(), pi)
    for got, ref, offs, cnt in ((dr.x_host(), xr, rk.offC, rk.m * rk.n), (dp.x_host(), xp, pv.offB, pv.n * pv.k)):
        for o, c in zip(offs, cnt):
            g, r = got[int(o):int(o) + int(c)], ref[int(o):int(o) + int(c)]
            assert np.linalg.norm(g - r) <= TOL * np.linalg.norm(r)
