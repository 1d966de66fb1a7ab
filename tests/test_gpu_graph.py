"""A batched call captured into a CUDA graph (the library allocates and
synchronises nothing on the solve path) replays with the same results, also
in SS_MODE_AUTO with several launch groups."""
import numpy as np
import pytest

from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import assert_parity, oracle_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op,mode", [("trsyl", ss.MODE_FP64), ("potrf", ss.MODE_FP32_REFINED),
                                     ("trlyap", ss.MODE_AUTO), ("trsyl", ss.MODE_DF), ("potrf", ss.MODE_DF)])
def test_graph_capture_and_replay(op, mode):
    from paper_1906_08613_gb300.device import DeviceBatch
    n = inputs.sizes_uniform(150, 1, 140, seed=51)
    pk = inputs.make_batch(op, n, seed=51)
    ref, rinfo = oracle_batch(op, pk)
    o = ss.OPS[op]
    if mode == ss.MODE_AUTO:
        ss.ss_set_auto_table(o, [ss.MODE_FP64, ss.MODE_FP32_REFINED] * 6 + [ss.MODE_FP64],
                             [-1] * ss.NUM_BINS)
    try:
        db = DeviceBatch(pk.n, pk.off, pk.ops, op)
        db.ensure_work(mode)
        torch.cuda.synchronize()            # buffer fills (default stream) before the side stream
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            db.solve(mode=mode, stream=st.cuda_stream)      # warm-up outside capture
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            db.solve(mode=mode, stream=st.cuda_stream)
        for _ in range(2):
            db.X.zero_()
            db.info.fill_(99)
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(db.info_host(), rinfo)
            assert_parity(op, pk, db.x_host(), ref)
    finally:
        ss.ss_set_auto_table(o, [], [])


def test_graph_capture_rect_and_posv():
    import oracle
    from paper_1906_08613_gb300.device import DevicePosvBatch, DeviceRectBatch
    rk = inputs.sylvester_rect_batch(inputs.sizes_uniform(90, 1, 100, seed=52),
                                     inputs.sizes_uniform(90, 1, 100, seed=53), seed=54)
    pv = inputs.posv_batch(inputs.sizes_uniform(90, 1, 100, seed=55), inputs.sizes_uniform(90, 1, 24, seed=56),
                           seed=57)
    xr, ri = oracle.solve_rect_packed(rk)
    xp, _, pi = oracle.solve_posv_packed(pv)
    dr, dp = DeviceRectBatch(rk), DevicePosvBatch(pv)
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        dr.solve(stream=st.cuda_stream)
        dp.solve(stream=st.cuda_stream)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        dr.solve(stream=st.cuda_stream)
        dp.solve(stream=st.cuda_stream)
    for _ in range(2):
        dr.X.fill_(0.5)
        dp.X.fill_(0.5)
        dr.info.fill_(99)
        dp.info.fill_(99)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(dr.info_host(), ri) and np.array_equal(dp.info_host(), pi)
        for got, ref, offs, cnt in ((dr.x_host(), xr, rk.offC, rk.m * rk.n), (dp.x_host(), xp, pv.offB, pv.n * pv.k)):
            for o, c in zip(offs, cnt):
                gg, rr = got[int(o):int(o) + int(c)], ref[int(o):int(o) + int(c)]
                assert np.linalg.norm(gg - rr) <= 1e-11 * max(np.linalg.norm(rr), 1e-300)
