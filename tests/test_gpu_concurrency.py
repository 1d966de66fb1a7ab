"""Two host threads driving the library at the same time, each on its own
stream and with its own workspace: the library's host state (configuration
and AUTO tables, the auxiliary-stream pool, the launch counter) is shared, the
calls are not ordered with respect to each other, and both must still give
the oracle's results."""
import threading

import numpy as np
import pytest

from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import assert_parity, oracle_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_two_threads_two_streams():
    from paper_1906_08613_gb300.device import DeviceBatch
    jobs = []
    for k, (op, mode) in enumerate((("trsyl", ss.MODE_FP64), ("trlyap", ss.MODE_AUTO),
                                    ("potrf", ss.MODE_FP32_REFINED), ("trsyl", ss.MODE_AUTO),
                                    ("trlyap", ss.MODE_DF), ("potrf", ss.MODE_DF))):
        n = inputs.sizes_uniform(200, 1, 150, seed=90 + k)
        pk = inputs.make_batch(op, n, seed=90 + k)
        ref, rinfo = oracle_batch(op, pk)
        jobs.append((op, mode, pk, ref, rinfo))
    # AUTO tables with two launch groups each, so calls use the auxiliary streams.
    for op in ("trsyl", "trlyap"):
        ss.ss_set_auto_table(ss.OPS[op], [ss.MODE_FP64, ss.MODE_FP32_REFINED] * 6 + [ss.MODE_FP64],
                             [-1] * ss.NUM_BINS)
    errors = []

    def worker(my_jobs):
        try:
            st = torch.cuda.Stream()
            for _ in range(3):
                for op, mode, pk, ref, rinfo in my_jobs:
                    with torch.cuda.stream(st):
                        # buffers filled on st, so the solve is ordered after them
                        db = DeviceBatch(pk.n, pk.off, pk.ops, op)
                        db.ensure_work(mode)
                        db.solve(mode=mode, stream=st.cuda_stream)
                    st.synchronize()
                    assert np.array_equal(db.info_host(), rinfo)
                    assert_parity(op, pk, db.x_host(), ref)
        except Exception as e:      # noqa: BLE001 - reported below
            errors.append(e)

    try:
        l0 = ss.ss_launch_count()
        th = [threading.Thread(target=worker, args=(jobs[i::2],)) for i in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors, errors
        assert ss.ss_launch_count() > l0
    finally:
        for op in ("trsyl", "trlyap"):
            ss.ss_set_auto_table(ss.OPS[op], [], [])
