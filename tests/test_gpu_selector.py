"""The committed selector evaluated by the CUDA forward kernel chooses the same
(mode, cfg) as the FP64 oracle forward, and its AUTO tables solve a mixed
batch within the FP64 gate."""
import os

import numpy as np
import pytest

from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import selector as sel
from paper_1906_08613_gb300 import smallsolve as ss
from paper_1906_08613_gb300 import tune

from common import assert_parity, oracle_batch
from test_selector import DB, WEIGHTS, choices_with_oracle_forward

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not os.path.exists(DB), reason="no tuning database")]


def test_cuda_inference_makes_the_oracle_choices():
    s = sel.Selector.load(WEIGHTS)
    s.batch_max = None                  # the network's own argmin, as the oracle forward computes it
    entries = tune.load(DB)["entries"]
    buckets = sorted({(e["op"], e["bin"], e["batch"]) for e in entries})
    got = [(m, c) for m, c, _ in s.choose_many([(op, sel.bin_center(k), b) for op, k, b in buckets])]
    ref = choices_with_oracle_forward(s.params.astype(np.float64), buckets, s.cfg_counts)
    same = sum(g == r for g, r in zip(got, ref))
    assert same >= len(buckets) - 1     # an FP32 near-tie may flip one choice


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
def test_selector_tables_solve_within_gate(op):
    s = sel.Selector.load(WEIGHTS)
    n = inputs.sizes_log_uniform(300, 4, 300, seed=41)
    pk = inputs.make_batch(op, n, seed=41)
    ref, rinfo = oracle_batch(op, pk)
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op)
    s.install(op, sel.counts_by_bin(n))
    try:
        db.solve(mode=ss.MODE_AUTO)
        torch.cuda.synchronize()
    finally:
        ss.ss_set_auto_table(ss.OPS[op], [], [])
    assert np.array_equal(db.info_host(), rinfo)
    assert_parity(op, pk, db.x_host(), ref)
