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


def reference_decision(op, counts, policy, X, Y, cfg_count):
    """The decision rule as the header states it, written out on the rows the
    library asked for (bins ascending, selector modes in order) and the
    network's outputs Y for them."""
    nb = len(counts)
    modes, cfgs = [-1] * nb, [-1] * nb
    rows = [(k, mi) for k in range(nb) if counts[k] > 0 for mi in range(5) if cfg_count[mi] > 0]
    assert len(rows) == len(X)
    scale = {}
    for r, (k, mi) in enumerate(rows):
        b = 2.0 ** (float(X[r][4]) * 14.0)
        scale[r] = counts[k] / round(b)
    if policy == ss.SELECTOR_PER_BIN:
        best = [np.inf] * nb
        for r, (k, mi) in enumerate(rows):
            c = int(np.argmin(Y[r, :cfg_count[mi]]))
            v = float(Y[r, c]) + np.log2(scale[r])
            if v < best[k]:
                best[k], modes[k], cfgs[k] = v, ss.SELECTOR_MODES[mi], c
        return modes, cfgs
    best = (np.inf, -1, -1)
    for mi in range(5):
        rs = [r for r, (_, m) in enumerate(rows) if m == mi]
        if not rs:
            continue
        tot = sum(scale[r] * np.exp2(Y[r, :cfg_count[mi]].astype(np.float64)) for r in rs)
        c = int(np.argmin(tot))
        if tot[c] < best[0]:
            best = (tot[c], ss.SELECTOR_MODES[mi], c)
    return [best[1]] * nb, [best[2]] * nb


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
def test_c_abi_selector_predict_follows_its_rule(op):
    s = sel.Selector.load(WEIGHTS)
    s.push()
    rng = np.random.default_rng(7)
    o = ss.OPS[op]
    cc = [min(ss.ss_config_count(o, m), int(s.cfg_counts.get(f"{op}:{mn}", 0)))
          for m, mn in zip(ss.SELECTOR_MODES, sel.MODE_ORDER)]
    for trial in range(20):
        counts = [int(c) if rng.random() < 0.5 else 0 for c in rng.integers(1, 3000, ss.NUM_BINS)]
        counts[int(rng.integers(2, 10))] += 5
        X = ss.ss_selector_queries(o, counts)
        Y = s.predict(X)                                    # the same CUDA forward kernel
        for policy in (ss.SELECTOR_PER_BIN, ss.SELECTOR_CALL):
            modes, cfgs, _ = ss.ss_selector_predict(o, counts, policy)
            assert (modes, cfgs) == reference_decision(op, counts, policy, X, Y, cc), (trial, policy)


def test_c_abi_selector_install_sets_the_auto_table():
    s = sel.Selector.load(WEIGHTS)
    s.push()
    n = inputs.sizes_log_uniform(200, 4, 200, seed=43)
    pk = inputs.make_batch("trsyl", n, seed=43)
    ref, rinfo = oracle_batch("trsyl", pk)
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl")
    ss.ss_selector_install(ss.OP_TRSYL, sel.counts_by_bin(n), ss.SELECTOR_PER_BIN)
    try:
        db.solve(mode=ss.MODE_AUTO)
        torch.cuda.synchronize()
    finally:
        ss.ss_set_auto_table(ss.OP_TRSYL, [], [])
    assert np.array_equal(db.info_host(), rinfo)
    assert_parity("trsyl", pk, db.x_host(), ref)


def test_c_abi_training_is_the_kernel_loop_and_keeps_the_bookkeeping():
    entries = tune.load(DB)["entries"]
    train, _ = sel.split_buckets(entries)
    X, T, M, _ = sel.dataset(entries, buckets=train)
    p0 = sel.init_params(3)
    steps = 150
    loss = ss.ss_selector_train(X, T, M, steps, 3e-3, init=p0)
    p_lib, cc, bm = ss.ss_selector_get()
    # The same steps by hand through ss_mlp_grad / ss_mlp_adam.
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")
    P, dX, dT, dM = dev(p0), dev(X), dev(T), dev(M)
    G, m1, m2 = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
    L = torch.zeros(1, dtype=torch.float32, device="cuda")
    wb = ss.ss_mlp_workspace_size(len(X))
    W = torch.empty(wb, dtype=torch.uint8, device="cuda")
    hand = []
    for step in range(1, steps + 1):
        ss.ss_mlp_grad(P.data_ptr(), len(X), dX.data_ptr(), dT.data_ptr(), dM.data_ptr(), float(M.sum()),
                       G.data_ptr(), L.data_ptr(), W.data_ptr(), wb)
        hand.append(float(L.item()))
        ss.ss_mlp_adam(P.data_ptr(), G.data_ptr(), m1.data_ptr(), m2.data_ptr(), step, 3e-3)
    torch.cuda.synchronize()
    assert np.array_equal(P.cpu().numpy(), p_lib)
    assert np.allclose(loss, hand, rtol=0, atol=0)
    assert loss[-1] < 0.5 * loss[0]
    s = sel.Selector(p_lib)
    s.pull()
    assert s.cfg_counts == {**{f"{o}:{m}": 0 for o in sel.OP_ORDER for m in sel.MODE_ORDER},
                            **sel.trained_cfg_counts(X, M)}
    assert s.batch_max == sel.trained_batch_max(X)


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
@pytest.mark.parametrize("mode", [ss.MODE_FP64, ss.MODE_DF])
def test_c_abi_autotune_times_every_configuration(op, mode):
    from paper_1906_08613_gb300.device import DeviceBatch
    n = tune.bucket_sizes(5, 300, seed=5)
    pk = inputs.make_batch(op, n, seed=5)
    db = DeviceBatch(pk.n, pk.off, pk.ops, op)
    ms, bad, best = db.autotune(mode, reps=3)
    assert len(ms) == ss.ss_config_count(ss.OPS[op], mode)
    assert all(t > 0 for t in ms) and all(b == 0 for b in bad)
    assert best == int(np.argmin(ms))
    # X holds the last configuration's solve.
    ref, rinfo = oracle_batch(op, pk)
    assert np.array_equal(db.info_host(), rinfo)
    assert_parity(op, pk, db.x_host(), ref)
