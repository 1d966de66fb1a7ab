"""Host logic of the autotuner and the learned selector, and what the trained
selector gains, evaluated on the tuning database measured on a GB300 (no GPU
needed: the committed network is evaluated with the oracle's FP64 forward)."""
import math
import json
import os

import numpy as np
import pytest

from oracle import mlp
from paper_1906_08613_gb300 import selector as sel
from paper_1906_08613_gb300 import smallsolve as ss
from paper_1906_08613_gb300 import tune

DATA = os.path.join(os.path.dirname(sel.__file__), "data")
DB = os.path.join(DATA, "tune_gb300.json")
WEIGHTS = os.path.join(DATA, "selector_gb300")


def test_features_and_bins():
    f = sel.features("trlyap", 128, 2048, "bf16_refined")
    assert list(f[:3]) == [0, 0, 1] and list(f[5:]) == [0, 0, 0, 1, 0]
    assert list(sel.features("potrf", 8, 64, "df")[5:]) == [0, 0, 0, 0, 1]
    assert math.isclose(f[3], 7 / 9, rel_tol=1e-6) and math.isclose(f[4], 11 / 14, rel_tol=1e-6)
    assert tune.bin_range(7) == (65, 128) and tune.bin_range(0) == (1, 1)
    for n in (1, 2, 3, 64, 65, 128, 129, 4096):
        k = ss.size_bin(n)
        lo, hi = tune.bin_range(k)
        assert lo <= n <= hi
    assert sel.counts_by_bin([1, 3, 4, 100, 128]) [:8] == [1, 0, 2, 0, 0, 0, 0, 2]


def synthetic_entries():
    # fp64 cfg 1 fastest in small bins, cfg 3 in large; one refined mode wins bin 6.
    out = []
    for k in range(2, 8):
        for mode, ncfg in (("fp64", 8), ("fp32_refined", 3)):
            for c in range(ncfg):
                ms = 1.0 + abs(c - (1 if k < 5 else 3)) + (0.5 if mode != "fp64" else 0.0)
                if k == 6 and mode == "fp32_refined" and c == 2:
                    ms = 0.5
                out.append(dict(op="trsyl", bin=k, batch=256, mode=mode, cfg=c, ms=ms, info_nonzero=0))
    return out


def test_dataset_exhaustive_table_and_regret():
    ent = synthetic_entries()
    X, T, M, keys = sel.dataset(ent)
    assert X.shape == (12, ss.MLP_IN) and M.sum() == 6 * (8 + 3)
    modes, cfgs = tune.exhaustive_table(ent, "trsyl", 256)
    assert modes[6] == ss.MODE_FP32_REFINED and cfgs[6] == 2
    assert modes[3] == ss.MODE_FP64 and cfgs[3] == 1 and cfgs[7] == 3 and modes[9] == -1
    buckets = [("trsyl", k, 256) for k in range(2, 8)]
    rep = sel.regret_report([("fp64", 1)] * 6, ent, buckets)
    assert rep["buckets"] == 6 and rep["max_regret"] > 0 and rep["mean_regret"] > 0


def choices_with_oracle_forward(params, buckets, cfg_counts):
    out = []
    for op, k, batch in buckets:
        best = None
        for mode in sel.MODE_ORDER:
            cnt = min(ss.ss_config_count(ss.OPS[op], ss.MODES[mode]), cfg_counts.get(f"{op}:{mode}", 0))
            if cnt <= 0:
                continue
            y, _ = mlp.forward(params, sel.features(op, sel.bin_center(k), batch, mode)[None, :])
            c = int(np.argmin(y[0, :cnt]))
            if best is None or y[0, c] < best[2]:
                best = (mode, c, y[0, c])
        out.append(best[:2])
    return out


@pytest.mark.skipif(not os.path.exists(DB), reason="no tuning database")
def test_trained_selector_gain_and_regret_on_measured_gb300_timings():
    entries = tune.load(DB)["entries"]
    params = np.load(WEIGHTS + ".npy").astype(np.float64)
    with open(WEIGHTS + ".json") as f:
        counts = json.load(f)["cfg_counts"]
    train, held = (sorted(x) for x in sel.split_buckets(entries))
    r_held = sel.regret_report(choices_with_oracle_forward(params, held, counts), entries, held)
    r_train = sel.regret_report(choices_with_oracle_forward(params, train, counts), entries, train)
    # The network never saw the held-out buckets; it must stay near the
    # exhaustive search there and beat the built-in FP64 default on both sets.
    assert r_held["buckets"] == len(held) > 0
    assert r_held["geomean_gain_over_default"] >= 1.0
    assert r_held["mean_regret"] <= 0.10
    assert r_train["geomean_gain_over_default"] >= 1.0
    assert r_train["mean_regret"] <= 0.05


def timings(entries):
    return {(e["op"], e["bin"], e["batch"], e["mode"], e["cfg"]): e["ms"]
            for e in entries if not e.get("info_nonzero", 0)}


def best_fixed_policy(T, op, buckets):
    """The single (mode, cfg) with the smallest geometric-mean time over the
    given buckets of op (among those measured in all of them): the method
    without a model, tuned on the same training data as the network."""
    bks = [b for b in buckets if b[0] == op]
    best = None
    for mc in sorted({k[3:] for k in T if k[0] == op}):
        ts = [T.get(b + mc) for b in bks]
        if any(t is None for t in ts):
            continue
        g = float(np.exp(np.mean(np.log(ts))))
        if best is None or g < best[1]:
            best = (mc, g)
    return best[0]


def test_best_fixed_policy_picks_the_cheapest_common_choice():
    T = {("trsyl", 2, 256, "fp64", 0): 1.0, ("trsyl", 2, 256, "df", 2): 0.5,
         ("trsyl", 3, 256, "fp64", 0): 2.0, ("trsyl", 3, 256, "df", 2): 3.0,
         ("trsyl", 3, 256, "df", 1): 0.1}                       # not measured in bin 2
    # Over both buckets: geomean(fp64 0) = sqrt(2) = 1.414, geomean(df 2) =
    # sqrt(1.5) = 1.225; df 1 is not measured in bin 2 and cannot be chosen.
    got = best_fixed_policy(T, "trsyl", [("trsyl", 2, 256), ("trsyl", 3, 256)])
    assert got == ("df", 2)
    assert best_fixed_policy(T, "trsyl", [("trsyl", 3, 256)]) == ("df", 1)
    assert best_fixed_policy(T, "trsyl", [("trsyl", 2, 256)]) == ("df", 2)


@pytest.mark.skipif(not os.path.exists(DB), reason="no tuning database")
def test_selector_beats_the_best_fixed_policy_on_heldout_buckets():
    """What the network itself adds: against the best single (mode, cfg) per
    operation, chosen on the training buckets only (so it includes "always
    the double-float default" if that is best there), on buckets neither of
    them was fitted on."""
    entries = tune.load(DB)["entries"]
    params = np.load(WEIGHTS + ".npy").astype(np.float64)
    with open(WEIGHTS + ".json") as f:
        counts = json.load(f)["cfg_counts"]
    train, held = (sorted(x) for x in sel.split_buckets(entries))
    assert not set(train) & set(held)
    T = timings(entries)
    fixed = {op: best_fixed_policy(T, op, train) for op in tune.OPS}
    gains = []
    for (op, k, b), (m, c) in zip(held, choices_with_oracle_forward(params, held, counts)):
        gains.append(T[(op, k, b) + fixed[op]] / T[(op, k, b, m, c)])
    g = float(np.exp(np.mean(np.log(gains))))
    assert g >= 1.0, (g, fixed)
    # per operation too
    for op in tune.OPS:
        sub = [x for (o, _, _), x in zip(held, gains) if o == op]
        assert float(np.exp(np.mean(np.log(sub)))) >= 1.0, (op, fixed[op])


def test_trained_cfg_counts_follow_the_mask():
    ent = synthetic_entries()
    X, T, M, keys = sel.dataset(ent)
    c = sel.trained_cfg_counts(X, M)
    for key in {f"{op}:{mode}" for op, _, _, mode in keys}:
        op, mode = key.split(":")
        want = 1 + max(e["cfg"] for e in ent if e["op"] == op and e["mode"] == mode)
        assert c[key] == want


def test_split_holds_out_every_third_cell_with_trained_neighbours():
    ent = [dict(op=op, bin=k, batch=b) for op in ("potrf", "trsyl") for k in range(2, 10)
           for b in ((256, 2048) if k <= 7 else (64, 256))]
    train, held = sel.split_buckets(ent)
    assert train and held and not (train & held)
    assert len(train | held) == len(ent)
    for op, k, b in held:
        assert any(t[0] == op and abs(t[1] - k) == 1 for t in train)
        assert any(t[0] == op and t[1] == k and t[2] != b for t in train)


def test_tuner_merge_replaces_only_swept_buckets():
    old = [dict(op="trsyl", bin=8, batch=256, mode="fp64", cfg=0, ms=1.0),
           dict(op="trsyl", bin=8, batch=256, mode="df", cfg=0, ms=2.0),
           dict(op="trsyl", bin=8, batch=1024, mode="df", cfg=0, ms=9.0),
           dict(op="potrf", bin=8, batch=1024, mode="df", cfg=0, ms=3.0)]
    new = [dict(op="trsyl", bin=8, batch=1024, mode="df", cfg=0, ms=4.0),
           dict(op="trsyl", bin=8, batch=1024, mode="df", cfg=1, ms=5.0)]
    got = tune.merge_entries(old, new)
    keys = [(e["op"], e["bin"], e["batch"], e["mode"], e["cfg"], e["ms"]) for e in got]
    assert ("trsyl", 8, 1024, "df", 0, 9.0) not in keys          # replaced
    assert ("trsyl", 8, 1024, "df", 0, 4.0) in keys and ("trsyl", 8, 1024, "df", 1, 5.0) in keys
    assert ("trsyl", 8, 256, "df", 0, 2.0) in keys and ("potrf", 8, 1024, "df", 0, 3.0) in keys
    assert len(got) == 5


def test_trained_batch_max_per_size_bin_and_mode():
    ent = [dict(op="trsyl", bin=8, batch=b, mode=m, cfg=0, ms=1.0, info_nonzero=0)
           for b, m in ((64, "fp64"), (256, "fp64"), (1024, "fp64"), (64, "df"), (256, "df"))]
    X, _, _, _ = sel.dataset(ent)
    bm = sel.trained_batch_max(X)
    assert bm == {"trsyl:8:fp64": 1024, "trsyl:8:df": 256}


def fixed_predictions(table):
    """A stand-in for the network: log2 ms per mode as a function of the
    batch feature, the same for every configuration slot."""
    def f(X):
        out = np.zeros((len(X), ss.MLP_OUT), dtype=np.float32)
        for i, x in enumerate(np.asarray(X)):
            mode = sel.MODE_ORDER[int(np.argmax(x[5:5 + len(sel.MODE_ORDER)]))]
            batch = 2.0 ** (float(x[4]) * 14.0)
            out[i, :] = table[mode](batch)
        return out
    return f


def test_selector_scales_predictions_beyond_the_trained_batch():
    # The library's decision (ss_selector_queries / ss_selector_decide, host
    # code) on predictions from a table.  In bin 8 the network saw DF only up
    # to 256 instances and FP64 up to 1024.  Its DF prediction flattens out
    # beyond 256 (a latency-bound time carried into the throughput-bound
    # regime); with batch_max the DF prediction is taken at 256 and scaled by
    # count / 256 instead.
    table = {"fp64": lambda b: math.log2(2.0 + 0.008 * b),
             "df": lambda b: math.log2(3.0 if b <= 256 else 3.0 + 0.0001 * b)}
    f = fixed_predictions(table)
    s = sel.Selector()
    s.cfg_counts = {"trsyl:fp64": 1, "trsyl:df": 1}
    counts = [0] * ss.NUM_BINS
    counts[8] = 200
    assert s.decide_with(f, "trsyl", counts, ss.SELECTOR_CALL)[0][8] == ss.MODE_DF   # 3.0 ms vs 3.6 ms
    counts[8] = 1024
    assert s.decide_with(f, "trsyl", counts, ss.SELECTOR_CALL)[0][8] == ss.MODE_DF   # unscaled: 3.1 vs 10.2 ms
    s.batch_max = {"trsyl:8:fp64": 1024, "trsyl:8:df": 256}
    modes, cfgs, ms = s.decide_with(f, "trsyl", counts, ss.SELECTOR_CALL)
    assert modes == [ss.MODE_FP64] * ss.NUM_BINS and cfgs == [0] * ss.NUM_BINS      # DF: 3 ms x 4 = 12 ms
    assert math.isclose(ms, 2.0 + 0.008 * 1024, rel_tol=1e-5)
    # The per-bin choice applies the same rule; bins without instances stay unset.
    modes, _, _ = s.decide_with(f, "trsyl", counts, ss.SELECTOR_PER_BIN)
    assert modes[8] == ss.MODE_FP64 and modes[7] == -1
    counts[8] = 200
    modes, _, _ = s.decide_with(f, "trsyl", counts, ss.SELECTOR_PER_BIN)
    assert modes[8] == ss.MODE_DF


def test_selector_decision_rows_and_argmin():
    # Rows: every (bin with instances, mode with configurations), features as
    # documented; the argmin picks the smallest slot within the mode's count.
    s = sel.Selector()
    s.cfg_counts = {"trlyap:fp64": 3, "trlyap:df": 2}
    counts = [0] * ss.NUM_BINS
    counts[3], counts[6] = 10, 300
    s.push()
    X = ss.ss_selector_queries(ss.OP_TRLYAP, counts)
    assert X.shape == (4, ss.MLP_IN)
    want = [sel.features("trlyap", sel.bin_center(k), counts[k], m) for k in (3, 6) for m in ("fp64", "df")]
    assert np.array_equal(X, np.array(want))
    Y = np.full((4, ss.MLP_OUT), 5.0, dtype=np.float32)
    Y[0, :] = [4, 3, 2, -9, -9, -9, -9, -9]    # bin 3 fp64: slot 2 (slots >= 3 are not configurations)
    Y[1, :2] = [2.5, 2.1]                       # bin 3 df: slot 1 (2.1 > 2.0)
    Y[2, :3] = [1, 0, 1]                        # bin 6 fp64: slot 1 (0)
    Y[3, :2] = [-1, 3]                          # bin 6 df: slot 0 (-1)
    modes, cfgs, ms = ss.ss_selector_decide(ss.OP_TRLYAP, counts, ss.SELECTOR_PER_BIN, Y)
    assert (modes[3], cfgs[3], modes[6], cfgs[6]) == (ss.MODE_FP64, 2, ss.MODE_DF, 0)
    assert math.isclose(ms, 2 ** 2 + 2 ** -1)
    # One choice for the call: fp64 totals 2^[4,3,2] + 2^[1,0,1]; df 2^[2.5,2.1] + 2^[-1,3].
    modes, cfgs, ms = ss.ss_selector_decide(ss.OP_TRLYAP, counts, ss.SELECTOR_CALL, Y)
    tot_fp = [2 ** 4 + 2, 2 ** 3 + 1, 2 ** 2 + 2]
    tot_df = [2 ** 2.5 + 0.5, 2 ** 2.1 + 8]
    assert min(tot_fp) < min(tot_df)
    assert modes == [ss.MODE_FP64] * ss.NUM_BINS and cfgs == [int(np.argmin(tot_fp))] * ss.NUM_BINS
    assert math.isclose(ms, min(tot_fp), rel_tol=1e-12)


def test_selector_save_load_roundtrip(tmp_path):
    s = sel.Selector.load(WEIGHTS) if os.path.exists(WEIGHTS + ".npy") else sel.Selector()
    s.push()
    path = str(tmp_path / "model.bin")
    ss.ss_selector_save(path)
    p0, cc0, bm0 = ss.ss_selector_get()
    ss.ss_selector_clear()
    with pytest.raises(ss.SmallSolveError):
        ss.ss_selector_get()
    ss.ss_selector_load(path)
    p1, cc1, bm1 = ss.ss_selector_get()
    assert np.array_equal(p0, p1) and cc0 == cc1 and bm0 == bm1
    assert np.array_equal(p1, s.params.astype(np.float32))
    bad = str(tmp_path / "short.bin")
    with open(path, "rb") as f, open(bad, "wb") as g:
        g.write(f.read()[:100])
    with pytest.raises(ss.SmallSolveError):
        ss.ss_selector_load(bad)


def test_tuning_grid():
    b = tune.default_buckets(9)
    for op in tune.OPS:
        for k in range(2, 10):
            got = sorted(x[2] for x in b if x[0] == op and x[1] == k)
            assert got == ([256, 1024, 2048] if k <= 7 else [64, 256, 1024])
    # The committed database covers the grid for FP64 and DF.
    entries = tune.load(DB)["entries"]
    have = {(e["op"], e["bin"], e["batch"], e["mode"]) for e in entries}
    for op, k, batch in b:
        assert (op, k, batch, "fp64") in have
        if op != "potrf" or ss.ss_config_count(ss.OP_POTRF, ss.MODE_DF) > 0:
            assert (op, k, batch, "df") in have
