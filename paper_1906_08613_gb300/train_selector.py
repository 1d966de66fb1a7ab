"""Train the learned selector on autotuner timings and measure what it gains.

Steps (one GPU):
  1. the autotuner's database (``--db``; ``--sweep`` measures it first);
  2. training rows = all (op, size bin, batch) buckets but every third
     (bin, batch rank) cell, which is held out (selector.split_buckets);
  3. the MLP is trained on the GPU by the library's own kernels;
  4. regret of the selector's choice against the exhaustive best, per bucket,
     on training and held-out buckets, and its gain over the FP64 default;
  5. the held-out stream: 16384 instances, operation uniform over the three,
     n log-uniform in [4, 512]; each operation's share is solved in one call
     with SS_MODE_AUTO driven by (a) the selector, (b) the exhaustive table,
     (c) FP64 with the default configuration, (d) the best single (mode, cfg)
     chosen on the training buckets, and all are timed.

Usage:  python -m paper_1906_08613_gb300.train_selector --db DB.json --out PREFIX [--sweep]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import inputs
from . import selector as sel
from . import smallsolve as ss
from . import tune


def stream_sizes(total: int, seed: int):
    """Operation and order of each instance of the held-out stream."""
    rng = np.random.default_rng([seed, 5])
    ops = rng.integers(0, 3, size=total)
    n = inputs.sizes_log_uniform(total, 4, 512, seed)
    return ops, n


def time_auto(db, reps=3):
    import torch
    db.solve(mode=ss.MODE_AUTO)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        db.solve(mode=ss.MODE_AUTO)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), db.info_host()


def evaluate_stream(selector, entries, total=16384, seed=2026, log=print):
    import torch
    from .device import DeviceBatch
    ops_idx, n = stream_sizes(total, seed)
    res = {}
    for oi, op in enumerate(sel.OP_ORDER):
        nn = n[ops_idx == oi]
        pk = inputs.make_batch(op, nn, seed=seed + oi)
        db = DeviceBatch(pk.n, pk.off, pk.ops, op)
        db.ensure_work(ss.MODE_AUTO)
        o = ss.OPS[op]
        row = {"instances": int(len(nn))}
        # (c) FP64 default configuration: an empty AUTO table.
        ss.ss_set_auto_table(o, [], [])
        row["fp64_default_ms"], info = time_auto(db)
        row["fp64_default_bad"] = int((info != 0).sum())
        counts = sel.counts_by_bin(nn)
        # (b) exhaustive autotune table.
        m, c = tune.exhaustive_table(entries, op, counts)
        ss.ss_set_auto_table(o, m, c)
        row["exhaustive_ms"], info = time_auto(db)
        row["exhaustive_table"] = list(zip(m, c))
        # (b') exhaustive search over single (mode, cfg) choices for the call.
        ex = tune.exhaustive_call_choice(entries, op, counts)
        if ex is not None:
            mm = [ss.MODES[ex[0]]] * ss.NUM_BINS
            cc = [ex[1]] * ss.NUM_BINS
            ss.ss_set_auto_table(o, mm, cc)
            row["exhaustive_call_ms"], _ = time_auto(db)
            row["exhaustive_call_choice"] = ex[:2]
        # (d) the best single (mode, cfg) chosen on the training buckets.
        train_set, _ = sel.split_buckets(entries)
        fx = sel.best_fixed_policy(entries, op, train_set)
        if fx is not None:
            ss.ss_set_auto_table(o, [ss.MODES[fx[0]]] * ss.NUM_BINS, [fx[1]] * ss.NUM_BINS)
            row["fixed_policy_ms"], _ = time_auto(db)
            row["fixed_policy"] = fx
        # (a) learned selector: per-bin table, and one choice for the call.
        m, c = selector.auto_table(op, counts)
        ss.ss_set_auto_table(o, m, c)
        row["selector_per_bin_ms"], _ = time_auto(db)
        row["selector_per_bin_table"] = list(zip(m, c))
        m, c = selector.call_table(op, counts)
        ss.ss_set_auto_table(o, m, c)
        row["selector_ms"], info = time_auto(db)
        row["selector_bad"] = int((info != 0).sum())
        row["selector_table"] = list(zip(m, c))
        ss.ss_set_auto_table(o, [], [])
        best_ex = min(row["exhaustive_ms"], row.get("exhaustive_call_ms", float("inf")))
        row["regret"] = row["selector_ms"] / best_ex - 1.0
        row["gain_over_fp64_default"] = row["fp64_default_ms"] / row["selector_ms"]
        if "fixed_policy_ms" in row:
            row["gain_over_fixed_policy"] = row["fixed_policy_ms"] / row["selector_ms"]
        log(f"stream {op}: {row['instances']} inst  fp64-default {row['fp64_default_ms']:.2f} ms  "
            f"exhaustive per-bin {row['exhaustive_ms']:.2f} ms  exhaustive call {row.get('exhaustive_call_ms', float('nan')):.2f} ms  "
            f"selector per-bin {row['selector_per_bin_ms']:.2f} ms  selector call {row['selector_ms']:.2f} ms  "
            f"regret {row['regret']:+.3f}  gain {row['gain_over_fp64_default']:.3f}")
        res[op] = row
        del db
        torch.cuda.empty_cache()
    tot = {k: sum(r.get(k, 0.0) for r in res.values())
           for k in ("fp64_default_ms", "exhaustive_ms", "exhaustive_call_ms", "selector_per_bin_ms", "selector_ms",
                     "fixed_policy_ms")}
    # Regret against the better exhaustive policy of each operation.
    best_ex = sum(min(r["exhaustive_ms"], r.get("exhaustive_call_ms", float("inf"))) for r in res.values())
    res["total"] = {**tot, "exhaustive_best_ms": best_ex, "regret": tot["selector_ms"] / best_ex - 1.0,
                    "gain_over_fp64_default": tot["fp64_default_ms"] / tot["selector_ms"],
                    "gain_over_fixed_policy": (tot["fixed_policy_ms"] / tot["selector_ms"]) if tot["fixed_policy_ms"] else None,
                    "solves_per_s_selector": total / (tot["selector_ms"] * 1e-3)}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--db", required=True)
    ap.add_argument("--out", required=True, help="prefix of the selector files (.npy/.json)")
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--report", default=None)
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--load", default=None, help="evaluate an existing selector instead of training")
    args = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)
    if args.sweep:
        t0 = time.time()
        entries = tune.sweep(tune.default_buckets(), log=log)
        tune.save(entries, args.db, {"sweep_seconds": time.time() - t0})
    entries = tune.load(args.db)["entries"]

    train_set, held_set = sel.split_buckets(entries)
    X, T, M, keys = sel.dataset(entries, buckets=train_set)
    log(f"training rows {len(keys)}, observed targets {int(M.sum())}")
    t0 = time.time()
    if args.load:
        s = sel.Selector.load(args.load)
        hist = [(0, float("nan"))]
    else:
        s = sel.Selector(sel.init_params(0))
        hist = s.train(X, T, M, steps=args.steps, lr=args.lr, log_every=500, log=log)
    train_s = time.time() - t0

    def report_for(bucket_set):
        buckets = sorted(bucket_set)
        choices = s.choose_many([(op, sel.bin_center(k), b) for op, k, b in buckets])
        return sel.regret_report([(m, c) for m, c, _ in choices], entries, buckets)

    rep = {"train_rows": len(keys), "train_seconds": train_s, "loss_history": hist,
           "train_buckets": report_for(train_set), "heldout_buckets": report_for(held_set)}
    for name in ("train_buckets", "heldout_buckets"):
        r = rep[name]
        if r.get("buckets"):
            log(f"{name}: {r['buckets']} buckets, mean regret {r['mean_regret']:.3f}, "
                f"max regret {r['max_regret']:.3f}, gain over FP64 default "
                f"{r['geomean_gain_over_default']:.3f}")
    if not args.no_stream:
        rep["stream"] = evaluate_stream(s, entries, log=log)
    s.save(args.out, trained_on=args.db, steps=args.steps, lr=args.lr,
           final_loss=hist[-1][1], split="every third (bin, batch rank) bucket held out")
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1, default=lambda o: o.tolist() if hasattr(o, "tolist") else str(o))
    return 0


if __name__ == "__main__":
    sys.exit(main())
