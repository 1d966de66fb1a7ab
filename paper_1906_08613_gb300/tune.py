"""Autotuner: exhaustive timing of every (precision mode, kernel configuration)
for buckets of (operation, size bin, batch), and the tuning database.

This is the search loop of the paper's generator ("Generator structure"
paragraph: autotuning selects the fastest code among alternative algorithms and
implementation parameters), over this library's axes: algorithm variant x block
size x threads per CTA x precision mode.  Only modes that meet the FP64
accuracy gate are candidates (FP64, the *_REFINED modes and DF).

A bucket's instances have order n uniform over the size bin
(2^(k-1), 2^k] and are solved in one call; the time is the median of a few
CUDA-event-timed calls after a warm-up (the library's ss_autotune).  The database is JSON:

    {"gpu": ..., "created": ..., "entries": [
        {"op": "trsyl", "bin": 7, "n_lo": 65, "n_hi": 128, "batch": 2048,
         "mode": "fp64", "cfg": 2, "ms": 1.23}, ...]}

Usage (on a GPU):  python -m paper_1906_08613_gb300.tune --out DB.json
            [--ops trsyl,trlyap --modes df --merge OLD.json]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import inputs
from . import smallsolve as ss

AUTO_MODES = ("fp64", "fp32_refined", "tf32_refined", "bf16_refined", "df")
OPS = ("potrf", "trsyl", "trlyap")


def bin_range(k: int):
    """Orders n with bin(n) = k: k = 0 -> {1}, else (2^(k-1), 2^k]."""
    if k == 0:
        return 1, 1
    return (1 << (k - 1)) + 1, 1 << k


def default_buckets(max_bin: int = 9):
    """(op, bin, batch) buckets: three batch counts per bin, 256 / 1024 / 2048
    up to n = 128 and 64 / 256 / 1024 above (a mixed stream of n up to 512
    puts several hundred instances in each of those bins, where the kernels
    move from latency- to throughput-bound).  With three counts per bin a
    held-out count has a trained one on either side or both, so the selector
    interpolates in batch where configurations of different occupancy cross."""
    out = []
    for op in OPS:
        for k in range(2, max_bin + 1):
            batches = (256, 1024, 2048) if k <= 7 else (64, 256, 1024)
            for b in batches:
                out.append((op, k, b))
    return out


def bucket_sizes(k: int, batch: int, seed: int) -> np.ndarray:
    lo, hi = bin_range(k)
    rng = np.random.default_rng([seed, k, batch])
    return rng.integers(lo, hi + 1, size=batch).astype(np.int32)


def sweep(buckets, modes=AUTO_MODES, seed: int = 99, reps: int = 3, log=print):
    """Time every (mode, cfg) on every bucket (the library's ss_autotune, one
    call per bucket and mode); returns the list of entries."""
    import torch
    from .device import DeviceBatch
    entries = []
    for (op, k, batch) in buckets:
        n = bucket_sizes(k, batch, seed)
        pk = inputs.make_batch(op, n, seed=seed + k)
        db = DeviceBatch(pk.n, pk.off, pk.ops, op)
        lo, hi = bin_range(k)
        for mname in modes:
            m = ss.MODES[mname]
            times, bads, _ = db.autotune(m, reps=reps)
            for cfg, (ms, bad) in enumerate(zip(times, bads)):
                entries.append(dict(op=op, bin=k, n_lo=lo, n_hi=hi, batch=batch, mode=mname,
                                    cfg=cfg, ms=ms, info_nonzero=bad))
                log(f"{op:6s} bin={k} n=({lo},{hi}] batch={batch:5d} {mname:13s} cfg={cfg} "
                    f"{ms:9.3f} ms bad={bad}")
        del db
        torch.cuda.empty_cache()
    return entries


def best_per_bucket(entries):
    """{(op, bin, batch): (mode, cfg, ms)} over entries whose solves all succeeded."""
    best = {}
    for e in entries:
        if e.get("info_nonzero", 0):
            continue
        key = (e["op"], e["bin"], e["batch"])
        if key not in best or e["ms"] < best[key][2]:
            best[key] = (e["mode"], e["cfg"], e["ms"])
    return best


def lookup(entries, op, k, batch, mode, cfg):
    """Measured ms of (mode, cfg) in the bucket of `op`, bin k closest in log batch."""
    cands = [e for e in entries if e["op"] == op and e["bin"] == k and e["mode"] == mode and e["cfg"] == cfg]
    if not cands:
        return None
    e = min(cands, key=lambda e: abs(math.log2(e["batch"]) - math.log2(max(batch, 1))))
    return e["ms"]


def exhaustive_table(entries, op, batch, nbins=ss.NUM_BINS):
    """Per-bin (mode, cfg) of the exhaustive search, from the bucket closest in
    log batch (`batch`: instances per bin, a list or one number); bins without
    measurements or instances stay unset (-1)."""
    best = best_per_bucket(entries)
    counts = list(batch) if hasattr(batch, "__len__") else [batch] * nbins
    modes, cfgs = [-1] * nbins, [-1] * nbins
    for k in range(nbins):
        cands = [(key, v) for key, v in best.items() if key[0] == op and key[1] == k]
        if not cands or counts[k] <= 0:
            continue
        key, v = min(cands, key=lambda kv: abs(math.log2(kv[0][2]) - math.log2(max(counts[k], 1))))
        modes[k] = ss.MODES[v[0]]
        cfgs[k] = v[1]
    return modes, cfgs


def exhaustive_call_choice(entries, op, batch, nbins=ss.NUM_BINS):
    """The single (mode, cfg) with the smallest measured total over the call's
    size bins (bucket closest in log batch per bin); None if unmeasured."""
    counts = list(batch) if hasattr(batch, "__len__") else [batch] * nbins
    pairs = sorted({(e["mode"], e["cfg"]) for e in entries if e["op"] == op and not e.get("info_nonzero", 0)})
    best = None
    for mode, cfg in pairs:
        tot = 0.0
        for k in range(nbins):
            if counts[k] <= 0:
                continue
            t = lookup(entries, op, k, counts[k], mode, cfg)
            if t is None:
                tot = None
                break
            tot += t
        if tot is not None and (best is None or tot < best[2]):
            best = (mode, cfg, tot)
    return best


def save(entries, path, extra=None):
    d = {"gpu": None, "created": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "entries": entries}
    try:
        import torch
        d["gpu"] = torch.cuda.get_device_name(0)
    except Exception:  # noqa: BLE001 - device name is informational
        pass
    if extra:
        d.update(extra)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=0)
    os.replace(tmp, path)


def load(path):
    with open(path) as f:
        return json.load(f)


def merge_entries(old, new):
    """The entries of `old` whose (op, bin, batch, mode) the sweep `new` did not
    measure, followed by all of `new`."""
    swept = {(e["op"], e["bin"], e["batch"], e["mode"]) for e in new}
    return [e for e in old if (e["op"], e["bin"], e["batch"], e["mode"]) not in swept] + list(new)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--max-bin", type=int, default=9)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--ops", default=",".join(OPS))
    ap.add_argument("--modes", default=",".join(AUTO_MODES))
    ap.add_argument("--min-bin", type=int, default=2)
    ap.add_argument("--batches", default=None, help="only these batch sizes of the default buckets")
    ap.add_argument("--merge", default=None,
                    help="existing database: keep its entries, replacing those of the swept (op, bin, batch, mode)")
    args = ap.parse_args(argv)
    ops = args.ops.split(",")
    modes = tuple(args.modes.split(","))
    batches = None if args.batches is None else {int(b) for b in args.batches.split(",")}
    buckets = [b for b in default_buckets(args.max_bin) if b[0] in ops and b[1] >= args.min_bin
               and (batches is None or b[2] in batches)]
    t0 = time.time()
    entries = sweep(buckets, modes=modes, reps=args.reps, log=lambda s: print(s, flush=True))
    extra = {"sweep_seconds": time.time() - t0}
    if args.merge:
        old = load(args.merge)
        entries = merge_entries(old["entries"], entries)
        what = f"{','.join(modes)} x {','.join(ops)}, bins >= {args.min_bin}" + (f", batches {args.batches}" if batches else "")
        extra["note"] = f"{old.get('note', '')}; swept {what} on {time.strftime('%Y-%m-%d')}".lstrip("; ")
    save(entries, args.out, extra)
    print(f"{len(entries)} entries in {time.time() - t0:.0f} s -> {args.out}")


if __name__ == "__main__":
    sys.exit(main())
