"""Learned selector: an MLP cost model that predicts, for an (operation, n,
batch, precision mode) bucket, the run time of every kernel configuration, so
that the fastest (mode, configuration) can be chosen without timing them.

The paper names this as future work: replacing the autotuning loops with a
model-based approach ("Limitations and future work" paragraph).  The network,
its training and the choice it makes run in the library (``ss_selector_train``,
``ss_selector_predict``, the CUDA kernels behind ``ss_mlp_*``); this module
builds the training rows from the tuning database, moves arrays and keeps the
model's files.  The exhaustive autotuner (``tune.py``) produces
the training table, stays the fallback, and is the yardstick of the selector's regret.

Features (SS_MLP_IN = 10): op one-hot (potrf, trsyl, trlyap), log2(n)/9,
log2(batch)/14, mode one-hot (fp64, fp32_refined, tf32_refined, bf16_refined,
df).
Targets: log2(milliseconds) per configuration id (SS_MLP_OUT = 8 slots, masked
to the configurations the mode has).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import smallsolve as ss
from . import tune

OP_ORDER = ("potrf", "trsyl", "trlyap")
MODE_ORDER = ("fp64", "fp32_refined", "tf32_refined", "bf16_refined", "df")


def heldout_bucket(k: int, batch: int, batches_of_bin) -> bool:
    """Buckets kept out of training to measure the selector on sizes and batch
    counts it has not seen: every third (size bin, batch rank) cell, so that
    each held-out bucket has trained neighbours in n (bins k-1, k+1) and in
    batch (the other batch count of its bin)."""
    r = sorted(set(batches_of_bin)).index(batch)
    return (k + r) % 3 == 0


def split_buckets(entries):
    """(training buckets, held-out buckets) of a tuning database, as sets of
    (op, bin, batch)."""
    buckets = {(e["op"], e["bin"], e["batch"]) for e in entries}
    per_bin = {}
    for op, k, b in buckets:
        per_bin.setdefault((op, k), set()).add(b)
    held = {(op, k, b) for op, k, b in buckets if heldout_bucket(k, b, per_bin[(op, k)])}
    return buckets - held, held


def features(op: str, n: float, batch: float, mode: str) -> np.ndarray:
    f = np.zeros(ss.MLP_IN, dtype=np.float32)
    f[OP_ORDER.index(op)] = 1.0
    f[3] = math.log2(max(n, 1.0)) / 9.0
    f[4] = math.log2(max(batch, 1.0)) / 14.0
    f[5 + MODE_ORDER.index(mode)] = 1.0
    return f


def bin_center(k: int) -> float:
    lo, hi = tune.bin_range(k)
    return math.sqrt(lo * hi)


def dataset(entries, bins=None, buckets=None):
    """Rows (features, log2-ms targets, mask, keys) from tuning entries,
    optionally restricted to size bins or to (op, bin, batch) buckets."""
    rows = {}
    for e in entries:
        if e.get("info_nonzero", 0) or e["mode"] not in MODE_ORDER:
            continue
        if bins is not None and e["bin"] not in bins:
            continue
        if buckets is not None and (e["op"], e["bin"], e["batch"]) not in buckets:
            continue
        key = (e["op"], e["bin"], e["batch"], e["mode"])
        rows.setdefault(key, {})[e["cfg"]] = e["ms"]
    keys = sorted(rows)
    X = np.zeros((len(keys), ss.MLP_IN), dtype=np.float32)
    T = np.zeros((len(keys), ss.MLP_OUT), dtype=np.float32)
    M = np.zeros((len(keys), ss.MLP_OUT), dtype=np.float32)
    for i, key in enumerate(keys):
        op, k, batch, mode = key
        X[i] = features(op, bin_center(k), batch, mode)
        for c, ms in rows[key].items():
            if c < ss.MLP_OUT:
                T[i, c] = math.log2(max(ms, 1e-6))
                M[i, c] = 1.0
    return X, T, M, keys


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    H, IN, OUT = ss.MLP_HIDDEN, ss.MLP_IN, ss.MLP_OUT
    parts = [rng.standard_normal(H * IN) * math.sqrt(2.0 / IN), np.zeros(H),
             rng.standard_normal(H * H) * math.sqrt(2.0 / H), np.zeros(H),
             rng.standard_normal(OUT * H) * math.sqrt(1.0 / H), np.zeros(OUT)]
    return np.concatenate(parts).astype(np.float32)


class Selector:
    def __init__(self, params=None, device="cuda"):
        self.params = init_params() if params is None else np.asarray(params, dtype=np.float32)
        assert self.params.shape == (ss.MLP_PARAMS,)
        self.device = device
        self.meta = {}
        # "op:mode" -> configurations with training targets; an output slot
        # that never had a target carries no information, so choices stay
        # within these (None: the library's count).
        self.cfg_counts = None
        # "op:bin:mode" -> the largest batch the network was trained on for
        # that size bin and mode.  Beyond it a prediction is taken at that
        # batch and scaled by count / batch (throughput-bound kernels), a
        # regime the network, trained on smaller batches there, does not
        # extrapolate to.
        self.batch_max = None

    def n_cfgs(self, op: str, mode: str) -> int:
        cnt = ss.ss_config_count(ss.OPS[op], ss.MODES[mode])
        if self.cfg_counts is not None:
            cnt = min(cnt, int(self.cfg_counts.get(f"{op}:{mode}", 0)))
        return cnt

    # ------------------------------------------------- the library's model
    def tables(self):
        """(cfg_count, batch_max) in the layout of ss_selector_set (None where
        this selector has no such record)."""
        cc = None
        if self.cfg_counts is not None:
            cc = [int(self.cfg_counts.get(f"{op}:{m}", 0)) for op in OP_ORDER for m in MODE_ORDER]
        bm = None
        if self.batch_max is not None:
            bm = [0] * (len(OP_ORDER) * ss.NUM_BINS * len(MODE_ORDER))
            for key, v in self.batch_max.items():
                op, k, m = key.split(":")
                bm[(OP_ORDER.index(op) * ss.NUM_BINS + int(k)) * len(MODE_ORDER) + MODE_ORDER.index(m)] = int(v)
        return cc, bm

    def push(self):
        """Make this the library's model (ss_selector_set); the choices below
        are the library's (ss_selector_predict)."""
        ss.ss_selector_set(self.params, *self.tables())

    def pull(self):
        """Take the library's model (after ss_selector_train)."""
        p, cc, bm = ss.ss_selector_get()
        self.params = p
        self.cfg_counts = {f"{op}:{m}": cc[i * len(MODE_ORDER) + j]
                           for i, op in enumerate(OP_ORDER) for j, m in enumerate(MODE_ORDER)}
        self.batch_max = {}
        for i, op in enumerate(OP_ORDER):
            for k in range(ss.NUM_BINS):
                for j, m in enumerate(MODE_ORDER):
                    v = bm[(i * ss.NUM_BINS + k) * len(MODE_ORDER) + j]
                    if v > 0:
                        self.batch_max[f"{op}:{k}:{m}"] = v

    # ----------------------------------------------------------- training
    def train(self, X, T, M, steps=3000, lr=3e-3, log_every=0, log=print):
        """Adam on the masked MSE by the library's kernels on the GPU
        (ss_selector_train, from this selector's parameters); returns the loss
        history as (step, loss) pairs."""
        loss = ss.ss_selector_train(X, T, M, steps, lr, init=self.params)
        self.pull()
        hist = [(s, float(loss[s - 1])) for s in range(1, steps + 1) if s == 1 or s % 50 == 0 or s == steps]
        if log_every:
            for s in range(log_every, steps + 1, log_every):
                log(f"step {s} loss {float(loss[s - 1]):.5f}")
        return hist

    # ---------------------------------------------------------- inference
    def predict(self, X):
        """log2-ms predictions [rows x SS_MLP_OUT] by the CUDA forward kernel."""
        import torch
        dev = torch.device(self.device)
        X = np.ascontiguousarray(X, dtype=np.float32)
        P = torch.as_tensor(self.params, device=dev)
        dX = torch.as_tensor(X, device=dev)
        Y = torch.zeros((X.shape[0], ss.MLP_OUT), dtype=torch.float32, device=dev)
        if X.shape[0]:
            ss.ss_mlp_forward(P.data_ptr(), X.shape[0], dX.data_ptr(), Y.data_ptr())
        torch.cuda.synchronize(dev)
        return Y.cpu().numpy()

    def _predict_table(self, op: str, counts, policy):
        self.push()
        return ss.ss_selector_predict(ss.OPS[op], list(counts), policy)

    def decide_with(self, predict_fn, op: str, counts, policy=ss.SELECTOR_PER_BIN):
        """The library's decision (ss_selector_queries / ss_selector_decide)
        on predictions from predict_fn(feature rows) instead of the network."""
        self.push()
        X = ss.ss_selector_queries(ss.OPS[op], list(counts))
        Y = np.asarray(predict_fn(X), dtype=np.float32).reshape(len(X), ss.MLP_OUT)
        return ss.ss_selector_decide(ss.OPS[op], list(counts), policy, Y)

    def choose_many(self, queries):
        """queries: list of (op, n, batch) -> list of (mode, cfg, predicted ms),
        each the library's per-bin choice for `batch` instances in bin(n)."""
        inv = {v: k for k, v in ss.MODES.items()}
        out = []
        for op, n, batch in queries:
            k = ss.size_bin(int(round(n)))
            counts = [0] * ss.NUM_BINS
            counts[k] = int(round(batch))
            modes, cfgs, ms = self._predict_table(op, counts, ss.SELECTOR_PER_BIN)
            out.append((inv[modes[k]], cfgs[k], ms))
        return out

    def auto_table(self, op: str, batch, nbins: int = ss.NUM_BINS):
        """Per-bin (mode ids, cfg ids) for ss_set_auto_table.  `batch` is the
        number of instances per size bin (a list, or one number for all);
        bins with no instances keep the library default (-1)."""
        counts = list(batch) if hasattr(batch, "__len__") else [batch] * nbins
        modes, cfgs, _ = self._predict_table(op, counts[:nbins], ss.SELECTOR_PER_BIN)
        return modes, cfgs

    def call_choice(self, op: str, batch, nbins: int = ss.NUM_BINS):
        """One (mode, cfg, predicted ms) for a whole call (SS_SELECTOR_CALL)."""
        counts = list(batch) if hasattr(batch, "__len__") else [batch] * nbins
        modes, cfgs, ms = self._predict_table(op, counts[:nbins], ss.SELECTOR_CALL)
        inv = {v: k for k, v in ss.MODES.items()}
        return inv[modes[0]], cfgs[0], ms

    def call_table(self, op: str, batch, nbins: int = ss.NUM_BINS):
        """AUTO table with the single call choice in every bin."""
        counts = list(batch) if hasattr(batch, "__len__") else [batch] * nbins
        modes, cfgs, _ = self._predict_table(op, counts[:nbins], ss.SELECTOR_CALL)
        return modes, cfgs

    def install(self, op: str, batch, per_bin: bool = False):
        modes, cfgs = (self.auto_table if per_bin else self.call_table)(op, batch)
        ss.ss_set_auto_table(ss.OPS[op], modes, cfgs)
        return modes, cfgs

    # ------------------------------------------------------------ storage
    def save(self, path: str, **meta):
        np.save(path + ".npy", self.params)
        with open(path + ".json", "w") as f:
            json.dump({"params": os.path.basename(path) + ".npy", "n_params": int(self.params.size),
                       "features": "op one-hot, log2(n)/9, log2(batch)/14, mode one-hot",
                       "op_order": OP_ORDER, "mode_order": MODE_ORDER,
                       "cfg_counts": self.cfg_counts, "batch_max": self.batch_max, **meta}, f, indent=1)

    @classmethod
    def load(cls, path: str, device="cuda"):
        s = cls(np.load(path + ".npy"), device=device)
        with open(path + ".json") as f:
            s.meta = json.load(f)
        s.cfg_counts = s.meta.get("cfg_counts")
        s.batch_max = s.meta.get("batch_max")
        return s


def trained_cfg_counts(X, M):
    """{"op:mode": 1 + the highest configuration id with a target} from the
    one-hot op and mode features of the training rows."""
    out = {}
    for x, m in zip(np.asarray(X), np.asarray(M)):
        op = OP_ORDER[int(np.argmax(x[0:3]))]
        mode = MODE_ORDER[int(np.argmax(x[5:5 + len(MODE_ORDER)]))]
        nz = np.nonzero(m > 0)[0]
        if nz.size:
            key = f"{op}:{mode}"
            out[key] = max(out.get(key, 0), int(nz[-1]) + 1)
    return out


def trained_batch_max(X):
    """{"op:bin:mode": the largest batch among the training rows of that size
    bin and mode} from the one-hot, log2(n) and log2(batch) features."""
    out = {}
    for x in np.asarray(X, dtype=np.float64):
        op = OP_ORDER[int(np.argmax(x[0:3]))]
        mode = MODE_ORDER[int(np.argmax(x[5:5 + len(MODE_ORDER)]))]
        k = ss.size_bin(int(round(2.0 ** (x[3] * 9.0))))
        b = int(round(2.0 ** (x[4] * 14.0)))
        key = f"{op}:{k}:{mode}"
        out[key] = max(out.get(key, 0), b)
    return out


def best_fixed_policy(entries, op: str, buckets):
    """The single (mode, cfg) with the smallest geometric-mean measured time
    over the given (op, bin, batch) buckets of `op`, among the pairs measured
    in all of them: the method without a model, tuned on the same data."""
    T = {(e["op"], e["bin"], e["batch"], e["mode"], e["cfg"]): e["ms"]
         for e in entries if not e.get("info_nonzero", 0)}
    bks = [b for b in buckets if b[0] == op]
    best = None
    for mc in sorted({k[3:] for k in T if k[0] == op}):
        ts = [T.get(tuple(b) + mc) for b in bks]
        if not ts or any(t is None for t in ts):
            continue
        g = float(np.exp(np.mean(np.log(ts))))
        if best is None or g < best[1]:
            best = (mc, g)
    return best[0] if best else None


def counts_by_bin(n, nbins: int = ss.NUM_BINS):
    """Number of instances of each order in each size bin."""
    c = [0] * nbins
    for v in np.asarray(n).ravel():
        c[ss.size_bin(int(v))] += 1
    return c


def regret_report(choices, entries, buckets):
    """For each bucket (op, bin, batch): the measured ms of the chosen
    (mode, cfg), of the exhaustive best and of the FP64 default; summary of
    regret (chosen / best - 1) and gain over the default (default / chosen)."""
    best = tune.best_per_bucket(entries)
    out = []
    for (op, k, batch), (mode, cfg) in zip(buckets, choices):
        key = (op, k, batch)
        if key not in best:
            continue
        t_c = tune.lookup(entries, op, k, batch, mode, cfg)
        t_b = best[key][2]
        dflt = default_fp64_cfg(1 << k, op, batch)
        t_d = tune.lookup(entries, op, k, batch, "fp64", dflt)
        if t_c is None or t_d is None:
            continue
        out.append(dict(op=op, bin=k, batch=batch, mode=mode, cfg=cfg, ms=t_c, best_ms=t_b,
                        best=best[key][:2], default_ms=t_d, regret=t_c / t_b - 1.0, gain=t_d / t_c))
    if not out:
        return {"buckets": 0}
    return {"buckets": len(out),
            "mean_regret": float(np.mean([o["regret"] for o in out])),
            "max_regret": float(np.max([o["regret"] for o in out])),
            "geomean_gain_over_default": float(np.exp(np.mean([math.log(o["gain"]) for o in out]))),
            "rows": out}


def default_fp64_cfg(max_n: int, op: str = "potrf", batch: int = 2048) -> int:
    """The library's built-in FP64 default (SS_CFG_DEFAULT) for a call with
    this largest order and batch."""
    if op == "potrf":
        if max_n <= 16:
            return 5
        return 0 if (max_n <= 128 and batch >= 1024) else 2
    if max_n <= 8:
        return 0
    if max_n <= 32:
        return 1
    if max_n <= 64:
        return 7
    return 6 if (max_n <= 128 and batch >= 1024) else 5
