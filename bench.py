"""Benchmark: batched small structured solves on GB300 (one JSON line).

Default workload: triangular Sylvester L X + X U = C, 4096 instances with
order n uniform in {4..128} (FP64 inputs and output), solved by the library's
C ABI (``trsyl_lu``) in one persistent launch per configuration group.  A step
is one batched solve of the whole workload.  Inputs are seeded synthetic data
(see paper_1906_08613_gb300/inputs.py); the operand buffers are larger than
the 129 MB L2, so no flush is needed between steps.

The headline path (``--path learned``, the default) is SS_MODE_AUTO driven by
the trained selector: each size bin runs in the (precision mode, kernel
configuration) the MLP cost model predicts fastest among FP64 and the refined
modes, all of which meet the 1e-11 accuracy gate.  Plain FP64 (built-in
default configuration, and the autotuner's best FP64 configuration per size
bin) is timed in the same run for comparison.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
        [--workload NAME] [--path learned|mode] [--mode fp64|fp32_refined|...]
        [--cfg C] [--graph]
For N > 1 launch with torch.distributed.run; each rank solves its own copy of
the workload (independent replicas, weak scaling, no collective on the data
path).  ``--impl reference`` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched solves/s and % roofline, mixed+learned vs plain FP64 GPU at 1e-11 error"
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07   # SMs x DFMA/clk/SM x flop/FMA x GHz = 1258.6
# Double-float ceiling of SS_MODE_DF: the FP32 pipe's instruction rate
# (152 SMs x 128 lanes x 2.07 GHz) over the 13 FP32 instructions of one
# double-float multiply-add (TwoProduct with cross terms, TwoSum, low-part
# update), counted as the 2 flops of the FP64 operation it replaces.
DF_OPS_PER_TERM = 13
DF_PEAK_GFLOPS = 152 * 128 * 2.07 / DF_OPS_PER_TERM * 2   # = 6196.0
# The same ceiling from the measured FP32 rate (an FFMA probe: 72 TFLOP/s =
# 36e12 FFMA/s) instead of the nominal lane rate.
DF_PEAK_MEASURED_FFMA_GFLOPS = 72000.0 / 2 / DF_OPS_PER_TERM * 2   # = 5538.5
GATE = 1e-11


# Arithmetic each precision mode computes in (the JSON line's dtype).
DTYPE_OF_MODE = {"fp64": "f64", "df": "f32x2 double-float block updates, f64 divisions / pivots",
                 "fp32_refined": "f32 solve + f32x2 double-float refinement",
                 "tf32_refined": "tf32 tensor-core updates + f32x2 refinement",
                 "bf16_refined": "bf16 tensor-core updates + f32x2 refinement"}


def inv_mode(m):
    from paper_1906_08613_gb300 import smallsolve as ss
    return {v: k for k, v in ss.MODES.items()}.get(int(m), str(m))


def flops_paper(op, n):
    """The paper's flop counts (Fig. 2 caption): n^3/3 for Cholesky, 2 n^3
    for Sylvester and Lyapunov."""
    n = np.asarray(n, dtype=np.float64)
    return float((n ** 3 / 3).sum()) if op == "potrf" else float((2 * n ** 3).sum())


def flops_algorithmic(op, n):
    """Multiply-add count x 2 of the solve as computed (Lyapunov exploits the
    symmetry of X: n^3)."""
    n = np.asarray(n, dtype=np.float64)
    if op == "potrf":
        return float((n ** 3 / 3).sum())
    if op == "trsyl":
        return float((2 * n ** 3).sum())
    return float((n ** 3).sum())


def bytes_algorithmic(op, n):
    """Stored triangles / full operands read once and X written once, FP64."""
    n = np.asarray(n, dtype=np.float64)
    tri = n * (n + 1) / 2
    if op == "potrf":
        return float((8 * (tri + tri)).sum())
    if op == "trsyl":
        return float((8 * (tri + tri + n * n + n * n)).sum())
    return float((8 * (tri + tri + tri)).sum())


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
        return dist, rank, world, local
    return None, rank, world, local


def barrier(dist, dev):
    import torch
    if dist is not None:
        if dev.type == "cuda":
            dist.barrier(device_ids=[dev.index])
        else:
            dist.barrier()
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)


def max_over_ranks(dist, value, dev):
    """The slowest rank's time (replicas: the job ends when the last rank does)."""
    import torch
    if dist is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, dev):
    """Units processed by all ranks together (whole-job throughput)."""
    import torch
    if dist is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(dist, units_per_rank, ms_per_rank, dev):
    """Whole-job units/s of independent replicas: all ranks' units over the
    slowest rank's time."""
    ms = max_over_ranks(dist, ms_per_rank, dev)
    return sum_over_ranks(dist, float(units_per_rank), dev) / (ms * 1e-3), ms


def read_traffic(key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (profiles/traffic.json, keyed workload:op:mode:cfg), if it was
    taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    from paper_1906_08613_gb300 import build as b
    ent = d.get(key)
    if not ent or ent.get("sources_sha") != b.sources_sha(ent.get("sources")):
        return None
    return ent.get("dram_bytes_per_launch")


def cpu_oracle_rate(op, pk, seconds: float, threads: int, indices=None):
    """Time the oracle on host threads over (a sample of) the batch, repeating
    passes until `seconds` elapsed; returns (solves/s, solves, elapsed, out)."""
    import oracle
    ops = {k: v for k, v in pk.ops.items() if k != "X0"}
    idx = np.arange(pk.batch) if indices is None else np.asarray(indices)
    done = 0
    out = None
    t0 = time.perf_counter()
    while True:
        out, _ = oracle.solve_packed_parallel(op, pk.n, pk.off, ops, threads=threads, indices=idx)
        done += len(idx)
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done / el, done, el, out


def launch_groups(table, max_n):
    """Solve launches per call: runs of equal (mode, cfg) over the size bins
    up to bin(max_n), from the largest bin down (one group without a table)."""
    if not table:
        return 1
    from paper_1906_08613_gb300 import smallsolve as ss
    pairs = list(zip(*table))[: ss.size_bin(max_n) + 1]
    runs, prev = 0, None
    for p in reversed(pairs):
        if p != prev:
            runs += 1
            prev = p
    return runs


def e2e_pipelined(dbs, host_in, solve, steps, dist, dev, batch):
    """End-to-end through the C ABI with host buffers, every step: H2D of the
    step's inputs from pinned memory, the solve, D2H of X.  Two device copies
    of the batch alternate between steps; H2D, the solve and D2H each have a
    stream, so the copies of step s+1 and of step s-1 run under the solve of
    step s (the GPU's copy engines work beside the SMs).  Returns (solves/s,
    bytes in per step, bytes out per step, last X on the host)."""
    import torch
    names = list(host_in)
    s_in, s_run, s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
    host_x = torch.empty_like(dbs[0].X, device="cpu").pin_memory()
    ev = lambda: torch.cuda.Event()
    h2d_done = [ev(), ev()]
    run_done = [ev(), ev()]
    d2h_done = [ev(), ev()]
    for e in h2d_done + run_done + d2h_done:
        e.record(s_run)

    def one(s):
        b = dbs[s % 2]
        s_in.wait_event(run_done[s % 2])              # step s-2 finished reading the inputs
        with torch.cuda.stream(s_in):
            for k in names:
                b.bufs[k].copy_(host_in[k], non_blocking=True)
        h2d_done[s % 2].record(s_in)
        s_run.wait_event(h2d_done[s % 2])
        s_run.wait_event(d2h_done[s % 2])             # X of step s-2 has reached the host
        with torch.cuda.stream(s_run):
            solve(b, s_run.cuda_stream)
        run_done[s % 2].record(s_run)
        s_out.wait_event(run_done[s % 2])
        with torch.cuda.stream(s_out):
            host_x.copy_(b.X, non_blocking=True)
        d2h_done[s % 2].record(s_out)

    for s in range(2):
        one(s)
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(s_run)
    s_in.wait_stream(s_run)
    s_out.wait_stream(s_run)
    for s in range(steps):
        one(s)
    s_run.wait_stream(s_out)
    s_run.wait_stream(s_in)
    f1.record(s_run)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(dist, f0.elapsed_time(f1), dev)
    value = sum_over_ranks(dist, float(batch * steps), dev) / (ms * 1e-3)
    h2d = sum(int(host_in[k].numel()) * 8 for k in names)
    d2h = int(host_x.numel()) * 8
    return value, h2d, d2h, host_x.numpy()


def sample_indices(pk, k, seed=7):
    rng = np.random.default_rng(seed)
    k = min(k, pk.batch)
    return np.sort(rng.choice(pk.batch, size=k, replace=False))


def run_reference(args):
    """The oracle arm: one step = the oracle over a bounded sample of the
    workload on all host cores."""
    dist, rank, world, _ = (None, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0)
    if rank != 0:
        return 0
    from paper_1906_08613_gb300 import inputs
    import oracle
    name = args.workload
    op = inputs.WORKLOADS[name]["op"]
    pk = inputs.make_workload(name, seed=args.seed)
    threads = os.cpu_count() or 1
    per_step = max(8, min(pk.batch, int(args.ref_sample)))
    ops = {k: v for k, v in pk.ops.items() if k != "X0"}
    for w in range(args.warmup):
        oracle.solve_packed_parallel(op, pk.n, pk.off, ops, threads=threads,
                                     indices=sample_indices(pk, per_step, seed=1000 + w))
    times = []
    solves = 0
    for s in range(args.steps):
        idx = sample_indices(pk, per_step, seed=s)
        t0 = time.perf_counter()
        oracle.solve_packed_parallel(op, pk.n, pk.off, ops, threads=threads, indices=idx)
        times.append(time.perf_counter() - t0)
        solves += len(idx)
    total = sum(times)
    value = solves / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "op": op, "batch_per_step": per_step,
                   "sizes": "sampled from the workload's size distribution"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} seeded random instances of {name} per step"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def extra_workload(name, seed, device):
    """The rectangular-Sylvester and SPD-solve workloads: (op label, packed
    batch, device batch, flops, algorithmic bytes, input names, oracle of one
    instance -> (X buffer offset, element count, reference values))."""
    import oracle
    from paper_1906_08613_gb300 import inputs
    from paper_1906_08613_gb300.device import DevicePosvBatch, DeviceRectBatch
    if name in inputs.RECT_WORKLOADS:
        pk = inputs.make_rect_workload(name, seed=seed)
        m, n = pk.m.astype(np.float64), pk.n.astype(np.float64)
        flops = float((m * n * (m + n)).sum())                       # m n (m + n): 2 n^3 when m = n
        nbytes = float((8 * (m * (m + 1) / 2 + n * (n + 1) / 2 + 2 * m * n)).sum())

        out = np.zeros_like(pk.ops["C"])

        def one(b):
            oracle.solve_rect_packed(pk, out=out, lo=b, hi=b + 1)
            o, c = int(pk.offC[b]), int(pk.m[b]) * int(pk.n[b])
            return o, c, out[o:o + c]
        return "trsyl_rect", pk, DeviceRectBatch(pk, device=device), flops, nbytes, ("L", "U", "C"), one
    pk = inputs.make_posv_workload(name, seed=seed)
    n, k = pk.n.astype(np.float64), pk.k.astype(np.float64)
    flops = float((n ** 3 / 3 + 2 * n * n * k).sum())                # factor + two triangular solves
    nbytes = float((8 * (n * (n + 1) + 2 * n * k)).sum())              # A and R triangles, B, X

    out_x, out_r = np.zeros_like(pk.ops["B"]), np.zeros_like(pk.ops["A"])

    def one(b):
        oracle.solve_posv_packed(pk, lo=b, hi=b + 1, out_x=out_x, out_r=out_r)
        o, c = int(pk.offB[b]), int(pk.n[b]) * int(pk.k[b])
        return o, c, out_x[o:o + c]
    return "posv_upper", pk, DevicePosvBatch(pk, device=device), flops, nbytes, ("A", "B"), one


def run_extra(args):
    """Rectangular Sylvester (trsyl_rect) or SPD solve (posv_upper) workload,
    FP64 or DF (--mode), with one explicit or the default configuration."""
    import torch
    from paper_1906_08613_gb300 import smallsolve as ss

    dist, rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    name = args.workload
    cfg = ss.CFG_DEFAULT if args.cfg is None else args.cfg
    mode = ss.MODES[args.mode]
    if mode not in (ss.MODE_FP64, ss.MODE_DF):
        raise SystemExit("trsyl_rect / posv_upper workloads run in fp64 or df")
    opname, pk, db, F, Balg, names, oracle_one = extra_workload(name, args.seed, dev)
    torch.cuda.synchronize(dev)         # buffer fills (default stream) before the side streams

    def step():
        db.solve(cfg=cfg, mode=mode, stream=sh)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    barrier(dist, dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = ss.ss_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(dist, dev)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
    stream.synchronize()
    barrier(dist, dev)
    launches = ss.ss_launch_count() - l0
    clk = clocks.stop()
    value, ms_total = job_throughput(dist, pk.batch * args.steps, e0.elapsed_time(e1), dev)
    ms_step = ms_total / args.steps
    info = db.info_host()

    host_in = {k: torch.from_numpy(pk.ops[k]).pin_memory() for k in names}
    _, _, db2, _, _, _, _ = extra_workload(name, args.seed, dev)
    torch.cuda.synchronize(dev)
    e2e_value, h2d, d2h, x_gpu = e2e_pipelined(
        [db, db2], host_in, lambda b, st: b.solve(cfg=cfg, mode=mode, stream=st), max(3, min(args.steps, 50)),
        dist, dev, pk.batch)
    del db2
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    # Whole call (pre-pass + solve launches) against the peak of the mode's
    # arithmetic.
    achieved = F / (ms_step * 1e-3) / 1e9
    if args.mode == "df":
        peak, peak_source = DF_PEAK_GFLOPS, ("derived: 152 SMs x 128 FP32 lanes x 2.07 GHz / 13 FP32 "
                                             "instructions per double-float multiply-add x 2 flop (of derived)")
    else:
        peak, peak_source = FP64_PEAK_GFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (of derived)"
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_OF_MODE[args.mode] + " (X in f64)", "data": "synthetic",
        "config": {"workload": name, "op": opname, "batch": pk.batch, "path": args.mode, "cfg": cfg,
                   "l2": f"operands {sum(int(v.numel()) * 8 for v in db.bufs.values()) / 1e6:.0f} MB "
                         "> 129 MB L2; no flush"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                     "frac": achieved / peak, "traffic": None, "fp64_equivalent_frac": achieved / FP64_PEAK_GFLOPS,
                     "kernel": f"{opname}: whole call (pre-pass and solve launches)", "call_ms": ms_step,
                     "algorithmic_bytes": Balg, "flops": F,
                     "peak_source": peak_source},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches), "launches_per_step": launches / args.steps, "clocks": clk,
        "info_nonzero": int((info != 0).sum()),
    }
    if not args.no_cpu:
        idx = sample_indices(pk, max(16, pk.batch // 8))
        done, t0, errs = 0, time.perf_counter(), []
        while True:
            for b in idx:
                o, c, ref = oracle_one(int(b))
                if done < len(idx):
                    errs.append(np.linalg.norm(x_gpu[o:o + c] - ref) / np.linalg.norm(ref))
                done += 1
            el = time.perf_counter() - t0
            if el >= args.cpu_seconds:
                break
        line["cpu_baseline"] = {"value": done / el, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                "sample": f"{len(idx)} seeded random instances of {name}, "
                                          f"repeated for {el:.1f} s ({done} solves), one thread"}
        line["accuracy"] = {"max_rel_fro_err_vs_oracle": float(max(errs)), "gate": GATE,
                            "instances_checked": len(idx), "pass": bool(max(errs) <= GATE)}
    print(json.dumps(line), flush=True)
    return 0


SIDE_WORKLOADS = ("potrf_1024x64", "trlyap_2048x128", "potrf_8192xLU8-256")


def measure_side_workloads(args, dev, stream):
    """The other measured configurations, each as the headline: mixed +
    learned (SS_MODE_AUTO with the selector's one choice for the call) against
    plain FP64 with the default configuration, on inputs resident in HBM;
    the learned path's accuracy against the oracle on a sample of 32
    instances and the roofline fraction of its dominant kernel."""
    import torch
    import oracle
    from paper_1906_08613_gb300 import inputs, selector as sel, smallsolve as ss
    from paper_1906_08613_gb300.device import DeviceBatch
    sh = stream.cuda_stream
    model = sel.Selector.load(os.path.join(ROOT, "paper_1906_08613_gb300", "data", "selector_gb300"), device=str(dev))
    inv = {v: k for k, v in ss.MODES.items()}
    out = {}
    for name in SIDE_WORKLOADS:
        op = inputs.WORKLOADS[name]["op"]
        o = ss.OPS[op]
        pk = inputs.make_workload(name, seed=args.seed)
        db = DeviceBatch(pk.n, pk.off, pk.ops, op, device=dev)
        table = model.install(op, sel.counts_by_bin(pk.n))
        torch.cuda.synchronize(dev)
        res = {}
        x_learned = None
        for label, mode in (("mixed_learned", ss.MODE_AUTO), ("fp64_default", ss.MODE_FP64)):
            db.ensure_work(mode)
            reps = max(3, min(args.steps, 20))
            with torch.cuda.stream(stream):
                for _ in range(3):
                    db.solve(mode=mode, stream=sh)
                ss.ss_profile_enable(True)
                ss.ss_profile_read()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    db.solve(mode=mode, stream=sh)
                e1.record(stream)
            stream.synchronize()
            kms, kc = ss.ss_profile_read()
            ss.ss_profile_enable(False)
            ms = e0.elapsed_time(e1) / reps
            res[label] = {"ms_per_step": ms, "value": pk.batch / (ms * 1e-3), "kernel_ms": kms / max(kc, 1)}
            if label == "mixed_learned":
                x_learned = db.x_host()
                res[label]["info_nonzero"] = int((db.info_host() != 0).sum())
        ss.ss_set_auto_table(o, [], [])
        idx = sample_indices(pk, 32, seed=11)
        ops = {k: v for k, v in pk.ops.items() if k != "X0"}
        ref, _ = oracle.solve_packed_parallel(op, pk.n, pk.off, ops, threads=os.cpu_count() or 1, indices=idx)
        errs = []
        for b in idx:
            nb, ob = int(pk.n[b]), int(pk.off[b])
            g = x_learned[ob:ob + nb * nb].reshape(nb, nb, order="F")
            r = ref[ob:ob + nb * nb].reshape(nb, nb, order="F")
            g, r = (np.triu(g), np.triu(r)) if op == "potrf" else ((np.tril(g), np.tril(r)) if op == "trlyap" else (g, r))
            errs.append(float(np.linalg.norm(g - r) / np.linalg.norm(r)))
        kbin = ss.size_bin(int(pk.n.max()))
        dm = inv.get(table[0][kbin], "fp64")
        peak = DF_PEAK_GFLOPS if dm == "df" else FP64_PEAK_GFLOPS
        achieved = flops_algorithmic(op, pk.n) / (res["mixed_learned"]["kernel_ms"] * 1e-3) / 1e9
        out[name] = {
            "op": op, "batch": pk.batch,
            "selector_choice": [dm, int(table[1][kbin])],
            "mixed_learned": res["mixed_learned"], "fp64_default": res["fp64_default"],
            "speedup_vs_fp64_default": res["mixed_learned"]["value"] / res["fp64_default"]["value"],
            "accuracy": {"max_rel_fro_err_vs_oracle": max(errs), "gate": GATE, "instances_checked": len(idx),
                         "pass": bool(max(errs) <= GATE)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                         "frac": achieved / peak, "fp64_equivalent_frac": achieved / FP64_PEAK_GFLOPS,
                         "peak_source": "derived (see the headline's roofline)"}}
        del db
        torch.cuda.empty_cache()
    return out


def measure_selector_stream():
    """The held-out stream of 16384 mixed instances (operation uniform over the
    three, n log-uniform in [4, 512]): each operation's share solved in one
    call under the selector, the exhaustive autotune tables, the best single
    (mode, cfg) chosen on the training buckets, and the FP64 default."""
    from paper_1906_08613_gb300 import selector as sel, train_selector as tsel, tune
    model = sel.Selector.load(os.path.join(ROOT, "paper_1906_08613_gb300", "data", "selector_gb300"))
    entries = tune.load(os.path.join(ROOT, "paper_1906_08613_gb300", "data", "tune_gb300.json"))["entries"]
    res = tsel.evaluate_stream(model, entries, total=16384, seed=2026, log=lambda _: None)
    keep = ("instances", "fp64_default_ms", "exhaustive_ms", "exhaustive_call_ms", "fixed_policy_ms", "fixed_policy",
            "selector_ms", "selector_table", "selector_bad", "regret", "gain_over_fp64_default",
            "gain_over_fixed_policy")
    out = {op: {k: v for k, v in r.items() if k in keep} for op, r in res.items() if op != "total"}
    out["total"] = res["total"]
    for r in out.values():
        if "selector_table" in r:
            r["selector_table"] = [list(map(int, r["selector_table"][0]))]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="graft", choices=["graft", "reference"])
    ap.add_argument("--workload", default="trsyl_4096xU4-128")
    ap.add_argument("--path", default="learned", choices=["learned", "mode"],
                    help="learned: SS_MODE_AUTO with the trained selector's tables (default); "
                         "mode: one explicit --mode/--cfg")
    ap.add_argument("--mode", default="fp64")
    ap.add_argument("--cfg", type=int, default=None)
    ap.add_argument("--graph", action="store_true", help="replay each step from a captured CUDA graph")
    ap.add_argument("--policy", default="call", choices=["per-bin", "call"],
                    help="selector policy: a (mode, cfg) per size bin, or one for the whole call")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP64 comparison runs")
    ap.add_argument("--seed", type=int, default=1234)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-sample", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the other configurations and the selector stream")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    from paper_1906_08613_gb300 import inputs as _inputs
    if args.workload in _inputs.RECT_WORKLOADS or args.workload in _inputs.POSV_WORKLOADS:
        return run_extra(args)

    import torch
    from paper_1906_08613_gb300 import inputs, smallsolve as ss
    from paper_1906_08613_gb300.device import DeviceBatch

    dist, rank, world, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream

    name = args.workload
    op = inputs.WORKLOADS[name]["op"]
    pk = inputs.make_workload(name, seed=args.seed)
    o = ss.OPS[op]
    learned = args.path == "learned"
    table = None
    if learned:
        from paper_1906_08613_gb300 import selector as sel
        s_model = sel.Selector.load(os.path.join(ROOT, "paper_1906_08613_gb300", "data", "selector_gb300"),
                                    device=str(dev))
        table = s_model.install(op, sel.counts_by_bin(pk.n), per_bin=args.policy == "per-bin")
        mode, cfg = ss.MODE_AUTO, ss.CFG_DEFAULT
    else:
        mode = ss.MODES[args.mode]
        cfg = ss.CFG_DEFAULT if args.cfg is None else args.cfg

    db = DeviceBatch(pk.n, pk.off, pk.ops, op, device=dev)
    db.ensure_work(mode)
    torch.cuda.synchronize(dev)         # buffer fills (default stream) before the side streams
    F = flops_paper(op, pk.n)
    Falg = flops_algorithmic(op, pk.n)
    Balg = bytes_algorithmic(op, pk.n)

    def step():
        db.solve(mode=mode, cfg=cfg, stream=sh)

    graph = None
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        if args.graph:
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                step()
            for _ in range(2):
                graph.replay()
    barrier(dist, dev)
    run_step = graph.replay if graph is not None else step

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ss.ss_profile_enable(True)
    ss.ss_profile_read()
    l0 = ss.ss_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(dist, dev)
    if graph is not None:
        ss.ss_profile_enable(False)     # events inside a graph are not re-recorded per replay
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            run_step()
        e1.record(stream)
    stream.synchronize()
    barrier(dist, dev)
    launches = ss.ss_launch_count() - l0
    kern_ms, kern_calls = ss.ss_profile_read()
    ss.ss_profile_enable(False)
    clk = clocks.stop()
    value, ms_total = job_throughput(dist, pk.batch * args.steps, e0.elapsed_time(e1), dev)
    if graph is not None:
        # Launches and kernel time inside graph replays are not seen by the
        # library's counters: one call launches 1 + (launch groups) kernels.
        launches = args.steps * (1 + launch_groups(table, int(pk.n.max())))
        kern_ms, kern_calls = ms_total, args.steps
    ms_step = ms_total / args.steps
    kern_avg_ms = kern_ms / max(kern_calls, 1)
    info = db.info_host()

    # End to end through the C ABI with host buffers (see e2e_pipelined).
    names = [k for k in ("A", "L", "U", "C", "S") if k in db.bufs]
    host_in = {k: torch.from_numpy(pk.ops[k]).pin_memory() for k in names}
    db2 = DeviceBatch(pk.n, pk.off, pk.ops, op, device=dev)
    db2.ensure_work(mode)
    torch.cuda.synchronize(dev)
    e2e_value, h2d, d2h, x_gpu = e2e_pipelined(
        [db, db2], host_in, lambda b, st: b.solve(mode=mode, cfg=cfg, stream=st),
        max(3, min(args.steps, 50)), dist, dev, pk.batch)
    del db2

    # Plain FP64 in the same run (the comparator): default configuration, and
    # the autotuner's best FP64 configuration per size bin (FP64-only table).
    compare = {}
    if not args.no_compare:
        from paper_1906_08613_gb300 import tune as tn
        from paper_1906_08613_gb300 import selector as sel2
        entries = tn.load(os.path.join(ROOT, "paper_1906_08613_gb300", "data", "tune_gb300.json"))["entries"]
        fp_entries = [e for e in entries if e["mode"] == "fp64"]
        fm, fc = tn.exhaustive_table(fp_entries, op, sel2.counts_by_bin(pk.n))
        variants = [("fp64_default", ss.MODE_FP64, ss.CFG_DEFAULT, None),
                    ("fp64_tuned", ss.MODE_AUTO, ss.CFG_DEFAULT, (fm, fc))]
        saved = table
        for label, md, cf, tab in variants:
            if tab is not None:
                ss.ss_set_auto_table(o, *tab)
            db.ensure_work(md)
            with torch.cuda.stream(stream):
                for _ in range(3):
                    db.solve(mode=md, cfg=cf, stream=sh)
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                reps = max(3, min(args.steps, 50))
                c0.record(stream)
                for _ in range(reps):
                    db.solve(mode=md, cfg=cf, stream=sh)
                c1.record(stream)
            stream.synchronize()
            cms = max_over_ranks(dist, c0.elapsed_time(c1) / reps, dev)
            compare[label] = {"ms_per_step": cms,
                              "value": sum_over_ranks(dist, float(pk.batch), dev) / (cms * 1e-3)}
        if saved is not None:
            ss.ss_set_auto_table(o, *saved)
        else:
            ss.ss_set_auto_table(o, [], [])

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # The dominant kernel: the (mode, cfg) of the largest size bin's group.
    if table:
        kbin = ss.size_bin(int(pk.n.max()))
        dm, dc = table[0][kbin], table[1][kbin]
        inv = {v: k for k, v in ss.MODES.items()}
        dominant_key = f"{name}:{op}:{inv.get(dm, 'fp64')}:{dc}"
    else:
        dominant_key = f"{name}:{op}:{args.mode}:{cfg}"
    achieved = Falg / (kern_avg_ms * 1e-3) / 1e9
    df_dominant = dominant_key.split(":")[2] == "df"
    if df_dominant:
        peak, peak_source = DF_PEAK_GFLOPS, (
            "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz / 13 FP32 instructions per double-float "
            "multiply-add x 2 flop (of derived; an FFMA probe measured 72 TFLOP/s, 89 % of the nominal "
            "FP32 rate)")
    else:
        peak, peak_source = FP64_PEAK_GFLOPS, ("derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz "
                                               "(of derived; a DFMA probe measured 1248 GFLOP/s)")
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
            "frac": achieved / peak,
            "traffic": read_traffic(dominant_key),
            "kernel": f"{op} persistent solve kernels ({'selector tables' if learned else args.mode})",
            "dominant": dominant_key,
            "peak_source": peak_source,
            "fp64_equivalent_frac": achieved / FP64_PEAK_GFLOPS,
            "frac_of_measured_ffma": (achieved / DF_PEAK_MEASURED_FFMA_GFLOPS) if df_dominant else None,
            "kernel_ms": kern_avg_ms, "algorithmic_bytes": Balg,
            "hbm_frac": Balg / (kern_avg_ms * 1e-3) / 6801.3e9}
    used = sorted({inv_mode(m) for m in table[0] if m >= 0}) if table else [args.mode]
    dtype = " + ".join(DTYPE_OF_MODE.get(m, m) for m in used) + " (X in f64)"

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": name, "op": op, "batch": pk.batch,
                   "sizes": f"n in [{int(pk.n.min())}, {int(pk.n.max())}], mean {float(pk.n.mean()):.1f}",
                   "path": (f"mixed+learned (SS_MODE_AUTO, trained selector, {args.policy} policy)"
                            if learned else args.mode),
                   "cfg": cfg, "graph": bool(args.graph),
                   "selector_table": [[int(m), int(c)] for m, c in zip(*table)] if table else None,
                   "l2": f"operands {sum(int(v.numel()) * 8 for v in db.bufs.values()) / 1e6:.0f} MB > 129 MB L2; no flush"},
        "gflops_paper_count": F / (ms_step * 1e-3) / 1e9,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "launches_per_step": launches / args.steps,
        "clocks": clk,
        "info_nonzero": int((info != 0).sum()),
        "plain_fp64": compare or None,
        "speedup_vs_plain_fp64_default": (value / compare["fp64_default"]["value"]) if compare else None,
        "speedup_vs_plain_fp64_tuned": (value / compare["fp64_tuned"]["value"]) if compare else None,
    }

    if not args.no_cpu:
        threads = os.cpu_count() or 1
        idx = sample_indices(pk, max(16, pk.batch // 8))
        rate, done, el, out = cpu_oracle_rate(op, pk, args.cpu_seconds, threads, indices=idx)
        # Accuracy of the GPU result on the oracle's sample.
        errs = []
        for b in idx:
            nb, o = int(pk.n[b]), int(pk.off[b])
            g = x_gpu[o:o + nb * nb].reshape(nb, nb, order="F")
            r = out[o:o + nb * nb].reshape(nb, nb, order="F")
            if op == "potrf":
                g, r = np.triu(g), np.triu(r)
            elif op == "trlyap":
                g, r = np.tril(g), np.tril(r)
            errs.append(np.linalg.norm(g - r) / np.linalg.norm(r))
        line["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": threads, "kind": "oracle",
                                "sample": f"{len(idx)} seeded random instances of {name}, "
                                          f"repeated for {el:.1f} s ({done} solves)"}
        line["accuracy"] = {"max_rel_fro_err_vs_oracle": float(max(errs)), "gate": GATE,
                            "instances_checked": len(idx), "pass": bool(max(errs) <= GATE)}
    if not args.no_side:
        line["workloads"] = measure_side_workloads(args, dev, stream)
        line["selector_stream"] = measure_selector_stream()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
