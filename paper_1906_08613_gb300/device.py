"""Device-memory plumbing for packed batches (allocation and pointer arrays).

PyTorch provides device memory and streams only; the solves themselves go
through the C ABI (``smallsolve``).  A ``DeviceBatch`` uploads a packed batch
(see ``inputs.Packed``), builds the per-instance pointer and size arrays the
entry points take, allocates X, info and the workspace, and calls the entry
point for its operation.
"""
from __future__ import annotations

import numpy as np
import torch

from . import smallsolve as ss

OPERANDS = {"potrf": ("A",), "trsyl": ("L", "U", "C"), "trlyap": ("L", "S")}


class DeviceBatch:
    def __init__(self, n, off, ops: dict, op: str, device="cuda", alias_rhs: bool = False,
                 x_fill: float = 0.0, max_n: int | None = None):
        self.op = op
        self.device = torch.device(device)
        n = np.ascontiguousarray(n, dtype=np.int32)
        off = np.ascontiguousarray(off, dtype=np.int64)
        self.batch = int(n.shape[0])
        self.max_n = int(n.max()) if (max_n is None and self.batch) else int(max_n or 0)
        self.n_host = n
        self.off_host = off
        self.d_n = torch.from_numpy(n).to(self.device)
        self.d_ld = torch.from_numpy(np.maximum(n, 1).astype(np.int32)).to(self.device)
        self.bufs = {k: torch.from_numpy(np.ascontiguousarray(ops[k])).to(self.device)
                     for k in OPERANDS[op]}
        rhs = {"potrf": "A", "trsyl": "C", "trlyap": "S"}[op]
        total = int(next(iter(ops.values())).shape[0])
        if alias_rhs:
            self.X = self.bufs[rhs]
        else:
            self.X = torch.full((total,), x_fill, dtype=torch.float64, device=self.device)
        offb = torch.from_numpy(off * 8).to(self.device)
        self.ptrs = {k: (v.data_ptr() + offb).contiguous() for k, v in self.bufs.items()}
        self.ptrs["X"] = (self.X.data_ptr() + offb).contiguous()
        self.info = torch.full((max(self.batch, 1),), 12345, dtype=torch.int32, device=self.device)
        self.work = None
        self.work_bytes = 0

    def ensure_work(self, mode: int) -> None:
        need = ss.ss_workspace_size(ss.OPS[self.op], self.batch, self.max_n, mode)
        if self.work is None or self.work_bytes < need:
            self.work = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            self.work_bytes = int(self.work.numel())

    def solve(self, mode: int = ss.MODE_FP64, cfg: int = ss.CFG_DEFAULT, stream: int = 0,
              check: bool = True) -> int:
        self.ensure_work(mode)
        p = self.ptrs
        ld = self.d_ld.data_ptr()
        w = self.work.data_ptr()
        common = dict(mode=mode, cfg=cfg, d_work=w, work_bytes=self.work_bytes, stream=stream,
                      check=check)
        if self.op == "potrf":
            return ss.potrf_upper(self.batch, self.max_n, self.d_n.data_ptr(), p["A"].data_ptr(), ld,
                                  p["X"].data_ptr(), ld, self.info.data_ptr(), **common)
        if self.op == "trsyl":
            return ss.trsyl_lu(self.batch, self.max_n, self.d_n.data_ptr(), p["L"].data_ptr(), ld,
                               p["U"].data_ptr(), ld, p["C"].data_ptr(), ld, p["X"].data_ptr(), ld,
                               self.info.data_ptr(), **common)
        return ss.trlyap_l(self.batch, self.max_n, self.d_n.data_ptr(), p["L"].data_ptr(), ld,
                           p["S"].data_ptr(), ld, p["X"].data_ptr(), ld, self.info.data_ptr(),
                           **common)

    def autotune(self, mode: int, reps: int = 3, stream: int = 0):
        """ss_autotune on this batch: (ms per configuration, bad instances per
        configuration, best configuration) of `mode`."""
        self.ensure_work(mode)
        p = self.ptrs
        ld = self.d_ld.data_ptr()
        names = {"potrf": ("A", None, None), "trsyl": ("L", "U", "C"), "trlyap": ("L", None, "S")}[self.op]
        a, b, c = (p[k] if k is not None else None for k in names)
        ptr = lambda t: t.data_ptr() if t is not None else 0
        return ss.ss_autotune(ss.OPS[self.op], mode, self.batch, self.max_n, self.d_n.data_ptr(), ptr(a), ld,
                              ptr(b), ld if b is not None else 0, ptr(c), ld if c is not None else 0,
                              p["X"].data_ptr(), ld, self.info.data_ptr(), self.work.data_ptr(), self.work_bytes,
                              reps=reps, stream=stream)

    def x_host(self) -> np.ndarray:
        return self.X.cpu().numpy()

    def info_host(self) -> np.ndarray:
        return self.info[: self.batch].cpu().numpy()


class DeviceRectBatch:
    """Device copy of a rectangular Sylvester batch (inputs.RectPacked) with the
    pointer and size arrays trsyl_rect takes; X is laid out like C."""

    def __init__(self, pk, device="cuda", alias_rhs: bool = False, x_fill: float = 0.0,
                 max_m: int | None = None, max_n: int | None = None):
        self.device = torch.device(device)
        self.batch = pk.batch
        m = np.ascontiguousarray(pk.m, dtype=np.int32)
        n = np.ascontiguousarray(pk.n, dtype=np.int32)
        self.max_m = int(m.max()) if (max_m is None and self.batch) else int(max_m or 0)
        self.max_n = int(n.max()) if (max_n is None and self.batch) else int(max_n or 0)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(self.device)
        self.d_m, self.d_n = to(m), to(n)
        self.d_ldm = to(np.maximum(m, 1).astype(np.int32))
        self.d_ldn = to(np.maximum(n, 1).astype(np.int32))
        self.bufs = {k: to(pk.ops[k]) for k in ("L", "U", "C")}
        self.X = self.bufs["C"] if alias_rhs else torch.full_like(self.bufs["C"], x_fill)
        off = {"L": pk.offL, "U": pk.offU, "C": pk.offC}
        self.ptrs = {k: (v.data_ptr() + to(off[k] * 8)).contiguous() for k, v in self.bufs.items()}
        self.ptrs["X"] = (self.X.data_ptr() + to(pk.offC * 8)).contiguous()
        self.info = torch.full((max(self.batch, 1),), 12345, dtype=torch.int32, device=self.device)
        # sized for SS_MODE_DF, which needs more than FP64 (its scale array)
        need = ss.ss_workspace_size(ss.OP_TRSYL, self.batch, max(self.max_m, self.max_n), ss.MODE_DF)
        self.work = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)

    def solve(self, cfg: int = ss.CFG_DEFAULT, mode: int = ss.MODE_FP64, stream: int = 0,
              check: bool = True) -> int:
        p = self.ptrs
        return ss.trsyl_rect(self.batch, self.max_m, self.max_n, self.d_m.data_ptr(), self.d_n.data_ptr(),
                             p["L"].data_ptr(), self.d_ldm.data_ptr(), p["U"].data_ptr(), self.d_ldn.data_ptr(),
                             p["C"].data_ptr(), self.d_ldm.data_ptr(), p["X"].data_ptr(), self.d_ldm.data_ptr(),
                             self.info.data_ptr(), mode=mode, cfg=cfg, d_work=self.work.data_ptr(),
                             work_bytes=int(self.work.numel()), stream=stream, check=check)

    def x_host(self) -> np.ndarray:
        return self.X.cpu().numpy()

    def info_host(self) -> np.ndarray:
        return self.info[: self.batch].cpu().numpy()


class DevicePosvBatch:
    """Device copy of an SPD-solve batch (inputs.PosvPacked) for posv_upper;
    R is laid out like A, X like B."""

    def __init__(self, pk, device="cuda", alias: bool = False, x_fill: float = 0.0,
                 max_n: int | None = None, max_k: int | None = None):
        self.device = torch.device(device)
        self.batch = pk.batch
        n = np.ascontiguousarray(pk.n, dtype=np.int32)
        k = np.ascontiguousarray(pk.k, dtype=np.int32)
        self.max_n = int(n.max()) if (max_n is None and self.batch) else int(max_n or 0)
        self.max_k = int(k.max()) if (max_k is None and self.batch) else int(max_k or 0)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(self.device)
        self.d_n, self.d_k = to(n), to(k)
        self.d_ld = to(np.maximum(n, 1).astype(np.int32))
        self.bufs = {"A": to(pk.ops["A"]), "B": to(pk.ops["B"])}
        self.R = self.bufs["A"] if alias else torch.full_like(self.bufs["A"], x_fill)
        self.X = self.bufs["B"] if alias else torch.full_like(self.bufs["B"], x_fill)
        oA, oB = to(pk.offA * 8), to(pk.offB * 8)
        self.ptrs = {"A": (self.bufs["A"].data_ptr() + oA).contiguous(), "R": (self.R.data_ptr() + oA).contiguous(),
                     "B": (self.bufs["B"].data_ptr() + oB).contiguous(), "X": (self.X.data_ptr() + oB).contiguous()}
        self.info = torch.full((max(self.batch, 1),), 12345, dtype=torch.int32, device=self.device)
        # sized for SS_MODE_DF, which needs more than FP64 (its scale array)
        need = ss.ss_workspace_size(ss.OP_POTRF, self.batch, self.max_n, ss.MODE_DF)
        self.work = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)

    def solve(self, cfg: int = ss.CFG_DEFAULT, mode: int = ss.MODE_FP64, stream: int = 0,
              check: bool = True) -> int:
        p, ld = self.ptrs, self.d_ld.data_ptr()
        return ss.posv_upper(self.batch, self.max_n, self.max_k, self.d_n.data_ptr(), self.d_k.data_ptr(),
                             p["A"].data_ptr(), ld, p["R"].data_ptr(), ld, p["B"].data_ptr(), ld,
                             p["X"].data_ptr(), ld, self.info.data_ptr(), mode=mode, cfg=cfg,
                             d_work=self.work.data_ptr(), work_bytes=int(self.work.numel()), stream=stream,
                             check=check)

    def x_host(self) -> np.ndarray:
        return self.X.cpu().numpy()

    def r_host(self) -> np.ndarray:
        return self.R.cpu().numpy()

    def info_host(self) -> np.ndarray:
        return self.info[: self.batch].cpu().numpy()
