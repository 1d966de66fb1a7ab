"""Seeded synthetic inputs for the three structured solves.

This module builds problem instances and nothing else: it holds none of the
solvers' arithmetic and imports neither the library binding nor the oracle.
Both sides of every parity check (the CUDA path and the CPU oracle) consume the
same arrays produced here.

Instances are packed into one flat float64 buffer per operand.  Instance ``b``
is an ``n[b] x n[b]`` column-major matrix with leading dimension ``n[b]`` that
starts at element offset ``off[b]``; offsets are multiples of 32 elements
(256 bytes) so that every instance starts on a 256-byte boundary.

Recipes (the paper's case studies are square double-precision matrices, Fig. 2
caption; the distributions below stand in for its size sweep, which used no
public dataset):

* Cholesky:  X0 upper triangular with N(0,1) entries (diagonal included),
  A = X0^T X0 + n I.  ``exact=True`` instead draws X0 with integer entries
  (off-diagonal in [-3, 3], diagonal in [1, 4]) and A = X0^T X0, which is exact
  in FP64, so the unique factor with positive diagonal is X0 itself.
* Sylvester: L lower and U upper triangular, off-diagonals N(0,1)/sqrt(n),
  diagonals uniform in [1, 2]; X0 ~ N(0,1); C = L X0 + X0 U.
* Lyapunov:  L as above; X0 symmetric (lower triangle of G ~ N(0,1) mirrored);
  M = L X0 and S = M + M^T, exactly symmetric.

Every instance draws from its own generator seeded with ``(seed, b)``, so a
single instance of a large batch can be regenerated on its own.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ALIGN_ELEMS = 32


@dataclasses.dataclass
class Packed:
    """A batch of square instances packed into flat float64 operand buffers."""

    n: np.ndarray            # int32 [batch]
    off: np.ndarray          # int64 [batch], element offsets
    total: int               # elements per operand buffer
    ops: dict                # name -> float64 [total]

    @property
    def batch(self) -> int:
        return int(self.n.shape[0])

    def view(self, name: str, b: int) -> np.ndarray:
        """Column-major n x n view of instance b of operand ``name``."""
        nb = int(self.n[b])
        o = int(self.off[b])
        return self.ops[name][o:o + nb * nb].reshape(nb, nb, order="F")


def pack_offsets(n: np.ndarray, align: int = ALIGN_ELEMS):
    n = np.asarray(n, dtype=np.int64)
    sizes = ((n * n + align - 1) // align) * align
    off = np.zeros_like(sizes)
    if len(sizes) > 1:
        off[1:] = np.cumsum(sizes)[:-1]
    total = int(sizes.sum()) if len(sizes) else 0
    return off, max(total, align)


def sizes_fixed(batch: int, n: int) -> np.ndarray:
    return np.full(batch, n, dtype=np.int32)


def sizes_uniform(batch: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n uniform over the integers lo..hi inclusive."""
    rng = np.random.default_rng([seed, 0x5151])
    return rng.integers(lo, hi + 1, size=batch).astype(np.int32)


def sizes_log_uniform(batch: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """n = round(exp(U(ln lo, ln hi))), clipped to [lo, hi]."""
    rng = np.random.default_rng([seed, 0x10a1])
    v = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=batch)))
    return np.clip(v, lo, hi).astype(np.int32)


def _instance_rng(seed: int, b: int) -> np.random.Generator:
    return np.random.default_rng([seed, 7919, b])


def _tri_factors(rng: np.random.Generator, n: int, lower: bool) -> np.ndarray:
    m = rng.standard_normal((n, n)) / math.sqrt(n)
    m = np.tril(m, -1) if lower else np.triu(m, 1)
    m[np.diag_indices(n)] = rng.uniform(1.0, 2.0, size=n)
    return m


def cholesky_instance(n: int, seed: int, b: int, exact: bool = False):
    rng = _instance_rng(seed, b)
    if exact:
        x0 = np.triu(rng.integers(-3, 4, size=(n, n)).astype(np.float64), 1)
        x0[np.diag_indices(n)] = rng.integers(1, 5, size=n).astype(np.float64)
        a = x0.T @ x0
    else:
        x0 = np.triu(rng.standard_normal((n, n)))
        a = x0.T @ x0 + n * np.eye(n)
        a = 0.5 * (a + a.T)
    return a, x0


def sylvester_instance(n: int, seed: int, b: int):
    rng = _instance_rng(seed, b)
    l = _tri_factors(rng, n, lower=True)
    u = _tri_factors(rng, n, lower=False)
    x0 = rng.standard_normal((n, n))
    c = l @ x0 + x0 @ u
    return l, u, c, x0


def lyapunov_instance(n: int, seed: int, b: int):
    rng = _instance_rng(seed, b)
    l = _tri_factors(rng, n, lower=True)
    g = rng.standard_normal((n, n))
    x0 = np.tril(g) + np.tril(g, -1).T
    m = l @ x0
    s = m + m.T
    return l, s, x0


def _pack(n: np.ndarray, names, make) -> Packed:
    n = np.asarray(n, dtype=np.int32)
    off, total = pack_offsets(n)
    ops = {k: np.zeros(total, dtype=np.float64) for k in names}
    for b, nb in enumerate(n):
        mats = make(int(nb), b)
        o = int(off[b])
        for k, m in zip(names, mats):
            ops[k][o:o + nb * nb] = np.asarray(m, dtype=np.float64).ravel(order="F")
    return Packed(n=n, off=off, total=total, ops=ops)


def cholesky_batch(n, seed: int, exact: bool = False) -> Packed:
    return _pack(n, ("A", "X0"), lambda nb, b: cholesky_instance(nb, seed, b, exact))


def sylvester_batch(n, seed: int) -> Packed:
    return _pack(n, ("L", "U", "C", "X0"), lambda nb, b: sylvester_instance(nb, seed, b))


def lyapunov_batch(n, seed: int) -> Packed:
    return _pack(n, ("L", "S", "X0"), lambda nb, b: lyapunov_instance(nb, seed, b))


# ---- rectangular Sylvester: L (m x m) lower, U (n x n) upper, C and X m x n ----

@dataclasses.dataclass
class RectPacked:
    """A batch of rectangular Sylvester instances.  Instance b has L at
    ``offL[b]`` (m x m, ld m), U at ``offU[b]`` (n x n, ld n) and C, X0 at
    ``offC[b]`` (m x n, ld m), each offset a multiple of 32 elements."""

    m: np.ndarray            # int32 [batch]
    n: np.ndarray            # int32 [batch]
    offL: np.ndarray         # int64 [batch]
    offU: np.ndarray
    offC: np.ndarray
    ops: dict                # "L", "U", "C", "X0" -> float64 buffers

    @property
    def batch(self) -> int:
        return int(self.m.shape[0])

    def view(self, name: str, b: int) -> np.ndarray:
        mb, nb = int(self.m[b]), int(self.n[b])
        rows, cols, o = {"L": (mb, mb, self.offL), "U": (nb, nb, self.offU)}.get(name, (mb, nb, self.offC))
        o = int(o[b])
        return self.ops[name][o:o + rows * cols].reshape(rows, cols, order="F")


def _offsets(elems: np.ndarray, align: int = ALIGN_ELEMS):
    sizes = ((np.asarray(elems, dtype=np.int64) + align - 1) // align) * align
    off = np.zeros_like(sizes)
    if len(sizes) > 1:
        off[1:] = np.cumsum(sizes)[:-1]
    return off, max(int(sizes.sum()) if len(sizes) else 0, align)


def sylvester_rect_instance(m: int, n: int, seed: int, b: int):
    """The square Sylvester recipe with an m x n unknown."""
    rng = _instance_rng(seed, b)
    l = _tri_factors(rng, m, lower=True)
    u = _tri_factors(rng, n, lower=False)
    x0 = rng.standard_normal((m, n))
    c = l @ x0 + x0 @ u
    return l, u, c, x0


def sylvester_rect_batch(m, n, seed: int) -> RectPacked:
    m = np.asarray(m, dtype=np.int32)
    n = np.asarray(n, dtype=np.int32)
    offL, tL = _offsets(m.astype(np.int64) ** 2)
    offU, tU = _offsets(n.astype(np.int64) ** 2)
    offC, tC = _offsets(m.astype(np.int64) * n)
    ops = {"L": np.zeros(tL), "U": np.zeros(tU), "C": np.zeros(tC), "X0": np.zeros(tC)}
    for b in range(len(m)):
        mb, nb = int(m[b]), int(n[b])
        l, u, c, x0 = sylvester_rect_instance(mb, nb, seed, b)
        ops["L"][offL[b]:offL[b] + mb * mb] = l.ravel(order="F")
        ops["U"][offU[b]:offU[b] + nb * nb] = u.ravel(order="F")
        ops["C"][offC[b]:offC[b] + mb * nb] = c.ravel(order="F")
        ops["X0"][offC[b]:offC[b] + mb * nb] = x0.ravel(order="F")
    return RectPacked(m=m, n=n, offL=offL, offU=offU, offC=offC, ops=ops)


# Rectangular Sylvester workloads: (m, n) pairs by name.
RECT_WORKLOADS = {
    # 4096 instances, m and n independent and uniform in {4..128}
    "trsyl_rect_4096xU4-128xU4-128": lambda s: (sizes_uniform(4096, 4, 128, s), sizes_uniform(4096, 4, 128, s + 1)),
}


def make_rect_workload(name: str, seed: int = 1234) -> RectPacked:
    m, n = RECT_WORKLOADS[name](seed)
    return sylvester_rect_batch(m, n, seed)


# ---- SPD solve A X = B through the Cholesky factor: A n x n, B and X n x k ----

@dataclasses.dataclass
class PosvPacked:
    """A batch of SPD solves.  Instance b has A at ``offA[b]`` (n x n, ld n) and
    B, X0 at ``offB[b]`` (n x k, ld n)."""

    n: np.ndarray
    k: np.ndarray
    offA: np.ndarray
    offB: np.ndarray
    ops: dict                # "A", "B", "X0"

    @property
    def batch(self) -> int:
        return int(self.n.shape[0])

    def view(self, name: str, b: int) -> np.ndarray:
        nb, kb = int(self.n[b]), int(self.k[b])
        rows, cols, o = (nb, nb, self.offA) if name == "A" else (nb, kb, self.offB)
        o = int(o[b])
        return self.ops[name][o:o + rows * cols].reshape(rows, cols, order="F")


def posv_instance(n: int, k: int, seed: int, b: int):
    """The Cholesky recipe's A (X0^T X0 + n I, X0 upper N(0,1)); a solution
    X0s ~ N(0,1) (n x k) and B = A X0s."""
    a, _ = cholesky_instance(n, seed, b)
    rng = np.random.default_rng([seed, 7907, b])
    xs = rng.standard_normal((n, k))
    return a, a @ xs, xs


def posv_batch(n, k, seed: int) -> PosvPacked:
    n = np.asarray(n, dtype=np.int32)
    k = np.asarray(k, dtype=np.int32)
    offA, tA = _offsets(n.astype(np.int64) ** 2)
    offB, tB = _offsets(n.astype(np.int64) * k)
    ops = {"A": np.zeros(tA), "B": np.zeros(tB), "X0": np.zeros(tB)}
    for b in range(len(n)):
        nb, kb = int(n[b]), int(k[b])
        a, bb, xs = posv_instance(nb, kb, seed, b)
        ops["A"][offA[b]:offA[b] + nb * nb] = a.ravel(order="F")
        ops["B"][offB[b]:offB[b] + nb * kb] = bb.ravel(order="F")
        ops["X0"][offB[b]:offB[b] + nb * kb] = xs.ravel(order="F")
    return PosvPacked(n=n, k=k, offA=offA, offB=offB, ops=ops)


POSV_WORKLOADS = {
    # 4096 SPD systems, n uniform in {8..128}, 16 right-hand sides each
    "posv_4096xU8-128xk16": lambda s: (sizes_uniform(4096, 8, 128, s), np.full(4096, 16, dtype=np.int32)),
}


def make_posv_workload(name: str, seed: int = 1234) -> PosvPacked:
    n, k = POSV_WORKLOADS[name](seed)
    return posv_batch(n, k, seed)


# The workloads measured and parity-checked by this project, by name.
WORKLOADS = {
    # plain FP64 upper Cholesky, 1024 instances of order 64
    "potrf_1024x64": dict(op="potrf", sizes=lambda s: sizes_fixed(1024, 64)),
    # FP64 triangular Sylvester, 4096 instances, n uniform in {4..128}
    "trsyl_4096xU4-128": dict(op="trsyl", sizes=lambda s: sizes_uniform(4096, 4, 128, s)),
    # triangular Lyapunov, 2048 instances of order 128
    "trlyap_2048x128": dict(op="trlyap", sizes=lambda s: sizes_fixed(2048, 128)),
    # mixed-size Cholesky, 8192 instances, n log-uniform in [8, 256]
    "potrf_8192xLU8-256": dict(op="potrf", sizes=lambda s: sizes_log_uniform(8192, 8, 256, s)),
    # quarter-size cases for detailed profiles (operands still > L2)
    "trsyl_1024xU4-128": dict(op="trsyl", sizes=lambda s: sizes_uniform(1024, 4, 128, s)),
    "trlyap_512x128": dict(op="trlyap", sizes=lambda s: sizes_fixed(512, 128)),
    "potrf_2048xLU8-256": dict(op="potrf", sizes=lambda s: sizes_log_uniform(2048, 8, 256, s)),
    # few large instances (one or two CTAs per SM): n uniform in {257..512}
    "trsyl_64xU257-512": dict(op="trsyl", sizes=lambda s: sizes_uniform(64, 257, 512, s)),
    "trsyl_256xU257-512": dict(op="trsyl", sizes=lambda s: sizes_uniform(256, 257, 512, s)),
    "trlyap_128xU257-512": dict(op="trlyap", sizes=lambda s: sizes_uniform(128, 257, 512, s)),
}


def make_workload(name: str, seed: int = 1234) -> Packed:
    w = WORKLOADS[name]
    n = w["sizes"](seed)
    return make_batch(w["op"], n, seed)


def make_batch(op: str, n, seed: int) -> Packed:
    if op == "potrf":
        return cholesky_batch(n, seed)
    if op == "trsyl":
        return sylvester_batch(n, seed)
    if op == "trlyap":
        return lyapunov_batch(n, seed)
    raise ValueError(f"unknown op {op!r}")


# ---- magnitude: instances rescaled by powers of two ----
#
# The problems are plain double precision (the paper's "Preliminary
# performance results" paragraph), so a solver must give the same accuracy on
# data of any magnitude.  Multiplying an instance's operands by powers of two
# is exact in FP64, which makes these scaled copies test inputs whose
# solutions are known exactly in terms of the unscaled ones.

RANGE_SHIFTS = (0, 70, -70, 100, -100, 130, -130)


def scale_instances(pk, op: str, shifts) -> None:
    """In place: instance b's operator by 2^s_op and its right-hand side by
    2^s_rhs, with shifts[b] = (s_op, s_rhs).  Sylvester / Lyapunov (Packed):
    L and U (or L) by 2^s_op, C (or S) by 2^s_rhs, so X becomes
    2^(s_rhs - s_op) X.  Cholesky (Packed): A by 2^s_op (s_op even, X by
    2^(s_op / 2)); s_rhs is unused.  Rectangular Sylvester (RectPacked): as
    Sylvester.  SPD solve (PosvPacked): A by 2^s_op, B by 2^s_rhs.  The stored
    X0 is scaled to match (Cholesky, SPD solve: left as it is)."""
    for b, (so, sr) in enumerate(shifts):
        if isinstance(pk, RectPacked):
            mb, nb = int(pk.m[b]), int(pk.n[b])
            for name, o, cnt, s in (("L", pk.offL, mb * mb, so), ("U", pk.offU, nb * nb, so),
                                    ("C", pk.offC, mb * nb, sr), ("X0", pk.offC, mb * nb, sr - so)):
                seg = slice(int(o[b]), int(o[b]) + cnt)
                pk.ops[name][seg] = np.ldexp(pk.ops[name][seg], s)
            continue
        if isinstance(pk, PosvPacked):
            nb, kb = int(pk.n[b]), int(pk.k[b])
            for name, o, cnt, s in (("A", pk.offA, nb * nb, so), ("B", pk.offB, nb * kb, sr)):
                seg = slice(int(o[b]), int(o[b]) + cnt)
                pk.ops[name][seg] = np.ldexp(pk.ops[name][seg], s)
            continue
        nb, o = int(pk.n[b]), int(pk.off[b])
        seg = slice(o, o + nb * nb)
        if op == "potrf":
            if so % 2:
                raise ValueError("a Cholesky operator shift must be even")
            pk.ops["A"][seg] = np.ldexp(pk.ops["A"][seg], so)
            pk.ops["X0"][seg] = np.ldexp(pk.ops["X0"][seg], so // 2)
            continue
        names = ("L", "U") if op == "trsyl" else ("L",)
        for name in names:
            pk.ops[name][seg] = np.ldexp(pk.ops[name][seg], so)
        rhs = "C" if op == "trsyl" else "S"
        pk.ops[rhs][seg] = np.ldexp(pk.ops[rhs][seg], sr)
        pk.ops["X0"][seg] = np.ldexp(pk.ops["X0"][seg], sr - so)


def range_shifts(batch: int, op: str, seed: int = 0):
    """Per-instance (s_op, s_rhs) pairs that mix well-scaled instances with
    instances scaled by 2^+-70, 2^+-100 and 2^+-130, cycling through those
    shifts s: instance b gets, by b mod 4, no scaling, (s, s) (the whole
    instance; X unchanged), (0, s) (the right-hand side; X by 2^s) or
    (s, -s) (X by 2^-2s).  Cholesky: (2s, 0), so that X moves by 2^s.  The
    start of the cycle depends on the seed."""
    nz = [s for s in RANGE_SHIFTS if s != 0]
    out = []
    for b in range(batch):
        s = nz[(b // 4 + seed) % len(nz)]
        if b % 4 == 0:
            out.append((0, 0))
        elif op == "potrf":
            out.append((2 * s, 0))
        elif b % 4 == 1:
            out.append((s, s))
        elif b % 4 == 2:
            out.append((0, s))
        else:
            out.append((s, -s))
    return out
