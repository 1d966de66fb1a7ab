"""The block schedule of the warp-specialised Sylvester / Lyapunov kernels,
modelled on the host.

The kernels solve blocks (I, J) of X in row-major order (Lyapunov: the lower
blocks J <= I only).  The block right-hand side is T_IJ = C_IJ - sum_{K<I}
L_IK X_KJ - sum_{K<J} X_IK U_KJ (Lyapunov: U = L^T, X symmetric, so X_KJ with
K < J is read as X_JK^T), the block form of the equations L X + X U = C and
L X + X L^T = S of the paper's case studies (Fig. 2 caption).  The update
warps form T_IJ in "bulk steps" from operands staged out of memory while the
diagonal warp still solves the previous block, then add the terms that need
that previous block from shared memory ("last phase") once it is final.
`plan` restates which operand tiles each step and the last phase take: the
selection in step_src / last_src_t of csrc/solve_fp64_ws.cu, including the
Lyapunov diagonal block and the single-block-column special cases.

Two properties are checked for square, rectangular and Lyapunov shapes:

* coverage - solving block by block with exactly these terms reproduces the
  oracle's X (numerically, with the small diagonal-block systems solved by
  scipy), so every term of every T_IJ is present once, with the right
  operand orientation;
* hand-off - every X block a bulk step reads was solved at least two blocks
  earlier (its copy in memory is complete before the "X final" arrival the
  update warps waited for at the end of the block before), and the last phase
  reads only the block solved just before, from shared memory.

The diagonal warp's double-float wavefront is modelled the same way: its lane
split gives every entry of every block shape all its terms exactly once, and
the per-part base offsets of the non-symmetric form address the same
shared-memory elements as the per-term operand selects they replace.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1906_08613_gb300 import inputs


def block_order(mb, nb, lyap):
    return [(I, J) for I in range(mb) for J in range(I + 1 if lyap else nb)]


def plan(I, J, nb, lyap):
    """(bulk steps, last-phase terms) of block (I, J).  A term is a pair of
    operand tiles (name, row block, column block, transposed); its
    contribution is op(a) op(b), subtracted from T_IJ."""
    ldiag = lyap and I == J and I > 0
    lfirst = J == 0 and I > 0 and (I == 1 if lyap else nb == 1)
    p1 = I - 1 if (ldiag or lfirst) else I
    has_last = J > 0 or lfirst
    nsteps = p1 + (J - 1 if J > 0 else 0)
    steps = []
    for s in range(nsteps):
        if s < p1:
            k = s
            a = ("L", I, k, False)
            if not lyap or s > J:
                b = ("X", k, J, False)
            elif s == J:
                b = ("Xsym", J, J, False)
            else:
                b = ("X", J, k, True)
        else:
            k = s - p1
            a = ("X", I, k, False)
            b = ("L", J, k, True) if lyap else ("U", k, J, False)
        steps.append((a, b))
    last = []
    if has_last:
        if J > 0:
            last.append((("X", I, J - 1, False), ("L", J, J - 1, True) if lyap else ("U", J - 1, J, False)))
            if ldiag:
                last.append((("L", I, I - 1, False), ("X", I, I - 1, True)))
        else:
            # Lyapunov (I = 1): X_00 is the symmetric block the diagonal warp
            # mirrored in shared memory.
            last.append((("L", I, I - 1, False), ("Xsym" if lyap else "X", I - 1, 0, False)))
    return steps, last


def tile(mats, ref, bs):
    name, r, c, tr = ref
    m = mats["X" if name == "Xsym" else name]
    t = m[r * bs:(r + 1) * bs, c * bs:(c + 1) * bs]
    if name == "Xsym":                       # lower triangle stored, mirrored
        t = np.tril(t) + np.tril(t, -1).T
    return t.T if tr else t


def blocked_solve(L, U, C, bs, lyap):
    """X by the modelled schedule: T from the planned terms, then the
    diagonal-block system L_II X_IJ + X_IJ U_JJ = T_IJ."""
    m, n = C.shape
    mb, nb = -(-m // bs), -(-n // bs)
    X = np.zeros((m, n))
    mats = {"L": L, "U": U, "X": X}
    for I, J in block_order(mb, nb, lyap):
        steps, last = plan(I, J, nb, lyap)
        T = C[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs].copy()
        if lyap and I == J:
            T = np.tril(T) + np.tril(T, -1).T
        for a, b in steps + last:
            T -= tile(mats, a, bs) @ tile(mats, b, bs)
        Lii = L[I * bs:(I + 1) * bs, I * bs:(I + 1) * bs]
        Ujj = (L[J * bs:(J + 1) * bs, J * bs:(J + 1) * bs].T if lyap
               else U[J * bs:(J + 1) * bs, J * bs:(J + 1) * bs])
        Y = scipy.linalg.solve_sylvester(Lii, Ujj, T)
        if lyap and I == J:
            Y = np.tril(Y)
        X[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = Y
    return X


SHAPES = [(1, 1), (4, 4), (5, 5), (16, 16), (33, 33), (40, 40), (4, 37), (37, 4), (23, 41), (41, 23), (8, 3)]


@pytest.mark.parametrize("bs", [4, 8])
@pytest.mark.parametrize("m,n", SHAPES)
def test_sylvester_terms_cover_the_block_recurrence(m, n, bs):
    L, U, C, _ = inputs.sylvester_rect_instance(m, n, 17, m * 100 + n)
    X = blocked_solve(L, U, C, bs, lyap=False)
    ref, info = oracle.trsyl_rect(L, U, C)
    assert info == 0
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("bs", [4, 8])
@pytest.mark.parametrize("n", [1, 4, 5, 8, 9, 16, 17, 33, 40])
def test_lyapunov_terms_cover_the_block_recurrence(n, bs):
    L, S, _ = inputs.lyapunov_instance(n, 19, n)
    X = blocked_solve(L, None, S, bs, lyap=True)
    ref, info = oracle.trlyap_l(L, S)
    assert info == 0
    assert np.linalg.norm(np.tril(X) - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("lyap", [False, True])
@pytest.mark.parametrize("mb,nb", [(1, 1), (1, 5), (5, 1), (2, 2), (3, 7), (7, 3), (8, 8), (16, 16)])
def test_hand_off_reads_only_final_blocks(mb, nb, lyap):
    if lyap and mb != nb:
        pytest.skip("Lyapunov blocks are square")
    order = block_order(mb, nb, lyap)
    pos = {blk: t for t, blk in enumerate(order)}
    for t, (I, J) in enumerate(order):
        steps, last = plan(I, J, nb, lyap)
        for a, b in steps:
            for name, r, c, _ in (a, b):
                if name in ("X", "Xsym"):
                    assert pos[(r, c)] <= t - 2, ((I, J), (r, c))
        for a, b in last:
            xs = [(r, c) for name, r, c, _ in (a, b) if name in ("X", "Xsym")]
            assert xs and all(pos[x] == t - 1 for x in xs), ((I, J), xs)


def test_the_special_cases_are_needed():
    """Without the Lyapunov-diagonal and single-column hand-offs the bulk
    steps would read the block solved just before, whose copy in memory is
    still being written: the model's hand-off check must see that."""
    def bulk_reads_previous(mb, nb, lyap):
        order = block_order(mb, nb, lyap)
        pos = {blk: t for t, blk in enumerate(order)}
        for t, (I, J) in enumerate(order):
            p1 = I                                   # no special case
            for k in range(p1):
                blk = (k, J) if (not lyap or k > J) else ((J, J) if k == J else (J, k))
                if pos[blk] == t - 1:
                    return True
        return False
    assert bulk_reads_previous(4, 4, True)           # X_{I,I-1} in the diagonal block's first sum
    assert bulk_reads_previous(4, 1, False)          # X_{I-1,0} with a single block column
    assert not bulk_reads_previous(4, 4, False)


# ---- the diagonal warp's wavefront (warp_diag_solve_df) ----------------------

def wf_step(d, m, nn, sym):
    """Per-step constants: first row, entry count and lanes per entry (a
    power of two: at most 32 / entries rounded down to a power of two, at most
    the largest power of two <= d)."""
    ilo = max((d + 1) // 2, d - nn + 1) if sym else max(0, d - nn + 1)
    cnt = min(d, m - 1) - ilo + 1
    by_cnt = 1 if cnt >= 32 else 32 >> (0 if cnt <= 1 else (cnt - 1).bit_length())
    by_len = 1 << (max(d, 1).bit_length() - 1)
    return ilo, cnt, min(by_cnt, by_len)


@pytest.mark.parametrize("B,LDT", [(16, 18), (32, 34)])
@pytest.mark.parametrize("sym", [False, True])
def test_wavefront_lanes_cover_each_entry_once(B, LDT, sym):
    for m in range(1, B + 1):
        for nn in ([m] if sym else range(1, B + 1)):
            seen = set()
            for d in range(m + nn - 1):
                ilo, cnt, split = wf_step(d, m, nn, sym)
                assert cnt * split <= 32 and split & (split - 1) == 0
                lg = split.bit_length() - 1
                terms = {}
                for lane in range(32):
                    idx, part = lane >> lg, lane & (split - 1)
                    if idx >= cnt:
                        continue
                    i = ilo + idx
                    j = d - i
                    assert 0 <= i < m and 0 <= j < nn and (not sym or i >= j)
                    terms.setdefault((i, j), []).extend(range(part, d, split))
                for e, ts in terms.items():
                    assert sorted(ts) == list(range(d)), (m, nn, d, e)
                    seen.add(e)
            want = {(i, j) for i in range(m) for j in range(nn) if not sym or i >= j}
            assert seen == want


@pytest.mark.parametrize("B,LDT", [(16, 18), (32, 34)])
def test_wavefront_base_offsets_match_the_operand_selects(B, LDT):
    """Non-symmetric blocks: term t of entry (i, j) reads sLU[i + t LDT] and
    sT[t + j LDT] for t < i, sT[i + (t - i) LDT] and sLU[(t - i) + j LDT]
    from t = i on; the kernel forms both as offsets from sT with bases that
    switch at t = i.  Same elements, all inside the two tiles."""
    dlu = -3 * B * LDT                      # sLU - sT in elements (any offset)
    for m in range(1, B + 1):
        for nn in range(1, B + 1):
            for d in range(m + nn - 1):
                ilo, cnt, split = wf_step(d, m, nn, False)
                for idx in range(cnt):
                    i = ilo + idx
                    j = d - i
                    aL, aU, bL, bU = dlu + i, i - i * LDT, j * LDT, dlu - i + j * LDT
                    for t in range(d):
                        a = (aL if t < i else aU) + t * LDT
                        b = (bL if t < i else bU) + t
                        ea = dlu + i + t * LDT if t < i else i + (t - i) * LDT
                        eb = t + j * LDT if t < i else dlu + (t - i) + j * LDT
                        assert (a, b) == (ea, eb)
                        for off in (a, b):
                            base = dlu if dlu <= off < dlu + B * LDT else 0
                            assert 0 <= off - base < B * LDT
                            r, c = (off - base) % LDT, (off - base) // LDT
                            assert r < B and c < B
