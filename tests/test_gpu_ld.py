"""Leading dimensions larger than the order (ld = n + pad, a different pad per
operand and per instance), for every entry point: the kernels must index each
operand with its own leading dimension and leave the padding rows untouched."""
import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAD_FILL = -3.5


def padded(mats, pads, dev):
    """Pack column-major matrices with leading dimension rows + pad into one
    device buffer; returns (buffer, pointer array, ld array, offsets, lds)."""
    offs, lds, total = [], [], 0
    for m, p in zip(mats, pads):
        r, c = m.shape
        ld = r + p
        offs.append(total)
        lds.append(ld)
        total += ((ld * max(c, 1) + 31) // 32) * 32
    host = np.full(max(total, 32), PAD_FILL)
    for m, o, ld in zip(mats, offs, lds):
        r, c = m.shape
        for j in range(c):
            host[o + j * ld:o + j * ld + r] = m[:, j]
    buf = torch.from_numpy(host).to(dev)
    ptr = (buf.data_ptr() + torch.tensor(offs, dtype=torch.int64, device=dev) * 8).contiguous()
    return buf, ptr, torch.tensor(lds, dtype=torch.int32, device=dev), offs, lds


def unpack(buf, offs, lds, shapes):
    host = buf.cpu().numpy()
    out = []
    for o, ld, (r, c) in zip(offs, lds, shapes):
        m = np.stack([host[o + j * ld:o + j * ld + r] for j in range(c)], axis=1) if c else np.zeros((r, 0))
        pad = np.concatenate([host[o + j * ld + r:o + (j + 1) * ld] for j in range(c)]) if c else np.zeros(0)
        out.append((m, pad))
    return out


def work(op, batch, max_n, mode=ss.MODE_FP64):
    return torch.empty(max(ss.ss_workspace_size(op, batch, max_n, mode), 256), dtype=torch.uint8, device="cuda")


SIZES = [1, 7, 16, 17, 40, 70]


@pytest.mark.parametrize("mode", [ss.MODE_FP64, ss.MODE_FP32_REFINED, ss.MODE_DF])
def test_padded_ld_sylvester_lyapunov_cholesky(mode):
    dev = torch.device("cuda")
    rng = np.random.default_rng(11)
    n = np.array(SIZES, dtype=np.int32)
    dn = torch.from_numpy(n).to(dev)
    info = torch.zeros(len(n), dtype=torch.int32, device=dev)
    pads = lambda: [int(p) for p in rng.integers(1, 6, len(n))]
    # Sylvester
    ls, us, cs = zip(*[inputs.sylvester_instance(int(k), 12, b)[:3] for b, k in enumerate(n)])
    L = padded(ls, pads(), dev); U = padded(us, pads(), dev); C = padded(cs, pads(), dev)
    X = padded([np.zeros((k, k)) for k in n], pads(), dev)
    w = work(ss.OP_TRSYL, len(n), int(n.max()), mode)
    ss.trsyl_lu(len(n), int(n.max()), dn.data_ptr(), L[1].data_ptr(), L[2].data_ptr(), U[1].data_ptr(), U[2].data_ptr(),
                C[1].data_ptr(), C[2].data_ptr(), X[1].data_ptr(), X[2].data_ptr(), info.data_ptr(), mode=mode,
                d_work=w.data_ptr(), work_bytes=int(w.numel()))
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for (x, pad), l, u, c in zip(unpack(X[0], X[3], X[4], [(k, k) for k in n]), ls, us, cs):
        ref, _ = oracle.trsyl_lu(l, u, c)
        assert np.linalg.norm(x - ref) <= TOL * np.linalg.norm(ref) and np.all(pad == PAD_FILL)
    # Lyapunov (FP64: X in place of S; refined modes need X separate)
    ll, ss_, _ = zip(*[inputs.lyapunov_instance(int(k), 13, b) for b, k in enumerate(n)])
    Lb = padded(ll, pads(), dev); S = padded(ss_, pads(), dev)
    Xl = S if mode in (ss.MODE_FP64, ss.MODE_DF) else padded([np.zeros((k, k)) for k in n], pads(), dev)
    w = work(ss.OP_TRLYAP, len(n), int(n.max()), mode)
    ss.trlyap_l(len(n), int(n.max()), dn.data_ptr(), Lb[1].data_ptr(), Lb[2].data_ptr(), S[1].data_ptr(),
                S[2].data_ptr(), Xl[1].data_ptr(), Xl[2].data_ptr(), info.data_ptr(), mode=mode,
                d_work=w.data_ptr(), work_bytes=int(w.numel()))
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for (x, pad), l, s in zip(unpack(Xl[0], Xl[3], Xl[4], [(k, k) for k in n]), ll, ss_):
        ref, _ = oracle.trlyap_l(l, s)
        assert np.linalg.norm(np.tril(x) - np.tril(ref)) <= TOL * np.linalg.norm(np.tril(ref))
        assert np.all(pad == PAD_FILL)
    # Cholesky
    aa = [inputs.cholesky_instance(int(k), 14, b)[0] for b, k in enumerate(n)]
    A = padded(aa, pads(), dev)
    Xc = padded([np.zeros((k, k)) for k in n], pads(), dev)
    w = work(ss.OP_POTRF, len(n), int(n.max()), mode)
    ss.potrf_upper(len(n), int(n.max()), dn.data_ptr(), A[1].data_ptr(), A[2].data_ptr(), Xc[1].data_ptr(),
                   Xc[2].data_ptr(), info.data_ptr(), mode=mode, d_work=w.data_ptr(), work_bytes=int(w.numel()))
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for (x, pad), a in zip(unpack(Xc[0], Xc[3], Xc[4], [(k, k) for k in n]), aa):
        ref, _ = oracle.potrf_upper(a)
        assert np.linalg.norm(np.triu(x) - ref) <= TOL * np.linalg.norm(ref) and np.all(pad == PAD_FILL)


@pytest.mark.parametrize("mode", [ss.MODE_FP64, ss.MODE_DF])
def test_padded_ld_rect_and_posv(mode):
    dev = torch.device("cuda")
    rng = np.random.default_rng(12)
    m = np.array([1, 20, 33, 5, 64], dtype=np.int32)
    n = np.array([9, 3, 33, 70, 17], dtype=np.int32)
    pads = lambda: [int(p) for p in rng.integers(1, 6, len(m))]
    ls, us, cs = zip(*[inputs.sylvester_rect_instance(int(a), int(b), 15, i)[:3] for i, (a, b) in enumerate(zip(m, n))])
    L = padded(ls, pads(), dev); U = padded(us, pads(), dev); C = padded(cs, pads(), dev)
    X = padded([np.zeros((int(a), int(b))) for a, b in zip(m, n)], pads(), dev)
    dm, dn = torch.from_numpy(m).to(dev), torch.from_numpy(n).to(dev)
    info = torch.zeros(len(m), dtype=torch.int32, device=dev)
    w = work(ss.OP_TRSYL, len(m), int(max(m.max(), n.max())), mode)
    ss.trsyl_rect(len(m), int(m.max()), int(n.max()), dm.data_ptr(), dn.data_ptr(), L[1].data_ptr(), L[2].data_ptr(),
                  U[1].data_ptr(), U[2].data_ptr(), C[1].data_ptr(), C[2].data_ptr(), X[1].data_ptr(), X[2].data_ptr(),
                  info.data_ptr(), mode=mode, d_work=w.data_ptr(), work_bytes=int(w.numel()))
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for (x, pad), l, u, c in zip(unpack(X[0], X[3], X[4], list(zip(m, n))), ls, us, cs):
        ref, _ = oracle.trsyl_rect(l, u, c)
        assert np.linalg.norm(x - ref) <= TOL * np.linalg.norm(ref) and np.all(pad == PAD_FILL)
    k = np.array([2, 16, 1, 40, 5], dtype=np.int32)
    nn = np.array([5, 33, 64, 17, 1], dtype=np.int32)
    aa, bb = zip(*[inputs.posv_instance(int(a), int(b), 16, i)[:2] for i, (a, b) in enumerate(zip(nn, k))])
    A = padded(aa, pads(), dev); R = padded([np.zeros((int(a), int(a))) for a in nn], pads(), dev)
    B = padded(bb, pads(), dev); Xp = padded([np.zeros((int(a), int(b))) for a, b in zip(nn, k)], pads(), dev)
    dnn, dk = torch.from_numpy(nn).to(dev), torch.from_numpy(k).to(dev)
    w = work(ss.OP_POTRF, len(nn), int(nn.max()), mode)
    ss.posv_upper(len(nn), int(nn.max()), int(k.max()), dnn.data_ptr(), dk.data_ptr(), A[1].data_ptr(), A[2].data_ptr(),
                  R[1].data_ptr(), R[2].data_ptr(), B[1].data_ptr(), B[2].data_ptr(), Xp[1].data_ptr(), Xp[2].data_ptr(),
                  info.data_ptr(), mode=mode, d_work=w.data_ptr(), work_bytes=int(w.numel()))
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for (x, pad), a, b in zip(unpack(Xp[0], Xp[3], Xp[4], list(zip(nn, k))), aa, bb):
        ref, _, _ = oracle.posv_upper(a, b)
        assert np.linalg.norm(x - ref) <= TOL * np.linalg.norm(ref) and np.all(pad == PAD_FILL)


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
def test_refined_modes_reject_in_place_raw_and_fp64_accept(op):
    from paper_1906_08613_gb300.device import DeviceBatch
    n = np.array([5, 33, 70], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=17)
    rhs = {"potrf": "A", "trsyl": "C", "trlyap": "S"}[op]
    for mode, want in ((ss.MODE_FP32_REFINED, ss.INFO_ALIASED), (ss.MODE_FP32_RAW, 0), (ss.MODE_FP64, 0),
                       (ss.MODE_DF, 0)):
        db = DeviceBatch(pk.n, pk.off, pk.ops, op, alias_rhs=True)
        db.ensure_work(mode)
        db.solve(mode=mode)
        torch.cuda.synchronize()
        assert np.all(db.info_host() == want), (mode, db.info_host())
        if want == ss.INFO_ALIASED:
            assert np.array_equal(db.x_host(), pk.ops[rhs])       # left untouched
