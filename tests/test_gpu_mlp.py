"""The CUDA MLP kernels (forward, loss gradient, Adam) against the FP64
oracle, through the C ABI.  FP32 kernels vs FP64 oracle: relative 1e-4 (the
gradient also element by element, against each layer's own scale)."""
import numpy as np
import pytest

from oracle import mlp
from paper_1906_08613_gb300 import smallsolve as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


LAYER_SIZES = (mlp.H * mlp.IN, mlp.H, mlp.H * mlp.H, mlp.H, mlp.OUT * mlp.H, mlp.OUT)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def data(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, mlp.IN))
    T = rng.standard_normal((rows, mlp.OUT))
    M = (rng.random((rows, mlp.OUT)) < 0.6).astype(float)
    M[0, 0] = 1.0
    return X, T, M


@pytest.mark.parametrize("rows", [1, 7, 130, 1000])
def test_forward_matches_oracle(rows):
    p = mlp.init_params(rows)
    X, _, _ = data(rows, 2)
    dp, dx = dev(p), dev(X)
    dy = torch.zeros((rows, mlp.OUT), dtype=torch.float32, device="cuda")
    ss.ss_mlp_forward(dp.data_ptr(), rows, dx.data_ptr(), dy.data_ptr())
    torch.cuda.synchronize()
    y, _ = mlp.forward(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    got = dy.cpu().numpy().astype(np.float64)
    assert np.abs(got - y).max() <= 1e-4 * max(1.0, np.abs(y).max())


@pytest.mark.parametrize("rows", [1, 33, 400])
def test_gradient_matches_oracle(rows):
    p = mlp.init_params(10 + rows)
    X, T, M = data(rows, 3)
    p32 = p.astype(np.float32).astype(np.float64)
    L, g = mlp.loss_and_grad(p32, X.astype(np.float32), T.astype(np.float32), M)
    dp, dx, dt, dm = dev(p), dev(X), dev(T), dev(M)
    dg = torch.zeros(mlp.NPARAM, dtype=torch.float32, device="cuda")
    dl = torch.zeros(1, dtype=torch.float32, device="cuda")
    wb = ss.ss_mlp_workspace_size(rows)
    dw = torch.empty(wb, dtype=torch.uint8, device="cuda")
    ss.ss_mlp_grad(dp.data_ptr(), rows, dx.data_ptr(), dt.data_ptr(), dm.data_ptr(), float(M.sum()),
                   dg.data_ptr(), dl.data_ptr(), dw.data_ptr(), wb)
    torch.cuda.synchronize()
    got = dg.cpu().numpy().astype(np.float64)
    assert abs(float(dl.item()) - L) <= 1e-4 * max(1.0, L)
    assert np.linalg.norm(got - g) <= 1e-4 * max(1e-6, np.linalg.norm(g))
    # Element by element, per parameter block: every entry within 1e-4 of its
    # own layer's largest gradient, so that a wrong slice of a layer with
    # small gradients (b1, W1) cannot hide under the large W3 entries.  The
    # seeds keep every pre-activation away from the ReLU kink (FP32 and FP64
    # then agree on which units are active).
    _, (a1, _, a2, _) = mlp.forward(p32, X.astype(np.float32).astype(np.float64))
    assert min(np.abs(a1).min(), np.abs(a2).min()) > 1e-5
    o = 0
    for name, k in zip(("W1", "b1", "W2", "b2", "W3", "b3"), LAYER_SIZES):
        ref, gpu = g[o:o + k], got[o:o + k]
        scale = max(np.abs(ref).max(), 1e-12)
        worst = int(np.argmax(np.abs(gpu - ref)))
        assert np.abs(gpu - ref).max() <= 1e-4 * scale, f"{name}[{worst}]: {gpu[worst]} vs {ref[worst]}"
        o += k
    assert o == mlp.NPARAM
    # Deterministic: a second evaluation is bit-identical.
    dg2 = torch.zeros_like(dg)
    ss.ss_mlp_grad(dp.data_ptr(), rows, dx.data_ptr(), dt.data_ptr(), dm.data_ptr(), float(M.sum()),
                   dg2.data_ptr(), dl.data_ptr(), dw.data_ptr(), wb)
    torch.cuda.synchronize()
    assert torch.equal(dg, dg2)


def test_adam_matches_oracle_and_training_descends():
    rows = 200
    p = mlp.init_params(7)
    X, T, M = data(rows, 4)
    dp, dx, dt, dm = dev(p), dev(X), dev(T), dev(M)
    dg = torch.zeros(mlp.NPARAM, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(dg)
    v = torch.zeros_like(dg)
    dl = torch.zeros(1, dtype=torch.float32, device="cuda")
    wb = ss.ss_mlp_workspace_size(rows)
    dw = torch.empty(wb, dtype=torch.uint8, device="cuda")
    po, mo, vo = p.astype(np.float32).astype(np.float64), np.zeros(mlp.NPARAM), np.zeros(mlp.NPARAM)
    losses = []
    for step in range(1, 61):
        ss.ss_mlp_grad(dp.data_ptr(), rows, dx.data_ptr(), dt.data_ptr(), dm.data_ptr(), float(M.sum()),
                       dg.data_ptr(), dl.data_ptr(), dw.data_ptr(), wb)
        if step <= 2:
            g_gpu = dg.cpu().numpy().astype(np.float64)
            po, mo, vo = mlp.adam_step(po, g_gpu, mo, vo, step, lr=1e-3)
        ss.ss_mlp_adam(dp.data_ptr(), dg.data_ptr(), m.data_ptr(), v.data_ptr(), step, 1e-3)
        torch.cuda.synchronize()
        losses.append(float(dl.item()))
        if step <= 2:
            got = dp.cpu().numpy().astype(np.float64)
            assert np.abs(got - po).max() <= 1e-6 + 1e-5 * np.abs(po).max()
    assert losses[-1] < 0.7 * losses[0]
