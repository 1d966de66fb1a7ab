"""The fifth-generation tensor-core path (tcgen05 MMA into tensor memory)
that the refined modes' trailing updates use, pinned tile by tile against a
host product: operand layout, shared-memory and instruction descriptors, the
accumulate flag, the negate-A bit, the TMEM load / store lane mapping and the
mbarrier completion.

Small-integer operands make every product and sum exact in FP32, so those
cases are compared bit for bit; random operands are compared with the host
product of the operands rounded as the library rounds them (TF32 to nearest
with ties away from zero, BF16 to nearest even)."""
import numpy as np
import pytest

from paper_1906_08613_gb300 import smallsolve as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KSTEP = {ss.UMMA_TF32: 8, ss.UMMA_BF16: 16}


def round_tf32(x):
    """Round FP32 to the 10-bit TF32 mantissa, ties away from zero."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000) & 0xFFFFFFFF
    return u.astype(np.uint32).view(np.float32)


def round_bf16(x):
    """Round FP32 to BF16 (8-bit significand), ties to even."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000) & 0xFFFFFFFF
    return u.astype(np.uint32).view(np.float32)


def run(kind, n, k, A, B, C, flags):
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")
    dA, dB = dev(A), dev(B)
    dC = dev(C) if C is not None else None
    dD = torch.full((128, n), np.nan, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ss.ss_umma_selftest(kind, n, k, dA.data_ptr(), dB.data_ptr(), dC.data_ptr() if dC is not None else 0,
                        dD.data_ptr(), flags, st.data_ptr())
    torch.cuda.synchronize()
    assert int(st.item()) == 0, "the bounded wait for the tile ran out"
    return dD.cpu().numpy()


SHAPES = [(16, None), (32, 32), (48, 64), (96, None), (128, 32), (256, 64), (256, None)]


@pytest.mark.parametrize("kind", [ss.UMMA_TF32, ss.UMMA_BF16])
@pytest.mark.parametrize("n,k", SHAPES)
@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_exact_tile(kind, n, k, flags):
    k = k or KSTEP[kind]
    rng = np.random.default_rng(1000 * n + 10 * k + flags + 7 * kind)
    A = rng.integers(-8, 9, (128, k)).astype(np.float32) / 4
    B = rng.integers(-8, 9, (n, k)).astype(np.float32) / 4
    C = rng.integers(-64, 65, (128, n)).astype(np.float32) if flags & 1 else None
    ref = (-A if flags & 2 else A).astype(np.float64) @ B.astype(np.float64).T
    if C is not None:
        ref = ref + C
    got = run(kind, n, k, A, B, C, flags)
    assert np.array_equal(got, ref.astype(np.float32))


@pytest.mark.parametrize("kind", [ss.UMMA_TF32, ss.UMMA_BF16])
@pytest.mark.parametrize("n,k", [(128, 32), (256, 64), (80, 48)])
def test_random_tile_matches_rounded_operands(kind, n, k):
    rng = np.random.default_rng(n + k + kind)
    A = rng.standard_normal((128, k)).astype(np.float32)
    B = rng.standard_normal((n, k)).astype(np.float32)
    C = rng.standard_normal((128, n)).astype(np.float32)
    rnd = round_tf32 if kind == ss.UMMA_TF32 else round_bf16
    Ar, Br = rnd(A).astype(np.float64), rnd(B).astype(np.float64)
    ref = C.astype(np.float64) + Ar @ Br.T
    got = run(kind, n, k, A, B, C, 1)
    bound = 1e-5 * (np.abs(C) + np.abs(Ar) @ np.abs(Br).T) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)
    # The rounding is the stated one: unrounded operands miss by far more.
    raw = C.astype(np.float64) + A.astype(np.float64) @ B.astype(np.float64).T
    assert np.max(np.abs(got - raw) / bound) > 10


def test_selftest_rejects_bad_shapes():
    for args in [(2, 16, 8), (0, 8, 8), (0, 24, 8), (0, 272, 8), (0, 16, 4), (1, 16, 8), (0, 16, 72)]:
        kind, n, k = args
        assert ss.ss_umma_selftest(kind, n, k, 1, 1, 1, 1, 0, 1, check=False) < 0
