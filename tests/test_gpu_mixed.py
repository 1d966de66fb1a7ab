"""Parity of the mixed-precision + FP64-refinement forms with the FP64 oracle.

Refined modes must meet the same gate as the FP64 path
(||X - X_oracle||_F / ||X_oracle||_F <= 1e-11 per instance).  Raw
(unrefined) modes are not gated; their error is checked against a loose bound
that the low precision explains (TF32/BF16 operand rounding, about 1e-3 and
1e-2 relative for these well-conditioned inputs, FP32 about 1e-6)."""
import numpy as np
import pytest

from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import assert_parity, oracle_batch, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 5, 8, 15, 16, 17, 31, 32, 33, 64, 65, 100, 128, 129]
REFINED = ["fp32_refined", "tf32_refined", "bf16_refined"]
RAW_BOUND = {"fp32_raw": 1e-5, "tf32_raw": 2e-2, "bf16_raw": 1e-1}
SENT = -3.5


def run(op, pk, mode, cfg=ss.CFG_DEFAULT, **kw):
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op, x_fill=SENT, **kw)
    db.solve(mode=ss.MODES[mode], cfg=cfg)
    torch.cuda.synchronize()
    return db.x_host(), db.info_host()


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
@pytest.mark.parametrize("mode", REFINED)
def test_refined_every_config(op, mode):
    n = np.array(SIZES, dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=31)
    ref, rinfo = oracle_batch(op, pk)
    for cfg in range(ss.ss_config_count(ss.OPS[op], ss.MODES[mode])):
        x, info = run(op, pk, mode, cfg=cfg)
        assert np.array_equal(info, rinfo), (mode, cfg, info)
        assert_parity(op, pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
@pytest.mark.parametrize("mode", sorted(RAW_BOUND))
def test_raw_modes_error_is_that_of_the_low_precision(op, mode):
    n = np.array([7, 40, 96], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=32)
    ref, _ = oracle_batch(op, pk)
    x, info = run(op, pk, mode)
    assert np.all(info == 0)
    errs = rel_errors(op, pk, x, ref)
    assert np.all(errs < RAW_BOUND[mode]), errs
    assert np.all(errs > 0)   # it is genuinely the low-precision result


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
@pytest.mark.parametrize("mode", REFINED)
def test_refinement_reports_non_convergence(op, mode):
    # A NaN in the right-hand side (the divisors are fine) keeps every
    # correction norm NaN, so the stopping test never passes and refinement
    # stops at the iteration cap with info = n + 1.  (An ill-conditioned but
    # finite problem is not a reliable trigger: with an FP64-accurate residual
    # the iteration still contracts and stops at the residual's precision.)
    n = np.array([24, 24], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=33)
    rhs = {"trsyl": "C", "trlyap": "S", "potrf": "A"}[op]
    if op == "potrf":
        # For the Cholesky factor the NaN reaches a pivot first, which is
        # reported as that leading minor's failure, exactly as the oracle does.
        pk.view(rhs, 1)[3, 20] = np.nan
        _, rinfo = oracle_batch(op, pk)
        _, info = run(op, pk, mode)
        assert list(info) == list(rinfo) and info[1] == 21
        return
    pk.view(rhs, 1)[20, 3] = np.nan
    _, info = run(op, pk, mode)
    assert info[0] == 0
    assert info[1] == 25


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
def test_singular_divisor_flagged(op):
    n = np.array([10], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=34)
    l = pk.view("L", 0)
    if op == "trsyl":
        pk.view("U", 0)[2, 2] = -l[6, 6]
    else:
        l[3, 3] = 0.0
    _, info = run(op, pk, "fp32_refined")
    assert info[0] == 1


def test_mixed_cholesky_failure_and_untouched_lower():
    n = np.array([5, 30, 40], dtype=np.int32)
    pk = inputs.cholesky_batch(n, seed=36)
    pk.view("A", 1)[12, 12] = -100.0            # leading minor 13 fails
    pk.view("A", 2)[np.tril_indices(40, -1)] = np.nan   # never read
    ref, rinfo = oracle_batch("potrf", pk)
    for mode in REFINED:
        x, info = run("potrf", pk, mode)
        assert list(info) == [0, 13, 0] == list(rinfo)
        for b in (0, 2):
            nb, o = int(n[b]), int(pk.off[b])
            g = x[o:o + nb * nb].reshape(nb, nb, order="F")
            r = ref[o:o + nb * nb].reshape(nb, nb, order="F")
            assert np.linalg.norm(np.triu(g - r)) <= 1e-11 * np.linalg.norm(np.triu(r))
            assert np.all(g[np.tril_indices(nb, -1)] == SENT)


@pytest.mark.parametrize("name,mode", [("potrf_1024x64", "fp32_refined"),
                                       ("potrf_8192xLU8-256", "bf16_refined"),
                                       ("potrf_8192xLU8-256", "fp32_refined"),
                                       ("trsyl_4096xU4-128", "fp32_refined"),
                                       ("trsyl_4096xU4-128", "tf32_refined"),
                                       ("trlyap_2048x128", "tf32_refined"),
                                       ("trlyap_2048x128", "fp32_refined")])
def test_refined_full_workloads(name, mode):
    op = inputs.WORKLOADS[name]["op"]
    pk = inputs.make_workload(name, seed=1234)
    x, info = run(op, pk, mode)
    ref, rinfo = oracle_batch(op, pk, threads=16)
    assert np.all(info == 0) and np.all(rinfo == 0)
    assert_parity(op, pk, x, ref, sentinel=SENT)


def test_workspace_too_small_is_reported():
    from paper_1906_08613_gb300.device import DeviceBatch
    n = np.array([64, 64, 64], dtype=np.int32)
    pk = inputs.make_batch("trsyl", n, seed=35)
    db = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl")
    need = ss.ss_workspace_size(ss.OP_TRSYL, 3, 64, ss.MODE_FP32_REFINED)
    # Enough for the scheduler but only two instances' scratch.
    short = need - 64 * 64 * 2 * 4 + 16
    db.work = torch.empty(need, dtype=torch.uint8, device="cuda")
    rc = ss.trsyl_lu(3, 64, db.d_n.data_ptr(), db.ptrs["L"].data_ptr(), db.d_ld.data_ptr(),
                     db.ptrs["U"].data_ptr(), db.d_ld.data_ptr(), db.ptrs["C"].data_ptr(),
                     db.d_ld.data_ptr(), db.ptrs["X"].data_ptr(), db.d_ld.data_ptr(),
                     db.info.data_ptr(), mode=ss.MODE_FP32_REFINED, d_work=db.work.data_ptr(),
                     work_bytes=short, check=False)
    assert rc == -16          # shorter than the bound: rejected on the host


@pytest.mark.parametrize("op", ["potrf", "trsyl", "trlyap"])
def test_auto_mode_mixes_modes_per_size_bin(op):
    """SS_MODE_AUTO with a different (mode, cfg) in every size bin (as the
    selector sets it) still meets the FP64 gate on every instance."""
    n = inputs.sizes_uniform(200, 1, 200, seed=37)
    pk = inputs.make_batch(op, n, seed=37)
    ref, rinfo = oracle_batch(op, pk)
    o = ss.OPS[op]
    cycle = [ss.MODE_FP64, ss.MODE_FP32_REFINED, ss.MODE_TF32_REFINED, ss.MODE_BF16_REFINED]
    modes, cfgs = [], []
    for k in range(ss.NUM_BINS):
        m = cycle[k % 4]
        modes.append(m)
        cfgs.append(k % ss.ss_config_count(o, m))
    ss.ss_set_auto_table(o, modes, cfgs)
    try:
        from paper_1906_08613_gb300.device import DeviceBatch
        db = DeviceBatch(pk.n, pk.off, pk.ops, op, x_fill=SENT)
        db.solve(mode=ss.MODE_AUTO)
        torch.cuda.synchronize()
        x, info = db.x_host(), db.info_host()
    finally:
        ss.ss_set_auto_table(o, [], [])
    assert np.array_equal(info, rinfo)
    assert_parity(op, pk, x, ref, sentinel=SENT)
