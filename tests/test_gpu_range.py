"""Magnitude edge cases of every mode that leaves the FP64 pipe, against the
CPU oracle through the C ABI.

The problems are plain double precision (the paper's "Preliminary performance
results" paragraph), so data far outside FP32's exponent range must be solved
as accurately as well-scaled data.  SS_MODE_DF and the refined modes compute in
FP32 arithmetic; they rescale each instance by powers of two first (exact in
binary floating point) and solve again in FP64 an instance whose double-float
solution left the range they are accurate in.  Every batch below mixes
well-scaled instances with instances whose operator, right-hand side or both
are multiplied by 2^+-70, 2^+-100 and 2^+-130 (inputs.range_shifts), so X moves
by up to 2^+-260.  Gate: ||X - X_oracle||_F / ||X_oracle||_F <= 1e-11 per
instance (the double-float mode's own bound, 1e-12), info codes as the
oracle's."""
import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import TOL, assert_parity, oracle_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENT = -7.25
DF_TOL = 1e-12
SIZES = [1, 2, 5, 16, 17, 33, 48, 64, 100, 128]
MODES = {"fp64": ss.MODE_FP64, "df": ss.MODE_DF, "fp32_refined": ss.MODE_FP32_REFINED,
         "tf32_refined": ss.MODE_TF32_REFINED, "bf16_refined": ss.MODE_BF16_REFINED}


def scaled_batch(op, count, seed):
    n = np.array([SIZES[(b * 7 + seed) % len(SIZES)] for b in range(count)], dtype=np.int32)
    pk = inputs.make_batch(op, n, seed=seed)
    inputs.scale_instances(pk, op, inputs.range_shifts(count, op, seed))
    return pk


def run(op, pk, mode, cfg=ss.CFG_DEFAULT, **kw):
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op, x_fill=SENT, **kw)
    db.solve(mode=mode, cfg=cfg)
    torch.cuda.synchronize()
    return db.x_host(), db.info_host()


def test_scaled_inputs_really_leave_fp32_range():
    pk = scaled_batch("trsyl", 56, seed=3)
    mags = [np.abs(pk.view("C", b)).max() for b in range(pk.batch)]
    assert max(mags) > 2.0 ** 128 and min(mags) < 2.0 ** -126


@pytest.mark.parametrize("op", ["trsyl", "trlyap", "potrf"])
@pytest.mark.parametrize("mode", list(MODES))
def test_scaled_instances(op, mode):
    pk = scaled_batch(op, 56, seed=11)
    ref, rinfo = oracle_batch(op, pk)
    x, info = run(op, pk, MODES[mode])
    assert np.array_equal(info, rinfo), (info, rinfo)
    errs = assert_parity(op, pk, x, ref, sentinel=SENT)
    if mode == "df":
        assert errs.max() <= DF_TOL, f"max rel err {errs.max():.3e}"


@pytest.mark.parametrize("op", ["trsyl", "trlyap", "potrf"])
def test_scaled_instances_every_df_config(op):
    pk = scaled_batch(op, 84, seed=12)
    ref, rinfo = oracle_batch(op, pk)
    for cfg in range(ss.ss_config_count(ss.OPS[op], ss.MODE_DF)):
        x, info = run(op, pk, ss.MODE_DF, cfg=cfg)
        assert np.array_equal(info, rinfo)
        errs = assert_parity(op, pk, x, ref, sentinel=SENT)
        assert errs.max() <= DF_TOL, f"cfg {cfg}: max rel err {errs.max():.3e}"


@pytest.mark.parametrize("op", ["trsyl", "trlyap", "potrf"])
def test_scaled_instances_auto_table(op):
    # SS_MODE_AUTO with a table that puts the size bins in different modes.
    pk = scaled_batch(op, 84, seed=13)
    ref, rinfo = oracle_batch(op, pk)
    o = ss.OPS[op]
    cycle = [ss.MODE_DF, ss.MODE_FP32_REFINED, ss.MODE_TF32_REFINED, ss.MODE_BF16_REFINED, ss.MODE_FP64]
    modes = [cycle[k % len(cycle)] for k in range(ss.NUM_BINS)]
    ss.ss_set_auto_table(o, modes, [-1] * ss.NUM_BINS)
    try:
        x, info = run(op, pk, ss.MODE_AUTO)
    finally:
        ss.ss_set_auto_table(o, [], [])
    assert np.array_equal(info, rinfo)
    assert_parity(op, pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("mode", ["fp64", "df"])
def test_scaled_rect(mode):
    from paper_1906_08613_gb300.device import DeviceRectBatch
    count = 56
    m = np.array([SIZES[(3 * b) % len(SIZES)] for b in range(count)], dtype=np.int32)
    n = np.array([SIZES[(5 * b + 1) % len(SIZES)] for b in range(count)], dtype=np.int32)
    pk = inputs.sylvester_rect_batch(m, n, seed=14)
    inputs.scale_instances(pk, "trsyl", inputs.range_shifts(count, "trsyl", 14))
    ref, rinfo = oracle.solve_rect_packed(pk)
    db = DeviceRectBatch(pk, x_fill=SENT)
    db.solve(mode=MODES[mode])
    torch.cuda.synchronize()
    x, info = db.x_host(), db.info_host()
    assert np.array_equal(info, rinfo)
    for b in range(count):
        o, c = int(pk.offC[b]), int(m[b]) * int(n[b])
        err = np.linalg.norm(x[o:o + c] - ref[o:o + c]) / np.linalg.norm(ref[o:o + c])
        assert err <= (DF_TOL if mode == "df" else TOL), (b, m[b], n[b], err)


@pytest.mark.parametrize("mode", ["fp64", "df"])
def test_scaled_posv(mode):
    from paper_1906_08613_gb300.device import DevicePosvBatch
    count = 56
    n = np.array([SIZES[(3 * b) % len(SIZES)] for b in range(count)], dtype=np.int32)
    k = np.array([(1, 5, 16, 17, 40)[b % 5] for b in range(count)], dtype=np.int32)
    pk = inputs.posv_batch(n, k, seed=15)
    # A by 2^(2s) (R by 2^s), B by 2^t: X by 2^(t - 2s).
    shifts = [(2 * a, r) for a, r in inputs.range_shifts(count, "trsyl", 15)]
    inputs.scale_instances(pk, "posv", shifts)
    ref_x, ref_r, rinfo = oracle.solve_posv_packed(pk)
    db = DevicePosvBatch(pk, x_fill=SENT)
    db.solve(mode=MODES[mode])
    torch.cuda.synchronize()
    x, r, info = db.x_host(), db.r_host(), db.info_host()
    assert np.array_equal(info, rinfo)
    tol = DF_TOL if mode == "df" else TOL
    for b in range(count):
        o, c = int(pk.offB[b]), int(n[b]) * int(k[b])
        err = np.linalg.norm(x[o:o + c] - ref_x[o:o + c]) / np.linalg.norm(ref_x[o:o + c])
        assert err <= tol, (b, n[b], k[b], shifts[b], err)
        nb, oa = int(n[b]), int(pk.offA[b])
        g = np.triu(r[oa:oa + nb * nb].reshape(nb, nb, order="F"))
        q = np.triu(ref_r[oa:oa + nb * nb].reshape(nb, nb, order="F"))
        assert np.linalg.norm(g - q) <= tol * np.linalg.norm(q), (b, "R")


def growth_batch(op):
    """Well-scaled data whose solution is about 1e26 times larger: two divisors
    l_ii + u_jj of 1e-13 (above the singularity threshold) in one dependency
    chain.  The double-float solve of instance 1 leaves its range."""
    pk = inputs.make_batch(op, np.array([20, 3, 40], dtype=np.int32), seed=16)
    if op == "trsyl":
        l = np.array([[1.0, 0, 0], [0, 1, 0], [0, 0, 1]])
        u = np.array([[-1 + 1e-13, 1, 0], [0, -1 + 1e-13, 1], [0, 0, 2]])
        pk.view("L", 1)[:] = l
        pk.view("U", 1)[:] = u
        pk.view("C", 1)[:] = 1.0
    else:
        l = np.array([[1.0, 0, 0], [1, -1 + 1e-13, 0], [1, 1, 1]])
        pk.view("L", 1)[:] = l
        pk.view("S", 1)[:] = 1.0
    return pk


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
def test_df_out_of_range_solution_is_solved_in_fp64(op):
    pk = growth_batch(op)
    ref, rinfo = oracle_batch(op, pk)
    assert np.all(rinfo == 0)
    assert np.abs(ref[int(pk.off[1]):int(pk.off[1]) + 9]).max() > 2.0 ** 80
    for cfg in range(ss.ss_config_count(ss.OPS[op], ss.MODE_DF)):
        x, info = run(op, pk, ss.MODE_DF, cfg=cfg)
        assert np.all(info == 0), info
        assert_parity(op, pk, x, ref, sentinel=SENT)


@pytest.mark.parametrize("op", ["trsyl", "trlyap"])
def test_df_out_of_range_in_place_reports(op):
    # X == C: the right-hand side is gone when the range is left, so the
    # instance is reported; the others are solved.
    pk = growth_batch(op)
    ref, _ = oracle_batch(op, pk)
    from paper_1906_08613_gb300.device import DeviceBatch
    db = DeviceBatch(pk.n, pk.off, pk.ops, op, alias_rhs=True)
    db.solve(mode=ss.MODE_DF)
    torch.cuda.synchronize()
    info = db.info_host()
    assert list(info) == [0, ss.INFO_RANGE, 0]
    assert_parity(op, pk, db.x_host(), ref, indices=[0, 2])


@pytest.mark.parametrize("op", ["trsyl", "trlyap", "potrf"])
def test_df_nonfinite_input_like_fp64(op):
    pk = inputs.make_batch(op, np.array([17, 33, 9], dtype=np.int32), seed=17)
    rhs = {"potrf": "A", "trsyl": "C", "trlyap": "S"}[op]
    pk.view(rhs, 1)[3, 2] = np.nan
    pk.view(rhs, 1)[2, 3] = np.nan
    xf, info_f = run(op, pk, ss.MODE_FP64)
    xd, info_d = run(op, pk, ss.MODE_DF)
    assert np.array_equal(info_f, info_d)
    ref, rinfo = oracle_batch(op, pk)
    assert np.array_equal(info_d, rinfo)
    assert_parity(op, pk, xd, ref, indices=[0, 2])
