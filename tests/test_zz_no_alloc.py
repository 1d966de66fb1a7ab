"""trsyl_lu_noalloc: the Sylvester solve for callers that cannot allocate
device memory (for example code that runs while a CUDA graph is being
captured, or a plugin whose host forbids allocation after start-up).

It must give the same X and info as trsyl_lu with a caller workspace, and
match the CPU oracle, on two calls in a row (the second reuses the library's
scratch area as the first left it).  This file is collected last, and passes
both alone in a fresh process and after every other test."""
import numpy as np
import pytest

from paper_1906_08613_gb300 import inputs
from paper_1906_08613_gb300 import smallsolve as ss

from common import TOL, oracle_batch, rel_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc_call(db):
    ld = db.d_ld.data_ptr()
    return ss.trsyl_lu_noalloc(db.batch, db.max_n, db.d_n.data_ptr(), db.ptrs["L"].data_ptr(), ld,
                               db.ptrs["U"].data_ptr(), ld, db.ptrs["C"].data_ptr(), ld,
                               db.ptrs["X"].data_ptr(), ld, db.info.data_ptr())


def test_noalloc_matches_the_workspace_entry_point_twice():
    from paper_1906_08613_gb300.device import DeviceBatch
    n = inputs.sizes_uniform(700, 1, 130, seed=77)
    pk = inputs.sylvester_batch(n, seed=77)

    ref = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl")
    ref.solve(mode=ss.MODE_FP64)
    torch.cuda.synchronize()
    x_ref, info_ref = ref.x_host(), ref.info_host()
    x_orc, info_orc = oracle_batch("trsyl", pk)
    assert np.array_equal(info_ref, info_orc)

    db = DeviceBatch(pk.n, pk.off, pk.ops, "trsyl", x_fill=-1.0)
    for call in range(2):
        db.X.fill_(-1.0)
        db.info.fill_(777)
        assert _noalloc_call(db) == 0
        torch.cuda.synchronize()
        x, info = db.x_host(), db.info_host()
        assert np.array_equal(info, info_ref), f"call {call}"
        errs = rel_errors("trsyl", pk, x, x_ref)
        assert np.all(errs <= TOL), f"call {call}: max rel err {errs.max():.3e}"
        errs = rel_errors("trsyl", pk, x, x_orc)
        assert np.all(errs <= TOL), f"call {call}: max rel err vs the oracle {errs.max():.3e}"


def test_noalloc_rejects_batches_beyond_its_scratch():
    rc = ss.trsyl_lu_noalloc(300000, 16, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, check=False)
    assert rc == ss.ERR_SCRATCH_LIMIT
    assert ss.trsyl_lu_noalloc(-1, 16, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, check=False) == -1
