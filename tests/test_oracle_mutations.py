"""The oracle's pins are sensitive: each test below plants one plausible
mistake in a private copy of oracle.c (a dropped term, a flipped sign, a
transposed operand, a wrong index), compiles it, and checks that the
independent pins of test_oracle.py's kind reject the mutant."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    # Cholesky
    "chol_drop_offdiag_sum": ("s = s - AT(X, ldx, k, i) * AT(X, ldx, k, j);", "s = s;"),
    "chol_transposed_read": ("double s = AT(A, lda, i, j);", "double s = AT(A, lda, j, i);"),
    "chol_wrong_pivot": ("AT(X, ldx, i, j) = s / AT(X, ldx, i, i);", "AT(X, ldx, i, j) = s / AT(X, ldx, j, j);"),
    "chol_diag_sign": ("d = d - AT(X, ldx, k, j) * AT(X, ldx, k, j);", "d = d + AT(X, ldx, k, j) * AT(X, ldx, k, j);"),
    # Sylvester
    "syl_drop_L_term": ("s = s - AT(L, ldl, i, k) * AT(X, ldx, k, j);", "s = s;"),
    "syl_sign_U_term": ("s = s - AT(X, ldx, i, k) * AT(U, ldu, k, j);", "s = s + AT(X, ldx, i, k) * AT(U, ldu, k, j);"),
    "syl_transposed_L": ("s = s - AT(L, ldl, i, k) * AT(X, ldx, k, j);", "s = s - AT(L, ldl, k, i) * AT(X, ldx, k, j);"),
    "syl_wrong_divisor": ("double d = AT(L, ldl, i, i) + AT(U, ldu, j, j);", "double d = AT(L, ldl, i, i) + AT(U, ldu, i, i);"),
    # Lyapunov
    "lya_drop_right_term": ("s = s - sym_lower(X, ldx, i, k) * AT(L, ldl, j, k);", "s = s;"),
    "lya_untransposed_L": ("s = s - sym_lower(X, ldx, i, k) * AT(L, ldl, j, k);", "s = s - sym_lower(X, ldx, i, k) * AT(L, ldl, k, j);"),
    "lya_no_symmetry": ("return r >= c ? AT(X, ldx, r, c) : AT(X, ldx, c, r);", "return AT(X, ldx, r, c);"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation anchor missing for {name}"
    p = tmp_path / f"{name}.c"
    p.write_text(text.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           "-o", str(so), str(p), "-lm"])
    return ctypes.CDLL(str(so))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pins_pass(lib, op):
    """Run the oracle pins for ``op`` against a (possibly mutated) library."""
    for n in (3, 5, 6):
        if op == "potrf":
            a, x0 = inputs.cholesky_instance(n, 5, n, exact=True)
            a = np.asfortranarray(a)
            a[np.tril_indices(n, -1)] = np.nan    # only the upper triangle may be read
            x = np.zeros((n, n), order="F")
            info = lib.oracle_potrf_upper(n, _dp(a), n, _dp(x), n)
            if info != 0 or not np.array_equal(x, x0):
                return False
        elif op == "trsyl":
            l, u, c, _ = (np.asfortranarray(m) for m in inputs.sylvester_instance(n, 1, 0))
            x = np.zeros((n, n), order="F")
            lib.oracle_trsyl_lu(n, _dp(l), n, _dp(u), n, _dp(c), n, _dp(x), n)
            m = np.kron(np.eye(n), l) + np.kron(u.T, np.eye(n))
            xk = np.linalg.solve(m, c.ravel(order="F")).reshape(n, n, order="F")
            if np.linalg.norm(x - xk) > 1e-12 * np.linalg.norm(xk):
                return False
        else:
            l, s, _ = (np.asfortranarray(m) for m in inputs.lyapunov_instance(n, 1, 0))
            x = np.zeros((n, n), order="F")
            lib.oracle_trlyap_l(n, _dp(l), n, _dp(s), n, _dp(x), n)
            m = np.kron(np.eye(n), l) + np.kron(l, np.eye(n))
            xk = np.linalg.solve(m, s.ravel(order="F")).reshape(n, n, order="F")
            if np.linalg.norm(x - np.tril(xk)) > 1e-12 * np.linalg.norm(xk):
                return False
    return True


def test_unmutated_oracle_passes_the_pins():
    lib = oracle.lib()
    for op in ("potrf", "trsyl", "trlyap"):
        assert pins_pass(lib, op)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(tmp_path, name):
    lib = build_mutant(tmp_path, name)
    op = {"chol": "potrf", "syl": "trsyl", "lya": "trlyap"}[name.split("_")[0]]
    assert not pins_pass(lib, op), f"mutant {name} survived the pins"
