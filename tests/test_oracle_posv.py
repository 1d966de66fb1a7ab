"""Pins of the oracle's SPD solve A X = B through the upper Cholesky factor,
each independent of the oracle's recurrences: numpy's dense solve and
Cholesky factor on the same problem, an integer case whose forward and back
substitutions are exact in FP64, closed forms (identity and diagonal A), the
non-SPD info code, and planted mistakes that the pins must reject."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle
from paper_1906_08613_gb300 import inputs


@pytest.mark.parametrize("n,k", [(1, 1), (2, 3), (7, 1), (16, 16), (33, 5), (64, 20)])
def test_posv_matches_numpy_solve_and_cholesky(n, k):
    a, b, _ = inputs.posv_instance(n, k, seed=3, b=n * 100 + k)
    x, r, info = oracle.posv_upper(a, b)
    assert info == 0
    ref = np.linalg.solve(a, b)
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.allclose(np.triu(r), np.linalg.cholesky(a).T, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n,k", [(3, 2), (8, 5), (20, 7)])
def test_posv_integer_case_is_exact(n, k):
    rng = np.random.default_rng([n, k])
    a, x0 = inputs.cholesky_instance(n, 9, n, exact=True)     # A = X0^T X0, integer, exact
    xs = rng.integers(-3, 4, size=(n, k)).astype(np.float64)
    b = a @ xs                                                # exact: small integers
    x, r, info = oracle.posv_upper(a, b)
    assert info == 0
    assert np.array_equal(np.triu(r), x0)
    assert np.array_equal(x, xs)


def test_posv_identity_and_diagonal():
    rng = np.random.default_rng(4)
    b = rng.standard_normal((6, 3))
    x, _, info = oracle.posv_upper(np.eye(6), b)
    assert info == 0 and np.array_equal(x, b)
    d = rng.uniform(1, 4, 6)
    x, _, _ = oracle.posv_upper(np.diag(d), b)
    assert np.allclose(x, b / d[:, None], rtol=4e-16, atol=0)


def test_posv_not_spd_reports_pivot_and_leaves_x():
    a = np.eye(4)
    a[2, 2] = -1.0
    x, _, info = oracle.posv_upper(a, np.ones((4, 2)))
    assert info == 3 and np.all(x == 0)


# ---------------------------------------------------------------- mutants

SRC = oracle.__file__.replace("__init__.py", "oracle.c")

MUTANTS = {
    "posv_drop_forward_term": ("s = s - AT(R, ldr, l, i) * AT(X, ldx, l, j);", "s = s;"),
    "posv_forward_untransposed": ("s = s - AT(R, ldr, l, i) * AT(X, ldx, l, j);",
                                  "s = s - AT(R, ldr, i, l) * AT(X, ldx, l, j);"),
    "posv_backward_transposed": ("s = s - AT(R, ldr, i, l) * AT(X, ldx, l, j);",
                                 "s = s - AT(R, ldr, l, i) * AT(X, ldx, l, j);"),
    "posv_backward_ascending": ("for (int i = n - 1; i >= 0; --i) {\n            double s = AT(X, ldx, i, j);\n            for (int l = i + 1; l < n; ++l)",
                                "for (int i = 0; i < n; ++i) {\n            double s = AT(X, ldx, i, j);\n            for (int l = i + 1; l < n; ++l)"),
    "posv_no_back_substitution": ("            AT(X, ldx, i, j) = s / AT(R, ldr, i, i);\n        }\n    }\n    return 0;",
                                  "        }\n    }\n    return 0;"),
}


def build(tmp_path, name, text):
    p = tmp_path / f"{name}.c"
    p.write_text(text)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           "-o", str(so), str(p), "-lm"])
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_posv_upper.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp,
                                      ctypes.c_int, dp, ctypes.c_int]
    return lib


def pins_pass(lib):
    dp = lambda v: v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for n, k in ((5, 3), (12, 2)):
        a, x0 = inputs.cholesky_instance(n, 9, n, exact=True)
        xs = np.random.default_rng([n, k, 1]).integers(-3, 4, size=(n, k)).astype(np.float64)
        b = np.asfortranarray(a @ xs)
        a = np.asfortranarray(a)
        r = np.zeros((n, n), order="F")
        x = np.zeros((n, k), order="F")
        info = lib.oracle_posv_upper(n, k, dp(a), n, dp(r), n, dp(b), n, dp(x), n)
        if info != 0 or not np.array_equal(x, xs):
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    assert pins_pass(build(tmp_path, "same", open(SRC).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    start = text.find("int oracle_posv_upper(")
    i = text.find(old, start)
    assert i >= 0, f"anchor of {name} not in the SPD solve"
    assert not pins_pass(build(tmp_path, name, text[:i] + new + text[i + len(old):]))
