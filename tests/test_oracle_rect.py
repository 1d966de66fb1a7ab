"""Pins of the oracle's rectangular Sylvester solve (L m x m lower, U n x n
upper, X m x n), each independent of the oracle's own recurrence: the
Kronecker form solved by a dense LU, scipy's Sylvester solver, closed forms
(diagonal factors; n = 1 and m = 1 reduce to one shifted triangular solve),
exact recovery of X0, and the singular-divisor threshold.  The last part
plants mistakes in a private copy of oracle.c and checks the pins reject
them."""
import ctypes
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1906_08613_gb300 import inputs

EPS = np.finfo(np.float64).eps


def rand_tri(rng, k, lower):
    a = rng.standard_normal((k, k)) / np.sqrt(k)
    a = np.tril(a, -1) if lower else np.triu(a, 1)
    a[np.diag_indices(k)] = rng.uniform(1.0, 2.0, size=k)
    return a


def kron_solve(l, u, c):
    """vec(L X + X U) = (I_n kron L + U^T kron I_m) vec(X), column-major vec."""
    m, n = c.shape
    k = np.kron(np.eye(n), l) + np.kron(u.T, np.eye(m))
    return np.linalg.solve(k, c.ravel(order="F")).reshape(m, n, order="F")


@pytest.mark.parametrize("m,n", [(1, 1), (1, 4), (4, 1), (2, 5), (5, 2), (3, 3), (6, 4)])
def test_rect_matches_kronecker_brute_force(m, n):
    rng = np.random.default_rng([m, n, 3])
    l, u = rand_tri(rng, m, True), rand_tri(rng, n, False)
    c = rng.standard_normal((m, n))
    x, info = oracle.trsyl_rect(l, u, c)
    ref = kron_solve(l, u, c)
    assert info == 0
    assert np.linalg.norm(x - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("m,n", [(40, 17), (17, 40), (64, 1), (1, 64)])
def test_rect_matches_scipy_sylvester(m, n):
    rng = np.random.default_rng([m, n, 4])
    l, u = rand_tri(rng, m, True), rand_tri(rng, n, False)
    c = rng.standard_normal((m, n))
    x, info = oracle.trsyl_rect(l, u, c)
    ref = sla.solve_sylvester(l, u, c)
    assert info == 0
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def test_rect_diagonal_factors_closed_form():
    rng = np.random.default_rng(5)
    m, n = 7, 3
    l = np.diag(rng.uniform(1, 2, m))
    u = np.diag(rng.uniform(1, 2, n))
    c = rng.standard_normal((m, n))
    x, info = oracle.trsyl_rect(l, u, c)
    assert info == 0
    assert np.array_equal(x, c / (np.diag(l)[:, None] + np.diag(u)[None, :]))


def test_rect_single_column_and_single_row_are_shifted_triangular_solves():
    rng = np.random.default_rng(6)
    l, u = rand_tri(rng, 9, True), rand_tri(rng, 1, False)
    c = rng.standard_normal((9, 1))
    x, _ = oracle.trsyl_rect(l, u, c)
    ref = sla.solve_triangular(l + u[0, 0] * np.eye(9), c, lower=True)
    assert np.allclose(x, ref, rtol=1e-13, atol=0)
    l, u = rand_tri(rng, 1, True), rand_tri(rng, 8, False)
    c = rng.standard_normal((1, 8))
    x, _ = oracle.trsyl_rect(l, u, c)
    # x (l00 I + U) = c  <=>  (l00 I + U)^T x^T = c^T, lower triangular
    ref = sla.solve_triangular((u + l[0, 0] * np.eye(8)).T, c.T, lower=True).T
    assert np.allclose(x, ref, rtol=1e-13, atol=0)


def test_rect_recovers_generated_solution():
    pk = inputs.sylvester_rect_batch([5, 33, 1, 70], [40, 2, 9, 70], seed=8)
    out, info = oracle.solve_rect_packed(pk)
    assert np.all(info == 0)
    for b in range(pk.batch):
        o, k = int(pk.offC[b]), int(pk.m[b]) * int(pk.n[b])
        x, x0 = out[o:o + k], pk.ops["X0"][o:o + k]
        assert np.linalg.norm(x - x0) <= 1e-12 * np.linalg.norm(x0)


def threshold_cases():
    # (L diag, U diag, expected info): divisors built exactly in FP64.
    return [
        # m = 5 > n = 2: delta = 5 eps * 1; divisor l00 + u00 = 3 eps -> singular
        (np.ones(5), np.array([-1 + 3 * EPS, 1.0]), 1),
        # maxdiag comes from U (8), delta = 2 eps * 8 = 16 eps; divisor 4 eps -> singular
        (np.array([0.5, 0.5]), np.array([-0.5 + 4 * EPS, 8.0]), 1),
        # divisor 40 eps > delta = 16 eps -> regular
        (np.array([0.5, 0.5]), np.array([-0.5 + 40 * EPS, 8.0]), 0),
        # NaN divisor
        (np.array([np.nan, 1.0, 1.0]), np.array([1.0]), 1),
    ]


@pytest.mark.parametrize("case", range(4))
def test_rect_singular_divisor_threshold(case):
    ld, ud, want = threshold_cases()[case]
    l, u = np.diag(ld), np.diag(ud)
    _, info = oracle.trsyl_rect(l, u, np.ones((len(ld), len(ud))))
    assert info == want


# ---------------------------------------------------------------- mutants

SRC = oracle.__file__.replace("__init__.py", "oracle.c")

# (anchor, replacement); the rectangular routine's copy of a shared line is
# its last occurrence in the file.
MUTANTS = {
    "rect_drop_L_term": ("s = s - AT(L, ldl, i, k) * AT(X, ldx, k, j);", "s = s;"),
    "rect_sign_U_term": ("s = s - AT(X, ldx, i, k) * AT(U, ldu, k, j);", "s = s + AT(X, ldx, i, k) * AT(U, ldu, k, j);"),
    "rect_threshold_n_only": ("divisor_threshold(m > n ? m : n, maxdiag)", "divisor_threshold(n, maxdiag)"),
    "rect_maxdiag_without_U": ("    for (int j = 0; j < n; ++j)\n        if (fabs(AT(U, ldu, j, j)) > maxdiag) maxdiag = fabs(AT(U, ldu, j, j));\n", ""),
    "rect_transposed_C": ("double s = AT(C, ldc, i, j);", "double s = AT(C, ldc, j < m ? j : 0, i < n ? i : 0);"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    i = text.rfind(old)
    assert i >= 0 and i > text.find("int oracle_trsyl_rect("), f"anchor of {name} not in the rectangular routine"
    p = tmp_path / f"{name}.c"
    p.write_text(text[:i] + new + text[i + len(old):])
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           "-o", str(so), str(p), "-lm"])
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_trsyl_rect.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp,
                                      ctypes.c_int, dp, ctypes.c_int]
    return lib


def rect_pins_pass(lib):
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def solve(l, u, c):
        m, n = c.shape
        l, u, c = (np.asfortranarray(a, dtype=np.float64) for a in (l, u, c))
        x = np.zeros((m, n), order="F")
        info = lib.oracle_trsyl_rect(m, n, dp(l), m, dp(u), n, dp(c), m, dp(x), m)
        return x, info

    for m, n in ((2, 5), (5, 2), (4, 4)):
        rng = np.random.default_rng([m, n, 11])
        l, u = rand_tri(rng, m, True), rand_tri(rng, n, False)
        c = rng.standard_normal((m, n))
        x, info = solve(l, u, c)
        ref = kron_solve(l, u, c)
        if info != 0 or not np.linalg.norm(x - ref) <= 1e-13 * np.linalg.norm(ref):
            return False
    for ld, ud, want in threshold_cases():
        _, info = solve(np.diag(ld), np.diag(ud), np.ones((len(ld), len(ud))))
        if info != want:
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    text = open(SRC).read()
    p = tmp_path / "same.c"
    p.write_text(text)
    so = tmp_path / "same.so"
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           "-o", str(so), str(p), "-lm"])
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_trsyl_rect.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp,
                                      ctypes.c_int, dp, ctypes.c_int]
    assert rect_pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(tmp_path, name):
    assert not rect_pins_pass(build_mutant(tmp_path, name))
