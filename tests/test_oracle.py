"""Pins for the CPU oracle: each check compares it with something other than
itself (a Kronecker brute-force solve, integer-exact factors, library routines
used as independent solvers, hand-worked examples, special cases, and the
structure of the problems in the paper's Fig. 2 caption)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1906_08613_gb300 import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def kron_sylvester(l, u, c):
    """Brute force: (I (x) L + U^T (x) I) vec X = vec C, vec stacking columns."""
    n = c.shape[0]
    m = np.kron(np.eye(n), l) + np.kron(u.T, np.eye(n))
    x = np.linalg.solve(m, c.ravel(order="F"))
    return x.reshape(n, n, order="F")


# --------------------------------------------------------------- hand-worked

def test_golden_worked_examples():
    g = json.load(open(GOLDEN))
    e = g["sylvester_2x2"]
    x, info = oracle.trsyl_lu(np.array(e["L"], float), np.array(e["U"], float), np.array(e["C"], float))
    assert info == 0 and np.array_equal(x, np.array(e["X"], float))
    e = g["lyapunov_2x2"]
    x, info = oracle.trlyap_l(np.array(e["L"], float), np.array(e["S"], float))
    assert info == 0 and np.array_equal(x, np.tril(np.array(e["X"], float)))
    e = g["cholesky_3x3"]
    x, info = oracle.potrf_upper(np.array(e["A"], float))
    assert info == 0 and np.array_equal(x, np.array(e["X"], float))
    e = g["cholesky_not_spd"]
    _, info = oracle.potrf_upper(np.array(e["A"], float))
    assert info == e["info"]


# ------------------------------------------------------- Kronecker brute force

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sylvester_kronecker(n, seed):
    l, u, c, _ = inputs.sylvester_instance(n, seed, 0)
    x, info = oracle.trsyl_lu(l, u, c)
    assert info == 0
    assert rel(x, kron_sylvester(l, u, c)) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_sylvester_kronecker_general_triangles(n):
    # Triangular factors with arbitrary (also negative) diagonals; l_ii + u_jj
    # kept away from zero.
    rng = np.random.default_rng(100 + n)
    l = np.tril(rng.standard_normal((n, n)))
    u = np.triu(rng.standard_normal((n, n)))
    l[np.diag_indices(n)] = rng.uniform(2, 3, n) * rng.choice([-1, 1])
    u[np.diag_indices(n)] = np.sign(l[0, 0]) * rng.uniform(2, 3, n)
    c = rng.standard_normal((n, n))
    x, info = oracle.trsyl_lu(l, u, c)
    assert info == 0
    assert rel(x, kron_sylvester(l, u, c)) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("seed", [0, 1])
def test_lyapunov_kronecker_and_symmetry(n, seed):
    l, s, _ = inputs.lyapunov_instance(n, seed, 0)
    xk = kron_sylvester(l, l.T, s)
    # The brute-force solution of a symmetric right-hand side is symmetric.
    assert np.abs(xk - xk.T).max() <= 1e-14 * max(np.abs(xk).max(), 1)
    x, info = oracle.trlyap_l(l, s)
    assert info == 0
    assert rel(x, np.tril(xk)) < 1e-13
    assert np.all(np.triu(x, 1) == 0)


# ----------------------------------------------------- exact Cholesky factors

@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33])
def test_cholesky_integer_exact(n):
    # A = X0^T X0 with small integers is exact in FP64, every intermediate of
    # the recurrence is an integer, so the factor must come back bit-exact.
    a, x0 = inputs.cholesky_instance(n, 5, n, exact=True)
    x, info = oracle.potrf_upper(a)
    assert info == 0
    assert np.array_equal(x, x0)


@pytest.mark.parametrize("n", [4, 17, 64])
def test_cholesky_vs_numpy_and_residual(n):
    a, _ = inputs.cholesky_instance(n, 11, 0)
    x, info = oracle.potrf_upper(a)
    assert info == 0
    assert np.all(np.tril(x, -1) == 0) and np.all(np.diag(x) > 0)
    assert rel(x, np.linalg.cholesky(a).T) < 1e-13
    assert np.linalg.norm(x.T @ x - a) / np.linalg.norm(a) < 4 * n * EPS


# ------------------------------------------------- library cross-checks

@pytest.mark.parametrize("n", [8, 31, 64])
def test_sylvester_vs_scipy(n):
    l, u, c, x0 = inputs.sylvester_instance(n, 3, 1)
    x, info = oracle.trsyl_lu(l, u, c)
    assert info == 0
    assert rel(x, scipy.linalg.solve_sylvester(l, u, c)) < 1e-12
    # C was built from the known X0, so the solution sits within rounding of it.
    assert rel(x, x0) < 1e-12
    r = c - l @ x - x @ u
    scale = (np.abs(l) @ np.abs(x) + np.abs(x) @ np.abs(u)).max()
    assert np.abs(r).max() < 4 * n * EPS * scale


@pytest.mark.parametrize("n", [8, 40])
def test_lyapunov_vs_scipy(n):
    l, s, x0 = inputs.lyapunov_instance(n, 4, 2)
    x, info = oracle.trlyap_l(l, s)
    assert info == 0
    xs = scipy.linalg.solve_continuous_lyapunov(l, s)   # solves A X + X A^H = Q
    assert rel(np.tril(x), np.tril(xs)) < 1e-12
    assert rel(np.tril(x), np.tril(x0)) < 1e-12


# ------------------------------------------------------------ special cases

def test_order_one():
    x, _ = oracle.trsyl_lu([[3.0]], [[5.0]], [[16.0]])
    assert x[0, 0] == 2.0
    x, _ = oracle.potrf_upper([[9.0]])
    assert x[0, 0] == 3.0
    x, _ = oracle.trlyap_l([[2.0]], [[12.0]])
    assert x[0, 0] == 3.0


def test_diagonal_factors():
    rng = np.random.default_rng(9)
    n = 7
    ld = rng.uniform(1, 2, n)
    ud = rng.uniform(1, 2, n)
    c = rng.standard_normal((n, n))
    x, _ = oracle.trsyl_lu(np.diag(ld), np.diag(ud), c)
    assert np.allclose(x, c / (ld[:, None] + ud[None, :]), rtol=1e-15, atol=0)


def test_identity_cholesky():
    x, info = oracle.potrf_upper(np.eye(12))
    assert info == 0 and np.array_equal(x, np.eye(12))


# -------------------------------------------------- which triangles are read

def test_reads_only_stated_triangles():
    n = 9
    a, _ = inputs.cholesky_instance(n, 2, 0)
    x_ref, _ = oracle.potrf_upper(a)
    a2 = a.copy()
    a2[np.tril_indices(n, -1)] = np.nan
    x2, info = oracle.potrf_upper(a2)
    assert info == 0 and np.array_equal(x2, x_ref)

    l, u, c, _ = inputs.sylvester_instance(n, 2, 0)
    x_ref, _ = oracle.trsyl_lu(l, u, c)
    l2, u2 = l.copy(), u.copy()
    l2[np.triu_indices(n, 1)] = np.nan
    u2[np.tril_indices(n, -1)] = np.nan
    x2, _ = oracle.trsyl_lu(l2, u2, c)
    assert np.array_equal(x2, x_ref)

    l, s, _ = inputs.lyapunov_instance(n, 2, 0)
    x_ref, _ = oracle.trlyap_l(l, s)
    l2, s2 = l.copy(), s.copy()
    l2[np.triu_indices(n, 1)] = np.nan
    s2[np.triu_indices(n, 1)] = np.nan
    x2, _ = oracle.trlyap_l(l2, s2)
    assert np.array_equal(x2, x_ref)


# ------------------------------------------------------------ failure codes

def test_failure_codes():
    a = np.diag([4.0, 1.0, -1.0, 2.0])
    _, info = oracle.potrf_upper(a)
    assert info == 3
    a = np.eye(3)
    a[1, 1] = np.nan
    _, info = oracle.potrf_upper(a)
    assert info == 2
    l = np.eye(3)
    u = np.eye(3)
    u[2, 2] = -1.0        # l_22 + u_22 = 0: singular Sylvester operator
    _, info = oracle.trsyl_lu(l, u, np.ones((3, 3)))
    assert info == 1
    l = np.diag([1.0, 0.0, 2.0])   # l_11 + l_11 = 0
    _, info = oracle.trlyap_l(l, np.eye(3))
    assert info == 1


# ------------------------------------------------------------ packed batches

def test_packed_batch_matches_single_calls():
    n = inputs.sizes_uniform(12, 1, 20, seed=3)
    pk = inputs.sylvester_batch(n, seed=3)
    out, info = oracle.solve_packed("trsyl", pk.n, pk.off, pk.ops)
    outp, infop = oracle.solve_packed_parallel("trsyl", pk.n, pk.off, pk.ops, threads=3)
    assert np.array_equal(out, outp) and np.all(info == 0) and np.all(infop == 0)
    for b in range(pk.batch):
        x, _ = oracle.trsyl_lu(pk.view("L", b), pk.view("U", b), pk.view("C", b))
        nb, o = int(pk.n[b]), int(pk.off[b])
        assert np.array_equal(out[o:o + nb * nb].reshape(nb, nb, order="F"), x)
