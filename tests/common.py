"""Helpers shared by the GPU parity tests: run the oracle on a packed batch
and compare the CUDA result instance by instance."""
import numpy as np

import oracle

RHS = {"potrf": "A", "trsyl": "C", "trlyap": "S"}
TOL = 1e-11          # ||X - X_oracle||_F / ||X_oracle||_F for FP64 and refined forms


def meaningful(op, m):
    if op == "potrf":
        return np.triu(m)
    if op == "trlyap":
        return np.tril(m)
    return m


def other_triangle(op, m):
    if op == "potrf":
        return m[np.tril_indices(m.shape[0], -1)]
    if op == "trlyap":
        return m[np.triu_indices(m.shape[0], 1)]
    return np.zeros(0)


def oracle_batch(op, pk, threads=8, indices=None):
    ops = {k: pk.ops[k] for k in pk.ops if k != "X0"}
    out, info = oracle.solve_packed_parallel(op, pk.n, pk.off, ops, threads=threads, indices=indices)
    return out, info


def instance(buf, pk, b):
    nb, o = int(pk.n[b]), int(pk.off[b])
    return buf[o:o + nb * nb].reshape(nb, nb, order="F")


def rel_errors(op, pk, x_gpu, x_ref, indices=None):
    idx = range(pk.batch) if indices is None else indices
    errs = []
    for b in idx:
        if pk.n[b] == 0:
            errs.append(0.0)
            continue
        g = meaningful(op, instance(x_gpu, pk, b))
        r = meaningful(op, instance(x_ref, pk, b))
        errs.append(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300))
    return np.array(errs)


def assert_parity(op, pk, x_gpu, x_ref, tol=TOL, indices=None, sentinel=None):
    errs = rel_errors(op, pk, x_gpu, x_ref, indices)
    worst = int(np.argmax(errs)) if len(errs) else 0
    assert np.all(errs <= tol), f"{op}: max rel err {errs.max():.3e} at instance {worst} (n={pk.n[worst] if indices is None else '?'})"
    if sentinel is not None:
        idx = range(pk.batch) if indices is None else indices
        for b in idx:
            rest = other_triangle(op, instance(x_gpu, pk, b))
            assert np.all(rest == sentinel), f"{op}: untouched triangle modified (instance {b})"
    return errs
