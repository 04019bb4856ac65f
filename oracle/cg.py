"""Conjugate gradient and dense solves for the oracle (test infrastructure only).

Section 2 of the paper: K = M^dag M is large and sparse and is inverted by
an iterative solver such as conjugate gradient, each iteration costing one
multiplication by K (the unit N_mat of the cost metric, Section 3.1).
This is textbook CG (Hestenes-Stiefel) for a Hermitian positive definite
operator; it stops when the TRUE residual |b - A x| / |b| <= tol, restarting
from the true residual whenever the recursive one claims convergence first.
The dense path builds the matrix of an operator column by column (2^4
lattices) for exact solves and determinants.
"""
import numpy as np


def vdot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def cg(A, b, tol, maxiter=100000, x0=None):
    """Solve A x = b; returns (x, info) with info = iterations, n_mat, true residual."""
    bnorm = np.sqrt(vdot(b, b).real)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bnorm == 0:
        return x, dict(iters=0, n_mat=0, rel_resid=0.0)
    r = b - A(x)
    n_mat = 1
    p = r.copy()
    rr = vdot(r, r).real
    it = 0
    while True:
        if np.sqrt(rr) <= tol * bnorm:
            r = b - A(x)
            n_mat += 1
            rr = vdot(r, r).real
            if np.sqrt(rr) <= tol * bnorm or it >= maxiter:
                break
            p = r.copy()
        if it >= maxiter:
            break
        Ap = A(p)
        n_mat += 1
        alpha = rr / vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, dict(iters=it, n_mat=n_mat, rel_resid=float(np.sqrt(rr) / bnorm))


def dense_matrix(op, support, dtype=np.complex128):
    """Matrix of a linear operator restricted to the entries where support is True.

    support: boolean array of the field's shape; columns are unit vectors on it."""
    idx = np.flatnonzero(support.reshape(-1))
    n = idx.size
    mat = np.zeros((n, n), dtype=dtype)
    e = np.zeros(support.size, dtype=dtype)
    for j, k in enumerate(idx):
        e[:] = 0
        e[k] = 1
        mat[:, j] = op(e.reshape(support.shape)).reshape(-1)[idx]
    return mat, idx
