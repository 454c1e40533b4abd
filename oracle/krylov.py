"""Oracle: Krylov solvers for A alpha = b (Sec. 4: GMRES with a preconditioner).

TEST INFRASTRUCTURE (see ``oracle/__init__``).  The paper names GMRES with a
block-Jacobi or an MgNet preconditioner but not its variant, restart or
orthogonalisation; the reading used here is right-preconditioned flexible
GMRES(m) (the preconditioner may change between iterations), x0 = 0 unless
given, Arnoldi by modified Gram-Schmidt with one full reorthogonalisation, and
convergence decided by the recomputed residual ||b - A x|| / ||b||.

Pins: dense LU solve (P7), Arnoldi orthonormality and finite termination (P15).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _givens(a, b):
    """Rotation (cs, sn) with [cs sn; -sn cs] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def fgmres(apply_A, b, precond, tol=1e-10, restart=50, max_iter=10000, x0=None,
           history=None):
    """Right-preconditioned flexible GMRES(restart).

    apply_A(v) -> A v ; precond(v, j) -> z (may vary with the iteration j).
    Vectors are flat float64.  Returns (x, info) with info = dict(iters,
    cycles, relres, converged).  The stopping test recomputes r = b - A x at
    the end of every cycle.
    """
    b = np.asarray(b, np.float64).ravel()
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64).ravel()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), dict(iters=0, cycles=0, relres=0.0, converged=True)
    total = 0
    cycles = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        relres = beta / bnorm
        if history is not None:
            history.append(relres)
        if relres <= tol or total >= max_iter:
            return x, dict(iters=total, cycles=cycles, relres=relres, converged=relres <= tol)
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j], total)
            w = apply_A(Z[j])
            # modified Gram-Schmidt, then one reorthogonalisation pass
            for _ in range(2):
                for i in range(j + 1):
                    hij = np.dot(V[i], w)
                    H[i, j] += hij
                    w = w - hij * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            # apply previous rotations to the new column, then a new one
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            total += 1
            k = j + 1
            if abs(gvec[j + 1]) / bnorm <= tol or total >= max_iter or breakdown:
                break
        y = sla.solve_triangular(H[:k, :k], gvec[:k], lower=False)
        x = x + Z[:k].T @ y
        cycles += 1


def arnoldi(apply_A, v0, steps):
    """Unpreconditioned Arnoldi (MGS + reorthogonalisation); returns V (steps+1, n), H."""
    n = v0.size
    V = np.zeros((steps + 1, n))
    H = np.zeros((steps + 1, steps))
    V[0] = v0 / np.linalg.norm(v0)
    for j in range(steps):
        w = apply_A(V[j])
        for _ in range(2):
            for i in range(j + 1):
                hij = np.dot(V[i], w)
                H[i, j] += hij
                w = w - hij * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            return V[:j + 1], H[:j + 1, :j]
        V[j + 1] = w / H[j + 1, j]
    return V, H


def dense_solve(A_sparse, b):
    """Reference solve by dense LU with partial pivoting (library primitive), small n only."""
    A = A_sparse.toarray()
    return sla.lu_solve(sla.lu_factor(A), np.asarray(b, np.float64).ravel())
