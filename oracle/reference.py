"""Reference discrete eigenvalues by a library eigensolver (test infrastructure).

The k smallest eigenpairs of the FE pencil A u = lambda M u (Section 2, the
discrete eigenproblem) computed with scipy's ARPACK in shift-invert mode
around 0 -- a solver independent of both PASM implementations.  Used to pin
the oracle on larger meshes than dense solves allow and to define the
algebraic error of the iterates (|lambda - lambda_h| / lambda_h)."""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def smallest_eigenvalues(A, M, count: int, extra: int = 8, tol: float = 1e-14):
    """The `count` smallest eigenvalues of (A, M), ascending."""
    vals = spla.eigsh(A.tocsc(), k=count + extra, M=M.tocsc(), sigma=0.0, which="LM",
                      return_eigenvectors=False, tol=tol)
    return np.sort(vals)[:count]


def smallest_eigenvalues_lobpcg(hier, count: int, extra: int = 8, tol: float = 1e-10, maxiter: int = 400,
                                seed: int = 0):
    """The `count` smallest eigenvalues of the finest pencil of a hierarchy by
    LOBPCG (scipy), for problems too large to factorise for shift-invert (the
    3D meshes).  Preconditioner: one multigrid V-cycle for A (oracle.pasm.vcycle
    with damped Jacobi) applied to the residual block.  The preconditioner
    changes only the speed of LOBPCG, not the eigenpairs it converges to, so
    the values stay independent of PASM.  Returns the values and the largest
    relative residual norm ||A x - lambda M x|| / (lambda ||M x||) over the
    `count` wanted pairs."""
    from . import pasm as op
    prob = op.Problem.from_hierarchy(hier)
    A, M = hier.fine.A, hier.fine.M
    L = len(hier.levels) - 1
    m = count + extra

    def precond(R):
        R = np.asarray(R)
        if R.ndim == 1:
            return op.vcycle(prob, L, R[:, None], np.zeros((R.shape[0], 1)))[:, 0]
        return op.vcycle(prob, L, R, np.zeros_like(R))

    Pinv = spla.LinearOperator(A.shape, matvec=precond, matmat=precond, dtype=np.float64)
    # start from the coarse eigenvectors prolongated to the finest level
    _, X0 = op.initial_state(prob, m)
    X0 = X0 + 1e-3 * np.random.default_rng(seed).standard_normal(X0.shape) * np.abs(X0).max()
    vals, vecs = spla.lobpcg(A, X0, B=M, M=Pinv, tol=tol, maxiter=maxiter, largest=False)
    order = np.argsort(vals)
    vals, vecs = vals[order][:count], vecs[:, order][:, :count]
    res = A @ vecs - (M @ vecs) * vals[None, :]
    rel = np.linalg.norm(res, axis=0) / (vals * np.linalg.norm(M @ vecs, axis=0))
    return vals, float(rel.max())
