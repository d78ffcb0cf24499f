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


def laplacian_inverse(dim: int, N: int):
    """A^{-1} for the constant-coefficient P1 stiffness of the uniform meshes
    (the 5-point stencil (4, -1) of the right-triangle mesh of the square,
    h times the 7-point stencil (6, -1) of the Kuhn mesh of the cube): the
    grid sine functions sin(m pi x) ... are its eigenvectors with eigenvalues
    sum_d (2 - 2 cos(m_d pi h)) (times h in 3D), so the inverse is a type-I
    discrete sine transform, a division, and the inverse transform.  Interior
    nodes x fastest, as meshgen numbers them."""
    import scipy.fft as sfft
    # 2 - 2 cos(t) = 4 sin^2(t / 2): the subtraction would lose the low modes' digits (relative
    # error ~1e-10 at t = pi / 2048)
    lam1 = 4.0 * np.sin(0.5 * np.pi * np.arange(1, N) / N) ** 2
    grids = np.meshgrid(*([lam1] * dim), indexing="ij")
    sym = sum(grids) * (1.0 / N if dim == 3 else 1.0)          # index order (z, y, x) or (y, x)
    shape = (N - 1,) * dim

    def apply(b):
        b = np.asarray(b, dtype=np.float64)
        cols = b.reshape(b.shape[0], -1).T.reshape((-1,) + shape)
        axes = tuple(range(1, dim + 1))
        x = sfft.idstn(sfft.dstn(cols, type=1, axes=axes) / sym[None], type=1, axes=axes)
        return x.reshape(x.shape[0], -1).T.reshape(b.shape)
    return apply


def smallest_eigenvalues_sine(dim: int, N: int, count: int, extra: int = 8, tol: float = 1e-14, seed: int = 0):
    """The `count` smallest eigenvalues of the constant-coefficient pencil by
    ARPACK in shift-invert mode around 0, with the exact sine-transform A^{-1}
    (meshes too large to factorise)."""
    import meshgen as mg
    A, M = mg.assemble(dim, N)
    n = A.shape[0]
    inv = laplacian_inverse(dim, N)
    op = spla.LinearOperator((n, n), matvec=inv, matmat=inv, dtype=np.float64)
    v0 = np.random.default_rng(seed).standard_normal(n)
    vals = spla.eigsh(A, k=count + extra, M=M, sigma=0.0, which="LM", OPinv=op, tol=tol, v0=v0,
                      return_eigenvectors=False)
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
