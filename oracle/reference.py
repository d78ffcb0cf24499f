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
