"""Host-side accuracy report for computed eigenpairs of A u = lambda M u.

The library returns eigenpairs of the finite-element pencil (Section 2, the
discrete eigenproblem).  This module measures how far they are from exact
discrete eigenpairs, given a table of reference eigenvalues (the k + a few
smallest, from any independent eigensolver):

* clusters: consecutive reference eigenvalues closer than 1e-4 (relative) form
  one cluster -- near-degenerate eigenvalues whose individual eigenvectors are
  not well defined, only their joint eigenspace;
* the relative eigenvalue error of pair i against the reference values of
  pair i's own cluster;
* the largest M-principal angle between the computed vectors of a cluster and
  the exact eigenspace of that cluster.  Without exact eigenvectors it is
  bounded by the Davis-Kahan sin(Theta) theorem applied to T = A^{-1} M,
  which is self-adjoint in the M inner product (see angle_bound); the bound
  is at most the gap ratio above the true angle, whatever the frequency
  content of the error (the residual of A - lambda M itself would weigh
  high-frequency error by the largest eigenvalue, ~1/h^2, and be useless);
* distinct slots: within one cluster, the computed vectors of the pairs that
  reached it must be linearly independent (two pairs on one eigenvector are a
  duplicate, not two converged pairs).

Plain numpy/scipy on the host; no part of the method runs here.
"""
from __future__ import annotations

import numpy as np

CLUSTER_GAP = 1e-4


def clusters(ref, gap: float = CLUSTER_GAP) -> np.ndarray:
    """Cluster id of each (ascending) reference eigenvalue."""
    ref = np.asarray(ref, dtype=np.float64)
    cid = np.zeros(len(ref), dtype=int)
    for i in range(1, len(ref)):
        cid[i] = cid[i - 1] + (1 if (ref[i] - ref[i - 1]) / ref[i] > gap else 0)
    return cid


def cluster_errors(lam, ref, gap: float = CLUSTER_GAP) -> np.ndarray:
    """Relative distance of each lam_i (i < len(ref)) to the nearest reference
    eigenvalue of pair i's cluster; NaN for pairs beyond the table."""
    ref = np.asarray(ref, dtype=np.float64)
    cid = clusters(ref, gap)
    out = np.full(len(lam), np.nan)
    for i, v in enumerate(np.asarray(lam, dtype=np.float64)):
        if i < len(ref):
            mem = ref[cid == cid[i]]
            out[i] = np.min(np.abs(v - mem) / mem)
    return out


def gram_min(M, X) -> float:
    """Smallest eigenvalue of the M-Gram matrix of the M-normalised columns of
    X: 1 for M-orthogonal columns, near 0 when two columns are the same
    vector up to sign."""
    X = np.asarray(X, dtype=np.float64)
    Xn = X / np.sqrt(np.einsum("ij,ij->j", X, M @ X))[None, :]
    G = Xn.T @ (M @ Xn)
    return float(np.linalg.eigvalsh(0.5 * (G + G.T)).min())


def m_orthonormal(M, X):
    """M-orthonormal basis of span(X) by Cholesky QR, twice (X of full rank)."""
    X = np.asarray(X, dtype=np.float64)
    Q = X / np.sqrt(np.einsum("ij,ij->j", X, M @ X))[None, :]
    for _ in range(2):
        G = Q.T @ (M @ Q)
        L = np.linalg.cholesky(0.5 * (G + G.T))
        Q = np.linalg.solve(L, Q.T).T
    return Q


def stencil_inverse(A, dim: int, N: int):
    """Exact A^{-1} for the constant-coefficient P1 stiffness matrices of the
    uniform meshes (the 5-point stencil (4, -1) on the right-triangle mesh of
    the square; h times the 7-point stencil (6, -1) on the Kuhn mesh of the
    cube): both are diagonalised by the type-I discrete sine transform over
    the interior nodes (x fastest).  Checks A against the stencil on a random
    vector first and raises ValueError if A is another matrix."""
    import scipy.fft as sfft
    # 2 - 2 cos(t) = 4 sin^2(t / 2): the subtraction would lose the low modes' digits (relative
    # error ~1e-10 at t = pi / 2048), and with them the smallest eigenpairs' accuracy
    c = 4.0 * np.sin(0.5 * np.arange(1, N) * np.pi / N) ** 2
    if dim == 2:
        sym = c[:, None] + c[None, :]
    elif dim == 3:
        sym = (c[:, None, None] + c[None, :, None] + c[None, None, :]) / N
    else:
        raise ValueError("dim must be 2 or 3")
    shape = (N - 1,) * dim
    axes = tuple(range(dim))

    def apply(B):
        B = np.asarray(B, dtype=np.float64)
        one = B.ndim == 1
        B2 = B.reshape(B.shape[0], -1)
        G = B2.T.reshape((-1,) + shape[::-1])        # (cols, z, y, x): x fastest
        ax = tuple(a + 1 for a in axes)
        Xh = sfft.dstn(G, type=1, axes=ax) / sym.T[None]
        X = sfft.idstn(Xh, type=1, axes=ax).reshape(B2.shape[1], -1).T
        return X[:, 0] if one else X

    x = np.random.default_rng(0).standard_normal(A.shape[0])
    if A.shape[0] != (N - 1) ** dim or np.abs(A @ apply(x) - x).max() > 1e-9 * np.abs(x).max():
        raise ValueError("A is not the constant-coefficient stencil of this mesh")
    return apply


def angle_bound(M, X, ref, members, ainv):
    """Davis-Kahan bound on the largest M-principal angle between span(X) and
    the eigenspace of the reference eigenvalues with indices `members` (one
    cluster; the table must extend past it).  The operator is T = A^{-1} M,
    self-adjoint in the M inner product with eigenvalues 1/lambda_j and the
    same eigenvectors: with Ritz values mu of T on span(X) and residual block
    T Y - Y diag(mu) of the Ritz vectors Y, the sine of the largest angle is
    at most ||T Y - Y diag(mu)||_M / delta, delta the distance from the Ritz
    values to every 1/lambda_j outside the cluster (those past the table lie
    in [0, 1/ref[last]]).  The bound exceeds the true angle by at most the
    gap ratio (1/lambda) / delta.  `ainv` applies A^{-1} to a block.
    Returns (bound, delta, ritz values in lambda units)."""
    ref = np.asarray(ref, dtype=np.float64)
    members = np.asarray(members)
    Q = m_orthonormal(M, X)
    Z = ainv(M @ Q)
    Hs = Q.T @ (M @ Z)
    mu, W = np.linalg.eigh(0.5 * (Hs + Hs.T))
    R = Z @ W - (Q @ W) * mu[None, :]
    G = R.T @ (M @ R)
    rnorm = float(np.sqrt(max(np.linalg.eigvalsh(0.5 * (G + G.T)).max(), 0.0)))
    if members.max() + 1 >= len(ref):
        raise ValueError("the reference table must extend past the cluster")
    lo = 1.0 / ref[:members.min()]                  # larger mu: the eigenvalues below the cluster
    hi_max = 1.0 / ref[members.max() + 1]           # every eigenvalue above has mu <= this
    delta = min((lo.min() - mu.max()) if len(lo) else np.inf, mu.min() - hi_max)
    theta = 1.0 / mu
    if not delta > 0:
        return np.inf, float(delta), theta
    return rnorm / delta, float(delta), theta


def angle_to(M, X, V):
    """Largest M-principal angle (its sine) from span(X) to span(V), computed
    directly from both bases (for when reference eigenvectors are known)."""
    Qx = m_orthonormal(M, X)
    Qv = m_orthonormal(M, V)
    Z = Qx - Qv @ (Qv.T @ (M @ Qx))
    G = Z.T @ (M @ Z)
    return float(np.sqrt(max(np.linalg.eigvalsh(0.5 * (G + G.T)).max(), 0.0)))


def reference_pairs(A, M, count: int, ainv, tol: float = 1e-13, seed: int = 0):
    """The `count` smallest eigenpairs of (A, M) by ARPACK's Lanczos in
    shift-invert mode around 0, with A^{-1} given by `ainv` (a library
    eigensolver, independent of the method): eigenvalues ascending and
    M-orthonormal eigenvectors."""
    import scipy.sparse.linalg as spla
    n = A.shape[0]
    op = spla.LinearOperator((n, n), matvec=ainv, matmat=ainv, dtype=np.float64)
    v0 = np.random.default_rng(seed).standard_normal(n)
    vals, vecs = spla.eigsh(A, k=count, M=M, sigma=0.0, which="LM", OPinv=op, tol=tol, v0=v0)
    order = np.argsort(vals)
    vals, vecs = vals[order], vecs[:, order]
    return vals, m_orthonormal(M, vecs)


def report(M, lam, U, ref, target: float = 1e-9, pairs=None, gap: float = CLUSTER_GAP, vecs=None, ainv=None,
           angle_max: float = 1e-6):
    """Per-pair and per-cluster accuracy of computed pairs (lam, U) against a
    reference table `ref` (ascending eigenvalues; `vecs`, if given, their
    M-orthonormal eigenvectors).  `pairs` restricts the check to a set of pair
    indices (default: every pair the table covers).

    A pair is within the target when its cluster error is at most `target`.
    For each cluster holding such pairs: the distinct-slot test (no more pairs
    than eigenvalues, linearly independent vectors) and the largest
    M-principal angle between their vectors and the cluster's eigenspace --
    measured against `vecs` when the cluster lies inside them, else the
    Davis-Kahan bound when `ainv` (A^{-1}) is given.  A pair passes when it
    is within the target and its cluster is distinct with angle <= angle_max.

    Returns a dict: err and angle (per pair; NaN where not evaluated),
    passed (indices), clusters (list of {pairs, members, angle, angle_kind,
    delta, gram_min, distinct, ok}), max_angle."""
    ref = np.asarray(ref, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    err = cluster_errors(lam, ref, gap)
    cid = clusters(ref, gap)
    cand = range(min(len(lam), len(ref))) if pairs is None else pairs
    within = [int(i) for i in cand if i < len(ref) and err[i] <= target]
    angle = np.full(len(lam), np.nan)
    out, passed = [], []
    for c in sorted({int(cid[i]) for i in within}):
        ps = [i for i in within if cid[i] == c]
        members = np.where(cid == c)[0]
        X = np.asarray(U)[:, ps]
        gmin = gram_min(M, X)
        distinct = len(ps) <= len(members) and gmin > 1e-3
        a, kind, delta = None, None, None
        if distinct and vecs is not None and members.max() < vecs.shape[1]:
            a, kind = angle_to(M, X, vecs[:, members]), "measured"
        elif distinct and ainv is not None and members.max() + 1 < len(ref):
            a, delta, _ = angle_bound(M, X, ref, members, ainv)
            kind = "bound"
        ok = bool(distinct and a is not None and a <= angle_max)
        if a is not None:
            angle[ps] = a
        if ok:
            passed += ps
        out.append({"pairs": ps, "members": [int(v) for v in members], "angle": a, "angle_kind": kind,
                    "delta": delta, "gram_min": gmin, "distinct": bool(distinct), "ok": ok})
    angles = [c["angle"] for c in out if c["angle"] is not None]
    return {"err": err, "angle": angle, "passed": sorted(passed), "within": within, "clusters": out,
            "max_angle": max(angles) if angles else None}
