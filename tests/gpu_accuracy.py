"""Helpers of the GPU tests that judge computed eigenpairs at full size: the
set of pairs the float64 oracle converges and holds, reference eigenvectors,
and the final-state check (eigenvalue within the target of the pair's own
cluster, no duplicate in a cluster, largest M-principal angle to the cluster's
eigenspace within the bound)."""
import json
import os

import numpy as np

from paper_1908_10251_gb300 import accuracy as acc

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_VECS = {}


def golden_table(name):
    return np.loadtxt(os.path.join(GOLDEN, name + ".txt"))


def history(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return np.array(json.load(f)["history"])


def stable_set(ref_all, hist_name, nofreeze_name=None, target=1e-9):
    """Pairs the float64 oracle drives within `target` of a reference
    eigenvalue of their cluster (frozen run), and -- when the oracle's run
    without freezing is stored -- still holds there at its end."""
    hist = history(hist_name)
    err = np.array([acc.cluster_errors(row, ref_all) for row in hist])
    keep = np.where(np.nanmin(err, axis=0) <= target)[0]
    if nofreeze_name:
        last = acc.cluster_errors(history(nofreeze_name)[-1], ref_all)
        keep = keep[last[keep] <= target]
    return keep


def reference_vectors(H, dim, N, ref_all, upto):
    """M-orthonormal eigenvectors of the finest pencil covering every cluster of
    pairs 0..upto (ARPACK shift-invert, exact sine-transform A^{-1}); cached per
    mesh.  Also checks the eigenvalues against the stored table."""
    cid = acc.clusters(ref_all)
    last = int(np.where(cid == cid[upto])[0].max())
    count = min(len(ref_all), last + 7)
    key = (dim, N)
    if key not in _VECS or _VECS[key].shape[1] < count:
        ainv = acc.stencil_inverse(H.fine.A, dim, N)
        vals, vecs = acc.reference_pairs(H.fine.A, H.fine.M, count, ainv)
        assert np.allclose(vals, ref_all[:count], rtol=1e-11), np.abs(vals / ref_all[:count] - 1).max()
        _VECS[key] = vecs
    return _VECS[key]


def lu_inverse(A):
    """A^{-1} by a sparse LU factorisation (small meshes, any coefficients)."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(A.tocsc())
    return lambda B: lu.solve(np.asarray(B, dtype=np.float64))


def check_final(M, lam, U, ref_all, vecs, pairs, target=1e-9, angle_max=1e-6):
    """Assert the final state: every pair of `pairs` within `target`, every
    cluster distinct with its largest M-principal angle <= angle_max.
    Returns the report."""
    rep = acc.report(M, lam, U, ref_all, target=target, pairs=pairs, vecs=vecs, angle_max=angle_max)
    bad = [int(i) for i in pairs if i not in rep["passed"]]
    detail = [(c["pairs"], c["angle"], c["distinct"]) for c in rep["clusters"] if not c["ok"]]
    assert not bad, ("pairs failing the final-state check", bad, rep["err"][bad], detail)
    return rep
