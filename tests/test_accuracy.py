"""The host-side accuracy report (paper_1908_10251_gb300/accuracy.py) against
exact eigenvectors from a dense solve: the Davis-Kahan angle bound is never
below the true largest M-principal angle and is within the gap ratio of it,
duplicates are detected, and the eigenvalue error uses the pair's own
cluster."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import meshgen as mg
import oracle
from paper_1908_10251_gb300 import accuracy as acc


def dense(N, count, dim=2):
    A, M = mg.assemble(dim, N)
    lam, V = sla.eigh(A.toarray(), M.toarray(), subset_by_index=[0, count - 1])
    return A, M, lam, V


def lu_inverse(A):
    lu = spla.splu(A.tocsc())
    return lambda B: lu.solve(np.asarray(B, dtype=np.float64))


@pytest.mark.parametrize("dim,N", [(2, 16), (2, 33), (3, 8)])
def test_stencil_inverse_is_exact(dim, N):
    """The sine-transform inverse of the constant-coefficient stiffness equals
    a sparse LU solve; another matrix is refused."""
    A, M = mg.assemble(dim, N)
    B = np.random.default_rng(1).standard_normal((A.shape[0], 3))
    X = acc.stencil_inverse(A, dim, N)(B)
    assert np.abs(X - lu_inverse(A)(B)).max() <= 1e-12 * np.abs(X).max()
    with pytest.raises(ValueError):
        acc.stencil_inverse(A + M, dim, N)


def test_clusters_of_the_square():
    """The (m, n) / (n, m) modes of the square are split only by the mesh
    (2.3e-6 relative at h = 1/1024): pairs 1, 2 form one cluster, pair 0 its
    own; at h = 1/16 the split (2e-2) is above the cluster gap."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "square_h1024_k72.txt")
    ref = np.loadtxt(path)
    cid = acc.clusters(ref)
    assert cid[0] != cid[1] and cid[1] == cid[2] and cid[2] != cid[3]
    e = acc.cluster_errors(ref[[0, 2, 1]], ref)
    assert np.all(e == 0.0)      # swapping within a cluster is no error
    e = acc.cluster_errors(ref[[1, 0]], ref)
    assert np.all(e > 0.5)       # a value of another cluster is
    A, M, lam, V = dense(16, 4)
    assert len(set(acc.clusters(lam))) == 4


def test_exact_vectors_have_zero_angle():
    A, M, lam, V = dense(16, 12)
    for members in ([0], [1, 2]):
        b, delta, theta = acc.angle_bound(M, V[:, members], lam, np.array(members), lu_inverse(A))
        assert b < 1e-12 and delta > 0
        assert np.allclose(np.sort(theta), lam[members], rtol=1e-13)
        assert acc.angle_to(M, V[:, members], V[:, members]) < 1e-7


def test_bound_brackets_a_known_rotation():
    """u = cos(phi) v_c + sin(phi) w with w M-orthonormal to the cluster (a mix
    of low and high modes): the true angle is phi; the bound lies between it
    and the gap ratio (1 / lambda_1) / delta times it."""
    A, M, lam, V = dense(16, 20)
    lam_all, V_all = sla.eigh(A.toarray(), M.toarray())
    W_hi = V_all[:, -10:]                  # the highest-frequency eigenvectors
    rng = np.random.default_rng(0)
    for members, phi in (([0], 1e-3), ([1, 2], 1e-5), ([3], 1e-7)):
        c = np.array(members)
        w = V[:, 5:20] @ rng.standard_normal(15) + W_hi @ rng.standard_normal(W_hi.shape[1])
        w /= np.sqrt(w @ (M @ w))
        X = V[:, c].copy()
        X[:, 0] = np.cos(phi) * X[:, 0] + np.sin(phi) * w
        true = acc.angle_to(M, X, V[:, c])
        assert abs(true - phi) <= 1e-6 * phi + 1e-12
        b, delta, _ = acc.angle_bound(M, X, lam, c, lu_inverse(A))
        assert b >= true * (1 - 1e-6)
        assert b <= true * (1.0 / lam[0]) / delta * 1.01


def test_duplicates_are_not_distinct():
    A, M, lam, V = dense(16, 12)
    U = V[:, :4].copy()
    U[:, 2] = -U[:, 1]            # pairs 1 and 2 on one eigenvector of their cluster
    rep = acc.report(M, lam[:4], U, lam, gap=1e-1, ainv=lu_inverse(A))
    c = [x for x in rep["clusters"] if x["pairs"] == [1, 2]][0]
    assert not c["distinct"] and not c["ok"] and c["angle"] is None
    ok = [x for x in rep["clusters"] if x["pairs"] == [0]][0]
    assert ok["distinct"] and ok["ok"] and ok["angle"] < 1e-10 and ok["angle_kind"] == "bound"
    assert rep["passed"] == [0, 3]


def test_oracle_converged_pairs_within_bound():
    """The oracle's PASM run for 30 steps without freezing on a small mesh: the
    true angle to the dense eigenspaces never exceeds the bound, and both are
    far below 1e-6 for the pairs within 1e-9 (pairs 1 and 2, split by 2.3e-3
    here, are separate clusters, where the bound is ~430 times the angle)."""
    H = mg.build_hierarchy(2, 32, 8)
    prob = oracle.Problem.from_hierarchy(H)
    k = 8
    lam, U, _, _ = oracle.solve(prob, k, tol=0.0, max_steps=30)
    A, M = H.fine.A, H.fine.M
    ref, V = sla.eigh(A.toarray(), M.toarray(), subset_by_index=[0, k + 7])
    ainv = acc.stencil_inverse(A, 2, 32)
    rep = acc.report(M, lam, U, ref, ainv=ainv)
    meas = acc.report(M, lam, U, ref, vecs=V)
    assert len(rep["within"]) >= 6 and rep["passed"] == rep["within"] == meas["passed"]
    for c, m in zip(rep["clusters"], meas["clusters"]):
        assert c["distinct"] and c["angle_kind"] == "bound" and m["angle_kind"] == "measured"
        true = acc.angle_to(M, U[:, c["pairs"]], V[:, c["members"]])
        assert abs(m["angle"] - true) <= 1e-15
        assert true <= c["angle"] * (1 + 1e-6) + 1e-12     # the dense vectors carry ~1e-14 themselves
        assert c["angle"] <= 1e-6, c
        assert c["angle"] <= 1e3 * max(true, 1e-12), c


def test_reference_pairs_match_dense():
    """ARPACK shift-invert with the sine-transform A^{-1}: eigenvalues and
    eigenspaces of the dense solve."""
    A, M, lam, V = dense(24, 10)
    vals, vecs = acc.reference_pairs(A, M, 12, acc.stencil_inverse(A, 2, 24))
    assert np.allclose(vals[:10], lam, rtol=1e-12)
    for c in np.unique(acc.clusters(lam)):
        mem = np.where(acc.clusters(lam) == c)[0]
        if mem.max() < 9:
            assert acc.angle_to(M, vecs[:, mem], V[:, mem]) < 1e-9


def test_stencil_inverse_keeps_the_low_modes_accurate():
    """The lowest grid sine mode through A then the sine-transform inverse at
    h = 1/1024 comes back to 1e-13 (the symbol is formed as 4 sin^2, not by
    the cancelling 2 - 2 cos)."""
    N = 1024
    A, _ = mg.assemble(2, N)
    t = np.arange(1, N) / N
    v = np.kron(np.sin(np.pi * t), np.sin(np.pi * t))
    back = acc.stencil_inverse(A, 2, N)(A @ v)
    assert np.abs(back - v).max() <= 1e-13 * np.abs(v).max()
