"""The general operator of the paper's Example 2 (Section 5.2):
-div(D grad u) + phi u = lambda u on the unit cube with D = I + (x-1/2)(x-1/2)^T
and phi = exp(prod_i (x_i - 1/2)), P1 elements on the Kuhn mesh
(meshgen.assemble_operator), and the oracle's PASM on it.  CPU only.

The element integrals use a degree-2 rule; pins: it reproduces the stencil
assembly for D = I, adds exactly c M for a constant potential, integrates D
exactly over the cube, and gives O(h^2) convergence to the closed-form
eigenvalues of a constant anisotropic D; the oracle's PASM on the Example 2
pencil reaches the dense generalized eigenvalues."""
import numpy as np
import pytest
import scipy.linalg as sla

import meshgen as mg
import oracle
from oracle import pasm as op


def identity(x):
    return np.broadcast_to(np.eye(x.shape[-1]), x.shape[:-1] + (x.shape[-1], x.shape[-1]))


@pytest.mark.parametrize("dim,N", [(2, 16), (3, 8)])
def test_identity_diffusion_matches_stencil_assembly(dim, N):
    A, M = mg.assemble_operator(dim, N, identity)
    A0, M0 = mg.assemble(dim, N)
    assert abs(A - A0).max() <= 1e-14 * abs(A0).max()
    assert abs(M - M0).max() <= 1e-14 * abs(M0).max()


def test_constant_potential_adds_mass():
    A, M = mg.assemble_operator(3, 8, identity, lambda x: np.full(x.shape[:-1], 2.5))
    A0, M0 = mg.assemble(3, 8)
    assert abs(A - (A0 + 2.5 * M0)).max() <= 1e-13 * abs(A).max()


def test_diffusion_integrates_exactly_over_the_cube():
    """sum over all simplices of vol * (simplex average of D) = int_cube D
    = I + diag(1/12) (the off-diagonal products of (x_i - 1/2) integrate to 0)."""
    avgs, vol = mg.element_averages(3, 6, mg.example2_diffusion)
    total = sum(a.sum(axis=(0, 1, 2)) for a in avgs) * vol
    assert np.abs(total - np.eye(3) * (1.0 + 1.0 / 12.0)).max() < 1e-14


def test_anisotropic_constant_diffusion_eigenvalue_order_h2():
    """D = diag(1, 2, 3): lambda_1 = pi^2 (1 + 2 + 3); the P1 error falls by ~4 per halving of h."""
    D = np.diag([1.0, 2.0, 3.0])
    exact = 6.0 * np.pi ** 2
    errs = []
    for N in (6, 12):
        A, M = mg.assemble_operator(3, N, lambda x: np.broadcast_to(D, x.shape[:-1] + (3, 3)))
        lam = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[0, 0])[0]
        assert lam > exact
        errs.append(lam - exact)
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_example2_pencil_is_spd_and_pasm_matches_dense():
    H = mg.build_hierarchy(3, 16, 8, operator=(mg.example2_diffusion, mg.example2_potential))
    A, M = H.fine.A, H.fine.M
    assert abs(A - A.T).max() < 1e-15 * abs(A).max()
    k = 4
    dense = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[0, k - 1])
    assert dense[0] > 0
    prob = oracle.Problem.from_hierarchy(H)
    lam, U, steps, _ = op.solve(prob, k, tol=1e-12, max_steps=60, history=True)
    assert np.abs(lam - dense).max() / dense.max() < 1e-10
