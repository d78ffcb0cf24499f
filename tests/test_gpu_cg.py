"""GPU parity of the conjugate-gradient smoother (the multigrid smoother of
the paper's experiments, Section 5.1) against the oracle's CG-smoothed PASM,
through the C ABI.

CG is nonlinear in its data (the step lengths come from the residuals), but
two or three steps are well conditioned, so float64 runs match the oracle to
the same tolerances as the Jacobi-smoothed path: the multigrid iterate to
1e-11, eigenvalues to 1e-10 and vectors to 1e-8 (relative) per step.  Mixed
precision (float32 CG inside the V-cycles, double-float outer residuals)
must reach the oracle's converged eigenvalues to 1e-9.
"""
import numpy as np
import pytest

import gpu_accuracy as ga
import meshgen as mg
import oracle
from paper_1908_10251_gb300 import accuracy as acc
from oracle import pasm as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def pg():
    from paper_1908_10251_gb300 import build
    build.build()
    import paper_1908_10251_gb300 as pkg
    pkg.load_library()
    return pkg


def setup_ctx(pg, H, **opts):
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    return pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(smoother=pg.PASM_CG, **opts),
                         torch.cuda.current_stream().cuda_stream)


def colrel(U, V):
    return max(np.abs(U[:, j] - V[:, j]).max() / np.abs(V[:, j]).max() for j in range(V.shape[1]))


@pytest.mark.parametrize("dim,Nf,Nc,k,nu", [(2, 64, 8, 6, 2), (2, 128, 16, 16, 3), (3, 16, 8, 5, 2)])
def test_cg_bvp_parity_fp64(pg, dim, Nf, Nc, k, nu):
    """Algorithm 1 step 1 with CG smoothing (nu steps pre and post): the
    multigrid iterate matches the oracle's."""
    H = mg.build_hierarchy(dim, Nf, Nc)
    ctx = setup_ctx(pg, H, precision=0, nu_pre=nu, nu_post=nu)
    prob = oracle.Problem.from_hierarchy(H, smoother="cg", nu_pre=nu, nu_post=nu)
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    Uh = np.zeros_like(U)
    pg.pasm_bvp(ctx, lam, U, Uh)
    assert colrel(Uh, op.bvp_solve(prob, lam, U)) < 1e-11


def test_cg_correction_steps_parity_fp64(pg):
    """The small unit-square workload (h = 1/64, H = 1/8, k = 8): five CG-smoothed correction
    steps from the same initial pairs match the oracle step by step."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H, precision=0)
    prob = oracle.Problem.from_hierarchy(H, smoother="cg")
    k = 8
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    for step in range(5):
        lam, U, _ = oracle.correction(prob, lam, U)
        pg.pasm_step(ctx)
        lg = np.zeros(k)
        Ug = np.zeros_like(U)
        pg.pasm_get(ctx, lg, Ug)
        assert np.allclose(lg, lam, rtol=1e-10), (step, np.abs(lg / lam - 1).max())
        assert colrel(Ug, U) < 1e-8, step


def test_cg_mixed_precision_final_state(pg):
    """Mixed precision with CG smoothing, 40 steps (pairs frozen at
    |d lambda| / lambda < 1e-13): at the end every pair the float64 oracle converges (without freezing, 40 steps)
    is within 1e-9 of the oracle's eigenvalue and of the ARPACK reference of
    its cluster, distinct, and within an M-principal angle of 1e-6 of both the
    reference eigenspace and the oracle's vectors."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H, precision=1, max_steps=40)
    prob = oracle.Problem.from_hierarchy(H, smoother="cg")
    k = 5
    lam_o, U_o, _, _ = oracle.solve(prob, k, tol=0.0, max_steps=40)
    A, M = H.fine.A, H.fine.M
    ref, vecs = acc.reference_pairs(A, M, k + 6, acc.stencil_inverse(A, 2, 64))
    pset = np.where(acc.cluster_errors(lam_o, ref) <= 1e-9)[0]
    assert len(pset) >= 4
    lam = np.zeros(k)
    U = np.zeros((H.fine.n, k))
    steps = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    pg.pasm_solve(ctx, k, 1e-13, None, None, lam, U, steps, status)
    assert np.allclose(lam[pset], lam_o[pset], rtol=1e-9)
    ga.check_final(M, lam, U, ref, vecs, pset)
    for i in pset:
        assert acc.angle_to(M, U[:, [i]], U_o[:, [i]]) <= 1e-6, i


def test_cg_zero_and_ragged_columns(pg):
    """k = 3 (one padded column in the block of 4): the padded column's CG
    stays at zero (zero right-hand side, no division by zero) and the real
    columns match the oracle."""
    H = mg.build_hierarchy(2, 32, 8)
    ctx = setup_ctx(pg, H, precision=0)
    prob = oracle.Problem.from_hierarchy(H, smoother="cg")
    k = 3
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    pg.pasm_step(ctx)
    lam_o, U_o, _ = oracle.correction(prob, lam, U)
    lg = np.zeros(k)
    Ug = np.zeros_like(U)
    pg.pasm_get(ctx, lg, Ug)
    assert np.all(np.isfinite(lg)) and np.all(np.isfinite(Ug))
    assert np.allclose(lg, lam_o, rtol=1e-10)
    assert colrel(Ug, U_o) < 1e-8
