"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle on
the same seeded inputs.

Tolerances (float64 mode): one correction step reproduces the oracle's
eigenvalues to 1e-10 relative and vectors to 1e-8 (max-norm relative); the
arithmetic differs only in summation order and in the form of the multigrid
iteration (defect correction from zero vs. the oracle's direct iteration from
u, identical in exact arithmetic), so the observed gap is ~1e-13.  Mixed
precision (float32 V-cycles under float64 residuals) must reach the oracle's
converged eigenvalues to 1e-9 relative.
"""
import numpy as np
import pytest

import meshgen as mg
import oracle
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
    return pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(**opts), torch.cuda.current_stream().cuda_stream)


def get_state(pg, ctx, n, k):
    lam = np.zeros(k)
    U = np.zeros((n, k))
    steps = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    pg.pasm_get(ctx, lam, U, steps, status)
    return lam, U, steps, status


def colrel(U, V):
    """max over columns of max|U - V| / max|V|"""
    return max(np.abs(U[:, j] - V[:, j]).max() / np.abs(V[:, j]).max() for j in range(V.shape[1]))


def align(U, V):
    """flip the columns of U to the sign of V"""
    s = np.sign(np.einsum("ij,ij->j", U, V))
    s[s == 0] = 1
    return U * s


# ----------------------------------------------------------------------------- setup (Algorithm 2 step 1)

@pytest.mark.parametrize("Nf,Nc", [(32, 8), (64, 16)])
def test_coarse_eigendecomposition(pg, Nf, Nc):
    H = mg.build_hierarchy(2, Nf, Nc)
    ctx = setup_ctx(pg, H)
    lam, Q = pg.pasm_coarse_eigs(ctx)
    prob = oracle.Problem.from_hierarchy(H)
    lo, Qo = oracle.coarse_eigenpairs(prob)
    assert np.allclose(lam, lo, rtol=1e-12)
    MH = H.levels[0].M.toarray()
    AH = H.levels[0].A.toarray()
    assert np.allclose(Q.T @ MH @ Q, np.eye(len(lam)), atol=1e-11)
    assert np.allclose(Q.T @ AH @ Q, np.diag(lam), atol=1e-9 * lam.max())


def test_coarse_initial_state(pg):
    H = mg.build_hierarchy(2, 32, 8)
    ctx = setup_ctx(pg, H)
    k = 5
    pg.pasm_init(ctx, k, 1e-10)
    lam, U, steps, status = get_state(pg, ctx, H.fine.n, k)
    prob = oracle.Problem.from_hierarchy(H)
    lo, Uo = oracle.initial_state(prob, k)
    assert np.allclose(lam, lo, rtol=1e-12)
    assert colrel(align(U, Uo), Uo) < 1e-10
    assert np.all(steps == 0) and np.all(status == 0)


# ----------------------------------------------------------------------------- Algorithm 1, split

@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-5)])
def test_bvp_step_parity(pg, precision, tol):
    """Algorithm 1 step 1: two V-cycles for A u^ = lambda M u from u."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H, precision=precision)
    prob = oracle.Problem.from_hierarchy(H)
    k = 6
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    Uh = np.zeros_like(U)
    pg.pasm_bvp(ctx, lam, U, Uh)
    Uo = op.bvp_solve(prob, lam, U)
    assert colrel(Uh, Uo) < tol


@pytest.mark.parametrize("Nf,Nc,k", [(32, 8, 4), (64, 8, 8), (64, 16, 12)])
def test_augmented_step_parity(pg, Nf, Nc, k):
    """Algorithm 1 step 2: bordered eigenproblem, selection and update, given
    the same u~ on both sides."""
    H = mg.build_hierarchy(2, Nf, Nc)
    ctx = setup_ctx(pg, H)
    prob = oracle.Problem.from_hierarchy(H)
    lam, U = oracle.initial_state(prob, k)
    Ut = op.bvp_solve(prob, lam, U)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    lam_g = np.zeros(k); U_g = np.zeros_like(U); beta = np.zeros(k); zeta = np.zeros(k)
    pg.pasm_augmented(ctx, lam, Ut, lam_g, U_g, beta, zeta)
    for i in range(k):
        b, c, be, ze = op.bordering(prob, Ut[:, i])
        assert beta[i] == pytest.approx(be, rel=1e-12)
        assert zeta[i] == pytest.approx(ze, rel=1e-12)
    lam_o = np.zeros(k); U_o = np.zeros_like(U)
    for i in range(k):
        theta, X, sv, ok = op.augmented_eigenproblem(prob, Ut[:, i])
        j = int(np.argmax(np.abs(sv)))
        x = X[:, j] if sv[j] >= 0 else -X[:, j]
        lam_o[i] = theta[j]
        U_o[:, i] = x[-1] * Ut[:, i] + prob.Pc @ x[:-1]
    assert np.allclose(lam_g, lam_o, rtol=1e-11)
    assert colrel(U_g, U_o) < 1e-8


# ----------------------------------------------------------------------------- whole correction steps

@pytest.mark.parametrize("use_graph", [1, 0])
def test_correction_steps_parity_fp64(pg, use_graph):
    """The small unit-square workload (h = 1/64, H = 1/8, k = 8): five correction steps from the
    same initial pairs match the oracle step by step."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H, use_graph=use_graph)
    prob = oracle.Problem.from_hierarchy(H)
    k = 8
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    for step in range(5):
        lam, U, _ = oracle.correction(prob, lam, U)
        pg.pasm_step(ctx)
        lg, Ug, steps, status = get_state(pg, ctx, H.fine.n, k)
        assert np.allclose(lg, lam, rtol=1e-10), (step, np.abs(lg / lam - 1).max())
        assert colrel(Ug, U) < 1e-8, step
        assert np.all(steps == step + 1)


def test_secular_counters(pg):
    """pasm_secular_stats after five steps at h = 1/64, H = 1/8, k = 8: every active pair solved
    its first window (root 0 and the roots around lambda^(l)) each step, no root
    iteration hit its cap, and the counters restart at pasm_init."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H)
    k = 8
    pg.pasm_init(ctx, k, 0.0)
    assert pg.pasm_secular_stats(ctx) == (0, 0, 0)
    for _ in range(5):
        pg.pasm_step(ctx)
    roots, failed, capped = pg.pasm_secular_stats(ctx)
    assert roots >= 5 * k * 2 and capped == 0 and failed >= 0
    pg.pasm_init(ctx, k, 0.0)
    assert pg.pasm_secular_stats(ctx) == (0, 0, 0)
    pg.pasm_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-3)])
def test_residual_report(pg, precision, tol):
    """pasm_residuals against the residual of the state pasm_get returns,
    recomputed on the CPU in float64: ||A u - lam M u|| / (|lam| ||u||_M) per
    pair, after 1 and after 8 steps (large and small residuals).  Mixed mode
    forms r in double-float (2^-46 of |A u|), so small residuals agree to
    1e-3 relative plus 1e-13."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H, precision=precision)
    k = 8
    pg.pasm_init(ctx, k, 0.0)
    A, M = H.fine.A, H.fine.M
    for steps in (1, 7):
        for _ in range(steps):
            pg.pasm_step(ctx)
        res = pg.pasm_residuals(ctx)
        lam, U, _, _ = get_state(pg, ctx, H.fine.n, k)
        R = A @ U - (M @ U) * lam
        ref = np.linalg.norm(R, axis=0) / (np.abs(lam) * np.sqrt(np.einsum("ij,ij->j", U, M @ U)))
        assert np.all(np.abs(res - ref) <= tol * ref + 1e-13), (res, ref)
    pg.pasm_destroy(ctx)


def test_residual_guarded_freeze(pg):
    """opts.res_tol: with a bound the converged pairs meet, pasm_solve ends as
    without it (every pair converged, eigenvalues to 1e-10, residuals below the
    bound); with a bound no pair can meet, no pair is reported converged and
    pasm_solve returns PASM_ENOTCONV at max_steps."""
    H = mg.build_hierarchy(2, 32, 8)
    k = 5

    def solve(**opts):
        ctx = setup_ctx(pg, H, **opts)
        lam = np.zeros(k); U = np.zeros((H.fine.n, k))
        steps = np.zeros(k, dtype=np.int32); status = np.zeros(k, dtype=np.int32)
        code = pg.pasm_solve(ctx, k, 1e-10, None, None, lam, U, steps, status)
        res = pg.pasm_residuals(ctx)
        pg.pasm_destroy(ctx)
        return code, lam, status, res

    code0, lam0, status0, _ = solve()
    assert code0 == 0 and np.all(status0 == 1)
    code1, lam1, status1, res1 = solve(res_tol=1e-6)
    assert code1 == 0 and np.all(status1 == 1) and np.all(res1 <= 1e-6)
    assert np.allclose(lam1, lam0, rtol=1e-10)
    code2, lam2, status2, _ = solve(res_tol=1e-300, max_steps=12)
    assert code2 == 5 and np.all(status2 == 0)
    assert np.allclose(lam2, lam0, rtol=1e-9)


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-11)])
def test_pairs_independent_of_the_batch(pg, precision, tol):
    """Pairs are independent (Section 3.2): three steps of k = 8 pairs in one
    block give each pair what the same pair gives alone (k = 1, padded to a
    block of 4), to rounding in the cross-row sums."""
    H = mg.build_hierarchy(2, 64, 8)
    prob = oracle.Problem.from_hierarchy(H)
    k = 8
    lam0, U0 = oracle.initial_state(prob, k)
    ctx = setup_ctx(pg, H, precision=precision)
    pg.pasm_init(ctx, k, 0.0, lam0, U0)
    for _ in range(3):
        pg.pasm_step(ctx)
    lam, U, _, _ = get_state(pg, ctx, H.fine.n, k)
    pg.pasm_destroy(ctx)
    for i in (0, 3, 7):
        c1 = setup_ctx(pg, H, precision=precision)
        pg.pasm_init(c1, 1, 0.0, lam0[i:i + 1].copy(), np.ascontiguousarray(U0[:, i:i + 1]))
        for _ in range(3):
            pg.pasm_step(c1)
        l1, U1, _, _ = get_state(pg, c1, H.fine.n, 1)
        pg.pasm_destroy(c1)
        assert abs(l1[0] / lam[i] - 1) <= tol, (i, l1[0], lam[i])
        assert np.abs(U1[:, 0] - U[:, i]).max() / np.abs(U[:, i]).max() <= 100 * tol, i


def test_solve_converges_like_oracle(pg):
    """pasm_solve from the coarse initial pairs: the pairs the oracle converges
    (to the brute-force eigenvalues) converge on the GPU to the same values,
    with the same per-pair step counts up to one."""
    H = mg.build_hierarchy(2, 32, 8)
    ctx = setup_ctx(pg, H)
    prob = oracle.Problem.from_hierarchy(H)
    k = 5
    lam_o, U_o, steps_o, _ = oracle.solve(prob, k, tol=1e-10, max_steps=60)
    lam = np.zeros(k); U = np.zeros((H.fine.n, k))
    steps = np.zeros(k, dtype=np.int32); status = np.zeros(k, dtype=np.int32)
    code = pg.pasm_solve(ctx, k, 1e-10, None, None, lam, U, steps, status)
    assert code == 0
    assert np.allclose(lam, lam_o, rtol=1e-10)
    assert np.all(np.abs(steps - steps_o) <= 1)
    assert np.all(status == 1)


def test_mixed_precision_reaches_oracle(pg):
    """Mixed mode (float32 V-cycles as a defect correction under float64
    residuals): the converged eigenvalues match the oracle's to 1e-9."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H, precision=1)
    prob = oracle.Problem.from_hierarchy(H)
    k = 5
    lam_o, U_o, _, _ = oracle.solve(prob, k, tol=1e-12, max_steps=80)
    lam = np.zeros(k); U = np.zeros((H.fine.n, k))
    steps = np.zeros(k, dtype=np.int32); status = np.zeros(k, dtype=np.int32)
    pg.pasm_solve(ctx, k, 1e-12, None, None, lam, U, steps, status)
    assert np.allclose(lam, lam_o, rtol=1e-9)
    A = H.fine.A
    for i in range(k):
        u = U[:, i] * np.sign(U[:, i] @ U_o[:, i])
        e = u - U_o[:, i]
        assert np.sqrt(e @ (A @ e)) < 1e-5


# ----------------------------------------------------------------------------- edge cases

@pytest.mark.parametrize("k", [1, 3, 5])
def test_ragged_k(pg, k):
    """k not a power of two (padded columns stay inert)."""
    H = mg.build_hierarchy(2, 32, 8)
    ctx = setup_ctx(pg, H)
    prob = oracle.Problem.from_hierarchy(H)
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    pg.pasm_step(ctx)
    lo, Uo, _ = oracle.correction(prob, lam, U)
    lg, Ug, _, _ = get_state(pg, ctx, H.fine.n, k)
    assert np.allclose(lg, lo, rtol=1e-10)
    assert colrel(Ug, Uo) < 1e-8


def test_non_dyadic_sizes(pg):
    """A hierarchy 6 -> 12 -> 24 (odd interior sizes 25, 121, 529 rows; the
    row grid does not divide the block)."""
    H = mg.build_hierarchy(2, 24, 6)
    ctx = setup_ctx(pg, H)
    prob = oracle.Problem.from_hierarchy(H)
    k = 3
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    for _ in range(3):
        lam, U, _ = oracle.correction(prob, lam, U)
        pg.pasm_step(ctx)
    lg, Ug, _, _ = get_state(pg, ctx, H.fine.n, k)
    assert np.allclose(lg, lam, rtol=1e-10)
    assert colrel(Ug, U) < 1e-8


def test_three_dimensional_kuhn(pg):
    """3D Kuhn mesh (h = 1/16, H = 1/4): step parity for the first pair."""
    H = mg.build_hierarchy(3, 16, 4)
    ctx = setup_ctx(pg, H)
    prob = oracle.Problem.from_hierarchy(H)
    k = 1
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    for _ in range(3):
        lam, U, _ = oracle.correction(prob, lam, U)
        pg.pasm_step(ctx)
    lg, Ug, _, _ = get_state(pg, ctx, H.fine.n, k)
    assert np.allclose(lg, lam, rtol=1e-10)
    assert colrel(Ug, U) < 1e-8


def test_single_level_is_degenerate(pg):
    """With V_h = V_H every u~ lies in V_H: the bordered mass matrix is
    singular, the pair is kept and flagged degenerate (no NaN)."""
    H = mg.build_hierarchy(2, 8, 8)
    ctx = setup_ctx(pg, H)
    k = 2
    pg.pasm_init(ctx, k, 0.0)
    lam0, U0, _, _ = get_state(pg, ctx, H.fine.n, k)
    pg.pasm_step(ctx)
    lam, U, steps, status = get_state(pg, ctx, H.fine.n, k)
    assert np.all(status == 2)
    assert np.array_equal(lam, lam0) and np.array_equal(U, U0)


def test_k_too_big(pg):
    H = mg.build_hierarchy(2, 16, 4)
    ctx = setup_ctx(pg, H)
    with pytest.raises(pg.PasmError) as ei:
        pg.pasm_init(ctx, 10, 1e-10)
    assert ei.value.code == 2


def test_maximum_k(pg):
    """The widest block the library takes, k = 256 (block-vector rows of 2 KB
    in float64), with a 16 x 16 coarse grid (N_H = 256, so k = N_H too): one
    float64 step matches the oracle for every pair; mixed precision runs the
    same step with finite results within 1e-6 of it for the first eigenvalue;
    k = 257 is refused."""
    H = mg.build_hierarchy(2, 68, 17)
    assert H.levels[0].A.shape[0] == 256
    k = 256
    prob = oracle.Problem.from_hierarchy(H)
    lam, U = oracle.initial_state(prob, k)
    lo, Uo, _ = oracle.correction(prob, lam, U)
    ctx = setup_ctx(pg, H)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    pg.pasm_step(ctx)
    lg, Ug, _, _ = get_state(pg, ctx, H.fine.n, k)
    pg.pasm_destroy(ctx)
    assert np.allclose(lg, lo, rtol=1e-10), np.abs(lg / lo - 1).max()
    assert colrel(Ug, Uo) < 1e-8
    ctx = setup_ctx(pg, H, precision=1)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    pg.pasm_step(ctx)
    lm, Um, _, _ = get_state(pg, ctx, H.fine.n, k)
    assert np.all(np.isfinite(lm)) and np.all(np.isfinite(Um))
    assert abs(lm[0] / lo[0] - 1) < 1e-6
    with pytest.raises(pg.PasmError) as ei:
        pg.pasm_init(ctx, 257, 0.0, np.zeros(257), np.zeros((H.fine.n, 257)))
    assert ei.value.code == pg.capi.PASM_EINVAL
    pg.pasm_destroy(ctx)


def test_device_pointers_and_stream(pg):
    """Inputs and outputs as torch CUDA tensors on the caller's stream."""
    H = mg.build_hierarchy(2, 32, 8)
    ctx = setup_ctx(pg, H)
    prob = oracle.Problem.from_hierarchy(H)
    k = 4
    lam, U = oracle.initial_state(prob, k)
    lam_d = torch.tensor(lam, device="cuda"); U_d = torch.tensor(U, device="cuda")
    pg.pasm_init(ctx, k, 0.0, lam_d, U_d)
    pg.pasm_step(ctx)
    lo, Uo, _ = oracle.correction(prob, lam, U)
    lg = torch.zeros(k, dtype=torch.float64, device="cuda"); Ug = torch.zeros_like(U_d)
    pg.pasm_get(ctx, lg, Ug)
    torch.cuda.synchronize()
    assert np.allclose(lg.cpu().numpy(), lo, rtol=1e-10)
    assert colrel(Ug.cpu().numpy(), Uo) < 1e-8


def test_nested_initial_state(pg):
    """Algorithm 2 step 2(A): one correction step on every intermediate level
    before the finest, GPU vs oracle (h = 1/64, H = 1/8, 4 grids)."""
    H = mg.build_hierarchy(2, 64, 8)
    ctx = setup_ctx(pg, H, init=1)
    prob = oracle.Problem.from_hierarchy(H)
    k = 6
    pg.pasm_init(ctx, k, 1e-10)
    lam, U, steps, status = get_state(pg, ctx, H.fine.n, k)
    lo, Uo = oracle.initial_state_nested(prob, k)
    assert np.allclose(lam, lo, rtol=1e-10)
    assert colrel(align(U, Uo), Uo) < 1e-8
    assert np.all(steps == 0) and np.all(status == 0)
