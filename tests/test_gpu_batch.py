"""GPU checks of the batch boundary (pasm_batch_*): problems of uneven size
and k -- including variable-coefficient ones, -div(kappa grad u) = lambda u
with kappa = exp(g), g a seeded Gaussian field -- solved together must give
exactly what each problem gives alone, and a kappa problem matches the
oracle step by step."""
import numpy as np
import pytest

import meshgen as mg
import oracle

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


def kappa_problem(N, seed):
    kap = mg.gaussian_log_field(N, seed)
    return mg.build_hierarchy(2, N, 8, kappa=kap)


def parts(H):
    return [lv.A for lv in H.levels], [lv.M for lv in H.levels], list(H.P)


def test_batch_equals_individual_solves(pg):
    probs = [mg.build_hierarchy(2, 32, 8), kappa_problem(64, 1001), kappa_problem(32, 1002),
             mg.build_hierarchy(2, 64, 16)]
    ks = [3, 5, 4, 8]
    opts = pg.pasm_default_opts(precision=1, max_steps=40)
    batch = pg.pasm_batch_setup([parts(H) for H in probs], opts, torch.cuda.current_stream().cuda_stream)
    code, lams, Us, steps, stats, rounds = pg.pasm_batch_solve(batch, ks, 1e-10)
    assert rounds >= max(int(s.max()) for s in steps)
    for H, k, lb, Ub, sb in zip(probs, ks, lams, Us, steps):
        A, M, P = parts(H)
        ctx = pg.pasm_setup(A, M, P, opts, torch.cuda.current_stream().cuda_stream)
        lam = np.zeros(k); U = np.zeros((H.fine.n, k)); st = np.zeros(k, dtype=np.int32)
        pg.pasm_solve(ctx, k, 1e-10, None, None, lam, U, st, None)
        assert np.array_equal(lam, lb) and np.array_equal(U, Ub) and np.array_equal(st, sb)
    pg.pasm_batch_destroy(batch)


def test_kappa_problem_step_parity(pg):
    """Variable coefficient (Galerkin coarse operators): float64 steps match
    the oracle's to 1e-10."""
    H = kappa_problem(64, 1003)
    prob = oracle.Problem.from_hierarchy(H)
    k = 4
    lam, U = oracle.initial_state(prob, k)
    A, M, P = parts(H)
    ctx = pg.pasm_setup(A, M, P, pg.pasm_default_opts(), torch.cuda.current_stream().cuda_stream)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    for _ in range(4):
        lam, U, _ = oracle.correction(prob, lam, U)
        pg.pasm_step(ctx)
    lg = np.zeros(k)
    pg.pasm_get(ctx, lg)
    assert np.allclose(lg, lam, rtol=1e-10)


def test_uneven_batch_full_size(pg):
    """The uneven batch at full size: 16 problems -div(kappa grad u) = lambda u,
    kappa = exp(g_p) with g_p a seeded Gaussian field (sigma 1, correlation 0.1,
    seed 1000 + p), fine grids 2^(8 + p mod 4) per side (65,025 to 4,190,209
    DoF), k_p = (8, 16, 32, 64, 128)[p mod 5], H = 1/16, mixed precision, all
    solved together by pasm_batch_solve (60 steps at most, tol 1e-10).

    No oracle runs at these sizes; checked instead, in float64 on the CPU:
      * every pair reported converged is a Ritz pair: its eigenvalue is the
        Rayleigh quotient u^T A u / u^T M u of its vector (1e-9);
      * pairs with relative residual ||A u - lambda M u|| / (lambda ||M u||)
        below 1e-3 are eigenpairs: on the four 256^2 problems each is within
        1e-9 of a shift-invert reference eigenvalue, and there are at least 60
        in the batch.  (A residual norm amplifies the float32 V-cycles'
        high-frequency error by up to lambda_max / lambda, so it is a coarse
        test.)  The other converged pairs are the method's spurious freezes: with
        this coarse space several pairs can select the same augmented Ritz pair,
        whose value then stops changing, and the paper's |delta lambda| test
        reads that as convergence -- the oracle freezes pairs 11-15 of problem 1
        at the same 232.7311330 (residual 4) as the GPU does;
      * problem 1 solved alone gives exactly what it gives in the batch."""
    from oracle.reference import smallest_eigenvalues
    probs, ks = [], []
    for p in range(16):
        N = 2 ** (8 + p % 4)
        kap = mg.gaussian_log_field(N, 1000 + p)
        probs.append(mg.build_hierarchy(2, N, 16, kappa=kap))
        ks.append((8, 16, 32, 64, 128)[p % 5])
    opts = pg.pasm_default_opts(precision=1, max_steps=60)
    batch = pg.pasm_batch_setup([parts(H) for H in probs], opts, torch.cuda.current_stream().cuda_stream)
    code, lams, Us, steps, stats, rounds = pg.pasm_batch_solve(batch, ks, 1e-10)
    pg.pasm_batch_destroy(batch)
    true_pairs = 0
    for p, (H, k, lam, U, st) in enumerate(zip(probs, ks, lams, Us, stats)):
        conv = st == 1
        A, M = H.fine.A, H.fine.M
        Uc = U[:, conv]
        MU = M @ Uc
        AU = A @ Uc
        rq = np.einsum("ij,ij->j", Uc, AU) / np.einsum("ij,ij->j", Uc, MU)
        assert np.max(np.abs(rq - lam[conv]) / lam[conv], initial=0.0) < 1e-9, p
        res = np.linalg.norm(AU - MU * lam[conv][None, :], axis=0) / (lam[conv] * np.linalg.norm(MU, axis=0))
        good = lam[conv][res < 1e-3]
        true_pairs += good.size
        if H.fine.N == 256:
            ref = smallest_eigenvalues(A, M, k + 8)
            err = np.array([np.min(np.abs(ref - v)) / v for v in good])
            assert err.max(initial=0.0) < 1e-9, (p, float(err.max()))
    assert true_pairs >= 60, true_pairs
    # problem 1 alone
    A, M, P = parts(probs[1])
    ctx = pg.pasm_setup(A, M, P, opts, torch.cuda.current_stream().cuda_stream)
    k = ks[1]
    lam = np.zeros(k)
    U = np.zeros((probs[1].fine.n, k))
    pg.pasm_solve(ctx, k, 1e-10, None, None, lam, U, None, None)
    assert np.array_equal(lam, lams[1]) and np.array_equal(U, Us[1])


def test_residual_guard_rejects_spurious_freezes(pg):
    """Problem 1 of the uneven batch (h = 1/512, kappa seed 1001, H = 1/16,
    k = 16, mixed precision), where the |delta lambda| test alone reports pairs
    converged at a value that is not an eigenvalue (residual about 4, see the
    test above).  With opts.res_tol = 1e-3, every pair pasm_solve reports
    converged has ||A u - lambda M u|| / (lambda ||u||_M) <= 1e-3, recomputed
    in float64 on the CPU, and the run ends with PASM_ENOTCONV if any pair is
    still iterating at max_steps."""
    N, k = 512, 16
    H = mg.build_hierarchy(2, N, 16, kappa=mg.gaussian_log_field(N, 1001))
    A, M, P = parts(H)

    def solve(res_tol):
        opts = pg.pasm_default_opts(precision=1, max_steps=60, res_tol=res_tol)
        ctx = pg.pasm_setup(A, M, P, opts, torch.cuda.current_stream().cuda_stream)
        lam = np.zeros(k)
        U = np.zeros((H.fine.n, k))
        steps = np.zeros(k, dtype=np.int32)
        status = np.zeros(k, dtype=np.int32)
        code = pg.pasm_solve(ctx, k, 1e-10, None, None, lam, U, steps, status)
        pg.pasm_destroy(ctx)
        Af, Mf = H.fine.A, H.fine.M
        MU = Mf @ U
        res = np.linalg.norm(Af @ U - MU * lam[None, :], axis=0) / (lam * np.sqrt(np.einsum("ij,ij->j", U, MU)))
        return code, status, res

    _, status0, res0 = solve(0.0)
    assert np.any((status0 == 1) & (res0 > 1e-3))           # the spurious freezes, unguarded
    code, status, res = solve(1e-3)
    conv = status == 1
    assert np.all(res[conv] <= 1e-3 * (1 + 1e-6)), res[conv]
    assert (code == 5) == bool(np.any(~conv))


def test_residual_guard_inside_the_step(pg):
    """The same problem driven by pasm_step alone (no host-side check): with
    opts.res_tol = 1e-3 the step itself freezes a pair only when the state it
    started from has relative residual <= 1e-3, so every pair reported
    converged after 40 steps has a small residual (recomputed in float64 on the
    CPU; the freezing step's own correction can only improve it, factor 2 of
    slack), while without the guard some converged pairs have residuals near 4."""
    N, k = 512, 16
    H = mg.build_hierarchy(2, N, 16, kappa=mg.gaussian_log_field(N, 1001))
    A, M, P = parts(H)

    def run(res_tol):
        opts = pg.pasm_default_opts(precision=1, res_tol=res_tol)
        ctx = pg.pasm_setup(A, M, P, opts, torch.cuda.current_stream().cuda_stream)
        pg.pasm_init(ctx, k, 1e-10)
        for _ in range(40):
            pg.pasm_step(ctx)
        lam = np.zeros(k)
        U = np.zeros((H.fine.n, k))
        steps = np.zeros(k, dtype=np.int32)
        status = np.zeros(k, dtype=np.int32)
        pg.pasm_get(ctx, lam, U, steps, status)
        pg.pasm_destroy(ctx)
        MU = H.fine.M @ U
        res = np.linalg.norm(H.fine.A @ U - MU * lam[None, :], axis=0) / (lam * np.sqrt(np.einsum("ij,ij->j", U, MU)))
        return status, res

    status0, res0 = run(0.0)
    assert np.any((status0 == 1) & (res0 > 1e-3))
    status, res = run(1e-3)
    conv = status == 1
    assert conv.any()
    assert np.all(res[conv] <= 2e-3), res[conv]
