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
