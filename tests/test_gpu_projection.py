"""The coarse projection b' = Q^T b, c' = Q^T c (the bordered matrix form of
Section 3.1 expressed in the coarse eigenbasis) on the tensor cores, through
pasm_project, against exact rational arithmetic.

Error bound of the digit-plane product (8 digits of 7 bits per operand,
products of weight 2^(-7 d), d <= 9, kept, summed exactly and rounded once):
slicing leaves < 2^(e_i - 56) per entry of row i of Q^T and < 2^(e_n - 56) per
entry of column n of b, and the dropped lighter products add < 8 2^-56 K
2^(e_i + e_n), where 2^e_i <= 2 max|Q_.i| and 2^e_n <= 2 max|b_.n|; the one
rounding adds half an ulp.  The tests use 2^-49 K max|Q_.i| max|b_.n| +
2^-52 |C|.  A float32 accumulator that lost bits would miss it by ~2^25.
"""
from fractions import Fraction

import numpy as np
import pytest

import meshgen as mg

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


def make_ctx(pg, dim, N, Nc, k, **opts):
    H = mg.build_hierarchy(dim, N, Nc)
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    ctx = pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(**opts), torch.cuda.current_stream().cuda_stream)
    pg.pasm_init(ctx, k, 1e-10)
    lam, Q = pg.pasm_coarse_eigs(ctx)
    return ctx, Q


def exact_entry(Q, b, i, n):
    return sum(Fraction(float(Q[j, i])) * Fraction(float(b[j, n])) for j in range(Q.shape[0]))


def bound(Q, b):
    K = Q.shape[0]
    return 2.0 ** -49 * K * np.outer(np.abs(Q).max(axis=0), np.abs(b).max(axis=0))


def check_against_exact(Q, b, got, rng, samples=160):
    """Sampled entries against exact rationals, all entries against float64."""
    NH, k = b.shape
    B = bound(Q, b)
    for _ in range(samples):
        i, n = int(rng.integers(NH)), int(rng.integers(k))
        ex = exact_entry(Q, b, i, n)
        err = abs(Fraction(float(got[i, n])) - ex)
        assert float(err) <= B[i, n] + 2.0 ** -52 * abs(float(ex)), (i, n, float(err), B[i, n])
    ref = Q.T @ b
    fp64_bound = Q.shape[0] * 2.0 ** -52 * (np.abs(Q).T @ np.abs(b))
    assert np.all(np.abs(got - ref) <= B + fp64_bound)


@pytest.mark.parametrize("dim,N,Nc,k", [(2, 32, 16, 64), (2, 16, 8, 16), (3, 16, 8, 32), (2, 32, 16, 4)])
def test_projection_matches_exact(pg, dim, N, Nc, k):
    ctx, Q = make_ctx(pg, dim, N, Nc, k)
    assert pg.pasm_projection_kind(ctx) == pg.PASM_PROJ_TENSOR
    NH = Q.shape[0]
    rng = np.random.default_rng(100 + dim * 10 + k)
    b = rng.standard_normal((NH, k)) * np.exp(rng.uniform(-20, 20, size=k))   # per-column scales
    c = rng.standard_normal((NH, k))
    bq = np.zeros((NH, k))
    cq = np.zeros((NH, k))
    pg.pasm_project(ctx, b, c, bq, cq)
    check_against_exact(Q, b, bq, rng)
    check_against_exact(Q, c, cq, rng)
    # a second call on the same context (the integer sums must start from zero again)
    bq2 = np.zeros((NH, k))
    cq2 = np.zeros((NH, k))
    pg.pasm_project(ctx, b, c, bq2, cq2)
    assert np.array_equal(bq, bq2) and np.array_equal(cq, cq2)


def test_projection_device_pointers_and_fp64_agree(pg):
    ctx, Q = make_ctx(pg, 2, 32, 16, 64)
    ctx64, Q64 = make_ctx(pg, 2, 32, 16, 64, projection=pg.PASM_PROJ_FP64)
    assert pg.pasm_projection_kind(ctx64) == pg.PASM_PROJ_FP64
    assert np.array_equal(Q, Q64)
    NH = Q.shape[0]
    rng = np.random.default_rng(7)
    b = torch.tensor(rng.standard_normal((NH, 64)), device="cuda")
    c = torch.tensor(rng.standard_normal((NH, 64)), device="cuda")
    out = [torch.zeros((NH, 64), dtype=torch.float64, device="cuda") for _ in range(4)]
    pg.pasm_project(ctx, b, c, out[0], out[1])
    pg.pasm_project(ctx64, b, c, out[2], out[3])
    torch.cuda.synchronize()
    bn, cn = b.cpu().numpy(), c.cpu().numpy()
    B = bound(Q, bn) + NH * 2.0 ** -52 * (np.abs(Q).T @ np.abs(bn))
    assert np.all(np.abs(out[0].cpu().numpy() - out[2].cpu().numpy()) <= 2 * B)
    C = bound(Q, cn) + NH * 2.0 ** -52 * (np.abs(Q).T @ np.abs(cn))
    assert np.all(np.abs(out[1].cpu().numpy() - out[3].cpu().numpy()) <= 2 * C)


def test_projection_degenerate_columns(pg):
    """Zero columns give exact zeros; a column holding a NaN gives NaN in that
    column only; wide exponent ranges across columns stay within the bound."""
    ctx, Q = make_ctx(pg, 2, 32, 16, 8)
    NH = Q.shape[0]
    rng = np.random.default_rng(11)
    b = rng.standard_normal((NH, 8))
    b[:, 1] = 0.0
    b[:, 2] *= 2.0 ** 600
    b[:, 3] *= 2.0 ** -600
    b[5, 4] = np.nan
    c = rng.standard_normal((NH, 8))
    c[:, 0] = 0.0
    bq = np.zeros((NH, 8))
    cq = np.zeros((NH, 8))
    pg.pasm_project(ctx, b, c, bq, cq)
    assert np.all(bq[:, 1] == 0.0) and np.all(cq[:, 0] == 0.0)
    assert np.all(np.isnan(bq[:, 4]))
    keep = [0, 1, 2, 3, 5, 6, 7]
    assert np.all(np.isfinite(bq[:, keep]))
    check_against_exact(Q, b[:, keep], bq[:, keep], rng, samples=60)
    check_against_exact(Q, c, cq, rng, samples=60)


def test_step_tensor_projection_matches_fp64_projection(pg):
    """Three correction steps of the whole path with either projection: the
    eigenvalues agree to 1e-13 and the vectors to 1e-10."""
    res = []
    for proj in (pg.PASM_PROJ_TENSOR, pg.PASM_PROJ_FP64):
        ctx, _ = make_ctx(pg, 2, 64, 16, 32, projection=proj)
        for _ in range(3):
            pg.pasm_step(ctx)
        n, _, _, _ = pg.pasm_sizes(ctx)
        lam = np.zeros(32)
        U = np.zeros((n, 32))
        pg.pasm_get(ctx, lam, U)
        res.append((lam, U))
    (l1, U1), (l2, U2) = res
    assert np.max(np.abs(l1 - l2) / l2) < 1e-13
    assert np.max(np.abs(U1 - U2)) / np.max(np.abs(U2)) < 1e-10


def test_bounded_wait_runs_out_and_context_recovers(pg):
    """The projection's MMA completion wait is bounded.  The test hook makes it
    run out safely -- no MMA is issued, so nothing arrives on the mbarrier and
    nothing is in flight when the CTA gives up and frees its TMEM: the call
    reports PASM_ETIMEOUT.  With the hook reset, the same context projects
    correctly again (the timed-out tiles still took part in the ticket
    protocol, so the integer accumulators were left cleared)."""
    ctx, Q = make_ctx(pg, 2, 32, 16, 16)
    NH = Q.shape[0]
    rng = np.random.default_rng(11)
    b = rng.standard_normal((NH, 16))
    c = rng.standard_normal((NH, 16))
    bq = np.zeros((NH, 16)); cq = np.zeros((NH, 16))
    pg.pasm_debug_waits(ctx, 1, 64)
    with pytest.raises(pg.PasmError) as ei:
        pg.pasm_project(ctx, b, c, bq, cq)
    assert ei.value.code == pg.PASM_ETIMEOUT
    pg.pasm_debug_waits(ctx, 0, 0)
    for _ in range(2):
        pg.pasm_project(ctx, b, c, bq, cq)
        check_against_exact(Q, b, bq, rng, samples=40)
        check_against_exact(Q, c, cq, rng, samples=40)
    # a whole correction step still runs on the context
    pg.pasm_step(ctx)
    with pytest.raises(pg.PasmError):
        pg.pasm_debug_waits(ctx, 0, -1)
