"""The tile autotuner: the shapes it picks are valid, and a context that uses
them computes the same correction steps as one with the default shapes.

Changing the number of columns a thread handles leaves every entry's own
arithmetic (its gather order and operations) unchanged; only the per-block
partial sums of the bordering dot products regroup, so in float64 eigenvalues
agree to 1e-13 and vectors to 1e-11 (relative).  In mixed precision the tuner
may also replace a fused float32 multigrid kernel by its unfused pair, whose
float32 roundings differ; the float64-accuracy outer iteration absorbs that to
well below the float32 level (eigenvalues 1e-7, vectors 1e-5 after 3 steps).
"""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_tiles_match_default(pg, precision):
    H = mg.build_hierarchy(2, 256, 16)   # finest level 65,025 rows: tuned
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    res = []
    for tune in (1, 0):
        opts = pg.pasm_default_opts(precision=precision, autotune=tune)
        ctx = pg.pasm_setup(A, M, H.P, opts, torch.cuda.current_stream().cuda_stream)
        pg.pasm_init(ctx, 32, 1e-12)
        tiles = pg.pasm_tiles(ctx, len(H.levels) - 1)
        assert all(v in (-1, 0, 1, 2, 4, 8) for v in tiles.values())
        assert tiles["restrict_first"] >= 0
        assert all(v >= 0 for kk, v in tiles.items() if kk not in ("jacobi2_zero", "resid_restrict", "prolong_sweep"))
        if precision == 0:
            assert tiles["restrict_first"] == 0
        rows = pg.pasm_tile_rows(ctx, len(H.levels) - 1)
        assert all(v in (0, 1, 4) for v in rows.values())
        if tune and precision == 1:
            assert rows["jacobi"] in (1, 4) and rows["prolong"] in (1, 4)   # float32 row kernels: chosen
            assert rows["outer_rhs"] in (1, 4) and rows["update"] in (1, 4)  # double-float row kernels too
            assert rows["border"] == 0                                       # grid-stride: not chosen
        if precision == 0:
            assert all(v == 0 for v in rows.values())     # float64 row kernels walk one row block
        if not tune:
            assert all(v == 0 for v in tiles.values())
            assert all(v == 0 for v in rows.values())
        assert all(v == 0 for v in pg.pasm_tiles(ctx, 1).values())   # 31 x 31: below the tuning size
        assert all(v == 0 for v in pg.pasm_tile_rows(ctx, 1).values())
        for _ in range(3):
            pg.pasm_step(ctx)
        n = H.fine.n
        lam = np.zeros(32)
        U = np.zeros((n, 32))
        pg.pasm_get(ctx, lam, U)
        res.append((lam, U))
    (l1, U1), (l0, U0) = res
    tl, tu = (1e-13, 1e-11) if precision == 0 else (1e-7, 1e-5)
    assert np.max(np.abs(l1 - l0) / l0) < tl
    assert np.max(np.abs(U1 - U0)) / np.max(np.abs(U0)) < tu


def test_saved_tiles_reproduce_the_tuned_run(pg):
    """A tuning cache: the shapes pasm_tiles / pasm_tile_rows report, set with
    pasm_set_tiles on an untuned context of the same hierarchy, read back the
    same and run the same kernels, so three steps agree bit for bit; values
    outside the documented sets are rejected."""
    H = mg.build_hierarchy(2, 256, 16)
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    runs = []
    for tune in (1, 0):
        opts = pg.pasm_default_opts(precision=1, autotune=tune)
        ctx = pg.pasm_setup(A, M, H.P, opts, torch.cuda.current_stream().cuda_stream)
        if not tune:
            for lv, (ch, rw) in saved.items():
                pg.pasm_set_tiles(ctx, lv, ch, rw)
        pg.pasm_init(ctx, 32, 1e-12)
        shapes = {lv: (pg.pasm_tiles(ctx, lv), pg.pasm_tile_rows(ctx, lv)) for lv in range(len(H.levels))}
        if tune:
            saved = shapes
        else:
            assert shapes == saved
        for _ in range(3):
            pg.pasm_step(ctx)
        lam = np.zeros(32)
        U = np.zeros((H.fine.n, 32))
        pg.pasm_get(ctx, lam, U)
        runs.append((lam, U))
        if not tune:
            bad = dict(saved[len(H.levels) - 1][0])
            bad["jacobi"] = 3
            with pytest.raises(RuntimeError):
                pg.pasm_set_tiles(ctx, len(H.levels) - 1, bad)
            bad = dict(saved[len(H.levels) - 1][0])
            bad["border"] = -1
            with pytest.raises(RuntimeError):
                pg.pasm_set_tiles(ctx, len(H.levels) - 1, bad)
            with pytest.raises(RuntimeError):
                pg.pasm_set_tiles(ctx, len(H.levels) - 1, saved[len(H.levels) - 1][0], {"jacobi": 2})
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("form", ["fused", "split", "restrict_first"])
def test_coarse_residual_forms_match_the_oracle_cycle(pg, form):
    """The three forms of the float32 coarse residual -- R (f - A e) with the
    fine residual recomputed per coarse row, the residual then the
    restriction, and R f - (R A) e with R A formed at setup -- set on every
    level through pasm_set_tiles, each give the oracle's two V-cycles of
    Algorithm 1 step 1 to float32 accuracy."""
    import oracle
    from oracle import pasm as op
    H = mg.build_hierarchy(2, 64, 8)
    opts = pg.pasm_default_opts(precision=1, autotune=0)
    ctx = pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P, opts,
                        torch.cuda.current_stream().cuda_stream)
    for lv in range(1, len(H.levels)):
        ch = {"resid_restrict": -1 if form == "split" else 0,
              "restrict_first": 2 if form == "restrict_first" else 0}
        rows = {"restrict_first": 4} if form == "restrict_first" else {}
        pg.pasm_set_tiles(ctx, lv, ch, rows)
    prob = oracle.Problem.from_hierarchy(H)
    k = 6
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    Uh = np.zeros_like(U)
    pg.pasm_bvp(ctx, lam, U, Uh)
    Uo = op.bvp_solve(prob, lam, U)
    err = max(np.abs(Uh[:, j] - Uo[:, j]).max() / np.abs(Uo[:, j]).max() for j in range(k))
    assert err < 1e-5, err
    # float64 contexts have no R A: the form is refused there
    ctx64 = pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P,
                          pg.pasm_default_opts(precision=0, autotune=0), torch.cuda.current_stream().cuda_stream)
    with pytest.raises(RuntimeError):
        pg.pasm_set_tiles(ctx64, len(H.levels) - 1, {"restrict_first": 2})
