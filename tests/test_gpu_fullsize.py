"""GPU parity at the benchmark's full size (unit square, h = 1/1024,
1,046,529 DoF, H = 1/16, k = 64) and on the 3D Kuhn mesh, against values the
oracle wrote (tests/golden, make_golden.py) and the ARPACK reference
eigenvalues."""
import json
import os

import numpy as np
import pytest

import gpu_accuracy as ga
import meshgen as mg
import oracle
from paper_1908_10251_gb300 import accuracy as acc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def pg():
    from paper_1908_10251_gb300 import build
    build.build()
    import paper_1908_10251_gb300 as pkg
    pkg.load_library()
    return pkg


@pytest.fixture(scope="module")
def square1024():
    return mg.build_hierarchy(2, 1024, 16)


def setup_ctx(pg, H, **opts):
    return pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P, pg.pasm_default_opts(**opts),
                         torch.cuda.current_stream().cuda_stream)


def test_fullsize_fp64_steps_match_oracle_history(pg, square1024):
    """Eight float64 correction steps, all 64 pairs, against the oracle's own
    iterates at the same size (1e-10 relative).  Both sides start from the
    oracle's coarse initial pairs.  The pairs that do not converge (the coarse
    space is too coarse for them) iterate chaotically: in the oracle itself a
    1e-15 relative perturbation of pair 10's start grows to 5e-11 by step 7
    and 2.6e-8 by step 8.  So steps 1-5 are compared for all 64 pairs and
    steps 6-8 for the pairs the oracle drives to 1e-9."""
    with open(os.path.join(GOLDEN, "square_h1024_H16_k64_history.json")) as f:
        hist = np.array(json.load(f)["history"])
    prob = oracle.Problem.from_hierarchy(square1024)
    k = 64
    lam0, U0 = oracle.initial_state(prob, k)
    ctx = setup_ctx(pg, square1024, precision=0)
    # the library's own coarse start agrees with the oracle's up to sign
    pg.pasm_init(ctx, k, 1e-10)
    lam = np.zeros(k)
    U = np.zeros_like(U0)
    pg.pasm_get(ctx, lam, U)
    assert np.allclose(lam, hist[0], rtol=1e-12)
    sgn = np.sign(np.einsum("ij,ij->j", U, U0))
    assert np.abs(U * sgn - U0).max() <= 1e-10 * np.abs(U0).max()
    ref = np.loadtxt(os.path.join(GOLDEN, "square_h1024_k72.txt"))[:64]
    stable = (np.abs(hist - ref) / ref <= 1e-9).any(axis=0)
    pg.pasm_init(ctx, k, 1e-10, lam0, U0)
    for step in range(1, 9):
        pg.pasm_step(ctx)
        pg.pasm_get(ctx, lam)
        rel = np.abs(lam - hist[step]) / hist[step]
        if step > 5:
            rel = rel[stable]
        assert rel.max() < 1e-10, (step, int(rel.argmax()), rel.max())
    pg.pasm_destroy(ctx)


def test_fullsize_nested_start_matches_oracle_history(pg, square1024):
    """The nested start (Algorithm 2 step 2(A): one correction step on each of
    the grids 1/32 .. 1/512 before the prolongation to h = 1/1024), float64,
    against the oracle's nested history at the same size: the start and four
    further steps agree to 1e-10 on the pairs the oracle drives to 1e-9; the
    other (chaotic) pairs are held only at the start, to 1e-8."""
    with open(os.path.join(GOLDEN, "square_h1024_H16_k64_nested_history.json")) as f:
        hist = np.array(json.load(f)["history"])
    k = 64
    ref = np.loadtxt(os.path.join(GOLDEN, "square_h1024_k72.txt"))[:64]
    stable = (np.abs(hist - ref) / ref <= 1e-9).any(axis=0)
    assert stable.sum() >= 10
    ctx = setup_ctx(pg, square1024, precision=0, init=pg.capi.PASM_INIT_NESTED)
    pg.pasm_init(ctx, k, 1e-10)
    lam = np.zeros(k)
    pg.pasm_get(ctx, lam)
    rel = np.abs(lam - hist[0]) / hist[0]
    assert rel.max() < 1e-8, (int(rel.argmax()), rel.max())
    assert rel[stable].max() < 1e-10
    for step in range(1, 5):
        pg.pasm_step(ctx)
        pg.pasm_get(ctx, lam)
        rel = (np.abs(lam - hist[step]) / hist[step])[stable]
        assert rel.max() < 1e-10, (step, rel.max())
    pg.pasm_destroy(ctx)


def cluster_err(lam, ref_all):
    """relative distance of each lam_i to the nearest reference eigenvalue of
    pair i's cluster (consecutive reference values closer than 1e-4 relative)"""
    cid = np.concatenate([[0], np.cumsum(np.diff(ref_all) / ref_all[1:] > 1e-4)])
    out = np.empty(len(lam))
    for i, v in enumerate(lam):
        mem = ref_all[cid == cid[i]]
        out[i] = np.min(np.abs(v - mem) / mem)
    return out


def test_fullsize_mixed_final_state_matches_reference(pg, square1024):
    """Mixed precision at full size, 40 correction steps, pairs frozen at
    |d lambda| / lambda < 1e-13 (the rounding floor; a looser threshold stops
    the vectors above the angle bound, none at all lets the fp32 noise rotate
    near-degenerate pairs away).  At the END every pair the float64 oracle
    converges and holds (its frozen
    run reaches 1e-9 of the ARPACK eigenvalues of the pair's own cluster; its
    run without freezing still holds it after 40 steps) is within 1e-9 of a
    reference eigenvalue of its cluster, no cluster holds a duplicate (pairs
    15/16 are split by 1.7e-11, 20/21 by 3.2e-9: only the joint eigenspace is
    defined), and each cluster's largest M-principal angle to the reference
    eigenspace is at most 1e-6; no eigenvalue drops below the first reference
    eigenvalue (Ritz values are upper bounds)."""
    ref_all = ga.golden_table("square_h1024_k72")
    pset = ga.stable_set(ref_all, "square_h1024_H16_k64_history", "square_h1024_H16_k64_nofreeze_history")
    assert len(pset) >= 10
    vecs = ga.reference_vectors(square1024, 2, 1024, ref_all, int(pset.max()))
    ctx = setup_ctx(pg, square1024, precision=1)
    k = 64
    pg.pasm_init(ctx, k, 1e-13)
    lam = np.zeros(k)
    for _ in range(40):
        pg.pasm_step(ctx)
        pg.pasm_get(ctx, lam)
        assert lam.min() >= ref_all[0] * (1 - 1e-11)   # Ritz upper bound, up to rounding
    U = np.zeros((square1024.fine.n, k))
    pg.pasm_get(ctx, lam, U)
    pg.pasm_destroy(ctx)
    ga.check_final(square1024.fine.M, lam, U, ref_all, vecs, pset)


def test_fullsize_3d_fp64_steps_match_oracle_history(pg):
    """The 3D workload at full size (Kuhn P1, h = 1/128, 2,048,383 DoF, H = 1/8,
    k = 32), float64: six correction steps from the oracle's coarse initial
    pairs against the oracle's own iterates (1e-10 relative) -- all 32 pairs
    for the first three steps, afterwards the pairs the oracle drives to 1e-9
    of the LOBPCG reference (of their own cluster), since the others iterate
    chaotically as in 2D."""
    with open(os.path.join(GOLDEN, "cube_h128_H8_k32_history.json")) as f:
        hist = np.array(json.load(f)["history"])
    ref_all = np.loadtxt(os.path.join(GOLDEN, "cube_h128_k40.txt"))
    stable = np.array([cluster_err(row, ref_all) for row in hist]).min(axis=0) <= 1e-9
    assert stable.sum() >= 4
    H = mg.build_hierarchy(3, 128, 8)
    prob = oracle.Problem.from_hierarchy(H)
    k = 32
    lam0, U0 = oracle.initial_state(prob, k)
    assert np.allclose(lam0, hist[0], rtol=1e-12)
    ctx = setup_ctx(pg, H, precision=0)
    pg.pasm_init(ctx, k, 1e-10, lam0, U0)
    lam = np.zeros(k)
    for step in range(1, 7):
        pg.pasm_step(ctx)
        pg.pasm_get(ctx, lam)
        rel = np.abs(lam - hist[step]) / hist[step]
        if step > 3:
            rel = rel[stable]
        assert rel.max() < 1e-10, (step, int(rel.argmax()), rel.max())
    pg.pasm_destroy(ctx)


def test_fullsize_3d_mixed_final_state_matches_reference(pg):
    """The 3D workload at full size: Kuhn P1 on the unit cube, h = 1/128
    (2,048,383 DoF), H = 1/8 (343), k = 32, mixed precision, 30 steps, pairs
    frozen at |d lambda| / lambda < 1e-13.  At the end every pair the float64
    oracle converges and holds (among them the simple first eigenvalue and the near-triple second,
    pi^2 (1 + 1 + 4) at the continuum level) is within 1e-9 of its cluster's
    reference eigenvalues (LOBPCG table), distinct, and within an M-principal
    angle of 1e-6 of the reference eigenspace (ARPACK shift-invert with the
    exact sine-transform inverse of the Kuhn stiffness); no pair ever drops
    below the smallest reference eigenvalue."""
    ref_all = ga.golden_table("cube_h128_k40")
    pset = ga.stable_set(ref_all, "cube_h128_H8_k32_history", "cube_h128_H8_k32_nofreeze_history")
    assert len(pset) >= 4 and np.all(pset[:4] == np.arange(4))
    H = mg.build_hierarchy(3, 128, 8)
    vecs = ga.reference_vectors(H, 3, 128, ref_all, int(pset.max()))
    ctx = setup_ctx(pg, H, precision=1)
    k = 32
    pg.pasm_init(ctx, k, 1e-13)
    lam = np.zeros(k)
    for _ in range(30):
        pg.pasm_step(ctx)
        pg.pasm_get(ctx, lam)
        assert lam.min() >= ref_all[0] * (1 - 1e-11)   # Ritz upper bound, up to rounding
    U = np.zeros((H.fine.n, k))
    pg.pasm_get(ctx, lam, U)
    pg.pasm_destroy(ctx)
    ga.check_final(H.fine.M, lam, U, ref_all, vecs, pset)


@pytest.mark.parametrize("precision", [0, 1])
def test_kuhn_3d_degenerate_coarse_pairs(pg, precision):
    """3D Kuhn mesh, h = 1/16, H = 1/4: the coarse pencil has exactly
    degenerate eigenvalues (axis-permutation symmetry).  Step parity with the
    oracle for 6 pairs (float64) / convergence of the first pairs to the
    oracle's converged values (mixed)."""
    H = mg.build_hierarchy(3, 16, 4)
    prob = oracle.Problem.from_hierarchy(H)
    lamH, _ = oracle.coarse_eigenpairs(prob)
    assert np.min(np.diff(lamH[:8]) / lamH[1:8]) < 1e-12      # a degenerate pair among the first
    ctx = setup_ctx(pg, H, precision=precision)
    k = 6
    lam, U = oracle.initial_state(prob, k)
    pg.pasm_init(ctx, k, 0.0, lam, U)
    if precision == 0:
        for step in range(4):
            lam, U, _ = oracle.correction(prob, lam, U)
            pg.pasm_step(ctx)
            lg = np.zeros(k)
            pg.pasm_get(ctx, lg)
            assert np.allclose(lg, lam, rtol=1e-10), (step, lg / lam - 1)
    else:
        lo, _, _, _ = oracle.solve(prob, k, tol=1e-13, max_steps=60, lam0=lam, U0=U)
        lg = np.zeros(k)
        for _ in range(60):
            pg.pasm_step(ctx)
        pg.pasm_get(ctx, lg)
        assert np.allclose(lg[:2], lo[:2], rtol=1e-9)
    pg.pasm_destroy(ctx)


@pytest.fixture(scope="module")
def square2048():
    return mg.build_hierarchy(2, 2048, 16)


def test_h2048_k128_fp64_step_sampled_oracle_parity(pg, square2048):
    """The largest 2D workload (h = 1/2048, 4,190,209 DoF, H = 1/16, 8 grids,
    k = 128) in the launch configuration of the solver: one float64 correction
    step for all 128 pairs from the oracle's coarse start; sampled pairs (the
    first, two middle and the last) match the oracle's correction of the same
    columns (pairs are independent, Section 3.2) to 1e-10 in the eigenvalue and
    1e-8 (relative) in the vector; the first eigenvalue does not increase
    (the augmented space contains the coarse space and u_1)."""
    H = square2048
    k = 128
    prob = oracle.Problem.from_hierarchy(H)
    lam0, U0 = oracle.initial_state(prob, k)
    ctx = setup_ctx(pg, H, precision=0)
    pg.pasm_init(ctx, k, 0.0, lam0, U0)
    pg.pasm_step(ctx)
    lam = np.zeros(k)
    U = np.zeros_like(U0)
    pg.pasm_get(ctx, lam, U)
    pg.pasm_destroy(ctx)
    assert np.all(np.isfinite(lam)) and lam[0] <= lam0[0] * (1 + 1e-14)
    cols = [0, 1, 63, 64, 127]
    lo, Uo, _ = oracle.correction(prob, lam0[cols], U0[:, cols])
    assert np.allclose(lam[cols], lo, rtol=1e-10), np.abs(lam[cols] / lo - 1).max()
    for q, j in enumerate(cols):
        assert np.abs(U[:, j] - Uo[:, q]).max() / np.abs(Uo[:, q]).max() < 1e-8, j


def test_h2048_k128_mixed_final_state(pg, square2048):
    """Mixed precision on the h = 1/2048, k = 128 workload, 40 steps, pairs
    frozen at |d lambda| / lambda < 1e-13: no eigenvalue ever drops below the
    smallest reference eigenvalue (Ritz values are upper bounds); at the end
    the simple first eigenvalue and the (1,2)/(2,1) cluster are within 1e-9 of
    the reference table (the 136 smallest eigenvalues: ARPACK shift-invert with
    the exact sine-transform inverse, agreeing with an independent LOBPCG
    table of 48 values to 1.4e-14), as are at least ten of the 128 pairs, and
    every pair of 0..41 that the float64 oracle converges and holds (stored
    histories of its runs with and without freezing) is within 1e-9, distinct
    in its cluster and within an M-principal angle of 1e-6 of the reference
    eigenspace."""
    ref_all = ga.golden_table("square_h2048_k136")
    H = square2048
    k = 128
    ctx = setup_ctx(pg, H, precision=1)
    pg.pasm_init(ctx, k, 1e-13)
    lam = np.zeros(k)
    for _ in range(40):
        pg.pasm_step(ctx)
        pg.pasm_get(ctx, lam)
        assert lam.min() >= ref_all[0] * (1 - 1e-11)   # Ritz upper bound, up to rounding
    U = np.zeros((H.fine.n, k))
    pg.pasm_get(ctx, lam, U)
    pg.pasm_destroy(ctx)
    err = acc.cluster_errors(lam, ref_all)
    within = np.where(err <= 1e-9)[0]
    assert np.all(err[:3] <= 1e-9), err[:3]
    assert len(within) >= 10, err
    # the vector check: the pairs among 0..41 that the float64 oracle converges and holds (its
    # frozen run reaches 1e-9 of their cluster; its run without freezing still holds it after 40
    # steps) -- a pair the oracle only passes on its way (an unstable fixed point of the correction)
    # keeps or leaves its eigenvector depending on where a freeze catches it
    pset = ga.stable_set(ref_all, "square_h2048_H16_k42_history", "square_h2048_H16_k42_nofreeze_history")
    assert len(pset) >= 8 and np.all(pset[:3] == np.arange(3))
    vecs = ga.reference_vectors(H, 2, 2048, ref_all, int(pset.max()))
    ga.check_final(H.fine.M, lam, U, ref_all, vecs, [int(i) for i in pset])
