"""GPU check of pasm_border_noalloc, the bordering entry point for callers
that cannot allocate device memory (a host that pre-reserves the device heap,
a latency-critical loop, memory owned by another allocator).  It must agree
with the bordering the regular context path computes (pasm_augmented's beta
and zeta) to the 1e-12 relative tolerance the other bordering tests use, on
two calls in a row -- the second one reusing the library's fixed scratch
array that the first call left behind.  Collected last on purpose."""
import numpy as np
import pytest

import meshgen as mg
import oracle
from oracle import pasm as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_border_noalloc_matches_context_path():
    from paper_1908_10251_gb300 import build
    build.build()
    import paper_1908_10251_gb300 as pg
    pg.load_library()
    H = mg.build_hierarchy(2, 64, 8)
    prob = oracle.Problem.from_hierarchy(H)
    k = 8
    stream = torch.cuda.current_stream()
    ctx = pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P, pg.pasm_default_opts(),
                        stream.cuda_stream)
    A, M = H.fine.A, H.fine.M
    n = A.shape[0]
    dev = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    Arp, Aci, Aval = dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64)
    Mrp, Mci, Mval = dev(M.indptr, torch.int32), dev(M.indices, torch.int32), dev(M.data, torch.float64)
    lam, U = oracle.initial_state(prob, k)
    inputs = [op.bvp_solve(prob, lam, U)]
    lam2, U2, _ = oracle.correction(prob, lam, U)
    inputs.append(op.bvp_solve(prob, lam2, U2))
    pg.pasm_init(ctx, k, 0.0, lam, U)
    for Ut in inputs:
        # the regular path: bordering inside pasm_augmented (context-owned scratch)
        beta_ref = np.zeros(k); zeta_ref = np.zeros(k)
        pg.pasm_augmented(ctx, lam, Ut, None, None, beta_ref, zeta_ref)
        # the allocation-free path
        X = dev(Ut, torch.float64)
        YA = torch.empty_like(X); YM = torch.empty_like(X)
        beta = torch.empty(k, dtype=torch.float64, device="cuda")
        zeta = torch.empty(k, dtype=torch.float64, device="cuda")
        pg.pasm_border_noalloc(n, Arp, Aci, Aval, Mrp, Mci, Mval, k, X, YA, YM, beta, zeta, stream.cuda_stream)
        torch.cuda.synchronize()
        assert np.allclose(beta.cpu().numpy(), beta_ref, rtol=1e-12, atol=0)
        assert np.allclose(zeta.cpu().numpy(), zeta_ref, rtol=1e-12, atol=0)
        assert np.allclose(YA.cpu().numpy(), A @ Ut, rtol=1e-12, atol=1e-14 * np.abs(A @ Ut).max())
        assert np.allclose(YM.cpu().numpy(), M @ Ut, rtol=1e-12, atol=1e-14 * np.abs(M @ Ut).max())
    pg.pasm_destroy(ctx)


def test_border_noalloc_rejects_bad_sizes():
    import paper_1908_10251_gb300 as pg
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    zi = torch.zeros(16, dtype=torch.int32, device="cuda")
    for kk in (3, 6, 512):
        with pytest.raises(pg.PasmError) as ei:
            pg.pasm_border_noalloc(2, zi, zi, z, zi, zi, z, kk, z, z, z, z, z)
        assert ei.value.code == 1


def test_border_noalloc_widest_block_capped_grid():
    """The widest block the entry point accepts (k = 256) on the h = 1/1024
    square (1,046,529 rows): the grid is capped by the fixed scratch (304
    blocks of 8 rows for 130,817 row groups), so every block walks many rows.
    Against scipy's A X, M X and float64 column dot products on the host, and
    against the bordering of the context path (pasm_augmented, H = 1/32 so
    that k <= N_H), on two calls in a row; a warm call changes the device's
    free memory by nothing."""
    from paper_1908_10251_gb300 import build
    build.build()
    import paper_1908_10251_gb300 as pg
    pg.load_library()
    H = mg.build_hierarchy(2, 1024, 32)
    A, M = H.fine.A, H.fine.M
    n, k = A.shape[0], 256
    stream = torch.cuda.current_stream()
    dev = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    Arp, Aci, Aval = dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64)
    Mrp, Mci, Mval = dev(M.indptr, torch.int32), dev(M.indices, torch.int32), dev(M.data, torch.float64)
    YA = torch.empty((n, k), dtype=torch.float64, device="cuda")
    YM = torch.empty_like(YA)
    beta = torch.empty(k, dtype=torch.float64, device="cuda")
    zeta = torch.empty(k, dtype=torch.float64, device="cuda")
    ctx = pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P, pg.pasm_default_opts(),
                        stream.cuda_stream)
    lam = np.linspace(20.0, 2000.0, k)
    pg.pasm_init(ctx, k, 0.0)
    for seed in (11, 12):
        Xh = np.random.default_rng(seed).standard_normal((n, k))
        X = dev(Xh, torch.float64)
        args = (n, Arp, Aci, Aval, Mrp, Mci, Mval, k, X, YA, YM, beta, zeta, stream.cuda_stream)
        pg.pasm_border_noalloc(*args)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        pg.pasm_border_noalloc(*args)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        ya_ref, ym_ref = A @ Xh, M @ Xh
        ya, ym = YA.cpu().numpy(), YM.cpu().numpy()
        assert np.abs(ya - ya_ref).max() <= 1e-13 * np.abs(ya_ref).max()
        assert np.abs(ym - ym_ref).max() <= 1e-13 * np.abs(ym_ref).max()
        del ya, ym
        b_ref = np.einsum("ij,ij->j", Xh, ya_ref)
        z_ref = np.einsum("ij,ij->j", Xh, ym_ref)
        assert np.allclose(beta.cpu().numpy(), b_ref, rtol=1e-12, atol=0)
        assert np.allclose(zeta.cpu().numpy(), z_ref, rtol=1e-12, atol=0)
        beta_ctx = np.zeros(k); zeta_ctx = np.zeros(k)
        pg.pasm_augmented(ctx, lam, Xh, None, None, beta_ctx, zeta_ctx)
        assert np.allclose(beta.cpu().numpy(), beta_ctx, rtol=1e-12, atol=0)
        assert np.allclose(zeta.cpu().numpy(), zeta_ctx, rtol=1e-12, atol=0)
        del Xh, X, ya_ref, ym_ref
    pg.pasm_destroy(ctx)
