"""Pins of the learned-smoother oracle (oracle/smoother.py): gradients against
central finite differences and against torch autograd over an independent
forward written with torch's conv2d, the homogeneity the odd bias-free
construction guarantees, and Adam against torch.optim.Adam."""
import numpy as np
import pytest

import meshgen as mg
from oracle import smoother as sm

torch = pytest.importorskip("torch")


def small_case(seed=0, N=8, k=2):
    A, M = mg.assemble(2, N)
    nx = ny = N - 1
    rng = np.random.default_rng(seed)
    R = rng.standard_normal((nx * ny, k))
    w = sm.init_weights(seed) * 3.0
    return A, R, w, nx, ny


def torch_forward(w, R, nx, ny):
    """N(r) with torch.nn.functional.conv2d (cross-correlation, NCHW)."""
    W1, W2, W3 = sm.unpack(w)
    def tw(W):  # [3][3][cin][cout] -> [cout][cin][3][3]
        return torch.tensor(np.transpose(W, (3, 2, 0, 1)))
    x = torch.tensor(np.asarray(R).T.reshape(-1, 1, ny, nx))
    F = torch.nn.functional
    def branch(z):
        a = F.relu(F.conv2d(z, tw(W1), padding=1))
        a = F.relu(F.conv2d(a, tw(W2), padding=1))
        return F.conv2d(a, tw(W3), padding=1)
    return 0.5 * (branch(x) - branch(-x))


def test_forward_matches_torch_conv2d():
    A, R, w, nx, ny = small_case()
    ours = sm.apply(w, sm.to_grid(R, nx, ny))
    ref = torch_forward(w, R, nx, ny).numpy()[:, 0]
    assert np.allclose(ours, ref, rtol=1e-12, atol=1e-12)


def test_gradient_matches_torch_autograd():
    A, R, w, nx, ny = small_case(1)
    L, g = sm.loss_and_grad(w, A, R, nx, ny)
    wt = torch.tensor(w, requires_grad=True)
    W1 = wt[:144].reshape(3, 3, 1, 16); W2 = wt[144:2448].reshape(3, 3, 16, 16); W3 = wt[2448:].reshape(3, 3, 16, 1)
    F = torch.nn.functional
    x = torch.tensor(R.T.reshape(-1, 1, ny, nx))
    def tw(W):
        return W.permute(3, 2, 0, 1)
    def branch(z):
        a = F.relu(F.conv2d(z, tw(W1), padding=1))
        a = F.relu(F.conv2d(a, tw(W2), padding=1))
        return F.conv2d(a, tw(W3), padding=1)
    D = (0.5 * (branch(x) - branch(-x))).reshape(R.shape[1], -1).T
    At = torch.tensor(A.toarray())
    Rt = torch.tensor(R)
    E = Rt - At @ D
    Lt = torch.mean((E * E).sum(0) / (Rt * Rt).sum(0))
    Lt.backward()
    assert L == pytest.approx(Lt.item(), rel=1e-12)
    assert np.allclose(g, wt.grad.numpy(), rtol=1e-9, atol=1e-12 * np.abs(g).max())


def test_gradient_matches_finite_differences():
    A, R, w, nx, ny = small_case(2)
    L, g = sm.loss_and_grad(w, A, R, nx, ny)
    rng = np.random.default_rng(3)
    for idx in rng.choice(len(w), 12, replace=False):
        h = 1e-6 * max(1.0, abs(w[idx]))
        wp, wm = w.copy(), w.copy()
        wp[idx] += h; wm[idx] -= h
        fd = (sm.loss_and_grad(wp, A, R, nx, ny)[0] - sm.loss_and_grad(wm, A, R, nx, ny)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=2e-5, abs=1e-9)


def test_odd_and_homogeneous():
    """N(s r) = s N(r) for every real s (bias-free ReLU net, odd part)."""
    A, R, w, nx, ny = small_case(4)
    r = sm.to_grid(R, nx, ny)
    base = sm.apply(w, r)
    for s in (2.5, -1.3, 1e-3):
        assert np.allclose(sm.apply(w, s * r), s * base, rtol=1e-12, atol=1e-15)


def test_adam_matches_torch():
    rng = np.random.default_rng(5)
    w = rng.standard_normal(50)
    m = np.zeros(50); v = np.zeros(50)
    wt = torch.tensor(w.copy(), requires_grad=True)
    opt = torch.optim.Adam([wt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 4):
        g = rng.standard_normal(50)
        w, m, v = sm.adam_step(w, g, m, v, t, lr=1e-2)
        opt.zero_grad(); wt.grad = torch.tensor(g); opt.step()
    assert np.allclose(w, wt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_zero_network_learned_sweep_is_jacobi_or_identity():
    """With all-zero weights N(r) = 0: x + N(r) = x keeps the residual, so every
    pair is accepted and the learned sweep leaves x unchanged."""
    import oracle
    from oracle import pasm as op
    H = mg.build_hierarchy(2, 16, 4)
    prob = oracle.Problem.from_hierarchy(H, nn_weights=np.zeros(sm.N_WEIGHTS),
                                         grids=[lv.N - 1 for lv in H.levels])
    rng = np.random.default_rng(0)
    f = rng.standard_normal((H.fine.n, 2)); x = rng.standard_normal((H.fine.n, 2))
    assert np.array_equal(op.learned_sweep(prob, prob.L, f, x), x)


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(9).standard_normal(1000) * 10.0 ** np.random.default_rng(10).integers(-5, 5, 1000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(sm.bf16(x), ref)


def torch_forward_bf16(w, R, nx, ny):
    """N(r) with the second convolution taking bfloat16 operands: torch rounds
    relu(+-z1) and W2 (via float32, round to nearest even), conv2d multiplies
    the rounded values exactly in float64; layers 1 and 3 stay float64."""
    W1, W2, W3 = sm.unpack(w)
    F = torch.nn.functional

    def tw(W):
        return torch.tensor(np.transpose(W, (3, 2, 0, 1)))

    def rb(t):
        return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)

    x = torch.tensor(np.asarray(R).T.reshape(-1, 1, ny, nx))
    z1 = F.conv2d(x, tw(W1), padding=1)
    W2b = rb(tw(W2))
    z2p = F.conv2d(rb(F.relu(z1)), W2b, padding=1)
    z2m = F.conv2d(rb(F.relu(-z1)), W2b, padding=1)
    h = 0.5 * (F.relu(z2p) - F.relu(z2m))
    return F.conv2d(h, tw(W3), padding=1)


def test_bf16_layer2_branch_matches_torch():
    """The tensor-core form of the network (layer 2 on bfloat16 operands,
    products exact and summed in high precision) against torch's rounding and
    conv2d of the same operands."""
    A, R, w, nx, ny = small_case(3, N=12, k=3)
    ours = sm.apply(w, sm.to_grid(R, nx, ny), bf16_layer2=True)
    ref = torch_forward_bf16(w, R, nx, ny).numpy()[:, 0]
    assert np.allclose(ours, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # the rounding is really applied: the plain network differs
    plain = sm.apply(w, sm.to_grid(R, nx, ny))
    assert np.abs(plain - ours).max() > 1e-6 * np.abs(plain).max()


def test_bf16_layer2_exact_when_operands_representable():
    """With weights and inputs on a coarse dyadic grid every operand of layer 2
    is already a bfloat16 number (small integers times powers of two), so the
    rounding is the identity and the bf16 form equals the float64 network
    exactly; odd symmetry N(-r) = -N(r) holds in both forms."""
    rng = np.random.default_rng(4)
    ws = [rng.integers(-3, 4, size=s).astype(np.float64) * 0.25 for s in sm.SHAPES]
    w = sm.pack(ws)
    nx = ny = 9
    r = rng.integers(-4, 5, size=(2, ny, nx)).astype(np.float64)
    a = sm.apply(w, r, bf16_layer2=True)
    b = sm.apply(w, r)
    assert np.array_equal(a, b)
    assert np.array_equal(sm.apply(w, -r, bf16_layer2=True), -a)


def test_bf16_gradient_equals_plain_where_rounding_is_exact():
    """With weights and inputs on a coarse dyadic grid the forward rounding is
    the identity: the bf16 form has the same loss and the same layer-3
    gradient (summed in another order: to 1e-12) as the float64 form; the
    layer-2 and layer-1 gradients differ, since the output gradients dL/dz2
    are not dyadic (the loss divides by |r|^2) and are rounded."""
    rng = np.random.default_rng(5)
    ws = [rng.integers(-3, 4, size=s).astype(np.float64) * 0.25 for s in sm.SHAPES]
    w = sm.pack(ws)
    A, M = mg.assemble(2, 10)
    nx = ny = 9
    R = rng.integers(-4, 5, size=(nx * ny, 2)).astype(np.float64)
    L1, g1 = sm.loss_and_grad(w, A, R, nx, ny)
    L2, g2 = sm.loss_and_grad_bf16(w, A, R, nx, ny)
    assert L1 == L2
    assert np.allclose(g1[2448:], g2[2448:], rtol=1e-12, atol=0)
    assert not np.allclose(g1[:2448], g2[:2448], rtol=1e-6, atol=0)


def test_bf16_gradient_within_first_order_bound():
    """|g_bf16 - g| <= the first-order bf16 bound of oracle.smoother
    (8 u G_abs, see bf16_gradient_bound), and the rounding does act."""
    A, R, w, nx, ny = small_case(6, N=10, k=3)
    _, g = sm.loss_and_grad(w, A, R, nx, ny)
    _, gb = sm.loss_and_grad_bf16(w, A, R, nx, ny)
    assert np.all(np.abs(gb - g) <= sm.bf16_gradient_bound(w, A, R, nx, ny))
    assert np.abs(gb - g).max() > 0


def _f32_fma(a, b, c):
    """float32 a*b + c with the product exact (float64) and one rounding of
    the sum to float32 through float64 (double rounding: within half a float64
    ulp of one float32 rounding)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def _bf16_trunc(x):
    """bfloat16 by truncation (a wrong rounding, for the planted-mistake check)."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32) & np.uint32(0xFFFF0000)
    return b.view(np.float32).astype(np.float64)


def float32_forward(w, r_grid, round_a=sm.bf16):
    """An independent float32 evaluation of N(r) in the order the fused
    tensor-core kernel uses: layer 1 as 9 FMAs per channel (taps row-major),
    relu(+-z1) of the float32 z1 rounded to bfloat16, layer 2 as float32 sums
    of the exact bfloat16 products, h in float32, layer 3 as 144 FMAs."""
    W1, W2, W3 = (np.asarray(x, np.float32) for x in sm.unpack(w))
    x = np.asarray(r_grid, np.float32)
    B, ny, nx = x.shape

    def pad(v):
        out = np.zeros((B, ny + 2, nx + 2) + v.shape[3:], np.float32)
        out[:, 1:-1, 1:-1] = v
        return out

    xp = pad(x)
    z1 = np.zeros((B, ny, nx, 16), np.float32)
    for tap in range(9):
        dy, dx = divmod(tap, 3)
        v = xp[:, dy:dy + ny, dx:dx + nx][..., None]
        z1 = _f32_fma(W1[dy, dx, 0][None, None, None, :], v, z1)
    W2b = sm.bf16(W2).astype(np.float32)
    z2 = []
    for s in (1.0, -1.0):
        a = pad(round_a(np.maximum(s * z1, 0.0)).astype(np.float32))
        acc = np.zeros((B, ny, nx, 16), np.float32)
        for tap in range(9):
            dy, dx = divmod(tap, 3)
            for ci in range(16):
                acc = acc + a[:, dy:dy + ny, dx:dx + nx, ci:ci + 1] * W2b[dy, dx, ci][None, None, None, :]
        z2.append(acc)
    h = np.float32(0.5) * (np.maximum(z2[0], np.float32(0)) - np.maximum(z2[1], np.float32(0)))
    hp = pad(h)
    d = np.zeros((B, ny, nx), np.float32)
    for tap in range(9):
        dy, dx = divmod(tap, 3)
        for c in range(16):
            d = _f32_fma(W3[dy, dx, c, 0], hp[:, dy:dy + ny, dx:dx + nx, c], d)
    return d.astype(np.float64)


def _bound_case(seed, scale=2.0, n=23, B=4):
    w = sm.init_weights(seed).astype(np.float32).astype(np.float64) * scale
    r = np.random.default_rng(seed + 10).standard_normal((B, n, n)).astype(np.float32).astype(np.float64)
    return w, r


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bf16_forward_bound_holds_for_a_float32_evaluation(seed):
    """The derived elementwise bound covers an independent float32 evaluation
    in the kernel's order, including outputs where the float32 z1 and the
    float64 z1 round relu(+-z1) to different bfloat16 neighbours."""
    w, r = _bound_case(seed)
    ref = sm.apply(w, r, bf16_layer2=True)
    got = float32_forward(w, r)
    bound = sm.bf16_forward_bound(w, r)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


def test_bf16_forward_bound_is_below_a_bfloat16_step():
    """Only the operands whose rounding boundary lies within the float32 error
    of z1 (about 1e-4 of them) contribute a bfloat16 step; elsewhere the bound
    is the worst-case float32 accumulation error, so the median output's bound
    stays below a quarter of a bfloat16 step of the largest output."""
    w, r = _bound_case(0)
    ref = sm.apply(w, r, bf16_layer2=True)
    bound = sm.bf16_forward_bound(w, r)
    assert np.median(bound) < 0.25 * 2.0 ** -8 * np.abs(ref).max()


def test_bf16_forward_bound_catches_a_wrong_rounding():
    """Planted mistake: relu(+-z1) truncated to bfloat16 instead of rounded to
    nearest; most outputs leave the bound."""
    w, r = _bound_case(0)
    ref = sm.apply(w, r, bf16_layer2=True)
    bad = float32_forward(w, r, round_a=_bf16_trunc)
    bound = sm.bf16_forward_bound(w, r)
    assert np.mean(np.abs(bad - ref) > bound) > 0.5
