"""Oracle of the learned multigrid post-smoother (test infrastructure only).

Not in the paper: the workload specification asks for a small convolutional
smoother standing in for damped Jacobi inside the V-cycles of Algorithm 1
step 1.  Reading (listed in the design notes): three bias-free 3x3
convolutions 1 -> 16 -> 16 -> 1 with ReLU after the first two, made odd,
    N(r) = (Nt(r) - Nt(-r)) / 2,
so that N(s r) = s N(r) for every real s (a bias-free ReLU net is positively
homogeneous; the odd part extends that to negative s) -- no normalisation of r
is needed.  It acts on the grid view of one level: the interior nodes of an
nx x ny grid (x fastest), zero outside (Dirichlet).  Training minimises the
residual left after the correction,
    L = mean_pairs |r - A N(r)|^2 / |r|^2,
over residuals r that the method's own V-cycles produce before
post-smoothing.  Float64 numpy, written directly from these definitions;
gradients by hand (chain rule), pinned against finite differences and
torch autograd in the tests.

Weight layout (float): W1[3][3][1][16], W2[3][3][16][16], W3[3][3][16][1],
concatenated in that order (144 + 2304 + 144 = 2592 values); index
[dy+1][dx+1][cin][cout] multiplies input pixel (y+dy, x+dx).
"""
from __future__ import annotations

import numpy as np

C = 16
SHAPES = ((3, 3, 1, C), (3, 3, C, C), (3, 3, C, 1))
N_WEIGHTS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(w[o:o + n].reshape(s))
        o += n
    return out


def pack(ws):
    return np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in ws])


def init_weights(seed: int = 0):
    """He-style random start, scaled so that N is small at first."""
    rng = np.random.default_rng(seed)
    ws = []
    for s in SHAPES:
        fan_in = s[0] * s[1] * s[2]
        ws.append(rng.standard_normal(s) * np.sqrt(2.0 / fan_in))
    ws[-1] *= 0.1
    return pack(ws)


def to_grid(v, nx, ny):
    """Block vector (n, k) with x fastest -> images (k, ny, nx)."""
    return np.asarray(v).T.reshape(-1, ny, nx)


def from_grid(g):
    k = g.shape[0]
    return g.reshape(k, -1).T


def conv(x, W):
    """x: (B, ny, nx, cin), W: (3, 3, cin, cout); zero padding (Dirichlet)."""
    B, ny, nx, cin = x.shape
    xp = np.zeros((B, ny + 2, nx + 2, cin))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((B, ny, nx, W.shape[3]))
    for dy in range(3):
        for dx in range(3):
            out += xp[:, dy:dy + ny, dx:dx + nx] @ W[dy, dx]
    return out


def conv_input_grad(g, W):
    """d(sum g * conv(x, W)) / dx for g: (B, ny, nx, cout)."""
    B, ny, nx, cout = g.shape
    gx = np.zeros((B, ny + 2, nx + 2, W.shape[2]))
    for dy in range(3):
        for dx in range(3):
            gx[:, dy:dy + ny, dx:dx + nx] += g @ W[dy, dx].T
    return gx[:, 1:-1, 1:-1]


def conv_weight_grad(x, g):
    """d(sum g * conv(x, W)) / dW."""
    B, ny, nx, cin = x.shape
    xp = np.zeros((B, ny + 2, nx + 2, cin))
    xp[:, 1:-1, 1:-1] = x
    gw = np.zeros((3, 3, cin, g.shape[3]))
    for dy in range(3):
        for dx in range(3):
            gw[dy, dx] = np.einsum("byxi,byxo->io", xp[:, dy:dy + ny, dx:dx + nx], g)
    return gw


def _branch(x, W1, W2, W3):
    z1 = conv(x, W1)
    a1 = np.maximum(z1, 0.0)
    z2 = conv(a1, W2)
    a2 = np.maximum(z2, 0.0)
    y = conv(a2, W3)
    return y, (x, z1, a1, z2, a2)


def _branch_back(gy, cache, W1, W2, W3):
    x, z1, a1, z2, a2 = cache
    gW3 = conv_weight_grad(a2, gy)
    ga2 = conv_input_grad(gy, W3)
    gz2 = ga2 * (z2 > 0)
    gW2 = conv_weight_grad(a1, gz2)
    ga1 = conv_input_grad(gz2, W2)
    gz1 = ga1 * (z1 > 0)
    gW1 = conv_weight_grad(x, gz1)
    return gW1, gW2, gW3


def bf16(x):
    """Round to bfloat16 (8-bit significand), round to nearest even, via float32."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def apply(w, r_grid, bf16_layer2: bool = False):
    """N(r) for images r_grid: (B, ny, nx) -> (B, ny, nx).  With bf16_layer2 the
    inputs of the second convolution (relu(+-z1) and W2) are rounded to
    bfloat16 first, as the tensor-core path computes that layer."""
    W1, W2, W3 = unpack(w)
    x = r_grid[..., None]
    if not bf16_layer2:
        yp, _ = _branch(x, W1, W2, W3)
        ym, _ = _branch(-x, W1, W2, W3)
        return 0.5 * (yp - ym)[..., 0]
    z1 = conv(x, W1)
    W2b = bf16(W2)
    z2p = conv(bf16(np.maximum(z1, 0.0)), W2b)
    z2m = conv(bf16(np.maximum(-z1, 0.0)), W2b)
    h = 0.5 * (np.maximum(z2p, 0.0) - np.maximum(z2m, 0.0))
    return conv(h, W3)[..., 0]


def _gamma(n, u):
    """n u / (1 - n u): the bound on the relative error of n rounded operations (Higham)."""
    return n * u / (1.0 - n * u)


def bf16_forward_bound(w, r_grid):
    """Elementwise bound on |N~(r) - apply(w, r, bf16_layer2=True)|, where N~ is
    any evaluation that computes layer 1 as 9 float32 FMAs per output in tap
    order (dy, then dx), rounds relu(+-z1) of its own float32 z1 to bfloat16,
    sums layer 2's exact products of those operands and of the bfloat16 W2 in
    float32 (144 terms, any order, rounded or truncated), forms h in float32
    and computes layer 3 as 144 float32 FMAs.  r is float32 on both sides.
      z1: the running error of the FMA chain, e_i <= (1 + u) e_(i-1) + u |s_i|
          with s_i the exact partial sums, gives |z1~ - z1| <= d1 =
          (1 + 10^-6) 2^-24 sum_i |s_i| + gamma_9(2^-53) (|W1| * |r|) (the
          second term: the oracle's own float64 z1);
      a = bf16(relu(+-z1)): relu and round-to-nearest are monotone, so both
          sides' a lie in [bf16(relu(+-z1 - d1)), bf16(relu(+-z1 + d1))]; the
          width da of that interval is zero unless a rounding boundary lies
          within d1 of +-z1, and then one bfloat16 step;
      z2: |dz2| <= |W2b| * da + gamma_144(2^-23) (|W2b| * (|a| + da));
      h = (relu(z2+) - relu(z2-)) / 2 (relu is 1-Lipschitz, one float32
          subtraction): |dh| <= (|dz2+| + |dz2-|) / 2 + 2^-23 (|h| + that);
      d: |dd| <= |W3| * dh + gamma_144(2^-24) (|W3| * (|h| + dh))
              + gamma_144(2^-53) (|W3| * |h|) (the oracle's own rounding).
    Returns the bound as images (B, ny, nx)."""
    W1, W2, W3 = unpack(w)
    u32, u64 = 2.0 ** -24, 2.0 ** -53
    x = np.asarray(r_grid, dtype=np.float64)[..., None]
    z1 = conv(x, W1)
    B, ny, nx, _ = x.shape
    xp = np.zeros((B, ny + 2, nx + 2, 1))
    xp[:, 1:-1, 1:-1] = x
    part, run = np.zeros(z1.shape), np.zeros(z1.shape)
    for tap in range(9):
        dy, dx = divmod(tap, 3)
        part = part + xp[:, dy:dy + ny, dx:dx + nx] * W1[dy, dx, 0]
        run += np.abs(part)
    d1 = (1.0 + 1e-6) * u32 * run + 2.0 * _gamma(9, u64) * conv(np.abs(x), np.abs(W1))
    W2b = np.abs(bf16(W2))
    dz2, a_abs = [], []
    for s in (1.0, -1.0):
        lo = bf16(np.maximum(s * z1 - d1, 0.0))
        hi = bf16(np.maximum(s * z1 + d1, 0.0))
        da = hi - lo
        a = bf16(np.maximum(s * z1, 0.0))
        dz2.append(conv(da, W2b) + _gamma(144, 2.0 * u32) * conv(a + da, W2b))
        a_abs.append(a)
    z2p, z2m = conv(a_abs[0], bf16(W2)), conv(a_abs[1], bf16(W2))
    h = 0.5 * (np.maximum(z2p, 0.0) - np.maximum(z2m, 0.0))
    dh = 0.5 * (dz2[0] + dz2[1])
    dh = dh + 2.0 * u32 * (np.abs(h) + dh)
    W3a = np.abs(W3)
    dd = conv(dh, W3a) + _gamma(144, u32) * conv(np.abs(h) + dh, W3a) + _gamma(144, u64) * conv(np.abs(h), W3a)
    return dd[..., 0]


def loss_and_grad(w, A, R, nx, ny):
    """L = mean_j |r_j - A N(r_j)|^2 / |r_j|^2 over the columns r_j of R (n, k)
    and its gradient with respect to the packed weights."""
    W1, W2, W3 = unpack(w)
    k = R.shape[1]
    x = to_grid(R, nx, ny)[..., None]
    yp, cp = _branch(x, W1, W2, W3)
    ym, cm = _branch(-x, W1, W2, W3)
    D = from_grid(0.5 * (yp - ym)[..., 0])
    E = R - A @ D
    nr2 = np.einsum("ij,ij->j", R, R)
    L = float(np.mean(np.einsum("ij,ij->j", E, E) / nr2))
    # dL/dD = -2 A^T E / (k |r|^2); A symmetric
    gD = -2.0 * (A.T @ (E / nr2)) / k
    gy = to_grid(gD, nx, ny)[..., None]
    g1 = _branch_back(0.5 * gy, cp, W1, W2, W3)
    g2 = _branch_back(-0.5 * gy, cm, W1, W2, W3)
    return L, pack([a + b for a, b in zip(g1, g2)])


def loss_and_grad_bf16(w, A, R, nx, ny):
    """loss_and_grad with the second convolution's products taken on bfloat16
    operands, as the tensor-core training path computes them: in the forward
    pass relu(+-z1) and W2 are rounded (as in apply(..., bf16_layer2=True));
    in the backward pass the two products of layer 2 -- its weight gradient
    sum a+- g+- and its input gradient g+- (*) W2 -- take a+- (already
    rounded), the rounded output gradients g+- = dL/dz2+- and the rounded W2.
    Everything else as in loss_and_grad (float64 here)."""
    W1, W2, W3 = unpack(w)
    k = R.shape[1]
    x = to_grid(R, nx, ny)[..., None]
    z1 = conv(x, W1)
    W2b = bf16(W2)
    ap, am = bf16(np.maximum(z1, 0.0)), bf16(np.maximum(-z1, 0.0))
    z2p, z2m = conv(ap, W2b), conv(am, W2b)
    h = 0.5 * (np.maximum(z2p, 0.0) - np.maximum(z2m, 0.0))
    D = from_grid(conv(h, W3)[..., 0])
    E = R - A @ D
    nr2 = np.einsum("ij,ij->j", R, R)
    L = float(np.mean(np.einsum("ij,ij->j", E, E) / nr2))
    gy = to_grid(-2.0 * (A.T @ (E / nr2)) / k, nx, ny)[..., None]
    gW3 = conv_weight_grad(h, gy)
    gh = conv_input_grad(gy, W3)
    gp = bf16(0.5 * gh * (z2p > 0))
    gm = bf16(-0.5 * gh * (z2m > 0))
    gW2 = conv_weight_grad(ap, gp) + conv_weight_grad(am, gm)
    gap, gam = conv_input_grad(gp, W2b), conv_input_grad(gm, W2b)
    gz1 = gap * (z1 > 0) - gam * (z1 < 0)
    gW1 = conv_weight_grad(x, gz1)
    return L, pack([gW1, gW2, gW3])


def bf16_gradient_bound(w, A, R, nx, ny):
    """First-order bound on |loss_and_grad_bf16 - loss_and_grad|, weight by
    weight: 8 u G_abs, u = 2^-9 (bf16 unit roundoff), G_abs = the gradient of
    the network evaluated on |W|, |r| and the absolute values of every
    activation and output gradient.  Each product of layer 2 carries at most
    four rounded factors along any path of the chain rule (forward a and W2,
    backward g and W2 or a): 4u to first order; the factor 2 covers
    second-order terms and ReLU switches near zero."""
    W1, W2, W3 = unpack(w)
    x = to_grid(R, nx, ny)[..., None]
    a = np.abs(conv(x, W1))
    W2a, W3a = np.abs(W2), np.abs(W3)
    z2 = conv(a, W2a)
    D = from_grid(conv(z2, W3a)[..., 0])
    absA = abs(A)
    E = np.abs(R) + absA @ D
    nr2 = np.einsum("ij,ij->j", R, R)
    gy = to_grid(2.0 * (absA.T @ (E / nr2)) / R.shape[1], nx, ny)[..., None]
    gh = conv_input_grad(gy, W3a)
    G2 = 2 * conv_weight_grad(a, gh)
    G1 = 2 * conv_weight_grad(np.abs(x), conv_input_grad(gh, W2a))
    return 8 * 2.0 ** -9 * pack([G1, G2, conv_weight_grad(z2, gy)])


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), t counted from 1.  Returns new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
