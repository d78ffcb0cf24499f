"""Seeded input generators: structured P1 finite-element hierarchies.

This module builds the INPUTS of the parallel augmented subspace method (PASM):
the level matrices A_l (stiffness), M_l (mass) and the interpolations P_l of a
nested sequence of uniform simplex meshes of the unit square or cube
(Section 2, the P1 space and the discrete pencil A u = lambda M u; Section 3.1,
nested meshes with refinement index beta = 2).  It holds none of the method's
arithmetic: no multigrid, no eigen-solve, no bordering.  Both the CPU oracle and
the CUDA path consume what it returns, which is why it lives on its own.

Meshes
  2D: the unit square cut into N x N cells, each split along its (1,1)
      diagonal into two right triangles.
  3D: the unit cube cut into N^3 cells, each split into the 6 Kuhn
      (Freudenthal) tetrahedra that share the cell's main diagonal.
  Both refine by halving h; the finer mesh is a red refinement of the coarser
  one, so the P1 spaces are nested and linear interpolation is exact.

Unknowns are the interior nodes (homogeneous Dirichlet data), numbered
lexicographically with x fastest: node (i, j[, l]) with 1 <= i, j, l <= N-1
gets index (i-1) + (N-1)*(j-1) [+ (N-1)^2*(l-1)].

Coefficient: -div(kappa grad u) = lambda u with kappa piecewise constant per
simplex (kappa = 1 by default), as in the model problem of Section 2.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Level", "Hierarchy", "reference_simplices", "assemble", "interpolation",
    "build_hierarchy", "gaussian_log_field", "continuous_eigenvalues",
    "assemble_operator", "element_averages", "example2_diffusion", "example2_potential",
]


@dataclass
class Level:
    """One mesh level: h = 1/N, the P1 stiffness A and mass M (CSR, float64)."""
    dim: int
    N: int
    A: sp.csr_matrix
    M: sp.csr_matrix

    @property
    def n(self) -> int:
        return self.A.shape[0]


@dataclass
class Hierarchy:
    """Nested levels, index 0 = coarsest (V_H), last = finest (V_h).

    P[l] (l = 0..L-1) is the interpolation from level l to level l+1,
    shape (n_{l+1}, n_l)."""
    levels: list
    P: list = field(default_factory=list)

    @property
    def fine(self) -> Level:
        return self.levels[-1]

    @property
    def coarse(self) -> Level:
        return self.levels[0]


def reference_simplices(dim: int):
    """Vertex offsets (0/1 integer vectors) of the simplices of one unit cell."""
    if dim == 2:
        return [np.array([[0, 0], [1, 0], [1, 1]]), np.array([[0, 0], [1, 1], [0, 1]])]
    if dim == 3:
        out = []
        for perm in itertools.permutations(range(3)):
            v = np.zeros(3, dtype=int)
            verts = [v.copy()]
            for ax in perm:
                v[ax] += 1
                verts.append(v.copy())
            out.append(np.array(verts))
        return out
    raise ValueError("dim must be 2 or 3")


def _local_matrices(offsets: np.ndarray, h: float):
    """P1 element stiffness and mass matrices of one simplex with vertices h*offsets."""
    dim = offsets.shape[1]
    X = h * offsets.astype(np.float64)
    B = (X[1:] - X[0]).T                       # columns: edge vectors from vertex 0
    vol = abs(np.linalg.det(B)) / float(np.prod(np.arange(1, dim + 1)))
    Binv = np.linalg.inv(B)
    G = np.zeros((dim + 1, dim))
    G[1:] = Binv                                # grad of barycentric lambda_i, i >= 1
    G[0] = -Binv.sum(axis=0)
    K = vol * (G @ G.T)
    K[np.abs(K) < 1e-13 * np.abs(K).max()] = 0.0   # exact zeros (right angles)
    Mloc = vol / ((dim + 1) * (dim + 2)) * (np.ones((dim + 1, dim + 1)) + np.eye(dim + 1))
    return K, Mloc


def _stencil_to_csr(dim: int, N: int, vals: dict) -> sp.csr_matrix:
    """Turn per-offset grid arrays (indexed by the row node, full grid incl. boundary)
    into a CSR matrix over the interior nodes, columns ascending."""
    m = N - 1
    n = m ** dim
    strides = [m ** a for a in range(dim)]     # x fastest
    offs = sorted(vals.keys(), key=lambda o: sum(o[a] * strides[a] for a in range(dim)))
    coords = np.stack(np.meshgrid(*[np.arange(1, N)] * dim, indexing="ij"), axis=0).reshape(dim, -1)
    coords = coords[:, np.lexsort(coords)]     # x fastest
    cols_l, vals_l, mask_l = [], [], []
    for o in offs:
        nb = coords + np.array(o)[:, None]
        ok = np.all((nb >= 1) & (nb <= N - 1), axis=0)
        lin = np.zeros(n, dtype=np.int64)
        for a in range(dim):
            lin += (nb[a] - 1) * strides[a]
        g = vals[o]
        v = g[tuple(coords[a] for a in range(dim))]
        ok &= v != 0.0
        cols_l.append(lin)
        vals_l.append(v)
        mask_l.append(ok)
    C = np.stack(cols_l, axis=1)
    V = np.stack(vals_l, axis=1)
    K = np.stack(mask_l, axis=1)
    counts = K.sum(axis=1)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    mat = sp.csr_matrix((V[K], C[K], indptr), shape=(n, n))
    mat.has_sorted_indices = True
    return mat


def assemble(dim: int, N: int, kappa=None):
    """Stiffness A and mass M of P1 elements on the uniform mesh with h = 1/N.

    kappa: None (kappa = 1) or an array of shape (n_simplex_types, N, ..., N)
    holding the coefficient of each simplex (type t of cell with lower corner
    index (i, j[, l]) at kappa[t, i, j(, l)])."""
    h = 1.0 / N
    simp = reference_simplices(dim)
    Avals, Mvals = {}, {}
    for t, offsets in enumerate(simp):
        K, Ml = _local_matrices(offsets, h)
        kap = 1.0 if kappa is None else np.asarray(kappa[t], dtype=np.float64)
        for a in range(dim + 1):
            for b in range(dim + 1):
                delta = tuple(int(x) for x in offsets[b] - offsets[a])
                sl = tuple(slice(int(offsets[a][ax]), int(offsets[a][ax]) + N) for ax in range(dim))
                for store, loc in ((Avals, K), (Mvals, Ml)):
                    if delta not in store:
                        store[delta] = np.zeros((N + 1,) * dim)
                    if loc[a, b] != 0.0:
                        store[delta][sl] += kap * loc[a, b]
    # drop offsets that never receive a value
    Avals = {o: g for o, g in Avals.items() if np.any(g != 0.0)}
    Mvals = {o: g for o, g in Mvals.items() if np.any(g != 0.0)}
    return _stencil_to_csr(dim, N, Avals), _stencil_to_csr(dim, N, Mvals)


# Degree-2 quadrature on a simplex: barycentric points and weights (fractions of
# the volume).  Tetrahedron: the symmetric 4-point rule (a, b, b, b),
# a = (5 + 3 sqrt 5) / 20, b = (5 - sqrt 5) / 20, exact for quadratics.
# Triangle: the 3 edge midpoints, exact for quadratics.
def _quadrature(dim: int):
    if dim == 3:
        a = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
        b = (5.0 - np.sqrt(5.0)) / 20.0
        pts = np.array([[a, b, b, b], [b, a, b, b], [b, b, a, b], [b, b, b, a]])
        return pts, np.full(4, 0.25)
    if dim == 2:
        pts = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
        return pts, np.full(3, 1.0 / 3.0)
    raise ValueError("dim must be 2 or 3")


def element_averages(dim: int, N: int, diffusion):
    """Per simplex type t and cell, the average of the diffusion tensor over the
    simplex by the degree-2 rule (exact for quadratic entries): a list over t of
    arrays of shape (N,)*dim + (dim, dim), and the simplex volume."""
    h = 1.0 / N
    pts, wts = _quadrature(dim)
    cells = np.stack(np.meshgrid(*[np.arange(N)] * dim, indexing="ij"), axis=-1).astype(np.float64)
    out = []
    for offsets in reference_simplices(dim):
        Xv = h * (cells[..., None, :] + offsets[None, :].astype(np.float64))   # (..., dim+1, dim)
        xq = np.einsum("qv,...vd->...qd", pts, Xv)                             # (..., q, dim)
        out.append(np.einsum("q,...qij->...ij", wts, diffusion(xq)))
    vol = h ** dim / float(np.prod(np.arange(1, dim + 1)))
    return out, vol


def assemble_operator(dim: int, N: int, diffusion, potential=None):
    """Stiffness A of a(u, v) = int grad v . D grad u + phi u v and the mass M of
    P1 elements on the uniform mesh with h = 1/N (the general second-order
    operator of the paper's Example 2, Section 5.2).

    diffusion(x): D at points x (array (..., dim)) -> (..., dim, dim), symmetric
    positive definite; potential(x) -> (...) or None.  Both element integrals
    use the degree-2 rule of `_quadrature`: exact for D with quadratic entries
    (so the stiffness part is exact) and for constant phi."""
    h = 1.0 / N
    pts, wts = _quadrature(dim)
    cells = np.stack(np.meshgrid(*[np.arange(N)] * dim, indexing="ij"), axis=-1).astype(np.float64)
    avgs, vol = element_averages(dim, N, diffusion)
    Avals, Mvals = {}, {}
    for t, offsets in enumerate(reference_simplices(dim)):
        X = h * offsets.astype(np.float64)
        B = (X[1:] - X[0]).T
        Binv = np.linalg.inv(B)
        G = np.zeros((dim + 1, dim))
        G[1:] = Binv
        G[0] = -Binv.sum(axis=0)
        Kloc = vol * np.einsum("ai,...ij,bj->...ab", G, avgs[t], G)            # (..., dim+1, dim+1)
        if potential is not None:
            Xv = h * (cells[..., None, :] + offsets[None, :].astype(np.float64))
            xq = np.einsum("qv,...vd->...qd", pts, Xv)
            phi = potential(xq)                                                   # (..., q)
            Kloc = Kloc + vol * np.einsum("q,...q,qa,qb->...ab", wts, phi, pts, pts)
        Ml = vol / ((dim + 1) * (dim + 2)) * (np.ones((dim + 1, dim + 1)) + np.eye(dim + 1))
        for a in range(dim + 1):
            for b in range(dim + 1):
                delta = tuple(int(x) for x in offsets[b] - offsets[a])
                sl = tuple(slice(int(offsets[a][ax]), int(offsets[a][ax]) + N) for ax in range(dim))
                for store, loc in ((Avals, Kloc[..., a, b]), (Mvals, Ml[a, b])):
                    if delta not in store:
                        store[delta] = np.zeros((N + 1,) * dim)
                    store[delta][sl] += loc
    Avals = {o: g for o, g in Avals.items() if np.any(g != 0.0)}
    Mvals = {o: g for o, g in Mvals.items() if np.any(g != 0.0)}
    return _stencil_to_csr(dim, N, Avals), _stencil_to_csr(dim, N, Mvals)


def example2_diffusion(x):
    """D(x) = I + (x - 1/2)(x - 1/2)^T (the paper's Example 2, Section 5.2)."""
    y = x - 0.5
    d = x.shape[-1]
    return np.eye(d) + y[..., :, None] * y[..., None, :]


def example2_potential(x):
    """phi(x) = exp(prod_i (x_i - 1/2)) (the paper's Example 2, Section 5.2)."""
    return np.exp(np.prod(x - 0.5, axis=-1))


def interpolation(dim: int, N_fine: int) -> sp.csr_matrix:
    """Linear interpolation from the mesh with N_fine/2 cells per side to N_fine.

    A fine node with integer coordinates x lies at the midpoint of the coarse
    edge from (x - p)/2 to (x + p)/2 where p = x mod 2 (a 0/1 vector; every 0/1
    direction is an edge of both meshes).  p = 0 means the node is a coarse node."""
    if N_fine % 2:
        raise ValueError("N_fine must be even")
    Nc = N_fine // 2
    mf, mc = N_fine - 1, Nc - 1
    nf = mf ** dim
    coords = np.stack(np.meshgrid(*[np.arange(1, N_fine)] * dim, indexing="ij"), axis=0).reshape(dim, -1)
    coords = coords[:, np.lexsort(coords)]     # x fastest
    p = coords % 2
    c0 = (coords - p) // 2
    c1 = (coords + p) // 2
    onepoint = ~np.any(p, axis=0)
    rows, cols, vals = [], [], []
    for cc, w in ((c0, 0.5), (c1, 0.5)):
        ok = np.all((cc >= 1) & (cc <= Nc - 1), axis=0)
        lin = np.zeros(nf, dtype=np.int64)
        for a in range(dim):
            lin += (cc[a] - 1) * mc ** a
        wt = np.where(onepoint, 0.5, w)          # coarse node: 0.5 + 0.5 = 1 on the same column
        rows.append(np.arange(nf)[ok]); cols.append(lin[ok]); vals.append(wt[ok])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nf, mc ** dim)).tocsr()
    P.sum_duplicates()
    P.sort_indices()
    return P


def build_hierarchy(dim: int, N_fine: int, N_coarse: int, kappa=None, galerkin: bool = False,
                    operator=None) -> Hierarchy:
    """Nested hierarchy N_coarse, 2 N_coarse, ..., N_fine (every dyadic level).

    kappa: fine-level per-simplex coefficient (see `assemble`) or None.  With a
    variable kappa (or galerkin=True) the coarser A_l, M_l are the Galerkin
    products P^T A P, P^T M P, so that every level is a subspace restriction of
    the finest pencil; with kappa = 1 and galerkin=False each level is assembled
    directly (the two agree to rounding because the spaces are nested).
    operator: (diffusion, potential) for `assemble_operator` on the finest
    level (e.g. the paper's Example 2), coarser levels by Galerkin products."""
    if N_fine % N_coarse or (N_fine // N_coarse) & (N_fine // N_coarse - 1):
        raise ValueError("N_fine / N_coarse must be a power of two")
    Ns = []
    N = N_fine
    while N >= N_coarse:
        Ns.append(N)
        N //= 2
    Ns = Ns[::-1]
    Ps = [interpolation(dim, Nf) for Nf in Ns[1:]]
    if kappa is None and not galerkin and operator is None:
        levels = [Level(dim, N, *assemble(dim, N)) for N in Ns]
    else:
        if operator is not None:
            Af, Mf = assemble_operator(dim, Ns[-1], *operator)
        else:
            Af, Mf = assemble(dim, Ns[-1], kappa)
        mats = [(Af, Mf)]
        for P in Ps[::-1]:
            A, M = mats[-1]
            Ac = (P.T @ A @ P).tocsr(); Mc = (P.T @ M @ P).tocsr()
            Ac.sort_indices(); Mc.sort_indices()
            mats.append((Ac, Mc))
        mats = mats[::-1]
        levels = [Level(dim, N, A, M) for N, (A, M) in zip(Ns, mats)]
    return Hierarchy(levels, Ps)


def gaussian_field_nodes(N: int, seed: int, sigma: float = 1.0, corr: float = 0.1) -> np.ndarray:
    """Seeded stationary Gaussian field g on the (N+1)^2 nodes of the unit square
    (node (i, j) at (i/N, j/N)): squared-exponential covariance
    sigma^2 exp(-d^2 / (2 corr^2)), synthesised spectrally on a periodic (2N)^2
    grid of spacing 1/N and cropped."""
    rng = np.random.default_rng(seed)
    L = 2 * N
    k = np.fft.fftfreq(L, d=1.0 / N) * 2 * np.pi          # angular wavenumbers
    kx, ky = np.meshgrid(k, k, indexing="ij")
    # spectral density of the squared-exponential kernel in 2D
    S = sigma ** 2 * 2 * np.pi * corr ** 2 * np.exp(-0.5 * corr ** 2 * (kx ** 2 + ky ** 2))
    dA = (2 * np.pi * N / L) ** 2
    noise = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    g = np.fft.ifft2(noise * np.sqrt(S * dA / (2 * np.pi) ** 2)) * L * L
    return np.real(g)[: N + 1, : N + 1]


def gaussian_log_field(N: int, seed: int, sigma: float = 1.0, corr: float = 0.1) -> np.ndarray:
    """The coefficient kappa = exp(g) of the variable-coefficient problems, g
    the field of `gaussian_field_nodes`: per triangle, kappa = exp(mean of g
    over the triangle's vertices), in the layout `assemble` expects: shape
    (2, N, N)."""
    g = gaussian_field_nodes(N, seed, sigma, corr)
    simp = reference_simplices(2)
    kap = np.empty((2, N, N))
    for t, offs in enumerate(simp):
        acc = np.zeros((N, N))
        for o in offs:
            acc += g[o[0]: o[0] + N, o[1]: o[1] + N]
        kap[t] = np.exp(acc / 3.0)
    return kap


def continuous_eigenvalues(dim: int, count: int) -> np.ndarray:
    """The `count` smallest eigenvalues of -Laplace on the unit square/cube with
    Dirichlet data: pi^2 (m^2 + n^2 [+ p^2]), m, n, p >= 1, with multiplicity."""
    top = int(np.ceil(np.sqrt(count))) + 3
    vals = [sum(q * q for q in idx) for idx in itertools.product(range(1, top + 1), repeat=dim)]
    vals = np.sort(np.array(vals, dtype=np.float64))
    return np.pi ** 2 * vals[:count]
