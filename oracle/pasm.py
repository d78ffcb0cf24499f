"""Oracle: Algorithms 1 and 2 of the parallel augmented subspace method, FP64 CPU.

Test infrastructure only (see the package docstring).  Notation follows the
paper: the pencil A u = lambda M u on the finest space V_h, a coarse space V_H
with matrices A_H, M_H, the augmented space V_{H,h} = V_H + span{u~}.  The
number of wanted eigenpairs is k here (the paper's m); mesh levels are l.

Readings of points the paper leaves open (listed with reasons in the design
notes of the repository):
  * multigrid for the boundary value problem of Algorithm 1 step 1 = V-cycles
    with damped Jacobi smoothing (omega = 2/3, nu_pre = nu_post = 2), exact
    solve on the coarsest level V_H, two V-cycles per correction step;
    optionally the paper's own smoother of Section 5.1, conjugate gradients
    (nu_pre / nu_post CG steps, unpreconditioned, restarted at every
    smoothing, each column its own CG);
  * the multigrid initial guess is the current eigenvector u^(l) (the
    contraction assumption of Theorem 3.1 measures from it);
  * initial pairs: the k smallest coarse eigenpairs of (A_H, M_H) prolongated
    to the finest level (Algorithm 2 step 1 with h_1 = H, then step 2(B));
  * selection score: |b(u_{H,h}, u~)| of the a-normalised Ritz vectors
    (Section 3.1, the rule after the bordered eigenproblem); ties go to the
    smaller Ritz value; the b-normalised score is an option;
  * sign: b(u^(l+1), u~) > 0;
  * a pair is frozen once |lambda^(l+1) - lambda^(l)| / lambda^(l+1) < tol;
  * degenerate bordering (u~ numerically inside V_H): the pair keeps its
    previous (lambda, u) for that step.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

SCORE_A = 0   # paper-literal: Ritz vectors normalised to a(u, u) = 1
SCORE_B = 1   # option: Ritz vectors normalised to b(u, u) = 1


@dataclass
class Problem:
    """A level hierarchy plus the method's parameters.

    A, M: lists of CSR matrices, index 0 = coarsest level (V_H).
    P: list of CSR interpolations, P[l] maps level l to level l+1."""
    A: list
    M: list
    P: list
    omega: float = 2.0 / 3.0
    nu_pre: int = 2
    nu_post: int = 2
    cycles: int = 2
    score: int = SCORE_A
    # learned post-smoother (oracle.smoother): packed weights and per-level grid
    # widths (0 / None = plain Jacobi on that level)
    nn_weights: object = None
    grids: object = None
    nn_bf16: bool = False          # round layer-2 inputs to bfloat16 (tensor-core path)
    smoother: str = "jacobi"       # "jacobi" (damped Jacobi) or "cg" (conjugate gradients)

    def __post_init__(self):
        self.L = len(self.A) - 1
        self.dinv = [1.0 / A.diagonal() for A in self.A]
        self.A_H = self.A[0].toarray()
        self.M_H = self.M[0].toarray()
        self._chol_H = sla.cho_factor(self.A_H, lower=True)
        # composite prolongation P_c = P[L-1] ... P[0] : V_H -> V_h (columns = coarse
        # basis functions phi_{j,H} written in the fine nodal basis)
        Pc = sp.identity(self.A[0].shape[0], format="csr")
        for P in self.P:
            Pc = (P @ Pc).tocsr()
        self.Pc = Pc

    @classmethod
    def from_hierarchy(cls, hier, **kw):
        return cls([lv.A for lv in hier.levels], [lv.M for lv in hier.levels], list(hier.P), **kw)

    @property
    def n(self) -> int:
        return self.A[-1].shape[0]

    @property
    def N_H(self) -> int:
        return self.A[0].shape[0]


# ----------------------------------------------------------------------------- Algorithm 2, step 1

def coarse_eigenpairs(prob: Problem):
    """Algorithm 2 step 1 on V_H: all eigenpairs of A_H q = Lambda M_H q,
    ascending, with Q^T M_H Q = I (library dense generalized eigensolver)."""
    lam, Q = sla.eigh(prob.A_H, prob.M_H)
    return lam, Q


def initial_state(prob: Problem, k: int):
    """Initial pairs: lambda_i = Lambda_H[i], u_i = P_c q_i a-normalised
    (a(u, u) = 1 as required by the weak eigenproblem of Section 2)."""
    if k > prob.N_H:
        raise ValueError("k exceeds the coarse space dimension N_H")
    lam, Q = coarse_eigenpairs(prob)
    U = prob.Pc @ (Q[:, :k] / np.sqrt(lam[:k]))
    return lam[:k].copy(), np.asarray(U)


def sub_problem(prob: Problem, l: int) -> Problem:
    """The hierarchy truncated at level l (V_H = level 0 stays the coarse space)."""
    return Problem(prob.A[:l + 1], prob.M[:l + 1], prob.P[:l], omega=prob.omega, nu_pre=prob.nu_pre,
                   nu_post=prob.nu_post, cycles=prob.cycles, score=prob.score, nn_weights=prob.nn_weights,
                   grids=None if prob.grids is None else prob.grids[:l + 1], nn_bf16=prob.nn_bf16,
                   smoother=prob.smoother)


def initial_state_nested(prob: Problem, k: int):
    """Algorithm 2 with h_1 = H: step 1 on V_H, then step 2(A) -- on every
    intermediate level one correction step (varpi = 1, the choice the paper
    recommends for the intermediate levels) started from the prolongated
    pairs of the level below -- and prolongation to the finest level."""
    lam, U = initial_state(sub_problem(prob, 0), k)      # pairs on V_H (u = q / sqrt(Lambda))
    for l in range(1, prob.L):
        U = prob.P[l - 1] @ U
        lam, U, _ = correction(sub_problem(prob, l), lam, U)
    return lam, prob.P[prob.L - 1] @ U if prob.L >= 1 else U


# ----------------------------------------------------------------------------- Algorithm 1, step 1

def jacobi(A, dinv, f, x, omega, nu):
    """nu damped Jacobi sweeps x <- x + omega D^{-1} (f - A x) (columns independent)."""
    for _ in range(nu):
        x = x + omega * (dinv[:, None] * (f - A @ x))
    return x


def cg(A, f, x, nu):
    """nu conjugate-gradient steps for A x = f started from x, each column an
    independent CG (Hestenes-Stiefel recurrences: residual r, direction p,
    step alpha = r.r / p.A p, then beta = r'.r' / r.r).  A column whose
    residual or curvature p.A p vanishes takes no step (alpha = beta = 0)."""
    r = f - A @ x
    p = r.copy()
    rr = np.einsum("ij,ij->j", r, r)
    for _ in range(nu):
        q = A @ p
        pq = np.einsum("ij,ij->j", p, q)
        alpha = np.divide(rr, pq, out=np.zeros_like(rr), where=pq > 0)
        x = x + alpha[None, :] * p
        r = r - alpha[None, :] * q
        rr_new = np.einsum("ij,ij->j", r, r)
        beta = np.divide(rr_new, rr, out=np.zeros_like(rr), where=rr > 0)
        p = r + beta[None, :] * p
        rr = rr_new
    return x


def smooth(prob: Problem, l: int, f, x, nu):
    """nu smoothing steps on level l with the problem's smoother."""
    if prob.smoother == "cg":
        return cg(prob.A[l], f, x, nu)
    return jacobi(prob.A[l], prob.dinv[l], f, x, prob.omega, nu)


def vcycle(prob: Problem, l: int, f, x):
    """One multigrid V-cycle for A_l x = f on level l: pre-smooth, restrict the
    residual with P^T, recurse from a zero guess, prolongate and correct,
    post-smooth.  Level 0 (V_H) is solved exactly (dense Cholesky)."""
    if l == 0:
        return sla.cho_solve(prob._chol_H, f)
    A, dinv, P = prob.A[l], prob.dinv[l], prob.P[l - 1]
    x = smooth(prob, l, f, x, prob.nu_pre)
    fc = P.T @ (f - A @ x)
    ec = vcycle(prob, l - 1, fc, np.zeros_like(fc))
    x = x + P @ ec
    nu = prob.nu_post
    if prob.nn_weights is not None and prob.grids is not None and prob.grids[l] and nu >= 1:
        x = learned_sweep(prob, l, f, x)
        nu -= 1
    x = smooth(prob, l, f, x, nu)
    return x


def learned_sweep(prob: Problem, l: int, f, x):
    """Learned post-smoothing step with a per-pair fallback: each column takes
    x + N(r) if that does not increase its residual norm, else one damped
    Jacobi step (the network is oracle.smoother.apply on the level's grid)."""
    from . import smoother as sm
    A, dinv = prob.A[l], prob.dinv[l]
    nx = prob.grids[l]
    ny = A.shape[0] // nx
    r = f - A @ x
    d = sm.from_grid(sm.apply(prob.nn_weights, sm.to_grid(r, nx, ny), bf16_layer2=prob.nn_bf16))
    xt = x + d
    rt = f - A @ xt
    ok = np.einsum("ij,ij->j", rt, rt) <= np.einsum("ij,ij->j", r, r)
    return np.where(ok[None, :], xt, x + prob.omega * dinv[:, None] * r)


def bvp_solve(prob: Problem, lam, U):
    """Algorithm 1 step 1: approximate u^ in a(u^, v) = lambda b(u, v), i.e.
    A u^ = lambda M u, by `cycles` V-cycles started from u.  Columns of U are
    independent pairs; lam holds one eigenvalue per column."""
    L = prob.L
    f = (prob.M[L] @ U) * np.asarray(lam)[None, :]
    x = np.array(U, dtype=np.float64, copy=True)
    for _ in range(prob.cycles):
        x = vcycle(prob, L, f, x)
    return x


# ----------------------------------------------------------------------------- Algorithm 1, step 2

def bordering(prob: Problem, ut):
    """Entries of the bordered eigenproblem on V_{H,h} = V_H + span{u~}
    (the matrix form of Section 3.1): b_j = a(phi_j, u~), c_j = b(phi_j, u~),
    beta = a(u~, u~), zeta = b(u~, u~) for one vector u~."""
    L = prob.L
    yA = prob.A[L] @ ut
    yM = prob.M[L] @ ut
    b = prob.Pc.T @ yA
    c = prob.Pc.T @ yM
    return np.asarray(b), np.asarray(c), float(ut @ yA), float(ut @ yM)


def augmented_eigenproblem(prob: Problem, ut, score=None):
    """All eigenpairs of the (N_H + 1) bordered pencil for one u~.

    Returns (theta, X, sv, ok): Ritz values ascending, a-normalised Ritz
    vectors X (columns [u_H; alpha]), signed selection scores
    sv_j = u_H . c + alpha zeta = b(u_{H,h}, u~) of the a-normalised (SCORE_A)
    or b-normalised (SCORE_B) Ritz vectors, and ok=False when the
    bordered mass matrix is numerically singular (u~ inside V_H)."""
    score = prob.score if score is None else score
    b, c, beta, zeta = bordering(prob, ut)
    N = prob.N_H
    Ab = np.empty((N + 1, N + 1)); Mb = np.empty((N + 1, N + 1))
    Ab[:N, :N] = prob.A_H; Ab[:N, N] = b; Ab[N, :N] = b; Ab[N, N] = beta
    Mb[:N, :N] = prob.M_H; Mb[:N, N] = c; Mb[N, :N] = c; Mb[N, N] = zeta
    # b-distance of u~ from V_H: zeta - c^T M_H^{-1} c (Schur complement of Mb)
    zeta_t = zeta - c @ np.linalg.solve(prob.M_H, c)
    if not zeta_t > 1e-14 * zeta:
        return None, None, None, False
    theta, X = sla.eigh(Ab, Mb)                  # X^T Mb X = I (b-normalised)
    sv = X[:N].T @ c + X[N] * zeta             # b(u_{H,h}, u~), signed, b-normalised
    X = X / np.sqrt(np.einsum("ij,ik,kj->j", X, Ab, X))   # a(u, u) = 1
    if score == SCORE_A:
        sv = X[:N].T @ c + X[N] * zeta
    return theta, X, sv, True


def correction(prob: Problem, lam, U, active=None):
    """One correction step (Algorithm 1) for every active pair (column).

    Returns (lam_new, U_new, info) where info holds the per-pair selected index
    and whether the bordered problem was degenerate."""
    lam = np.asarray(lam, dtype=np.float64)
    k = U.shape[1]
    active = np.ones(k, dtype=bool) if active is None else np.asarray(active, dtype=bool)
    Ut = bvp_solve(prob, lam, U)
    lam_new = lam.copy()
    U_new = np.array(U, copy=True)
    sel = np.full(k, -1)
    degenerate = np.zeros(k, dtype=bool)
    N = prob.N_H
    for i in range(k):
        if not active[i]:
            continue
        ut = Ut[:, i]
        theta, X, sv, ok = augmented_eigenproblem(prob, ut)
        if not ok:
            degenerate[i] = True
            continue
        j = int(np.argmax(np.abs(sv)))            # first maximum = smallest theta on ties
        x = X[:, j] if sv[j] >= 0 else -X[:, j]
        U_new[:, i] = x[N] * ut + prob.Pc @ x[:N]
        lam_new[i] = theta[j]
        sel[i] = j
    return lam_new, U_new, {"selected": sel, "degenerate": degenerate, "u_tilde": Ut}


# ----------------------------------------------------------------------------- Algorithm 2, step 2(B)

def solve(prob: Problem, k: int, tol: float = 1e-10, max_steps: int = 100,
          lam0=None, U0=None, history: bool = False, nested: bool = False):
    """Correction steps on the finest level until every pair is frozen
    (|d lambda| / lambda < tol) or max_steps.  Returns (lam, U, steps, hist)
    with steps = per-pair number of correction steps taken."""
    if lam0 is None:
        lam, U = initial_state_nested(prob, k) if nested else initial_state(prob, k)
    else:
        lam, U = np.array(lam0, dtype=np.float64), np.array(U0, dtype=np.float64)
    active = np.ones(k, dtype=bool)
    steps = np.zeros(k, dtype=int)
    hist = [lam.copy()] if history else None
    for _ in range(max_steps):
        if not active.any():
            break
        lam_new, U, _ = correction(prob, lam, U, active)
        steps[active] += 1
        done = np.abs(lam_new - lam) < tol * np.abs(lam_new)
        lam = lam_new
        active &= ~done
        if history:
            hist.append(lam.copy())
    return lam, U, steps, hist
