"""CPU FP64 oracle of the parallel augmented subspace method (PASM).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the tests, the smoke check and the CPU-baseline leg
of the benchmark use it.  It shares no code with the CUDA library; both sides
read their inputs from `meshgen`, which holds none of the method's arithmetic.

The oracle is a plain, slow, obviously correct restatement of the paper's
Algorithm 1 (one correction step) and Algorithm 2 (the parallel scheme) in
float64 with numpy/scipy, following the paper's order and notation.  Library
primitives serve as single steps: sparse matrix products, a dense Cholesky
solve, and the dense generalized symmetric eigensolver (scipy.linalg.eigh).

Every function is pinned by tests against what the paper and mathematics fix
(brute-force dense eigensolves, closed-form continuum eigenvalues, Galerkin
nestedness, fixed points, Ritz upper bounds, multigrid contraction), not
against itself.
"""
from .pasm import (  # noqa: F401
    Problem, coarse_eigenpairs, jacobi, vcycle, bvp_solve, bordering,
    augmented_eigenproblem, correction, initial_state, initial_state_nested, solve,
    SCORE_A, SCORE_B,
)
