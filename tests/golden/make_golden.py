"""Write the reference eigenvalue tables under tests/golden/ (calls only
meshgen and oracle/).  Run: python tests/golden/make_golden.py [name ...]

Run: python tests/golden/make_golden.py [name ...] [--procs=P]  (P processes
split the pairs of an iteration history; pairs are independent.)

Each table holds the smallest discrete eigenvalues of one synthetic workload
(the P1 pencil of Section 2 on the named mesh), from oracle.reference
(ARPACK shift-invert in 2D; in 3D, where the factorisation of the 2M-DoF
matrix does not fit in memory, LOBPCG with a multigrid preconditioner, checked
against shift-invert on the 32^3 and 64^3 meshes; for the largest 2D mesh,
ARPACK shift-invert with the exact sine-transform inverse of the stiffness), one value per line with %.17g."""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import meshgen as mg  # noqa: E402
from oracle.reference import smallest_eigenvalues, smallest_eigenvalues_lobpcg, smallest_eigenvalues_sine  # noqa: E402

TABLES = {
    # name: (dim, N_fine, count, method)
    "square_h1024_k72": (2, 1024, 72, "shift-invert"),
    "square_h64_k16": (2, 64, 16, "shift-invert"),
    "cube_h128_k40": (3, 128, 40, "lobpcg"),
    "square_h2048_k48": (2, 2048, 48, "lobpcg"),
    "square_h2048_k136": (2, 2048, 136, "sine"),
}


def write(name):
    dim, N, count, method = TABLES[name]
    t = time.time()
    if method == "sine":
        vals = smallest_eigenvalues_sine(dim, N, count)
        how = "ARPACK shift-invert, exact sine-transform inverse of the stiffness"
    elif method == "lobpcg":
        Nc = 8 if dim == 3 else 16     # a coarse space large enough to seed count + 8 vectors
        vals, res = smallest_eigenvalues_lobpcg(mg.build_hierarchy(dim, N, Nc), count, tol=1e-9)
        how = "LOBPCG, multigrid preconditioner, max relative residual %.1e" % res
    else:
        A, M = mg.assemble(dim, N)
        vals = smallest_eigenvalues(A, M, count)
        how = "ARPACK shift-invert"
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write("# smallest eigenvalues of the P1 pencil, dim=%d, h=1/%d, %d values\n" % (dim, N, count))
        f.write("# written by tests/golden/make_golden.py via oracle.reference (%s)\n" % how)
        for v in vals:
            f.write("%.17g\n" % v)
    print(name, "%.1fs" % (time.time() - t), flush=True)


HISTORIES = {
    # name: (dim, N_fine, N_coarse, k, tol, max_steps, nested start)
    "square_h64_H8_k8_history": (2, 64, 8, 8, 1e-10, 60, False),
    "square_h64_H8_k8_nofreeze_history": (2, 64, 8, 8, 0.0, 40, False),
    "square_h1024_H16_k64_history": (2, 1024, 16, 64, 1e-10, 40, False),
    "square_h1024_H16_k64_nested_history": (2, 1024, 16, 64, 1e-10, 40, True),
    "cube_h128_H8_k32_history": (3, 128, 8, 32, 1e-10, 30, False),
    # no freezing (tol 0): shows which converged pairs are stable fixed points of the correction
    "cube_h128_H8_k32_nofreeze_history": (3, 128, 8, 32, 0.0, 40, False),
    "square_h1024_H16_k64_nofreeze_history": (2, 1024, 16, 64, 0.0, 40, False),
    # h = 1/2048: the pairs of the clusters the vector check covers (0..41)
    "square_h2048_H16_k42_history": (2, 2048, 16, 42, 1e-10, 40, False),
    "square_h2048_H16_k42_nofreeze_history": (2, 2048, 16, 42, 0.0, 40, False),
}


def _history_chunk(args):
    """The oracle's iteration for one chunk of pairs (pairs are independent,
    Section 3.2): eigenvalue history and per-pair step counts."""
    name, cols = args
    import oracle
    dim, N, Nc, k, tol, max_steps, nested = HISTORIES[name]
    H = mg.build_hierarchy(dim, N, Nc)
    prob = oracle.Problem.from_hierarchy(H)
    lam0, U0 = (oracle.pasm.initial_state_nested if nested else oracle.initial_state)(prob, k)
    lam, U, steps, hist = oracle.solve(prob, len(cols), tol=tol, max_steps=max_steps, history=True,
                                       lam0=lam0[cols], U0=U0[:, cols])
    return cols, [list(map(float, row)) for row in hist], [int(v) for v in steps]


def write_history(name, procs=1):
    """Eigenvalue iterates of the oracle's PASM (float64, coarse initial pairs,
    two V-cycles per step) on one workload: one row per step, one column per
    pair; pairs freeze once their relative change is below tol.  With procs >
    1 the pairs are split over that many processes (spawned)."""
    import json
    dim, N, Nc, k, tol, max_steps, nested = HISTORIES[name]
    t = time.time()
    procs = max(1, min(procs, k))
    chunks = [list(range(k))[p::procs] for p in range(procs)]
    if procs == 1:
        outs = [_history_chunk((name, chunks[0]))]
    else:
        import multiprocessing as mp
        # one BLAS thread per worker (the spawned interpreters read this when they import numpy)
        os.environ["OPENBLAS_NUM_THREADS"] = "1"
        os.environ["OMP_NUM_THREADS"] = "1"
        with mp.get_context("spawn").Pool(procs) as pool:
            outs = pool.map(_history_chunk, [(name, c) for c in chunks])
    rows = max(len(h) for _, h, _ in outs)
    hist = [[0.0] * k for _ in range(rows)]
    steps = [0] * k
    for cols, h, st in outs:
        for r in range(rows):
            row = h[min(r, len(h) - 1)]          # a chunk that stopped early keeps its last values
            for j, c in enumerate(cols):
                hist[r][c] = row[j]
        for j, c in enumerate(cols):
            steps[c] = st[j]
    out = {"dim": dim, "N_fine": N, "N_coarse": Nc, "k": k, "tol": tol, "max_steps": max_steps, "nested": nested,
           "steps": steps, "history": hist, "seconds": time.time() - t}
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f)
    print(name, "%.1fs" % (time.time() - t), flush=True)


if __name__ == "__main__":
    procs = 1
    names = []
    for a in sys.argv[1:]:
        if a.startswith("--procs="):
            procs = int(a.split("=")[1])
        else:
            names.append(a)
    for n in (names or list(TABLES) + list(HISTORIES)):
        if n in HISTORIES:
            write_history(n, procs)
        else:
            write(n)
