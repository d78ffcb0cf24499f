"""How many of k pairs does the oracle's PASM converge, and under which settings?

A study on a reduced analogue of the paper's Example 1 (Section 5.1: the unit
cube, H = 1/16, 200 or 1000 pairs): Kuhn P1 on the unit cube, h = 1/32
(29,791 interior DoF), H = 1/8 (N_H = 343), k = 100 pairs, so N_H / k = 3.4 as
in Example 1 with 1000 pairs (N_H = 15^3 = 3375).  Calls only meshgen and
oracle/ (test infrastructure); the reference eigenvalues come from ARPACK
shift-invert (oracle.reference).  Writes tests/golden/convergence_study.json.

Settings (the oracle's PASM, float64, pairs run independently):
  base     two V-cycles per step, damped Jacobi omega = 2/3, 2 pre / 2 post,
           selection by the a-normalised score, pairs freeze at
           |d lambda| / lambda < 1e-10 (the workload's configuration);
  paper    the paper's Section 5.1 settings: one V-cycle with 2 CG steps pre and
           post, pairs stop at ||A x - lambda M x||_2 / |lambda| <= 1e-8 with x
           M-normalised;
  score_b  as base with the b-normalised selection score;
  finer_H  as base with H = 1/16 (N_H = 3375, N_H / k = 34).

For each setting and pair: the first step within 1e-9 (relative) of a
reference eigenvalue of its own cluster (consecutive reference values closer
than 1e-4 relative), the error at the end, the step and error at which the
paper's residual test was first met.  At the end the pairs within 1e-9 are
checked for distinct slots: no cluster holds more such pairs than it has
eigenvalues, and the final vectors of the pairs of one cluster are linearly
independent (smallest singular value of their M-Gram matrix, vectors
M-normalised, above 1e-3).

Run: python tests/golden/convergence_study.py [setting ...] [--procs P]
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

DIM, N_FINE, K = 3, 32, 100
TARGET = 1e-9
SETTINGS = {
    # name: (N_coarse, Problem keyword arguments, stop rule, max steps)
    "base": (8, {}, "dlambda", 40),
    "paper": (8, {"cycles": 1, "smoother": "cg"}, "residual", 40),
    "score_b": (8, {"score": 1}, "dlambda", 40),
    "finer_H": (16, {}, "dlambda", 20),
}


def clusters(ref, gap=1e-4):
    import numpy as np
    cid = np.zeros(len(ref), dtype=int)
    for i in range(1, len(ref)):
        cid[i] = cid[i - 1] + (1 if (ref[i] - ref[i - 1]) / ref[i] > gap else 0)
    return cid


def cluster_error(lam, ref, cid, i):
    """relative distance of lam to the reference eigenvalues of pair i's cluster"""
    import numpy as np
    mem = ref[cid == cid[i]]
    return float(np.min(np.abs(lam - mem) / mem))


def _worker(args):
    """Run the correction steps of one chunk of pairs; returns per-pair histories
    of the eigenvalue and of the paper's relative residual, and the final vectors."""
    name, cols = args
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    import numpy as np

    import meshgen as mg
    import oracle
    from oracle import pasm as op
    Nc, kw, stop, max_steps = SETTINGS[name]
    H = mg.build_hierarchy(DIM, N_FINE, Nc)
    prob = oracle.Problem.from_hierarchy(H, **kw)
    lam_all, U_all = oracle.initial_state(prob, K)
    lam, U = lam_all[cols].copy(), U_all[:, cols].copy()
    A, M = H.fine.A, H.fine.M

    def residual(lam, U):
        Un = U / np.sqrt(np.einsum("ij,ij->j", U, M @ U))
        R = A @ Un - (M @ Un) * lam[None, :]
        return np.linalg.norm(R, axis=0) / np.abs(lam)

    active = np.ones(len(cols), dtype=bool)
    hl, hr = [lam.copy()], [residual(lam, U)]
    for _ in range(max_steps):
        if not active.any():
            break
        lam_new, U, _ = op.correction(prob, lam, U, active)
        res = residual(lam_new, U)
        if stop == "dlambda":
            done = np.abs(lam_new - lam) < 1e-10 * np.abs(lam_new)
        else:
            done = res <= 1e-8
        lam = lam_new
        active &= ~done
        hl.append(lam.copy())
        hr.append(res)
    return cols, np.array(hl), np.array(hr), U


def run(name, procs, ref):
    import numpy as np

    import meshgen as mg
    t0 = time.time()
    chunks = [list(range(K))[p::procs] for p in range(procs)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        outs = pool.map(_worker, [(name, c) for c in chunks])
    steps = max(o[1].shape[0] for o in outs)
    hl = np.full((steps, K), np.nan)
    hr = np.full((steps, K), np.nan)
    U = None
    for cols, l, r, Uc in outs:
        # a frozen pair keeps its value: pad its history with the last row
        l = np.vstack([l, np.repeat(l[-1:], steps - l.shape[0], axis=0)])
        r = np.vstack([r, np.repeat(r[-1:], steps - r.shape[0], axis=0)])
        hl[:, cols] = l
        hr[:, cols] = r
        if U is None:
            U = np.zeros((Uc.shape[0], K))
        U[:, cols] = Uc
    cid = clusters(ref)
    err = np.array([[cluster_error(hl[s, i], ref, cid, i) for i in range(K)] for s in range(steps)])
    first = [int(np.argmax(err[:, i] <= TARGET)) if (err[:, i] <= TARGET).any() else -1 for i in range(K)]
    final_ok = err[-1] <= TARGET
    # distinct slots among the pairs within the target at the end
    M = mg.build_hierarchy(DIM, N_FINE, SETTINGS[name][0]).fine.M
    dup = []
    for c in np.unique(cid[:K]):
        mem = [i for i in range(K) if final_ok[i] and cid[i] == c]
        size = int((cid == c).sum())
        if not mem:
            continue
        X = U[:, mem] / np.sqrt(np.einsum("ij,ij->j", U[:, mem], M @ U[:, mem]))
        smin = float(np.linalg.svd(X.T @ (M @ X), compute_uv=False).min()) if len(mem) > 1 else 1.0
        if len(mem) > size or smin < 1e-3:
            dup.append({"cluster_pairs": mem, "cluster_size": size, "gram_smin": smin})
    res_first = [int(np.argmax(hr[:, i] <= 1e-8)) if (hr[:, i] <= 1e-8).any() else -1 for i in range(K)]
    res_err = [float(err[s, i]) if s >= 0 else None for i, s in enumerate(res_first)]
    out = {
        "setting": name, "N_coarse": SETTINGS[name][0], "problem": SETTINGS[name][1], "stop": SETTINGS[name][2],
        "max_steps": SETTINGS[name][3], "steps_run": steps - 1, "seconds": time.time() - t0,
        "reached_1e-9": int(sum(f >= 0 for f in first)), "final_within_1e-9": int(final_ok.sum()),
        "final_distinct_violations": dup,
        "met_residual_1e-8": int(sum(s >= 0 for s in res_first)),
        "met_residual_and_within_1e-9": int(sum(1 for e in res_err if e is not None and e <= TARGET)),
        "met_residual_and_within_1e-6": int(sum(1 for e in res_err if e is not None and e <= 1e-6)),
        "first_step_within_1e-9": first, "final_error": [float(v) for v in err[-1]],
        "first_step_residual_1e-8": res_first, "error_when_residual_met": res_err,
    }
    return out


def main():
    import numpy as np

    import meshgen as mg
    from oracle.reference import smallest_eigenvalues
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    procs = 6
    for a in sys.argv[1:]:
        if a.startswith("--procs="):
            procs = int(a.split("=")[1])
    names = args or list(SETTINGS)
    path = os.path.join(HERE, "convergence_study.json")
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    if "reference" not in data:
        A, M = mg.assemble(DIM, N_FINE)
        data["reference"] = [float(v) for v in smallest_eigenvalues(A, M, K + 16)]
    ref = np.array(data["reference"])
    data["workload"] = {"dim": DIM, "N_fine": N_FINE, "k": K, "target": TARGET,
                        "reference": "ARPACK shift-invert, %d smallest eigenvalues" % len(ref)}
    for name in names:
        data.setdefault("settings", {})[name] = run(name, procs, ref)
        r = data["settings"][name]
        print(name, "reached %d, final %d, residual-met %d (within 1e-9: %d), %.0fs" % (
            r["reached_1e-9"], r["final_within_1e-9"], r["met_residual_1e-8"], r["met_residual_and_within_1e-9"],
            r["seconds"]), flush=True)
        with open(path, "w") as f:
            json.dump(data, f)


if __name__ == "__main__":
    main()
