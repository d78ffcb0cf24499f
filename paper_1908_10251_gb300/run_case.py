"""Run a few PASM correction steps on one synthetic mesh and print the
per-kernel-class event times of one eager step: the small, self-contained
workload that profiler captures wrap.

    python -m paper_1908_10251_gb300.run_case --dim 2 --N 512 --NH 16 --k 64 --steps 3

The mesh is the P1 Laplacian hierarchy of the unit square (dim 2) or the Kuhn
cube (dim 3), every dyadic grid from 1/NH to 1/N; the start is the
prolongated coarse eigenpairs.  The steps replay the captured step graph, as
the solver does.
"""
import argparse
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--N", type=int, default=512, help="fine grid: h = 1/N")
    ap.add_argument("--NH", type=int, default=16, help="coarse grid: H = 1/NH")
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--smoother", default="jacobi", choices=["jacobi", "cg"])
    ap.add_argument("--launches", action="store_true", help="also list every launch of the traced step")
    ap.add_argument("--learned", action="store_true",
                    help="mixed precision with the learned post-smoothing step on every 2D grid (seeded random weights)")
    args = ap.parse_args(argv)

    import torch
    import meshgen as mg
    import paper_1908_10251_gb300 as pg

    pg.load_library()
    H = mg.build_hierarchy(args.dim, args.N, args.NH)
    stream = torch.cuda.current_stream()
    opts = pg.pasm_default_opts(precision=pg.PASM_MIXED if args.precision == "mixed" else pg.PASM_FP64,
                                smoother=pg.PASM_CG if args.smoother == "cg" else pg.PASM_JACOBI)
    if args.learned:
        opts = pg.pasm_default_opts(precision=pg.PASM_MIXED, smoother=1)
    ctx = pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P, opts, stream.cuda_stream)
    if args.learned:
        # He-style random weights of the 1 -> 16 -> 16 -> 1 network (the kernels' cost does not depend on them)
        rng = np.random.default_rng(0)
        w = [rng.standard_normal(sh) * np.sqrt(2.0 / (sh[0] * sh[1] * sh[2]))
             for sh in ((3, 3, 1, 16), (3, 3, 16, 16), (3, 3, 16, 1))]
        w[2] *= 0.1
        pg.pasm_nn_setup(ctx, np.array([lv.N - 1 for lv in H.levels], dtype=np.int32),
                         np.concatenate([x.ravel() for x in w]).astype(np.float32))
    pg.pasm_init(ctx, args.k, 0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pg.pasm_step_async(ctx)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / max(args.steps, 1) * 1e3
    lam = np.zeros(args.k)
    pg.pasm_get(ctx, lam)
    stats = pg.pasm_secular_stats(ctx)
    trace = pg.pasm_trace_step(ctx)
    launches = pg.pasm_trace_launches(ctx) if args.launches else []
    pg.pasm_destroy(ctx)
    print("n=%d k=%d %s: %.3f ms per step (wall); lambda_1 = %.12g" % (H.fine.n, args.k, args.precision, wall,
                                                                          lam[0]))
    print("secular: %d window roots, %d failed certificates, %d capped iterations over %d steps"
          % (stats + (args.steps,)))
    for name, (t_ms, by, fl, n) in sorted(trace.items(), key=lambda kv: -kv[1][0]):
        print("  %-14s %3d launches %8.3f ms %8.1f GB/s" % (name, n, t_ms, by / max(t_ms, 1e-9) / 1e6))
    for name, rows, t_ms, by, fl in launches:
        print("    %-14s rows %9d %9.1f us %8.1f GB/s" % (name, rows, t_ms * 1e3, by / max(t_ms, 1e-9) / 1e6))


if __name__ == "__main__":
    main()
