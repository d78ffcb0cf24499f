#!/usr/bin/env python
"""Benchmark of the PASM hot path on GB300: eigenpairs/s to 1e-9 relative
eigenvalue error, and the achieved bandwidth / arithmetic rate of the dominant
kernel against the measured peak.

Workload (synthetic, regenerated exactly): -Laplace u = lambda u on the unit
square, P1 elements on the (1,1)-split right-triangle mesh, fine h = 1/1024
(1,046,529 interior DoF), coarse H = 1/16 (225 DoF), 7 grids, k = 64 pairs,
initial pairs = prolongated coarse eigenpairs, damped Jacobi (omega = 2/3,
2 pre / 2 post), 2 V-cycles per correction step, pairs freeze at relative
eigenvalue change < 1e-10.

A step is one correction step (Algorithm 1) for all k pairs: one replay of
the captured CUDA graph.  value = pairs that reach 1e-9 relative error
against the reference eigenvalues (tests/golden, ARPACK shift-invert) divided
by the time of the S steps the slowest of them needs (S from an untimed
calibration run of the same iteration).  Block vectors are 536 MB each, far
above the 129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import os

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import meshgen as mg  # noqa: E402

WORK = {"dim": 2, "N": 1024, "NH": 16, "k": 64, "tol": 1e-10, "target": 1e-9,
        "golden": "square_h1024_k72", "history": "square_h1024_H16_k64_history"}
WORKLOAD_NAME = "unit-square P1 h=1/1024 (1046529 DoF), H=1/16 (225 DoF), 7 grids, k=64"
# the 3D workload (a variant of the bench line): Kuhn P1 on the unit cube
WORK3D = {"dim": 3, "N": 128, "NH": 8, "k": 32, "tol": 1e-10, "target": 1e-9,
          "golden": "cube_h128_k40", "history": "cube_h128_H8_k32_history",
          "stable_history": "cube_h128_H8_k32_nofreeze_history"}
# the h = 1/2048 workload (4,190,209 DoF, H = 1/16, 8 grids, k = 128): its reference table holds the
# 48 smallest eigenvalues, so only pairs 0..47 can be counted; no oracle history at this size
WORK_H2048 = {"dim": 2, "N": 2048, "NH": 16, "k": 128, "tol": 1e-10, "target": 1e-9,
         "golden": "square_h2048_k48", "history": None}
METRIC = "eigenpairs/s to 1e-9 rel. eigenvalue error"
FP64_PEAK_TFLOPS = 1.259   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (measured 1.198)
# kernel classes whose arithmetic is float64 in mixed mode (the V-cycle classes are float32 there)
FP64_CLASSES = ("outer_rhs", "outer_res", "border", "update", "axpy", "secular")


def load_golden(name):
    with open(os.path.join(ROOT, "tests", "golden", name + ".txt")) as f:
        return np.array([float(x) for x in f if not x.startswith("#") and x.strip()])


def load_traffic():
    """Per-launch DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the
    profiled kernels, from the committed ncu summary (profiles/)."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        return json.load(f)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def hierarchy():
    return mg.build_hierarchy(WORK["dim"], WORK["N"], WORK["NH"])


def clusters(ref, gap=1e-4):
    """cluster id of each reference eigenvalue: consecutive values closer than
    `gap` (relative) share a cluster (near-degenerate pairs such as the
    (m, n)/(n, m) modes of the square, split here by 1e-11 .. 1e-9)"""
    cid = np.zeros(len(ref), dtype=int)
    for i in range(1, len(ref)):
        cid[i] = cid[i - 1] + (1 if (ref[i] - ref[i - 1]) / ref[i] > gap else 0)
    return cid


def first_reach(hist, ref, target, ref_all=None):
    """per pair: first step index at which its eigenvalue is within `target`
    (relative) of a reference eigenvalue of its own cluster (or -1)"""
    ref_all = ref if ref_all is None else ref_all
    cid = clusters(ref_all)
    out = np.full(hist.shape[1], -1)
    for i in range(min(hist.shape[1], len(ref_all))):
        members = ref_all[cid == cid[i]]
        err = np.min(np.abs(hist[:, i][:, None] - members[None, :]) / members[None, :], axis=1)
        ok = np.where(err <= target)[0]
        if ok.size:
            out[i] = int(ok[0])
    return out


def reference_set(work=None):
    """the pairs the oracle's own iteration drives to 1e-9 on this workload
    (tests/golden history); None if the table is missing"""
    w = WORK if work is None else work
    if not w.get("history"):
        return None
    p = os.path.join(ROOT, "tests", "golden", w["history"] + ".json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ref_all = load_golden(w["golden"])
    reach = first_reach(np.array(d["history"]), ref_all[:w["k"]], w["target"], ref_all)
    out = np.where(reach >= 0)[0]
    # where the oracle's run without freezing is available, keep only the pairs that are still
    # within the target at its end (stable fixed points of the correction)
    ps = os.path.join(ROOT, "tests", "golden", w.get("stable_history", "") + ".json")
    if w.get("stable_history") and os.path.exists(ps):
        with open(ps) as f:
            last = np.array(json.load(f)["history"])[-1:]
        ok = first_reach(last, ref_all[:w["k"]], w["target"], ref_all) >= 0
        out = np.array([i for i in out if ok[i]], dtype=int)
    return out


def max_over_ranks(torch, x):
    """The maximum of a float over all ranks, then a barrier (the job's time is
    its slowest replica's); the value itself on a single process.  CUDA tensors
    with NCCL, CPU tensors with gloo."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return x
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.barrier()
    return float(t.item())


def job_value(world, converged, steps_to_target, ms_step, start_ms=0.0):
    """Whole-job throughput of N replicas: every rank converges `converged`
    pairs in steps_to_target steps of ms_step (the max over ranks) plus an
    optional start cost, so the job delivers world * converged pairs in that time."""
    return world * converged / ((steps_to_target * ms_step + start_ms) / 1e3)


def time_to_target(reach, refset, cap):
    """(pairs counted, steps S): over the reference set when known -- every set
    pair must reach the target, a missing one costs the whole step cap -- else
    over the pairs that reached it"""
    if refset is None:
        conv = int((reach >= 0).sum())
        return conv, (int(reach.max()) if conv else cap)
    r = reach[refset]
    if np.all(r >= 0):
        return len(refset), int(r.max())
    return int((r >= 0).sum()), cap


# ----------------------------------------------------------------------------- our arm

def run_mode(pg, torch, H, ref, precision, steps, warmup, rank, calib_steps=60, nn_weights=None, init=0,
             smoother=None, nn_widths=None, work=None):
    w = WORK if work is None else work
    k = w["k"]
    stream = torch.cuda.current_stream()
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    t0 = time.perf_counter()
    if smoother is None:
        smoother = 1 if nn_weights is not None else 0
    opts = pg.pasm_default_opts(precision=precision, smoother=smoother, init=init)
    ctx = pg.pasm_setup(A, M, H.P, opts, stream.cuda_stream)
    if nn_weights is not None:
        pg.pasm_nn_setup(ctx, grid_widths(H) if nn_widths is None else nn_widths, nn_weights)
    setup_s = time.perf_counter() - t0
    # cost of the start: a nested start (Algorithm 2 step 2(A)) runs correction steps on the
    # intermediate levels; it is timed as the difference to a coarse start of the same context
    # the first pasm_init of a context runs the tile autotuner (kept for later inits): untimed
    t0 = time.perf_counter()
    pg.pasm_init(ctx, k, w["tol"]); torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    tiles = pg.pasm_tiles(ctx, len(H.levels) - 1)
    init_ms = 0.0
    if init:
        torch.cuda.synchronize()
        t0 = time.perf_counter(); pg.pasm_init(ctx, k, w["tol"]); torch.cuda.synchronize()
        t_nested = time.perf_counter() - t0
        ctx0 = pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(precision=precision), stream.cuda_stream)
        pg.pasm_init(ctx0, k, w["tol"]); torch.cuda.synchronize()
        t0 = time.perf_counter(); pg.pasm_init(ctx0, k, w["tol"]); torch.cuda.synchronize()
        t_coarse = time.perf_counter() - t0
        pg.pasm_destroy(ctx0)
        init_ms = max(0.0, (t_nested - t_coarse) * 1e3)
    # calibration (untimed): iterate from the start, record eigenvalues per step
    pg.pasm_init(ctx, k, w["tol"])
    lam = np.zeros(k)
    hist = [None]
    pg.pasm_get(ctx, lam)
    hist[0] = lam.copy()
    for _ in range(calib_steps):
        act = pg.pasm_step(ctx)
        pg.pasm_get(ctx, lam)
        hist.append(lam.copy())
        if act == 0:
            break
    hist = np.array(hist)
    ref_all = load_golden(w["golden"])
    reach = first_reach(hist, ref, w["target"], ref_all)
    refset = reference_set(w)
    conv, S = time_to_target(reach, refset, calib_steps)
    missed = [] if refset is None else [int(i) for i in refset if reach[i] < 0]
    # the paper's stopping quantity at the end of the calibration run, over the counted pairs
    res = pg.pasm_residuals(ctx)
    counted = np.where(reach >= 0)[0] if refset is None else np.array([i for i in refset if reach[i] >= 0], dtype=int)
    res_max = float(res[counted].max()) if counted.size else None
    launches = pg.pasm_last_launches(ctx)
    # timed: W warm-up steps then exactly K steps of the captured graph
    pg.pasm_init(ctx, k, w["tol"])
    for _ in range(warmup):
        pg.pasm_step_async(ctx)
    torch.cuda.synchronize()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as cs:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            pg.pasm_step_async(ctx)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(torch, e0.elapsed_time(e1))
    ms_step = ms / steps
    # per-kernel-class event timing of a few eager steps (same arithmetic)
    trace = {}
    fine_jacobi = []
    fine_sweep_update = []
    for _ in range(3):
        for name, (t_ms, by, fl, n) in pg.pasm_trace_step(ctx).items():
            a = trace.setdefault(name, [0.0, 0.0, 0.0, 0])
            a[0] += t_ms; a[1] += by; a[2] += fl; a[3] += n
        launches_list = pg.pasm_trace_launches(ctx)
        fine_jacobi += [(t, b) for name, rows, t, b, f in launches_list if name == "jacobi" and rows == H.fine.n]
        fine_sweep_update += [(t, b) for name, rows, t, b, f in launches_list
                              if name == "sweep_update" and rows == H.fine.n]
    accepted = pg.pasm_nn_accepted(ctx, k).tolist() if nn_weights is not None else None
    pg.pasm_destroy(ctx)
    return {"setup_s": setup_s, "S": S, "converged": conv, "reach": reach.tolist(), "ms_per_step": ms_step,
            "launches_per_step": launches, "trace": trace, "clocks": cs.summary(), "final_lam": hist[-1].tolist(),
            "fine_jacobi": fine_jacobi, "accepted": accepted, "init_ms": init_ms, "missed": missed,
            "tiles": tiles, "first_init_s": tune_s, "fine_sweep_update": fine_sweep_update,
            "residual_max": res_max,
            "reached_outside_set": [int(i) for i in np.where(reach >= 0)[0]
                                    if refset is not None and i not in set(refset.tolist())]}


def init_weights(seed):
    """He-style random start of the 2592 smoother weights (last layer scaled by 0.1)."""
    rng = np.random.default_rng(seed)
    shapes = ((3, 3, 1, 16), (3, 3, 16, 16), (3, 3, 16, 1))
    out = []
    for i, sh in enumerate(shapes):
        w = rng.standard_normal(sh) * np.sqrt(2.0 / (sh[0] * sh[1] * sh[2]))
        out.append(w * (0.1 if i == 2 else 1.0))
    return np.concatenate([x.ravel() for x in out]).astype(np.float32)


def grid_widths(H):
    return np.array([lv.N - 1 for lv in H.levels], dtype=np.int32)


def train_smoother(pg, torch, H, epochs=10, iters=20, lr=3e-3):
    """Train the learned post-smoother on residuals the method's own first
    V-cycles produce on this workload (captured on the level with h = 4 h_fine;
    the network is h-independent), from the coarse start and two later steps."""
    k = WORK["k"]
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    ctx = pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(precision=1), torch.cuda.current_stream().cuda_stream)
    pg.pasm_nn_setup(ctx, grid_widths(H), init_weights(0))
    lvl = len(H.levels) - 3
    t0 = time.perf_counter()
    pg.pasm_init(ctx, k, WORK["tol"])
    batches = []
    for _ in range(3):
        R = np.zeros((H.levels[lvl].n, k), dtype=np.float32)
        pg.pasm_nn_capture_residuals(ctx, lvl, R)
        batches.append(R)
        pg.pasm_step(ctx)
    losses = []
    for _ in range(epochs):
        for R in batches:
            losses.append(float(pg.pasm_nn_train(ctx, lvl, R, iters, lr)[-1]))
    w = pg.pasm_nn_get_weights(ctx)
    pg.pasm_destroy(ctx)
    return w, time.perf_counter() - t0, losses


def run_e2e(pg, torch, H, S, precision):
    """End to end through pasm_solve with host buffers: the initial pairs go in
    from pinned host memory, the eigenpairs come back to pinned host memory."""
    k = WORK["k"]
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    ctx = pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(precision=precision, max_steps=S),
                        torch.cuda.current_stream().cuda_stream)
    n = H.fine.n
    pg.pasm_init(ctx, k, WORK["tol"])
    lam0 = torch.zeros(k, dtype=torch.float64).pin_memory()
    U0 = torch.zeros((n, k), dtype=torch.float64).pin_memory()
    pg.pasm_get(ctx, lam0.numpy(), U0.numpy())
    lam = torch.zeros(k, dtype=torch.float64).pin_memory()
    U = torch.zeros((n, k), dtype=torch.float64).pin_memory()
    steps = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    pg.pasm_solve(ctx, k, WORK["tol"], lam0.numpy(), U0.numpy(), lam.numpy(), U.numpy(), steps, status)  # warm
    torch.cuda.synchronize()
    times = []
    for _ in range(3):     # median of three solves
        t0 = time.perf_counter()
        pg.pasm_solve(ctx, k, WORK["tol"], lam0.numpy(), U0.numpy(), lam.numpy(), U.numpy(), steps, status)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    pg.pasm_destroy(ctx)
    nbytes_in = (n * k + k) * 8
    nbytes_out = (n * k + k) * 8 + 2 * k * 4
    return dt, nbytes_in, nbytes_out


def oracle_sample(H, k_sample, n_steps):
    """CPU baseline: the oracle (test infrastructure) on a bounded sample of the
    same workload -- k_sample pairs for n_steps correction steps."""
    import oracle
    prob = oracle.Problem.from_hierarchy(H)
    lam, U = oracle.initial_state(prob, k_sample)
    t0 = time.perf_counter()
    for _ in range(n_steps):
        lam, U, _ = oracle.correction(prob, lam, U)
    return (time.perf_counter() - t0) / n_steps


def reference_counts():
    """steps to 1e-9 and converged pairs of the oracle's own iteration on the
    full workload (tests/golden, written by the oracle)."""
    p = os.path.join(ROOT, "tests", "golden", WORK["history"] + ".json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ref_all = load_golden(WORK["golden"])
    reach = first_reach(np.array(d["history"]), ref_all[:WORK["k"]], WORK["target"], ref_all)
    conv = int((reach >= 0).sum())
    return (int(reach.max()) if conv else len(d["history"]) - 1), conv


def main_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    from paper_1908_10251_gb300 import build
    build.build()
    import paper_1908_10251_gb300 as pg
    H = hierarchy()
    ref = load_golden(WORK["golden"])[:WORK["k"]]
    res = {}
    modes = {"both": (("mixed", 1), ("fp64", 0)), "mixed": (("mixed", 1),), "fp64": (("fp64", 0),)}[args.mode]
    for name, prec in modes:
        res[name] = run_mode(pg, torch, H, ref, prec, args.steps, args.warmup, rank, args.calib_steps)
    res["mixed_nested"] = run_mode(pg, torch, H, ref, 1, args.steps, args.warmup, rank, args.calib_steps, init=1)
    # the smoother of the paper's experiments (Section 5.1): 2 CG steps pre and post
    res["mixed_cg"] = run_mode(pg, torch, H, ref, 1, args.steps, args.warmup, rank, args.calib_steps, smoother=2)
    # the 3D workload: Kuhn P1 on the cube, h = 1/128 (2,048,383 DoF), H = 1/8 (343), k = 32, mixed
    if not args.no_3d:
        H3 = mg.build_hierarchy(3, WORK3D["N"], WORK3D["NH"])
        ref3 = load_golden(WORK3D["golden"])[:WORK3D["k"]]
        res["cube_h128_H8_k32_mixed"] = run_mode(pg, torch, H3, ref3, 1, args.steps, args.warmup, rank,
                                                 args.calib_steps, work=WORK3D)
        del H3
    # the h = 1/2048, k = 128 workload (when its reference table is present)
    H2048 = None
    if not args.no_h2048 and os.path.exists(os.path.join(ROOT, "tests", "golden", WORK_H2048["golden"] + ".txt")):
        H2048 = mg.build_hierarchy(WORK_H2048["dim"], WORK_H2048["N"], WORK_H2048["NH"])
        ref2048 = load_golden(WORK_H2048["golden"])
        res["square_h2048_H16_k128_mixed"] = run_mode(pg, torch, H2048, ref2048, 1, args.steps, args.warmup, rank,
                                                      args.calib_steps, work=WORK_H2048)
    training = None
    if args.learned:
        w, train_s, losses = train_smoother(pg, torch, H)
        res["mixed_learned"] = run_mode(pg, torch, H, ref, 1, args.steps, args.warmup, rank, args.calib_steps,
                                        nn_weights=w)
        # the learned step only on the grids up to h = 4 h_fine (the two finest levels keep Jacobi)
        coarse = grid_widths(H)
        coarse[-2:] = 0
        res["mixed_learned_coarse"] = run_mode(pg, torch, H, ref, 1, args.steps, args.warmup, rank,
                                               args.calib_steps, nn_weights=w, nn_widths=coarse)
        if H2048 is not None:
            # the same network (the 2D stencil is h-independent) on the h = 1/2048 workload
            coarse2048 = grid_widths(H2048)
            coarse2048[-2:] = 0
            res["square_h2048_H16_k128_learned_coarse"] = run_mode(
                pg, torch, H2048, load_golden(WORK_H2048["golden"]), 1, args.steps, args.warmup, rank, args.calib_steps,
                nn_weights=w, nn_widths=coarse2048, work=WORK_H2048)
        training = {"seconds": train_s, "loss_first": losses[0], "loss_last": losses[-1]}
    H2048 = None
    primary, primary_prec = modes[0]
    main = res[primary]
    S, conv, ms_step = main["S"], main["converged"], main["ms_per_step"]
    value = job_value(world, conv, S, ms_step)
    if args.no_e2e:
        e2e_s, bin_, bout, e2e_value = None, 0, 0, None
    else:
        e2e_s, bin_, bout = run_e2e(pg, torch, H, S, primary_prec)
        e2e_value = world * conv / e2e_s
    # dominant kernel class of the primary mode
    tr = main["trace"]
    dom = max(tr, key=lambda q: tr[q][0])
    d_ms, d_bytes, d_flops, d_n = tr[dom]
    hbm, peak_kind = load_peaks()
    gbs = d_bytes / (d_ms * 1e-3) / 1e9
    tfs = d_flops / (d_ms * 1e-3) / 1e12
    fp64_heavy = dom in FP64_CLASSES and tfs / FP64_PEAK_TFLOPS > gbs / hbm
    if fp64_heavy:
        ach = tfs
        roof = {"bound": "alu", "kernel": dom, "achieved": round(ach, 4), "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s (fp64)", "frac": round(ach / FP64_PEAK_TFLOPS, 4), "traffic": None,
                "achieved_gbs": round(d_bytes / (d_ms * 1e-3) / 1e9, 1),
                "peak_note": "fp64 FMA peak derived from 2 FMA/clk/SM x 152 SMs x 2.07 GHz"}
    else:
        ach = d_bytes / (d_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": None, "peak_note": "of %s" % peak_kind}
    roof["launches_per_step"] = d_n / 3.0
    roof["avg_launch_us"] = round(d_ms / d_n * 1e3, 2)
    prof = load_traffic()
    if dom in prof:
        roof["traffic"] = prof[dom]["dram_bytes_per_launch"]
        roof["traffic_source"] = prof[dom]["source"]
    dominant_class = roof
    # the V-cycle's own roofline: finest-level float32 Jacobi sweeps (the metric's "V-cycle HBM GB/s")
    # finest-level k_rowop Jacobi sweeps only (the fused two-sweep kernel of the same class moves
    # fewer algorithmic bytes per launch and is left out)
    fj = main["fine_jacobi"]
    if fj:
        bmax = max(b for _, b in fj)
        fj = [(t, b) for t, b in fj if b >= 0.99 * bmax]
    vcyc = None
    if fj:
        t_avg = sum(t for t, _ in fj) / len(fj)
        b_avg = sum(b for _, b in fj) / len(fj)
        ach = b_avg / (t_avg * 1e-3) / 1e9
        vcyc = {"bound": "hbm", "kernel": "k_rowop<float,JACOBI> finest level", "achieved": round(ach, 1),
                "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4), "avg_launch_us": round(t_avg * 1e3, 1),
                "algorithmic_bytes_per_launch": b_avg,
                "traffic": prof.get("jacobi_fine", {}).get("dram_bytes_per_launch"),
                "launches_timed": len(fj), "peak_note": "of %s" % peak_kind}
    # the fused last sweep + outer update (k_jacobi_axpy_ff), finest level
    fsu = main.get("fine_sweep_update") or []
    sweep_update = None
    if fsu:
        t_avg = sum(t for t, _ in fsu) / len(fsu)
        b_avg = sum(b for _, b in fsu) / len(fsu)
        ach = b_avg / (t_avg * 1e-3) / 1e9
        sweep_update = {"bound": "hbm", "kernel": "k_jacobi_axpy_ff finest level (last sweep + x += e)",
                        "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                        "avg_launch_us": round(t_avg * 1e3, 1), "algorithmic_bytes_per_launch": b_avg,
                        "traffic": prof.get("sweep_update_fine", {}).get("dram_bytes_per_launch"),
                        "launches_timed": len(fsu), "peak_note": "of measured"}
    # the reported roofline kernel: the finest-level float32 Jacobi sweep, the V-cycle kernel the
    # metric names and the largest HBM-bound kernel of the step; the dominant class stays alongside
    roof = dict(vcyc) if vcyc else dominant_class
    if vcyc:
        roof["traffic_source"] = prof.get("jacobi_fine", {}).get("source")
        roof["launches_per_step"] = round(len(fj) / 3.0, 2)
    classes = {q: {"ms_per_step": round(v[0] / 3, 4), "GBps": round(v[1] / (v[0] * 1e-3) / 1e9, 1) if v[0] else 0,
                   "GFLOPs": round(v[2] / (v[0] * 1e-3) / 1e9, 1) if v[0] else 0, "launches": v[3] // 3}
               for q, v in sorted(tr.items(), key=lambda kv: -kv[1][0])}
    # CPU baseline (oracle), bounded sample on rank 0
    cpu = None
    if rank == 0 and not args.no_cpu:
        ks = 2
        t_step = oracle_sample(H, ks, 1)
        cpu_val = conv / ((WORK["k"] / ks) * S * t_step)
        cpu = {"value": cpu_val, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle",
               "sample": "oracle correction step on %d of %d pairs of the same workload, 1 step (%.1f s); "
                         "scaled by k/%d x S=%d steps" % (ks, WORK["k"], t_step, ks, S)}
    out = {
        "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if primary == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME,
                   "precision": ("mixed: f32 V-cycles under double-float (f32 pair) outer residuals"
                                 if primary == "mixed" else "f64"),
                   "pairs_converged": conv, "pairs": WORK["k"], "steps_to_1e-9": S,
                   "pair_set": "the pairs the float64 oracle drives to 1e-9 on this workload (cluster-aware)",
                   "missed": main["missed"],
                   "eigen_residual_max": main["residual_max"],
                   "l2": "inputs larger than L2 (536 MB block vectors)", "parallelism": "replicas",
                   "tiles_finest": {kk: v for kk, v in main["tiles"].items() if v},
                   "first_init_s": round(main["first_init_s"], 3)},
        "e2e": {"value": e2e_value, "unit": "eigenpairs/s", "h2d_bytes_per_step": bin_ // max(S, 1),
                "d2h_bytes_per_step": bout // max(S, 1), "seconds": e2e_s,
                "note": "pasm_solve with pinned host inputs/outputs, S steps per call"},
        "roofline": roof,
        "roofline_dominant_class": dominant_class,
        "roofline_sweep_update": sweep_update,
        "smoother_training": training,
        "cpu_baseline": cpu,
        "gpu_launches": int(args.steps * main["launches_per_step"]),
        "clocks": main["clocks"],
        "kernels": classes,
        "variants": {name: {"value": job_value(world, r["converged"], r["S"], r["ms_per_step"], r["init_ms"]),
                            "ms_per_step": r["ms_per_step"], "steps_to_1e-9": r["S"], "init_ms": r["init_ms"],
                            "pairs_converged": r["converged"], "missed": r["missed"], "clocks": r["clocks"],
                            "eigen_residual_max": r["residual_max"],
                            "learned_steps_accepted": r["accepted"]}
                     for name, r in res.items() if name != primary},
        "setup_s": main["setup_s"],
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def main_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    H = hierarchy()
    counts = reference_counts()
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration history table missing"}))
        return
    S, conv = counts
    ks = 2
    times = [oracle_sample(H, ks, 1) for _ in range(max(args.steps, 1))]
    t_step = statistics.median(times)
    value = conv / ((WORK["k"] / ks) * S * t_step)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 * WORK["k"] / ks,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "precision": "f64 oracle", "pairs_converged": conv,
                   "steps_to_1e-9": S},
        "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle",
                         "sample": "%d of %d pairs per step, %d steps; scaled by k/%d x S" % (ks, WORK["k"],
                                                                                              len(times), ks)},
        "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--mode", default="both", choices=["both", "mixed", "fp64"],
                    help="precision modes to run (the first one listed is the primary)")
    ap.add_argument("--calib-steps", type=int, default=60, help="step cap of the calibration run")
    ap.add_argument("--learned", dest="learned", action="store_true", default=True,
                    help="also train the learned post-smoother and run the mixed mode with it (default)")
    ap.add_argument("--no-learned", dest="learned", action="store_false")
    ap.add_argument("--no-3d", dest="no_3d", action="store_true", help="skip the 3D workload variant")
    ap.add_argument("--no-h2048", dest="no_h2048", action="store_true", help="skip the h = 1/2048, k = 128 variant")
    args = ap.parse_args()
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
