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

# tol = the freeze threshold of the GPU runs: a pair stops at |d lambda| / lambda < tol.  1e-10 stops
# the vectors at M-principal angles up to ~1e-5, above the 1e-6 the counting rule asks for; with no
# freezing at all (0) the fp32 noise of mixed precision slowly rotates the pairs of near-degenerate
# clusters away; 1e-13 freezes a pair once its eigenvalue sits at the rounding floor (angles measured
# below 4e-7 on this workload)
WORK = {"dim": 2, "N": 1024, "NH": 16, "k": 64, "tol": 1e-13, "target": 1e-9,
        "golden": "square_h1024_k72", "history": "square_h1024_H16_k64_history",
        "stable_history": "square_h1024_H16_k64_nofreeze_history"}
WORKLOAD_NAME = "unit-square P1 h=1/1024 (1046529 DoF), H=1/16 (225 DoF), 7 grids, k=64"
# the 3D workload (a variant of the bench line): Kuhn P1 on the unit cube
WORK3D = {"dim": 3, "N": 128, "NH": 8, "k": 32, "tol": 1e-13, "target": 1e-9,
          "golden": "cube_h128_k40", "history": "cube_h128_H8_k32_history",
          "stable_history": "cube_h128_H8_k32_nofreeze_history"}
# the h = 1/2048 workload (4,190,209 DoF, H = 1/16, 8 grids, k = 128): its reference table holds the
# 136 smallest eigenvalues (every pair can be judged); the oracle's histories cover pairs 0..41 (the
# higher ones do not converge with this coarse space), so its reference set is the stable pairs among them
WORK_H2048 = {"dim": 2, "N": 2048, "NH": 16, "k": 128, "tol": 1e-13, "target": 1e-9,
              "golden": "square_h2048_k136", "history": "square_h2048_H16_k42_history",
              "stable_history": "square_h2048_H16_k42_nofreeze_history"}
# the small latency-bound workload: unit square h = 1/64 (3969 DoF), H = 1/8 (49), 4 grids, k = 8,
# float64, pairs judged at 1e-10 (its stop rule is |d lambda| / lambda < 1e-10)
WORK_C1 = {"dim": 2, "N": 64, "NH": 8, "k": 8, "tol": 1e-13, "target": 1e-10, "stop_tol": 1e-10,
           "golden": "square_h64_k16", "history": "square_h64_H8_k8_history",
           "stable_history": "square_h64_H8_k8_nofreeze_history"}
METRIC = "eigenpairs/s to 1e-9 rel. eigenvalue error"
FP64_PEAK_TFLOPS = 1.259   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (measured 1.198)
# kernel classes whose arithmetic is float64 in mixed mode (the V-cycle classes are float32 there)
FP64_CLASSES = ("outer_rhs", "outer_res", "border", "update", "axpy", "secular")


_T0 = time.perf_counter()


def log(msg):
    """Progress of the bench run on stderr (the JSON line stays alone on stdout)."""
    print("[bench %7.1fs] %s" % (time.perf_counter() - _T0, msg), file=sys.stderr, flush=True)


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


ANGLE_MAX = 1e-6
_REFERENCE_PAIRS = {}


class VectorCheck:
    """The vector part of the bench's counting rule for one workload: reference
    eigenvectors (ARPACK shift-invert with the exact sine-transform A^{-1} of
    the constant-coefficient stiffness; computed once per workload and kept),
    then per call the accuracy report of the pairs `pset` (eigenvalue within
    the target of their own cluster, distinct slots, largest M-principal angle
    to the cluster's eigenspace <= ANGLE_MAX)."""

    def __init__(self, w, H, ref_all, pset):
        from paper_1908_10251_gb300 import accuracy as acc
        self.acc = acc
        self.w, self.M, self.ref_all, self.pset = w, H.fine.M, ref_all, [int(i) for i in pset]
        key = w["golden"]
        if key not in _REFERENCE_PAIRS:
            cid = acc.clusters(ref_all)
            top = max(self.pset) if self.pset else 0
            last = int(np.where(cid == cid[top])[0].max())           # the whole cluster of the last pair
            count = min(len(ref_all), last + 1 + 6)
            ainv = acc.stencil_inverse(H.fine.A, w["dim"], w["N"])
            t0 = time.perf_counter()
            vals, vecs = acc.reference_pairs(H.fine.A, H.fine.M, count, ainv)
            _REFERENCE_PAIRS[key] = (vecs, time.perf_counter() - t0,
                                     float(np.max(np.abs(vals - ref_all[:count]) / ref_all[:count])))
        self.vecs, self.seconds, self.table_diff = _REFERENCE_PAIRS[key]

    def __call__(self, lam, U):
        return self.acc.report(self.M, lam, U, self.ref_all, target=self.w["target"], pairs=self.pset,
                               vecs=self.vecs, angle_max=ANGLE_MAX)


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
    log("mode %s precision %d smoother %s init %d" % (w["golden"], precision, smoother, init))
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
    tile_rows = pg.pasm_tile_rows(ctx, len(H.levels) - 1)
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
    # calibration (untimed), two passes over the same iteration from the start.
    # Pass 1 runs to the step cap, recording the eigenvalues, and judges the final state: F = the
    # pairs of the set that are then within the target of a reference eigenvalue of their cluster,
    # in clusters without duplicates and with largest M-principal angle <= ANGLE_MAX to the
    # reference eigenspace.  Pass 2 re-runs the iteration and finds S, the first step at which
    # every pair of F passes the same check (tried from the first step after which F's
    # eigenvalues stay within the target).  Set pairs outside F are reported as missed.
    pg.pasm_init(ctx, k, w["tol"])
    lam = np.zeros(k)
    U = np.zeros((H.fine.n, k))
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
    T = len(hist) - 1
    ref_all = load_golden(w["golden"])
    reach = first_reach(hist, ref, w["target"], ref_all)
    refset = reference_set(w)
    if refset is None:
        # no oracle set at this size: the pairs within the target at the end of pass 1
        pset = np.where(first_reach(hist[-1:], ref, w["target"], ref_all) >= 0)[0]
    else:
        pset = refset
    conv_eig, S_eig = time_to_target(reach, refset if refset is not None else pset, calib_steps)
    checker = VectorCheck(w, H, ref_all, pset)
    pg.pasm_get(ctx, lam, U)
    rep = checker(lam, U)
    F = list(rep["passed"])
    checks = 1
    S = T
    if F:
        errs = np.array([checker.acc.cluster_errors(row, ref_all)[F] for row in hist])
        bad = np.where(~np.all(errs <= w["target"], axis=1))[0]
        s0 = int(bad.max()) + 1 if bad.size else 0
        pg.pasm_init(ctx, k, w["tol"])
        for s in range(1, T + 1):
            pg.pasm_step(ctx)
            if s < s0:
                continue
            pg.pasm_get(ctx, lam, U)
            checks += 1
            r = checker(lam, U)
            if set(F) <= set(r["passed"]):
                S, rep = s, r
                break
    conv = len(F)
    missed = [int(i) for i in pset if i not in F]
    if F:
        # the eigenvalue-only step count over the same counted pairs, for comparison with S
        conv_eig, S_eig = time_to_target(reach, np.array(F), calib_steps)
    accuracy = {"step": S, "vector_checks": checks, "angle_max_allowed": ANGLE_MAX,
                "pairs": [int(i) for i in pset], "counted": [int(i) for i in F],
                "eig_err": [float(rep["err"][i]) for i in pset],
                "angle": [None if np.isnan(rep["angle"][i]) else float(rep["angle"][i]) for i in pset],
                "max_eig_err": float(np.nanmax(rep["err"][F])) if F else None,
                "max_angle": float(np.nanmax(rep["angle"][F])) if F else None,
                "angle_kind": "measured against ARPACK eigenvectors"}
    # the paper's stopping quantity at step S, over the counted pairs
    res = pg.pasm_residuals(ctx)
    res_max = float(res[F].max()) if F else None
    launches = pg.pasm_last_launches(ctx)
    # timed: W warm-up steps, then a fresh start (untimed) and exactly K steps of the captured
    # graph, so that the timed steps are steps 1..K of the trajectory the count was taken on
    pg.pasm_init(ctx, k, w["tol"])
    for _ in range(warmup):
        pg.pasm_step_async(ctx)
    pg.pasm_init(ctx, k, w["tol"])
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
            "S_eig": S_eig, "converged_eig": conv_eig, "accuracy": accuracy,
            "launches_per_step": launches, "trace": trace, "clocks": cs.summary(), "final_lam": hist[-1].tolist(),
            "fine_jacobi": fine_jacobi, "accepted": accepted, "init_ms": init_ms, "missed": missed,
            "tiles": tiles, "tile_rows": tile_rows, "first_init_s": tune_s, "fine_sweep_update": fine_sweep_update,
            "residual_max": res_max,
            "reached_outside_set": [int(i) for i in np.where(reach >= 0)[0]
                                    if refset is not None and i not in set(refset.tolist())]}


def solve_latency(pg, torch, H, w, precision, repeats=5):
    """Wall-clock latency of pasm_solve with device-resident start and result
    buffers and the workload's stop rule (|d lambda| / lambda < stop_tol), from
    the coarse start: median over `repeats` solves after one warm solve."""
    k = w["k"]
    ctx = pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P,
                        pg.pasm_default_opts(precision=precision, max_steps=60), torch.cuda.current_stream().cuda_stream)
    pg.pasm_init(ctx, k, w["stop_tol"])
    lam0 = torch.zeros(k, dtype=torch.float64, device="cuda")
    U0 = torch.zeros((H.fine.n, k), dtype=torch.float64, device="cuda")
    pg.pasm_get(ctx, lam0, U0)
    lam = torch.zeros_like(lam0)
    U = torch.zeros_like(U0)
    steps = np.zeros(k, dtype=np.int32)
    status = np.zeros(k, dtype=np.int32)
    pg.pasm_solve(ctx, k, w["stop_tol"], lam0, U0, lam, U, steps, status)
    times = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pg.pasm_solve(ctx, k, w["stop_tol"], lam0, U0, lam, U, steps, status)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    pg.pasm_destroy(ctx)
    return {"solve_ms": statistics.median(times) * 1e3, "steps": [int(v) for v in steps],
            "stop_tol": w["stop_tol"]}


def _build_kappa_problem(p):
    """Problem p of the uneven batch: -div(kappa grad u) = lambda u on the unit
    square, kappa = exp(g), g the seeded Gaussian field (sigma 1, correlation
    0.1, seed 1000 + p), fine grid 2^(8 + p mod 4) per side, H = 1/16, Galerkin
    coarse operators."""
    N = 2 ** (8 + p % 4)
    H = mg.build_hierarchy(2, N, 16, kappa=mg.gaussian_log_field(N, 1000 + p))
    return [lv.A for lv in H.levels], [lv.M for lv in H.levels], list(H.P)


BATCH_K = (8, 16, 32, 64, 128)


def run_uneven_batch(pg, torch, repeats=2):
    """The uneven batch: 16 kappa problems (65,025 to 4,190,209 DoF), k_p =
    (8, 16, 32, 64, 128)[p mod 5], mixed precision, pairs freeze at
    |d lambda| / lambda < 1e-10 unless their relative residual exceeds 1e-3
    (opts.res_tol; the guard against spurious freezes).  Wall-clock of
    pasm_batch_solve (one graph replay per batch step) against the same
    problems solved one after another with pasm_solve; pairs counted = frozen
    pairs whose residual, recomputed in float64 on the host, is below 1e-3."""
    import multiprocessing as mp
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, host_cores())) as pool:
        probs = pool.map(_build_kappa_problem, range(16))
    build_s = time.perf_counter() - t0
    ks = [BATCH_K[p % 5] for p in range(16)]
    stream = torch.cuda.current_stream().cuda_stream
    opts = pg.pasm_default_opts(precision=1, max_steps=60, res_tol=1e-3)
    batch = pg.pasm_batch_setup(probs, opts, stream)
    pg.pasm_batch_solve(batch, ks, 1e-10)                  # warm: autotuner, graph capture
    times = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code, lams, Us, steps, stats, rounds = pg.pasm_batch_solve(batch, ks, 1e-10)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    captures = pg.pasm_batch_captures(batch)
    pg.pasm_batch_destroy(batch)
    good = 0
    for (A, M, _), lam, U, st in zip(probs, lams, Us, stats):
        conv = st == 1
        MU = M[-1] @ U[:, conv]
        res = np.linalg.norm(A[-1] @ U[:, conv] - MU * lam[conv][None, :], axis=0) / (
            lam[conv] * np.sqrt(np.einsum("ij,ij->j", U[:, conv], MU)))
        good += int((res <= 1e-3 * (1 + 1e-6)).sum())
    seq = 0.0
    for (A, M, P), k in zip(probs, ks):
        ctx = pg.pasm_setup(A, M, P, opts, stream)
        pg.pasm_solve(ctx, k, 1e-10)                       # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pg.pasm_solve(ctx, k, 1e-10)
        torch.cuda.synchronize()
        seq += time.perf_counter() - t0
        pg.pasm_destroy(ctx)
    batch_s = statistics.median(times)
    return {"value": good / batch_s, "unit": "eigenpairs/s", "pairs_counted": good, "pairs": int(sum(ks)),
            "batch_s": batch_s, "sequential_s": seq, "speedup_vs_sequential": seq / batch_s,
            "batch_steps": rounds, "graph_captures": captures, "build_s": build_s,
            "rule": "frozen pairs with relative residual <= 1e-3 (float64, host)",
            "workload": "16 kappa = exp(g) problems, 2^(8 + p mod 4) per side, k = (8,16,32,64,128)[p mod 5], "
                        "H = 1/16, mixed"}


def run_per_pair(pg, torch, H, conv, S, steps=10):
    """The same workload with one launch sequence per pair: k problems of one
    pair each (k = 1, each its own context and graph branch) stepped together
    by the batch driver; per-step time from (T(steps) - T(0)) / steps (T(steps)
    includes the one capture of the step graph)."""
    k = WORK["k"]
    parts = ([lv.A for lv in H.levels], [lv.M for lv in H.levels], list(H.P))
    stream = torch.cuda.current_stream().cuda_stream

    b = pg.pasm_batch_setup([parts] * k, pg.pasm_default_opts(precision=1, max_steps=steps), stream)
    pg.pasm_batch_solve(b, [1] * k, 0.0)                   # warm: autotuner, capture

    def timed(nsteps):
        pg.pasm_batch_set_max_steps(b, nsteps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pg.pasm_batch_solve(b, [1] * k, 0.0)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    ms = (timed(steps) - timed(0)) / steps * 1e3
    pg.pasm_batch_destroy(b)
    return {"ms_per_step": ms, "value": conv / (S * ms * 1e-3), "unit": "eigenpairs/s",
            "note": "%d single-pair contexts in one batch graph per step; pairs and S as the block path" % k}


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
    V-cycles produce on this workload (captured in a damped-Jacobi run on the
    level with h = 4 h_fine, from the coarse start and two later steps; the
    network is h-independent), in a learned-smoother context, whose training
    runs layer 2 on the tensor cores."""
    k = WORK["k"]
    A = [lv.A for lv in H.levels]
    M = [lv.M for lv in H.levels]
    stream = torch.cuda.current_stream().cuda_stream
    ctx = pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(precision=1), stream)
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
    pg.pasm_destroy(ctx)
    ctx = pg.pasm_setup(A, M, H.P, pg.pasm_default_opts(precision=1, smoother=1), stream)
    pg.pasm_nn_setup(ctx, grid_widths(H), init_weights(0))
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
    for _ in range(5):     # median of five solves
        t0 = time.perf_counter()
        pg.pasm_solve(ctx, k, WORK["tol"], lam0.numpy(), U0.numpy(), lam.numpy(), U.numpy(), steps, status)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    log("end to end: solves %s ms" % ", ".join("%.1f" % (t * 1e3) for t in times))
    pg.pasm_destroy(ctx)
    nbytes_in = (n * k + k) * 8
    nbytes_out = (n * k + k) * 8 + 2 * k * 4
    return dt, nbytes_in, nbytes_out


def host_cores():
    """Cores this process may run on (the affinity mask, else the CPU count)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(conn, work, cols):
    """One worker of the oracle pool: the oracle's correction steps for the
    pairs `cols` of the workload (the oracle is test infrastructure; only the
    CPU-baseline legs of this file run it).  Replies to "step" with the pairs'
    eigenvalues after the step and the step's time in the worker."""
    import oracle
    H = mg.build_hierarchy(work["dim"], work["N"], work["NH"])
    prob = oracle.Problem.from_hierarchy(H)
    lam, U = oracle.initial_state(prob, work["k"])
    lam, U = lam[cols].copy(), np.ascontiguousarray(U[:, cols])
    active = np.ones(len(cols), dtype=bool)
    conn.send(("ready", lam))
    while True:
        msg = conn.recv()
        if msg != "step":
            break
        t0 = time.perf_counter()
        if active.any():
            lam_new, U, _ = oracle.correction(prob, lam, U, active)
            active &= ~(np.abs(lam_new - lam) < work["tol"] * np.abs(lam_new))
            lam = lam_new
        conn.send((lam, time.perf_counter() - t0))
    conn.close()


class OraclePool:
    """The oracle run pair-parallel on the host: P worker processes (spawned,
    one per core), the k pairs split as evenly as possible over them -- the
    paper's one-process-per-pair scheme of Algorithm 2 with its load-balancing
    remark when there are fewer processes than pairs.  step() runs one
    correction step of every pair and returns the wall-clock time it took."""

    def __init__(self, work, procs=None):
        import multiprocessing as mp
        k = work["k"]
        self.procs = max(1, min(procs or host_cores(), k))
        self.cols = [list(range(k))[p::self.procs] for p in range(self.procs)]
        ctx = mp.get_context("spawn")
        self.conns, self.workers = [], []
        t0 = time.perf_counter()
        for c in self.cols:
            a, b = ctx.Pipe()
            w = ctx.Process(target=_oracle_worker, args=(b, work, c), daemon=True)
            w.start()
            self.conns.append(a)
            self.workers.append(w)
        self.lam = np.zeros(k)
        for c, conn in zip(self.cols, self.conns):
            tag, lam = conn.recv()
            self.lam[c] = lam
        self.setup_s = time.perf_counter() - t0
        self.history = [self.lam.copy()]

    def step(self):
        t0 = time.perf_counter()
        for conn in self.conns:
            conn.send("step")
        for c, conn in zip(self.cols, self.conns):
            lam, _ = conn.recv()
            self.lam[c] = lam
        dt = time.perf_counter() - t0
        self.history.append(self.lam.copy())
        return dt

    def close(self):
        for conn in self.conns:
            try:
                conn.send("quit")
            except (BrokenPipeError, OSError):
                pass
        for w in self.workers:
            w.join(timeout=30)
            if w.is_alive():
                w.terminate()


def oracle_reach(hist, work):
    """(pairs counted, steps S) of an oracle eigenvalue history under the
    bench's eigenvalue rule (cluster-aware, over the oracle's own reference
    set), or None if the history is too short to show every set pair arrive."""
    ref_all = load_golden(work["golden"])
    reach = first_reach(np.array(hist), ref_all[:work["k"]], work["target"], ref_all)
    refset = reference_set(work)
    conv, S = time_to_target(reach, refset, len(hist) - 1)
    if refset is not None and np.any(reach[refset] < 0):
        return None
    return conv, S


def reference_counts():
    """steps to 1e-9 and converged pairs of the oracle's own iteration on the
    full workload (tests/golden, written by the oracle), over the reference
    set (the pairs it reaches and, without freezing, still holds)."""
    p = os.path.join(ROOT, "tests", "golden", WORK["history"] + ".json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ref_all = load_golden(WORK["golden"])
    reach = first_reach(np.array(d["history"]), ref_all[:WORK["k"]], WORK["target"], ref_all)
    refset = reference_set(WORK)
    if refset is not None:
        reach = reach[refset]
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
    modes = {"both": (("mixed", 1), ("fp64", 0)), "mixed": (("mixed", 1),), "fp64": (("fp64", 0),)}[
        "both" if args.mode == "both" else args.mode]
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
    # the uneven batch, and the bench workload with one launch sequence per pair
    log("uneven batch")
    batch_c4 = None if args.no_batch else run_uneven_batch(pg, torch)
    log("per-pair launches")
    per_pair = None if args.no_batch else run_per_pair(pg, torch, H, res[modes[0][0]]["converged"],
                                                       res[modes[0][0]]["S"])
    # the small latency-bound workload (h = 1/64, k = 8, float64)
    log("h = 1/64 latency")
    H1 = mg.build_hierarchy(WORK_C1["dim"], WORK_C1["N"], WORK_C1["NH"])
    c1 = run_mode(pg, torch, H1, load_golden(WORK_C1["golden"])[:WORK_C1["k"]], 0, args.steps, args.warmup, rank,
                  args.calib_steps, work=WORK_C1)
    c1["latency"] = solve_latency(pg, torch, H1, WORK_C1, 0)
    res["square_h64_H8_k8_fp64"] = c1
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
    log("end to end")
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
    # CPU baseline (oracle), bounded sample on rank 0: every pair of the workload, pair-parallel
    # over the host's cores, for two correction steps; scaled only by the step count S
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        log("cpu baseline")
        counts = reference_counts()
        cpu = cpu_baseline(*(counts[::-1] if counts else (conv, S)))
    log("done")
    out = {
        "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if primary == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME,
                   "precision": ("mixed: f32 V-cycles under double-float (f32 pair) outer residuals"
                                 if primary == "mixed" else "f64"),
                   "pairs_converged": conv, "pairs": WORK["k"], "steps_to_1e-9": S,
                   "steps_to_1e-9_eigenvalue_only": main["S_eig"],
                   "pair_set": "the pairs the float64 oracle drives to 1e-9 on this workload and still holds "
                               "after 40 steps without freezing (cluster-aware)",
                   "counting_rule": "the set pairs that pass at the end of a 60-step run count: within 1e-9 of "
                                    "a reference eigenvalue of their cluster, no duplicate in a cluster, largest "
                                    "M-principal angle to the ARPACK eigenspace <= 1e-6; S = the first step from "
                                    "which they all pass",
                   "freeze_tol": WORK["tol"],
                   "missed": main["missed"],
                   "eigen_residual_max": main["residual_max"],
                   "l2": "inputs larger than L2 (536 MB block vectors)", "parallelism": "replicas",
                   "tiles_finest": {kk: v for kk, v in main["tiles"].items() if v},
                   "rows_per_block_finest": {kk: v for kk, v in main["tile_rows"].items() if v},
                   "first_init_s": round(main["first_init_s"], 3)},
        "e2e": {"value": e2e_value, "unit": "eigenpairs/s", "h2d_bytes_per_step": bin_ // max(S, 1),
                "d2h_bytes_per_step": bout // max(S, 1), "seconds": e2e_s,
                "note": "pasm_solve with pinned host inputs/outputs, S steps per call"},
        "accuracy": main["accuracy"],
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
                            "steps_to_1e-9_eigenvalue_only": r["S_eig"],
                            "max_eig_err": (r["accuracy"] or {}).get("max_eig_err"),
                            "max_angle": (r["accuracy"] or {}).get("max_angle"),
                            "missed_detail": {str(i): {"eig_err": r["accuracy"]["eig_err"][j],
                                                       "angle": r["accuracy"]["angle"][j]}
                                              for j, i in enumerate(r["accuracy"]["pairs"]) if i in r["missed"]}
                            if r.get("accuracy") else None,
                            "learned_steps_accepted": r["accepted"],
                            **({"time_to_target_ms": r["S"] * r["ms_per_step"], "target": WORK_C1["target"],
                                "solve_latency": r["latency"]} if "latency" in r else {})}
                     for name, r in res.items() if name != primary},
        "setup_s": main["setup_s"],
        "uneven_batch": batch_c4,
        "per_pair_launches": per_pair,
    }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(conv, S, steps=2):
    """The oracle on the host, pair-parallel (OraclePool), timed for `steps`
    correction steps of all k pairs; eigenpairs/s = conv / (S x median step),
    conv and S from the oracle's own stored full-size iteration (eigenvalue
    rule, as the reference arm)."""
    pool = OraclePool(WORK)
    try:
        times = [pool.step() for _ in range(steps)]
    finally:
        pool.close()
    t_step = statistics.median(times)
    return {"value": conv / (S * t_step), "unit": "eigenpairs/s", "cores": pool.procs, "kind": "oracle",
            "sample": "%d correction steps of all %d pairs, %d worker processes (pairs split evenly), median "
                      "step %.2f s wall-clock, setup %.1f s untimed; value = %d pairs / (S=%d steps x step)"
                      % (steps, WORK["k"], pool.procs, t_step, pool.setup_s, conv, S),
            "step_s": times, "host_cores": host_cores()}


def main_reference(args):
    """The reference arm: the oracle (a plain CPU float64 PASM) pair-parallel on
    all host cores.  W untimed and K timed correction steps of all k pairs from
    the coarse start; value = pairs counted / (S x median timed step), with the
    count and S from the arm's own eigenvalues when its W + K steps show every
    set pair arrive, else from the oracle's stored full-size history."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    counts = reference_counts()
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration history table missing"}))
        return
    pool = OraclePool(WORK)
    try:
        for _ in range(args.warmup):
            pool.step()
        times = [pool.step() for _ in range(max(args.steps, 1))]
        hist = list(pool.history)
    finally:
        pool.close()
    own = oracle_reach(hist, WORK)
    S, conv = (own[1], own[0]) if own else counts
    t_step = statistics.median(times)
    value = conv / (S * t_step)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": 1,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "precision": "f64 oracle", "pairs_converged": conv,
                   "steps_to_1e-9": S, "counted_from": "own run" if own else "stored oracle history",
                   "rule": "eigenvalue within 1e-9 of its cluster (no vector check)"},
        "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": pool.procs, "kind": "oracle",
                         "sample": "%d timed correction steps of all %d pairs on %d worker processes (one per "
                                   "core, pairs split evenly), after %d untimed; setup %.1f s untimed"
                                   % (len(times), WORK["k"], pool.procs, args.warmup, pool.setup_s),
                         "host_cores": host_cores()},
        "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main_case(args):
    """One small synthetic case for a few correction steps (the command the
    profiler summaries wrap): the P1 Laplacian hierarchy of the unit square
    (dim 2) or the Kuhn cube (dim 3), every dyadic grid from 1/NH to 1/N,
    coarse start, replays of the captured step graph; prints the wall time per
    step and the per-kernel-class event times of one eager step."""
    import torch
    from paper_1908_10251_gb300 import build
    build.build()
    import paper_1908_10251_gb300 as pg
    dim, N, NH, k = (int(v) for v in args.case.split(","))
    H = mg.build_hierarchy(dim, N, NH)
    stream = torch.cuda.current_stream()
    smoother = {"jacobi": 0, "learned": 1, "cg": 2}[args.case_smoother]
    # --case-tiles: the tile shapes a plain run saved (--case-tiles-save), so that a profiled run
    # (whose launches the profiler slows unevenly) runs the shapes the autotuner picked unprofiled
    opts = pg.pasm_default_opts(precision=0 if args.mode == "fp64" else 1, smoother=smoother,
                                autotune=0 if args.case_tiles else 1)
    ctx = pg.pasm_setup([lv.A for lv in H.levels], [lv.M for lv in H.levels], H.P, opts, stream.cuda_stream)
    if args.case_tiles:
        with open(args.case_tiles) as f:
            for lv, sh in json.load(f).items():
                pg.pasm_set_tiles(ctx, int(lv), sh["chunks"], sh["rows"])
    if smoother == 1:
        pg.pasm_nn_setup(ctx, grid_widths(H), init_weights(0))   # cost does not depend on the weights
    pg.pasm_init(ctx, k, 0.0)
    if args.case_tiles_save:
        with open(args.case_tiles_save, "w") as f:
            json.dump({lv: {"chunks": pg.pasm_tiles(ctx, lv), "rows": pg.pasm_tile_rows(ctx, lv)}
                       for lv in range(len(H.levels))}, f)
    if args.case_train:
        lvl = len(H.levels) - 1
        R = np.random.default_rng(0).standard_normal((H.levels[lvl].n, k)).astype(np.float32)
        pg.pasm_nn_train(ctx, lvl, R, args.case_train, 1e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.case_steps):
        pg.pasm_step_async(ctx)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / max(args.case_steps, 1) * 1e3
    trace = pg.pasm_trace_step(ctx)
    fine = H.levels[-1].n
    finest = [(name, round(t * 1e3, 1)) for name, rows, t, b, f in pg.pasm_trace_launches(ctx) if rows == fine]
    shapes = {lv: {"chunks": {kk: v for kk, v in pg.pasm_tiles(ctx, lv).items() if v},
                   "rows": {kk: v for kk, v in pg.pasm_tile_rows(ctx, lv).items() if v}}
              for lv in range(1, len(H.levels))}
    pg.pasm_destroy(ctx)
    print(json.dumps({"case": {"dim": dim, "N": N, "NH": NH, "k": k, "mode": args.mode,
                               "smoother": args.case_smoother, "train_iters": args.case_train},
                      "ms_per_step_wall": wall,
                      "classes": {name: {"ms": t, "launches": n, "GBps": by / max(t, 1e-9) / 1e6}
                                  for name, (t, by, fl, n) in sorted(trace.items(), key=lambda kv: -kv[1][0])},
                      "finest_launches_us": finest, "tile_shapes": shapes}))


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
    ap.add_argument("--no-batch", dest="no_batch", action="store_true",
                    help="skip the uneven batch and the per-pair-launch comparison")
    ap.add_argument("--case", default=None, help="dim,N,NH,k: run one small case for profiling (no bench line)")
    ap.add_argument("--case-steps", type=int, default=3)
    ap.add_argument("--case-smoother", default="jacobi", choices=["jacobi", "learned", "cg"])
    ap.add_argument("--case-train", type=int, default=0, help="Adam steps of the smoother before the case's steps")
    ap.add_argument("--case-tiles-save", default=None, help="write the autotuned tile shapes of the case to this file")
    ap.add_argument("--case-tiles", default=None, help="run the case with the tile shapes of this file (no autotuning)")
    args = ap.parse_args()
    if args.case:
        main_case(args)
        return
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
