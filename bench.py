#!/usr/bin/env python3
"""Benchmark of the PP-PC hot path (batched fine propagators, jumps, coarse
linearisation, time-axis DFT, harmonic solves, inverse DFT + update).

Default: the large coax workload, 499 001 DOFs, N = 256 subintervals of 200
implicit-Euler steps, Brauer steel sheath with sigma = 3e7 S/m, 40 A at
50 Hz + 8 A at 150 Hz, mixed precision, multigrid-preconditioned fine PCG and
harmonic COCG.  One PP-PC iteration there takes minutes, so a "step" is a
fixed slice of it: 4 fine levels of all 256 subintervals (continuing the
first iteration's sweep from U = 0) plus one complete coarse update.
value = fine DOF-steps per second (N * 4 * ndof per step) over the timed
steps, device time from CUDA events on the library's stream; every state is
larger than L2.  Also reported: one whole PP-PC iteration timed once, the
time to periodic steady state at rel_res 1e-8 extrapolated from it and from
the iteration count measured on a 50 x 100 mesh with the same time grid,
the e2e rate through the C ABI with host buffers, the roofline of the fine
propagator kernel, and the CPU oracle on a bounded sample.

--workload medium: the medium coax workload (19 801 DOFs, N = 64, 50 fine
steps, sigma = 2e7, 10 A at 50 Hz); a step is one pppc_iterate() call.

Multi-GPU: the method runs on one GPU; with --gpus N each rank runs an
independent replica (weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s to periodic steady state at rel res 1e-8; fine DOF-steps/s; HBM % of peak"
UNIT = "fine DOF-steps/s"
WORKLOAD = "medium"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--newton-schedule", type=int, default=0, choices=[0, 1],
                    help="timed steps: 1 = inexact PP-PC (fine Newton tolerance tied to the previous rel res)")
    ap.add_argument("--tts-schedule", type=int, default=1, choices=[0, 1],
                    help="time-to-steady-state run: 1 = inexact PP-PC (same fixed point, final iterates at the "
                         "full Newton tolerance)")
    ap.add_argument("--tol-coarse", type=float, default=1e-3,
                    help="relative tolerance of the harmonic (COCG) solves of the medium run (their right-hand "
                         "side is the jumps, so a relative tolerance shrinks the absolute error with them)")
    ap.add_argument("--predictor", type=int, default=2, choices=[0, 1, 2],
                    help="Newton start: 0 previous level, 1 linear, 2 quadratic extrapolation")
    ap.add_argument("--precond", default="tridiag", choices=["jacobi", "tridiag", "amg"],
                    help="fine PCG preconditioner")
    ap.add_argument("--coarse-at", default="U", choices=["U", "F"],
                    help="freeze the coarse stiffness at U^k or at the fine results F^k")
    ap.add_argument("--workload", default="large", choices=["large", "medium"],
                    help="large: 499001 DOFs, N=256, 200 fine steps (the headline); medium: 19801 DOFs, N=64, 50")
    ap.add_argument("--no-full", action="store_true", help="large: skip the full PP-PC iteration")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-steady-state run")
    ap.add_argument("--profile-case", default=None, choices=["medium-short", "midsize"],
                    help="instead of the benchmark: a short case for ncu captures (medium-short: the medium mesh "
                         "with 2 fine steps, two PP-PC iterations from rest; midsize: a 250 x 500 mesh (124 501 "
                         "DOFs) with N=256, one fine level of every subinterval and one coarse update, states "
                         "larger than L2); fixed lane split, so no tuning launches")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--compare-methods", action="store_true",
                    help="instead of the benchmark: PP-PC vs PP-IC iterations to 1e-6 on the paper-shaped case")
    ap.add_argument("--batched", action="store_true",
                    help="instead of the medium benchmark: 32 uneven cables in one batch (two graphs per iteration)")
    ap.add_argument("--adjoint", action="store_true",
                    help="instead of the medium benchmark: periodic solve + adjoint gradient on the adjoint workload")
    ap.add_argument("--batched-tts", action="store_true",
                    help="with --batched: also solve all 32 cables from rest to rel res 1e-8")
    return ap.parse_args()


def compare_methods(args, local):
    """Sec. 4's comparison, paper-shaped: PP-PC with the multi-harmonic coarse
    solve against PP-IC (Eq. 5), both from U = 0 to rel res < 1e-6 on the
    2269-unknown coax case with N = 20 and 100 fine steps per subinterval.
    Prints one JSON line: iterations, device seconds and residual histories."""
    import numpy as np
    import torch

    from paper_1905_13076_gb300 import from_problem
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    prob = workload("paper")
    out = {"workload": "paper", "ndof": None, "N": prob.N, "n_fine": prob.n_fine, "tol": 1e-6,
           "precision": args.precision, "paper_iterations": {"pppc": 3, "ppic": 19}}
    states = {}
    for method in ("pppc", "ppic"):
        with from_problem(prob, precision=args.precision, method=method, stream=stream) as s:
            out["ndof"] = s.ndof
            s.set_state(np.zeros((prob.N, prob.mesh.n_nodes)))
            hist = []
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            it = 0
            while it < 60:
                rr = s.iterate()
                hist.append(rr)
                if rr < 1e-6:
                    break
                it += 1
            e1.record(stream)
            torch.cuda.synchronize(dev)
            st = s.stats()
            # rel res of U^k is returned by the k-th call (it measures the state going in)
            out[method] = {"iterations": it, "seconds": e0.elapsed_time(e1) * 1e-3,
                           "rel_res": [float(f"{h:.3e}") for h in hist], "cocg_iters_last": st["cocg_iters"]}
            states[method] = s.get_state()
    out["rel_diff_pppc_ppic"] = float(np.linalg.norm(states["pppc"] - states["ppic"])
                                      / np.linalg.norm(states["pppc"]))
    print(json.dumps(out), flush=True)


def run_adjoint(args, local):
    """The adjoint workload: coax nr=160 x ntheta=320 (50 881 unknowns), N =
    128, 40 fine steps, sheath sigma 2e7.  Periodic solve from rest to rel res
    1e-10, then the loss and dP/d(sigma, k1, k2, k3) of the sheath by the
    periodic adjoint to rel res 1e-10 (device times from the library's
    events; the adjoint's includes the forward trajectory sweep)."""
    import torch

    from paper_1905_13076_gb300 import from_problem
    from synth import REGION_SHEATH, workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    prob = workload("adjoint")
    s = from_problem(prob, precision=args.precision, precond=args.precond, predictor=args.predictor,
                     tol_coarse=args.tol_coarse, newton_schedule=bool(args.tts_schedule), stream=stream)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        its, rr = s.solve_periodic(tol=1e-10, kmax=80, raise_on_fail=False)
        t_fwd_host = time.perf_counter() - t0
        fst = s.stats()
        t0 = time.perf_counter()
        loss, grad, info = s.adjoint(REGION_SHEATH, tol=1e-10, kmax=80)
        t_adj_host = time.perf_counter() - t0
        ast = s.stats()
    units = prob.N * prob.n_fine * s.ndof
    fwd_s = (fst["fine_ms"] + fst["coarse_ms"]) * 1e-3
    adj_s = (ast["fine_ms"] + ast["coarse_ms"]) * 1e-3
    adj_sweeps = info["iterations"] + 1
    line = {
        "metric": "s to periodic steady state and adjoint gradient", "value": fwd_s + adj_s, "unit": "s",
        "higher_is_better": False, "n_gpus": 1, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": "coax adjoint case: nr=160 x ntheta=320 (50881 DOFs), N=128, 40 fine steps, "
                               "sigma=2e7, Brauer steel, 10 A 50 Hz", "precision": args.precision,
                   "precond": args.precond, "newton_schedule": args.tts_schedule, "predictor": args.predictor,
                   "tol_coarse": args.tol_coarse},
        "forward": {"seconds": fwd_s, "host_seconds": t_fwd_host, "pppc_iterations": its, "rel_res": rr,
                    "fine_dof_steps_per_s": units * (its + 1) / (fst["fine_ms"] * 1e-3)},
        "adjoint": {"seconds": adj_s, "host_seconds": t_adj_host, "pppc_iterations": info["iterations"],
                    "rel_res": info["rel_res"], "forward_rel_res": info["forward_rel_res"],
                    "refinement_passes": ast["newton_iters"], "pcg_iters": ast["pcg_iters"],
                    "fine_dof_steps_per_s": units * (adj_sweeps + 1) / (ast["fine_ms"] * 1e-3)},
        "loss_w_per_m": loss, "grad": {"sigma": grad[0], "k1": grad[1], "k2": grad[2], "k3": grad[3]},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    s.close()


def run_batched(args, local):
    """The many-instance workload: 32 independent coax cables drawn from a
    seed (nr 20-200, ntheta 40-400, 1-50 A, sheath sigma 1e6-3e7 S/m, N in
    {16, 32, 64}, 20-50 fine steps), all in one batch: per iteration one
    cooperative launch of every cable's fine sweep (one team of blocks per
    cable) and one of every cable's harmonic solves, from two CUDA graphs.
    A step is one batch iteration over all cables from their current states.
    Also timed: the same cables iterated one handle after another, and, with
    --batched-tts, the solve of all cables from rest to rel res 1e-8."""
    import numpy as np
    import torch

    from paper_1905_13076_gb300 import PPPCBatch, from_problem
    from synth import batched_cables

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    probs = batched_cables()
    # Kbar frozen at the fine results: a cold start of a 50 A cable linearised at
    # U = 0 (small-field reluctivity) sends the first coarse update far past saturation
    members = [from_problem(p, precision=args.precision, coarse_at="F", max_newton=100, precond=args.precond,
                            predictor=args.predictor, tol_coarse=args.tol_coarse, stream=stream)
               for p in probs]
    units = sum(p.N * p.n_fine * m.ndof for p, m in zip(probs, members))
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    hbm_peak, peak_src = peaks()
    mixed = args.precision == "mixed"

    def fine_bytes(ms):
        tot = 0.0
        for p, m in zip(probs, ms):
            mc = m.mesh_counts()
            bpr = pcg_bytes_per_row_lane(mixed, mc["special_rows"] / mc["ndof"], mc["nnz"] / mc["ndof"], p.N,
                                         tri=args.precond == "tridiag")
            # lane-vectors the PCG streamed (all lane teams of the member)
            tot += bpr * mc["ndof"] * m.stats()["pcg_lane_rounds"]
        return tot

    batch = PPPCBatch(members, autotune=True)
    for _ in range(max(3, args.warmup)):
        batch.iterate()
    dev_ms, fine_ms, kernels, retunes, fbytes = [], 0.0, 0, 0, 0.0
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize(dev)
            batch.iterate()
            st = batch.stats()
            dev_ms.append(st["fine_ms"] + st["coarse_ms"])
            fine_ms += st["fine_ms"]
            kernels += st["kernel_launches"]
            retunes += st["retunes"]
            fbytes += fine_bytes(members)
    value = units * args.steps / (sum(dev_ms) * 1e-3)
    achieved = fbytes / (fine_ms * 1e-3) / 1e9
    fteams, cteams = batch.teams()
    blanes, bteams = batch.lanes()
    batch.close()

    # the same cables, one handle after another, one iteration each
    seq_ms = 0.0
    for m in members:
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(dev)
        m.iterate()
        st = m.stats()
        seq_ms += st["fine_ms"] + st["coarse_ms"]
    seq_value = units / (seq_ms * 1e-3)

    tts = None
    if args.batched_tts:
        for p, m in zip(probs, members):
            m.set_state(np.zeros((p.N, p.mesh.n_nodes)))
        with PPPCBatch(members, autotune=True) as b2:
            t0 = time.perf_counter()
            its, rr = b2.solve_periodic(tol=1e-8, kmax=60, raise_on_fail=False)
            host_s = time.perf_counter() - t0
            st = b2.stats()
        tts = {"seconds": (st["fine_ms"] + st["coarse_ms"]) * 1e-3, "host_seconds": host_s,
               "batch_iterations": st["iterations"], "iterations_per_cable": [int(i) for i in its],
               "max_rel_res": float(np.max(rr)), "retunes": st["retunes"]}
    line = {
        "metric": "fine DOF-steps/s, 32-cable batch", "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(dev_ms) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": "32 coax cables, seed 2026: nr 20-200, ntheta 40-400, 1-50 A, sigma 1e6-3e7, "
                               "N in {16,32,64}, 20-50 fine steps", "precision": args.precision,
                   "precond": args.precond, "predictor": args.predictor, "tol_coarse": args.tol_coarse,
                   "fine_dof_steps_per_step": units, "l2": "flushed between steps (512 MB write)"},
        "sequential_single_handles": {"value": seq_value, "unit": UNIT, "ms": seq_ms},
        "batched_over_sequential": value / seq_value,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                     "kernel": "fine_batch_kernel"},
        "teams": {"fine": [int(x) for x in fteams], "cocg": [int(x) for x in cteams],
                  "lanes_per_team": [int(x) for x in blanes], "lane_teams": [int(x) for x in bteams]},
        "retunes_timed": retunes, "gpu_launches": kernels, "clocks": clk.summary(),
        "time_to_steady_state": tts,
    }
    print(json.dumps(line), flush=True)
    for m in members:
        m.close()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 rate of a GB300 (recipe figure); the FP64 path is bound by it.
FP64_PEAK_TFLOPS = 1.25


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def pcg_bytes_per_row_lane(mixed: bool, special_frac: float, nnz_row: float, NB: int, tri: bool = False) -> float:
    """Algorithmic bytes of one PCG iteration per (row, lane) of the fine
    propagator (single-reduction CG, two phases): phase A reads z, r and
    writes w; phase B reads z, w, p, s, r, u and writes p, s, r, z, u.  Vectors
    are FP32 in the mixed path (u stays FP64).  Matrix: per-lane values on the
    special rows, shared values and column indices amortised over the lanes.
    With the tridiagonal-chunk preconditioner phase B also reads the
    multiplier and inverse pivot of every row and writes and re-reads the
    forward-substituted vector, in place of the Jacobi diagonal."""
    v = 4.0 if mixed else 8.0
    phase_a = 3 * v
    phase_b = 5 * v + 8.0 + 4 * v + 8.0
    diag = special_frac * v + (1 - special_frac) * v / NB
    if tri:
        diag = 2 * v + 2 * v
    matrix = special_frac * nnz_row * v + (1 - special_frac) * nnz_row * (v + 4.0) / NB \
        + special_frac * nnz_row * 4.0 / NB
    return phase_a + phase_b + diag + matrix


# ---- the large workload (headline) -------------------------------------------
LARGE_LEVELS = 4   # fine implicit-Euler levels of every subinterval per timed step
# DRAM bytes (read + written) per row and lane-iteration of the multigrid
# fine team kernel, measured with ncu on a 250 x 500 mesh with the large
# workload's N = 256 (working set above L2): 579.1 GB over 124 501 rows x
# 33 968 lane-iterations.  The traffic grows in proportion to rows and
# lane-iterations once the working set exceeds L2.
TRAFFIC_PER_ROW_LANE_ITER = 136.9
LARGE_DESC = ("coax large: nr=500 x ntheta=1000 (499001 DOFs), N=256, 200 fine steps, sigma=3e7, Brauer steel, "
              "40 A @ 50 Hz + 8 A @ 150 Hz")


def fine_bytes_per_row_lane_round(mixed: bool, special_frac: float, N: int, amg_rows) -> dict:
    """Algorithmic bytes of one preconditioned PCG iteration per (row, lane)
    of the fine propagator, FP32 vectors in the mixed path (s = 4 bytes).
    pcg: the plain CG model, 7 s phi + 7 (s (1 - phi) + 4) / N + 13 s (matrix
    values per lane on the special rows, shared values and indices amortised
    over the N lanes; 13 vector passes), phi = special-row fraction.
    vcycle: one multigrid V-cycle, on the fine level 11 vector passes (smooth:
    read r, write y; residual: read y, r, write q; restriction reads q;
    prolongation reads and writes y; post-smoothing reads y, r, writes z) plus
    the per-lane Jacobian of the special rows twice and their l1 norms (16 s
    phi), and on every coarse level 10 passes of its own length (counted
    against the fine rows: 10 s n_l / n_0), coarse matrices not counted."""
    s = 4.0 if mixed else 8.0
    phi = special_frac
    pcg = 7 * s * phi + 7 * (s * (1 - phi) + 4) / N + 13 * s
    coarse = sum(amg_rows[1:]) / amg_rows[0] if amg_rows else 0.0
    vcycle = 11 * s + 16 * s * phi + 10 * s * coarse if amg_rows else 0.0
    return {"pcg": pcg, "vcycle": vcycle, "total": pcg + vcycle}


def run_large(args, world, rank, local):
    """The large workload: a step is LARGE_LEVELS fine implicit-Euler levels of
    all 256 subintervals (continuing the first PP-PC iteration's fine sweep
    from U = 0: the windows chain through the subintervals) plus one coarse
    update (jumps, Kbar, DFT, all harmonic solves, inverse DFT + update) on
    the fine values reached.  A whole PP-PC iteration (200 levels + coarse)
    takes minutes here, so it is timed once beside the steps, and the time to
    steady state is extrapolated from it."""
    import numpy as np
    import torch

    from paper_1905_13076_gb300 import from_problem
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    prob = workload("large")
    mixed = args.precision == "mixed"
    opts = dict(precision=args.precision, precond="amg", predictor=args.predictor, tol_coarse=args.tol_coarse,
                coarse_at=args.coarse_at, stream=stream)
    t0 = time.perf_counter()
    s = from_problem(prob, **opts)
    setup_s = time.perf_counter() - t0
    N, n_nodes, ndof, nf = prob.N, prob.mesh.n_nodes, s.ndof, prob.n_fine
    units_per_step = N * LARGE_LEVELS * ndof
    with torch.cuda.stream(stream):
        U0 = torch.zeros((N, n_nodes), dtype=torch.float64, device=dev)   # U^0 = 0
    torch.cuda.synchronize(dev)
    state = {"F": U0, "level": 0}

    def step():
        """One window of the sweep (restarting from U^0 after the last level)
        and the coarse update of U^0 with the values reached."""
        if state["level"] + LARGE_LEVELS > nf:
            state["F"], state["level"] = U0, 0
        with torch.cuda.stream(stream):
            F = s.propagate_fine_window(state["F"], state["level"], LARGE_LEVELS)
            a = s.stats()
            Unew, rr = s.coarse_update(U0, F)
            b = s.stats()
        state["F"], state["level"] = F, state["level"] + LARGE_LEVELS
        return {"fine_ms": a["fine_ms"], "pcg": a["pcg_iters"], "lane_rounds": a["pcg_lane_rounds"],
                "lane_iters": a["pcg_lane_iters"], "newton": a["newton_iters"], "coarse_ms": b["coarse_ms"],
                "cocg": b["cocg_iters"], "launches": a["launches"] + b["launches"]}

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    t0 = time.perf_counter()
    for _ in range(max(3, args.warmup)):
        step()
    warmup_s = time.perf_counter() - t0
    plan = s.fine_plan()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    per = []
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            per.append(step())
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, t_max = aggregate(sum(step_ms), units_per_step, args.steps)

    # roofline of the fine team kernel: algorithmic bytes / its event time
    mc = s.mesh_counts()
    bpr = fine_bytes_per_row_lane_round(mixed, mc["special_rows"] / mc["ndof"], N, plan["amg_rows"])
    fine_s = sum(p["fine_ms"] for p in per) * 1e-3
    lane_rounds = sum(p["lane_rounds"] for p in per)
    alg_bytes = bpr["total"] * ndof * lane_rounds
    hbm_peak, peak_src = peaks()
    achieved = alg_bytes / fine_s / 1e9
    launches = max(1, len(per))   # one fine launch per step
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": TRAFFIC_PER_ROW_LANE_ITER * ndof * lane_rounds / launches if mixed else None,
            "traffic_source": "ncu dram__bytes on the 250 x 500 mesh, N = 256, scaled per row and lane-iteration",
            "algorithmic_bytes_per_launch": alg_bytes / launches,
            "peak_source": peak_src, "kernel": "fine_batch_kernel<float>" if mixed else "fine_batch_kernel<double>",
            "bytes_per_row_lane_iteration": bpr, "pcg_lane_iterations": lane_rounds, "kernel_seconds": fine_s}

    # parity at full size on sampled outputs: one fine level of two
    # subintervals (where the current is high) from rest, against the
    # oracle's implicit-Euler/Newton step with sparse LU
    parity = None
    if not args.no_cpu:
        with torch.cuda.stream(stream):
            F1 = s.propagate_fine_window(U0, 0, 1)
        F1h = F1.cpu().numpy()
        free = prob.mesh.dirichlet == 0
        lanes = (64, 200)
        try:
            import multiprocessing as mp

            with mp.get_context("spawn").Pool(len(lanes)) as pool:
                ref = pool.map_async(_oracle_large_level1, [n + 1 for n in lanes], chunksize=1).get(timeout=900)
            errs = {n: float(np.linalg.norm(F1h[n][free] - u) / np.linalg.norm(u)) for n, u in zip(lanes, ref)}
            parity = {"fine_level_rel_err": max(errs.values()), "per_lane": errs,
                      "tol": 1e-7 if mixed else 1e-9,
                      "what": "level 1 of subintervals 65 and 201 from U=0 vs the oracle's Newton step (sparse LU)"}
        except Exception as exc:
            parity = {"unavailable": str(exc)[:200]}

    # end to end through the C ABI with host buffers: inputs from pinned host
    # memory every step, results read back; the same window and coarse update
    n_e2e = min(args.steps, 3)
    Fh = torch.empty((N, n_nodes), dtype=torch.float64).pin_memory()
    Fh.copy_(state["F"].cpu())
    U0h = torch.zeros((N, n_nodes), dtype=torch.float64).pin_memory()
    lev0 = state["level"] if state["level"] + LARGE_LEVELS <= nf else 0
    if lev0 == 0:
        Fh.zero_()
    e2e_t = []
    for k in range(n_e2e):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        F2 = s.propagate_fine_window(Fh.numpy(), lev0, LARGE_LEVELS)
        Un, rr = s.coarse_update(U0h.numpy(), F2)
        e2e_t.append(time.perf_counter() - t0)
    state_bytes = N * n_nodes * 8
    e2e_value = units_per_step * n_e2e * world / sum(e2e_t)

    # one whole PP-PC iteration from U = 0 (all 200 levels, then the coarse update)
    full = None
    if not args.no_full:
        s.set_state(np.zeros((N, n_nodes)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        rr_full = s.iterate()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st = s.stats()
        full = {"seconds": e0.elapsed_time(e1) * 1e-3, "fine_s": st["fine_ms"] * 1e-3,
                "coarse_s": st["coarse_ms"] * 1e-3, "pcg_rounds": st["pcg_iters"], "newton_rounds": st["newton_iters"],
                "cocg_iters": st["cocg_iters"], "rel_res_of_U0": rr_full,
                "fine_dof_steps_per_s": N * nf * ndof / (st["fine_ms"] * 1e-3 + st["coarse_ms"] * 1e-3)}
    s.close()

    # iterations to rel res 1e-8 with this time grid and excitation, measured
    # on a 50 x 100 mesh (PP-PC's iteration count hardly depends on the mesh)
    tts = None
    if not args.no_tts:
        small = workload("large", nr=50, ntheta=100)
        with from_problem(small, precision=args.precision, precond="tridiag", predictor=args.predictor,
                          tol_coarse=args.tol_coarse, newton_schedule=bool(args.tts_schedule),
                          stream=stream) as ts:
            ts.set_state(np.zeros((N, small.mesh.n_nodes)))
            t0 = time.perf_counter()
            iters, rr = ts.solve_periodic(tol=1e-8, kmax=60, raise_on_fail=False)
            small_s = time.perf_counter() - t0
        tts = {"iterations": iters, "rel_res": rr, "iterations_from": "50 x 100 mesh (4901 DOFs), same N, n_fine, "
               "materials and excitation, inexact Newton schedule " + str(args.tts_schedule),
               "small_mesh_seconds": small_s}
        if full is not None:
            # k updates need k + 1 fine sweeps and k coarse updates
            tts["seconds_extrapolated"] = (iters + 1) * full["fine_s"] + iters * full["coarse_s"]
            tts["label"] = "extrapolated: measured iterations x measured full-iteration times"

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        try:
            cpu = cpu_baseline_large(cores=None)
        except Exception as exc:
            cpu = {"unavailable": str(exc)[:200]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": LARGE_DESC, "precision": args.precision, "parallelism": "replicas only",
                   "step": f"{LARGE_LEVELS} fine levels of all {N} subintervals (window of the first PP-PC "
                           "iteration's sweep from U=0) + one coarse update (jumps, Kbar, DFT, harmonic solves, "
                           "inverse DFT)",
                   "l2": "inputs larger than L2 (each state 1.02 GB)", "precond": "amg",
                   "lane_team": plan["lanes_per_team"], "teams": plan["teams"], "amg_rows": plan["amg_rows"],
                   "tol_coarse": args.tol_coarse, "predictor": args.predictor, "coarse_at": args.coarse_at},
        "setup_s": setup_s, "warmup_s_incl_tuning": warmup_s,
        "per_step": {k: sum(p[k] for p in per) / len(per) for k in per[0]} | {"step_ms": step_ms},
        "full_iteration": full,
        "time_to_steady_state": tts,
        "error_vs_oracle": parity,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * state_bytes,
                "d2h_bytes_per_step": 2 * state_bytes, "steps": n_e2e,
                "calls": "pppc_propagate_fine_window + pppc_coarse_update with host arrays"},
        "gpu_launches": sum(p["launches"] for p in per),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def _oracle_large_step(n):
    """One implicit-Euler step (Newton, sparse LU) of subinterval n of the
    large workload from rest: the oracle's first fine level (a pool worker)."""
    import numpy as np

    from oracle.fem import FEModel
    from oracle.stepping import ie_step
    from synth import workload

    prob = workload("large")
    m = _oracle_large_step.model = getattr(_oracle_large_step, "model", None) or FEModel(prob)
    dt = prob.T / (prob.N * prob.n_fine)
    t0 = time.perf_counter()
    ie_step(m, np.zeros(m.ndof), ((n - 1) * prob.n_fine + 1) * dt, dt)
    return m.ndof, time.perf_counter() - t0


def _oracle_large_level1(n):
    """The oracle's first implicit-Euler step of subinterval n of the large
    workload from rest (free nodes)."""
    import numpy as np

    from oracle.fem import FEModel
    from oracle.stepping import ie_step
    from synth import workload

    prob = workload("large")
    m = FEModel(prob)
    dt = prob.T / (prob.N * prob.n_fine)
    u, _ = ie_step(m, np.zeros(m.ndof), ((n - 1) * prob.n_fine + 1) * dt, dt)
    return u


def cpu_baseline_large(cores=None, pool=None):
    """The FP64 oracle as it stands on every host core, on a bounded sample of
    the large workload: the first implicit-Euler step of one subinterval per
    core (one sparse LU of 499 001 unknowns per Newton iteration), each
    process single-threaded.  The rate is the summed work over the longest
    step; building the FE model is not timed."""
    import multiprocessing as mp

    cores = max(1, min(cores or os.cpu_count() or 1, 256))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        own = pool is None
        if own:
            pool = mp.get_context("spawn").Pool(cores)
        try:
            res = pool.map_async(_oracle_large_step, list(range(1, cores + 1)), chunksize=1).get(timeout=900)
        finally:
            if own:
                pool.close()
                pool.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    units = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": units / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} subintervals x 1 implicit-Euler/Newton step with sparse LU on 499001 DOFs, "
                      f"one single-threaded process per core, from rest ({wall:.1f} s, the longest of them)"}


def cpu_baseline(prob, max_seconds=20.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    fine propagators of whole subintervals from rest (Eqs. 2-3), one core."""
    import numpy as np

    from oracle.fem import FEModel
    from oracle.stepping import propagate

    m = FEModel(prob)
    steps = 0
    t0 = time.perf_counter()
    n = 1
    while True:
        propagate(m, n, np.zeros(m.ndof), prob.N, prob.n_fine, prob.T)
        steps += prob.n_fine
        n += 1
        el = time.perf_counter() - t0
        if el > max_seconds * 0.5 or n > prob.N:
            break
    return {"value": steps * m.ndof / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n - 1} subinterval(s) x {prob.n_fine} implicit-Euler/Newton steps with sparse LU, "
                      f"{m.ndof} DOFs, from rest ({el:.1f} s)"}


def _oracle_subinterval(args):
    """One subinterval's fine propagator of the oracle (a worker of the pool)."""
    name, n = args
    import numpy as np

    from oracle.fem import FEModel
    from oracle.stepping import propagate
    from synth import workload

    prob = workload(name)
    m = FEModel(prob)
    t0 = time.perf_counter()
    propagate(m, n, np.zeros(m.ndof), prob.N, prob.n_fine, prob.T)
    return prob.n_fine * m.ndof, time.perf_counter() - t0


def cpu_baseline_pool(name, cores=None):
    """The same oracle on every host core: independent subintervals' fine
    propagators, one per process of a spawned pool (safe after GPU work),
    each process single-threaded.  The rate is the summed work over the
    longest propagation (they run at the same time); building the FE model
    in each process is not timed, as for the one-core figure."""
    import multiprocessing as mp

    from synth import workload

    prob = workload(name)
    cores = max(1, min(cores or os.cpu_count() or 1, prob.N))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            res = pool.map_async(_oracle_subinterval, [(name, n) for n in range(1, cores + 1)],
                                 chunksize=1).get(timeout=600)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    units = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": units / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} subintervals x {prob.n_fine} implicit-Euler/Newton steps with sparse LU, "
                      f"one single-threaded process per core, from rest ({wall:.1f} s, the longest of them)"}


def aggregate(total_ms: float, units_per_step: float, steps: int):
    """Whole-job rate of independent replicas: the work of all ranks divided
    by the slowest rank's time (max over ranks).  Returns (value, t_max_ms)."""
    world = 1
    t_max = total_ms
    try:
        import torch
        import torch.distributed as dist

        if dist.is_available() and dist.is_initialized():
            world = dist.get_world_size()
            t = torch.tensor([total_ms], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_max = float(t.item())
    except ImportError:
        pass
    return units_per_step * steps * world / (t_max * 1e-3), t_max


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return world, rank, local


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle timed as it stands on the host's cores
    (rank 0 only): each step runs, in a process pool, one subinterval's fine
    propagation per core (large: the first implicit-Euler step; medium: the
    whole subinterval); the value is the median over the steps."""
    if rank != 0:
        return
    from synth import workload

    if args.workload == "large":
        import multiprocessing as mp

        # each step is one implicit-Euler step of one subinterval (one sparse
        # LU of 499 001 unknowns per Newton iteration, ~20-100 s); the K steps
        # run concurrently on the host cores, one single-threaded process each
        t_all = time.perf_counter()
        K = max(1, args.steps)
        cores = max(1, min(os.cpu_count() or 1, K))
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        with mp.get_context("spawn").Pool(cores) as pool:
            t0 = time.perf_counter()
            res = pool.map_async(_oracle_large_step, [1 + (7 * j) % 256 for j in range(K)], chunksize=1).get(
                timeout=3000)
            wall = time.perf_counter() - t0
        value = sum(r[0] for r in res) / wall
        base = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{K} implicit-Euler/Newton steps with sparse LU on 499001 DOFs (one per timed step, "
                          f"subintervals spread over the period, from rest) on {cores} single-threaded processes "
                          f"({wall:.1f} s in all, building the FE models included)"}
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": LARGE_DESC, "parallelism": "replicas only"},
                "cpu_baseline": base,
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": time.perf_counter() - t_all}
        print(json.dumps(line))
        return

    prob = workload(WORKLOAD)
    for _ in range(args.warmup):
        pass
    vals = []
    t_all = time.perf_counter()
    base = None
    one_core = cpu_baseline(prob, max_seconds=min(20.0, 60.0 / max(1, args.steps)))
    for _ in range(max(1, args.steps)):
        base = cpu_baseline_pool(WORKLOAD)
        vals.append(base["value"])
    value = statistics.median(vals)
    base["value"] = value
    base["sample"] += f"; median of {len(vals)} such samples"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "coax medium: nr=100 x ntheta=200 (19801 DOFs), N=64, 50 fine steps, "
                                   "sigma=2e7, Brauer steel, 10 A 50 Hz", "parallelism": "replicas only"},
            "cpu_baseline": base, "cpu_baseline_one_core": one_core,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line))


def profile_case(args):
    """Short runs for ncu captures (see --profile-case); prints their counts."""
    import numpy as np

    from paper_1905_13076_gb300 import from_problem
    from synth import workload

    if args.profile_case == "medium-short":
        prob = workload("medium", n_fine=2)
        with from_problem(prob, precision=args.precision, precond=args.precond, lane_team=32, predictor=2,
                          tol_coarse=args.tol_coarse) as s:
            s.set_state(np.zeros((prob.N, prob.mesh.n_nodes)))
            for _ in range(2):
                rr = s.iterate()
                print(json.dumps({"case": args.profile_case, "rel_res": rr} | s.stats()), flush=True)
        return
    prob = workload("large", nr=250, ntheta=500)
    with from_problem(prob, precision=args.precision, precond="amg", lane_team=16, predictor=2,
                      tol_coarse=args.tol_coarse) as s:
        U = np.zeros((prob.N, prob.mesh.n_nodes))
        F = s.propagate_fine_window(U, 0, 1)
        print(json.dumps({"case": args.profile_case, "window": 1} | s.stats()), flush=True)
        Un, rr = s.coarse_update(U, F)
        print(json.dumps({"case": args.profile_case, "coarse": 1, "rel_res": rr} | s.stats()), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.profile_case:
        if rank == 0:
            profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.compare_methods:
        if rank == 0:
            compare_methods(args, local)
        return
    if args.batched:
        if rank == 0:
            run_batched(args, local)
        return
    if args.adjoint:
        if rank == 0:
            run_adjoint(args, local)
        return
    if args.workload == "large":
        run_large(args, world, rank, local)
        return
    import numpy as np
    import torch

    from paper_1905_13076_gb300 import from_problem
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    prob = workload(WORKLOAD)
    mixed = args.precision == "mixed"
    solver = from_problem(prob, precision=args.precision, coarse_at=args.coarse_at,
                          newton_schedule=bool(args.newton_schedule), precond=args.precond,
                          tol_coarse=args.tol_coarse, predictor=args.predictor, stream=stream)
    ndof = solver.ndof
    units_per_step = prob.N * prob.n_fine * ndof
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- warm-up (also the first PP-PC iterations from U = 0)
    solver.set_state(np.zeros((prob.N, prob.mesh.n_nodes)))
    for _ in range(max(3, args.warmup)):
        solver.iterate()
    U_start = solver.get_state()   # the timed steps and every e2e step start from here

    # ---- timed region: K iterations, L2 flushed between them
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fine_ms, pcg, newton, launches = [], 0, 0, 0
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[k][0].record(stream)
            solver.iterate()
            ev[k][1].record(stream)
            st = solver.stats()
            fine_ms.append(st["fine_ms"])
            pcg += st["pcg_iters"]
            newton += st["newton_iters"]
            launches += st["launches"]
        torch.cuda.synchronize(dev)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, t_max = aggregate(sum(step_ms), units_per_step, args.steps)

    # ---- roofline of the fine-propagator kernel (the dominant kernel)
    mc = solver.mesh_counts()
    nnz_row = mc["nnz"] / mc["ndof"]
    sp_frac = mc["special_rows"] / mc["ndof"]
    if args.precond == "amg":
        bpr = fine_bytes_per_row_lane_round(mixed, sp_frac, prob.N, solver.fine_plan()["amg_rows"])["total"]
    else:
        bpr = pcg_bytes_per_row_lane(mixed, sp_frac, nnz_row, prob.N, tri=args.precond == "tridiag")
    fine_s = sum(fine_ms) * 1e-3
    pcg_bytes = bpr * ndof * prob.N * pcg
    hbm_peak, peak_src = peaks()
    if mixed:
        achieved = pcg_bytes / fine_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                "kernel": "fine_sweep_kernel<float>"}
    else:
        flops_row = 2 * nnz_row + 6 + 9
        achieved = flops_row * ndof * prob.N * pcg / fine_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "peak_source": "recipe FP64 rate",
                "kernel": "fine_sweep_kernel<double>", "hbm_gbs_equiv": pcg_bytes / fine_s / 1e9}

    # ---- end to end through the C ABI with host buffers
    # every e2e step repeats the first timed step's work: the same input state
    # (from pinned host memory) each time, the result read back to the host
    pinned_in = torch.from_numpy(np.ascontiguousarray(U_start)).pin_memory()
    pinned_out = torch.zeros_like(pinned_in).pin_memory()
    U_in, U_out = pinned_in.numpy(), pinned_out.numpy()
    e2e_times = []
    for k in range(args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        solver.set_state(U_in)
        solver.iterate()
        U_out[:] = solver.get_state()
        e2e_times.append(time.perf_counter() - t0)
    e2e_units = units_per_step
    e2e_value = e2e_units * args.steps * world / sum(e2e_times)
    # the device-timed rate of that same first step, for comparison with e2e
    first_step_value = units_per_step / (step_ms[0] * 1e-3)
    state_bytes = prob.N * prob.mesh.n_nodes * 8

    # ---- time to periodic steady state from U = 0
    tts = None
    if not args.no_tts:
        tsolver = from_problem(prob, precision=args.precision, coarse_at=args.coarse_at,
                               newton_schedule=bool(args.tts_schedule), precond=args.precond,
                               tol_coarse=args.tol_coarse, predictor=args.predictor, stream=stream)
        tsolver.set_state(np.zeros((prob.N, prob.mesh.n_nodes)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e0.record(stream)
        iters, rr = tsolver.solve_periodic(tol=1e-8, kmax=60, raise_on_fail=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st = tsolver.stats()
        tts = {"seconds": e0.elapsed_time(e1) * 1e-3, "host_seconds": time.perf_counter() - t0,
               "pppc_iterations": iters, "rel_res": rr, "newton_iters": st["newton_iters"],
               "pcg_iters": st["pcg_iters"], "cocg_iters": st["cocg_iters"],
               "newton_schedule": args.tts_schedule}
        tsolver.close()

    if rank != 0:
        solver.close()
        return
    cpu = cpu_pool = None
    if not args.no_cpu:
        cpu = cpu_baseline(prob)
        try:
            cpu_pool = cpu_baseline_pool(WORKLOAD)
        except Exception as exc:   # a host without process support still reports the 1-core figure
            cpu_pool = {"unavailable": str(exc)[:200]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": "coax medium: nr=100 x ntheta=200 (19801 DOFs), N=64, 50 fine steps, "
                               "sigma=2e7, Brauer steel, 10 A 50 Hz", "precision": args.precision,
                   "parallelism": "replicas only", "l2": "flushed between steps (512 MB write)",
                   "coarse_at": args.coarse_at, "newton_schedule": args.newton_schedule,
                   "precond": args.precond, "tol_coarse": args.tol_coarse, "predictor": args.predictor},
        "time_to_steady_state": tts,
        "per_step": {"pcg_iters": pcg / args.steps, "newton_iters": newton / args.steps,
                     "fine_ms": sum(fine_ms) / args.steps, "step_ms": step_ms},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "repeats": "the first timed step (same input state) each time",
                "device_rate_of_that_step": first_step_value},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "cpu_baseline": cpu_pool if cpu_pool is not None and "value" in cpu_pool else cpu,
        "cpu_baseline_one_core": cpu,
    }
    print(json.dumps(line))
    solver.close()


if __name__ == "__main__":
    main()
