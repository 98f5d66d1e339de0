"""Benchmark of the fused split-form SBP RHS + RK4 stage path on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--no-drift] [--size N]

One bench step = one classical RK4 time step (4 fused RHS+stage launches) of
the large periodic workload: 8192 x 8192 nodes, dx = dy = 0.1, bathymetry
-1 + a 64-mode random Fourier field (rms 0.1), 16 Gaussian humps, lambda = 500,
g = 9.81; the job is 500 such steps.  The metric is cell-stage updates per
second (one node through one RK stage); the headline precision is FP64, with
FP32 and FP32-state/FP64-accumulator variants, their HBM/ALU roofline
fractions, and the energy drift and FP32-vs-FP64 errors of the full 500-step
job reported beside it.

The state (2.7 GB in FP64) is far larger than the 126 MB L2, so no flush is
needed between timed steps.  Timing uses CUDA events on the stream the kernels
run on, with a synchronize on both sides, after W warm-up steps; SM clocks and
throttle reasons are sampled with nvidia-smi during the timed region.

Under torchrun (N > 1) every rank runs its own replica of the workload (the
path has no exchange in this configuration: replicas only), the timed region is
bracketed by barriers and the slowest rank's time is used.

--impl reference times the CPU oracle (tests' reference implementation, plain
FP64 C, one thread) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2601_02540_b300 import inputs  # noqa: E402

METRIC = "cell-stage updates/s"
UNIT = "cell-stages/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
FP64_NOMINAL_TFLOPS = 1.25     # B300 dense FP64 (nominal; no measured entry)
# Algorithmic bytes per cell-stage of the three-register RK4 stage kernels
# (each plane read or written once per stage, halos from cache), FP64 and df64:
#   stage 1: read q, b; write acc, Q             16 planes
#   stages 2, 3: read Q, b, q, acc; write acc, Q  26 planes
#   stage 4: read Q, b, acc; write q              16 planes   -> 84 planes per step
# The FP32 mode advances two stages per launch (sgn_set_stage_fusion):
#   stages 1-2: read q, b; write acc, Q3          16 planes
#   stages 3-4: read Q3, b, q, acc; write q'      21 planes   -> 37 planes per step
# and, one launch per stage, runs stages 1 and 2 as S1K / S2K:
#   stage 1: read q, b; write k1                  11 planes
#   stage 2: read q, k1, b; write acc, Q          21 planes   -> 74 planes per step
# The mixed mode: q and acc double, Q and b float, the 84-plane scheme (536 B per step).
BYTES_PER_CELL_STAGE = {"f64": 84 * 8 / 4, "f32": 37 * 4 / 4, "f32_unfused": 74 * 4 / 4,
                        "f32_f64acc": 536 / 4,
                        "df64": 84 * 8 / 4}     # df64: stage states as float pairs, 8 bytes
# (launches per step, stages per launch, kernel) of each timed path
LAUNCH_SHAPE = {"f64": (4, 1, "k_stage (RK4 stage, 4 launches/step)"),
                "f32": (2, 2, "k_fused (two RK4 stages per launch, 2 launches/step)"),
                "f32_unfused": (4, 1, "k_stage (RK4 stage, 4 launches/step)"),
                "f32_f64acc": (4, 1, "k_stage (RK4 stage, 4 launches/step)"),
                "df64": (4, 1, "k_stage (RK4 stage, 4 launches/step)")}
# Algorithmic floating-point operations per cell-stage of the implemented
# formulation (an FMA counts 2; 1/h counts 1): pointwise operands (1/h, eta/h,
# eta + 3/2 b, P2 = 2g h(h+b) - lam/3 eta^2/h) 10, products 7, coefficients 5,
# 20 differences, the fluxes A_x, A_y 6, h 3, u 16, v 16, w 15, eta 6, stage
# algebra 17.5 (average of 20, 20, 20, 10).
FLOPS_PER_CELL_STAGE = 121.5
# The same arithmetic counted in FP64 pipe operations (an FMA is one; 1/h is
# one): operands 15, the node's RHS 60, stage algebra 8.75.  The FP64 pipe of
# a B300 SM issues two thread-operations per clock.
FP64_OPS_PER_CELL_STAGE = 83.75
FP64_OPS_PER_SM_CLOCK = 2
DTYPE_NAME = {"f64": "f64", "f32": "f32", "f32_unfused": "f32 (one launch per stage)", "f32_f64acc": "f32+f64acc",
              "df64": "df64 (float pairs)"}


def _peaks() -> tuple[float, str]:
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("sgn_kernels.cuh", "sgn_fused.cuh")


def _kernel_hash(text: str | None = None) -> str:
    """Hash of the sources that define the stage kernels (one and two stages
    per launch) and their tile shapes, with // comments, trailing blanks and
    empty lines removed (so that edits of comments do not invalidate a
    capture)."""
    if text is None:
        parts = []
        for name in KERNEL_SOURCES:
            with open(os.path.join(ROOT, "paper_2601_02540_b300", "csrc", name)) as fh:
                parts.append(fh.read())
        text = "\n".join(parts)
    lines = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


# The grid the committed per-launch traffic is stated for (the 4096^2 capture x 4).
TRAFFIC_CELLS = 8192 * 8192


def _ncu_traffic(prec: str, cells: int) -> float | None:
    """DRAM bytes per launch of the stage kernel from the committed ncu summary,
    or None when the kernels changed since it was captured or the grid is not
    the one the figure is stated for."""
    if cells != TRAFFIC_CELLS:
        return None
    path = os.path.join(ROOT, "profiles", "k_stage_traffic_4096.md")
    if not os.path.exists(path):
        return None
    vals, khash = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith("kernel_hash"):
                khash = line.split()[-1]
            elif line.startswith("traffic_bytes_per_launch"):
                parts = line.split()
                vals[parts[1]] = float(parts[2])
    if khash != _kernel_hash():
        return None
    return vals.get(prec)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------------------- GPU arm
def _time_steps(torch, solver, q, dt, steps, warmup, dist=None):
    from paper_2601_02540_b300 import sgn
    for _ in range(warmup):
        solver.step(q, dt, 1)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n0 = sgn.sgn_launch_count()
    torch.cuda.synchronize()
    e0.record(stream)
    solver.step(q, dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = sgn.sgn_launch_count() - n0
    ms = e0.elapsed_time(e1)
    if dist is not None:
        ms = max_over_ranks(torch, dist, ms, "cuda")
        dist.barrier()
    return ms, launches


def max_over_ranks(torch, dist, ms: float, device: str) -> float:
    """The slowest rank's time (replicas: the job ends when the last rank does)."""
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(cells: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job cell-stage rate of `world` independent replicas, each advancing
    `cells` nodes by `steps` RK4 steps (4 stages), over the slowest rank's time."""
    return 4.0 * cells * steps * world / (ms_max * 1e-3)


def measure_fp64_peak(torch, local: int, iters: int = 16384, reps: int = 3) -> dict:
    """The FP64 FMA rate of this GPU, measured by the library's FMA-chain
    kernel (sgn_measure_fp64_fma: independent chains, 8 blocks of 256 threads
    per SM), best of `reps` launches after one warm-up, with the SM clock
    sampled while it runs.  The SM count is read from the device."""
    from paper_2601_02540_b300 import sgn
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sgn.sgn_measure_fp64_fma(iters)
    best = 0.0
    with ClockSampler(local) as clk:
        for _ in range(reps):
            n, sec = sgn.sgn_measure_fp64_fma(iters)
            best = max(best, n / sec)
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz")
    return {"fma_per_s": best, "tflops": 2.0 * best / 1e12, "sms": sms, "sm_mhz": mhz,
            "fma_per_sm_clock": best / (sms * mhz * 1e6) if mhz else None,
            "reasons": clocks.get("reasons"),
            "how": f"sgn_measure_fp64_fma: {iters} iterations of 16 independent FMA chains per thread, "
                   f"8 x 256 threads per SM, best of {reps} launches (CUDA events)"}


def _roofline(prec: str, cells: int, ms_total: float, steps: int,
              hbm_peak: float, hbm_kind: str, fp64: dict | None = None) -> dict:
    launches_per_step, stages_per_launch, kernel = LAUNCH_SHAPE[prec]
    launch_ms = ms_total / (launches_per_step * steps)
    traffic = _ncu_traffic(prec, cells)
    if prec == "f64":
        # FP64 is ALU-bound on B300: the roofline is the FP64 pipe, whose
        # issue slots each take one FMA, add or multiply.  achieved = the
        # formulation's algorithmic FP64 operations per launch (FMA = 1) over
        # the launch time; peak = the FMA rate measured on this GPU by
        # measure_fp64_peak.  The flop form is given beside it.
        ops = FP64_OPS_PER_CELL_STAGE * cells / (launch_ms * 1e-3) / 1e9
        peak_ops = fp64["fma_per_s"] / 1e9
        flops = FLOPS_PER_CELL_STAGE * cells / (launch_ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ops, "peak": peak_ops,
                "unit": "G FP64 ops/s (FMA, add, mul = 1 each)", "frac": ops / peak_ops, "traffic": traffic,
                "peak_kind": (f"measured: FP64 FMA-chain kernel, {fp64['fma_per_s'] / 1e9:.1f} G FMA/s on "
                              f"{fp64['sms']} SMs at {fp64['sm_mhz']} MHz = {fp64['fma_per_sm_clock']:.3f} per "
                              f"SM-clock (unit count: 2; nominal {FP64_NOMINAL_TFLOPS} TFLOP/s)"),
                "algorithmic_ops_per_cell_stage": FP64_OPS_PER_CELL_STAGE,
                "fp64_peak": fp64,
                "kernel": kernel,
                "launch_ms": launch_ms,
                "flops": {"achieved": flops, "peak": fp64["tflops"], "unit": "TFLOP/s",
                          "frac": flops / fp64["tflops"], "flop_per_cell_stage": FLOPS_PER_CELL_STAGE},
                "hbm": {"achieved": BYTES_PER_CELL_STAGE[prec] * cells / (launch_ms * 1e-3) / 1e9,
                        "peak": hbm_peak, "unit": "GB/s",
                        "frac": BYTES_PER_CELL_STAGE[prec] * cells / (launch_ms * 1e-3) / 1e9 / hbm_peak,
                        "peak_kind": hbm_kind}}
    achieved = BYTES_PER_CELL_STAGE[prec] * stages_per_launch * cells / (launch_ms * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
           "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": hbm_kind,
           "kernel": kernel, "launch_ms": launch_ms,
           "algorithmic_bytes_per_cell_stage": BYTES_PER_CELL_STAGE[prec]}
    if stages_per_launch > 1:
        # two stages per launch halve the bytes and are bound by instruction
        # issue: their rate against the roof of one launch per stage
        out["single_stage_hbm_roof"] = _single_stage_roof(4.0 * cells * steps / (ms_total * 1e-3), hbm_peak)
    return out


def _cpu_baseline(p_full: inputs.Problem) -> dict:
    import oracle as orc
    n = 1024
    nst = 4
    p = inputs.workload3(n, n)
    g = orc.Grid(p.nx, p.ny, p.xmin, p.xmax, p.ymin, p.ymax, p.bc, p.g, p.lam)
    q0 = orc.init_aux(g, p.b, p.q0)
    t0 = time.perf_counter()
    ref = orc.rk4(g, p.b, q0, p_full.dt, nst)
    sec = time.perf_counter() - t0
    # the same oracle source built with OpenMP, on all host cores (same results)
    cores = len(os.sched_getaffinity(0))
    os.environ["OMP_NUM_THREADS"] = str(cores)
    om = orc.openmp()
    t0 = time.perf_counter()
    par = om.rk4(g, p.b, q0, p_full.dt, nst)
    sec_par = time.perf_counter() - t0
    return {"value": 4 * n * n * nst / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"same recipe at {n}x{n} (dx = 0.1), {nst} RK4 steps, single-threaded C, "
                      f"{sec:.1f} s",
            "all_cores": {"value": 4 * n * n * nst / sec_par, "cores": cores,
                          "same_result": bool((ref == par).all()),
                          "sample": f"the same sample, OpenMP build of the oracle, {sec_par:.1f} s"}}


def run_ours(args) -> None:
    import torch
    from paper_2601_02540_b300 import sgn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)

    p = inputs.workload3(args.size, args.size)
    cells = p.nx * p.ny
    hbm_peak, hbm_kind = _peaks()
    fp64 = measure_fp64_peak(torch, local)
    results = {}
    finals = {}
    drift = {}
    for prec in ("f64", "f32", "f32_f64acc", "df64"):
        s = sgn.Solver.from_problem(p, prec=prec)
        q = s.state(p.q0)
        s.init_aux(q)
        q_init = q.clone()
        if prec == "f64":
            with ClockSampler(local) as clk:
                ms, launches = _time_steps(torch, s, q, p.dt, args.steps, args.warmup, dist)
            clocks = clk.summary()
        else:
            ms, launches = _time_steps(torch, s, q, p.dt, args.steps, args.warmup, dist)
        results[prec] = {"value": replica_rate(cells, args.steps, ms, world), "ms_per_step": ms / args.steps,
                         "gpu_launches": launches,
                         "roofline": _roofline(prec, cells, ms, args.steps, hbm_peak, hbm_kind, fp64)}
        if prec == "f32":
            # the same FP32 steps with one launch per stage, for comparison
            s.set_stage_fusion(False)
            qu = q_init.clone()
            msu, lu = _time_steps(torch, s, qu, p.dt, args.steps, args.warmup, dist)
            s.set_stage_fusion(True)
            results["f32_unfused"] = {"value": replica_rate(cells, args.steps, msu, world),
                                      "ms_per_step": msu / args.steps, "gpu_launches": lu,
                                      "roofline": _roofline("f32_unfused", cells, msu, args.steps, hbm_peak,
                                                            hbm_kind, fp64)}
            del qu
        if not args.no_drift:
            # the full job, outside the timed region: energy drift and final state
            q.copy_(q_init)
            d0 = s.mass_energy(q)
            s.step(q, p.dt, p.nsteps)
            d1 = s.mass_energy(q)
            drift[prec] = {"energy": abs(d1["energy"] - d0["energy"]) / abs(d0["energy"]),
                           "energy_shifted": abs(d1["energy_shifted"] - d0["energy_shifted"])
                           / abs(d0["energy_shifted"]),
                           "mass": abs(d1["mass"] - d0["mass"]) / abs(d0["mass"]),
                           "steps": p.nsteps}
            finals[prec] = q.double()
        if prec == "f64":
            e2e = _e2e(torch, s, p, q_init, args.steps)
        del q, q_init
        s.close()
        torch.cuda.empty_cache()

    errors = {}
    if "f64" in finals:
        ref = finals["f64"]
        for prec in ("f32", "f32_f64acc", "df64"):
            if prec in finals:
                d = (finals[prec] - ref).abs().amax(dim=(1, 2))
                den = ref.abs().amax(dim=(1, 2)).clamp_min(1e-3 * float(ref[0].abs().max()))
                errors[prec] = {f: float(v) for f, v in zip(("h", "u", "v", "w", "eta"),
                                                             (d / den).tolist())}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = _cpu_baseline(p) if world == 1 and not args.no_cpu else None
    ens = None if args.no_extra else _ensemble(torch, 1000, 5)
    adj = None if args.no_extra else _adjoint(torch)
    adapt = None if args.no_extra else _adaptive(torch, args.size, results["f64"]["ms_per_step"])
    relax = None if args.no_extra else _relaxed(torch, args.size, results["f64"]["ms_per_step"])
    mms = None if args.no_extra else _manufactured(torch)
    refl = None if args.no_extra else _reflecting(torch)
    small = None if args.no_extra else _small_grids(torch)
    obst = None if args.no_extra else {"f64": _gaussian_obstacle(torch, "f64"),
                                       "df64": _gaussian_obstacle(torch, "df64"),
                                       "f64_bs3": _gaussian_obstacle(torch, "f64", "bs3")}
    head = results["f64"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"periodic {p.nx}x{p.ny} SGN split-form SBP, RK4 (4 fused stages/step)",
                   "nx": p.nx, "ny": p.ny, "bc": "periodic", "dx": 0.1, "lambda": p.lam,
                   "g": p.g, "dt": p.dt, "job_steps": p.nsteps, "cells": cells,
                   "l2": f"inputs larger than L2 ({5 * cells * 8 / 1e9:.2f} GB FP64 state), no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": head["roofline"],
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": head["gpu_launches"],
        "clocks": clocks,
        "variants": {DTYPE_NAME[k]: {"value": v["value"], "ms_per_step": v["ms_per_step"],
                                     "roofline": v["roofline"]} for k, v in results.items()
                     if k != "f64"},
        "ensemble": ens,
        "adjoint": adj,
        "adaptive": adapt,
        "relaxed": relax,
        "manufactured": mms,
        "gaussian_obstacle": obst,
        "reflecting": refl,
        "small_grids": small,
        "energy_drift": drift,
        "errors_vs_f64_after_job": errors,
        "kernel_hash": _kernel_hash(),
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def _ensemble(torch, steps: int, warmup: int, loop_steps: int = 50) -> dict:
    """Ragged ensemble (256 instances, N in {128,...,512}, half periodic, half
    reflecting, FP32 state, each with its own dt): the batched path (one
    launch per stage, or per two stages, over all instances, graph replays,
    autotuned tiling: tile height, per-tile or persistent kernel, two stages
    per launch) over `steps` steps (the job's 1000 by default), against a
    per-instance launch loop over `loop_steps`, both timed with CUDA events."""
    from paper_2601_02540_b300 import sgn
    probs = inputs.workload5()
    cells = sum(p.nx * p.ny for p in probs)
    bs = sgn.BatchSolver(probs, prec="f32")
    q = bs.pack([p.q0 for p in probs])
    bs.init_aux(q)
    # every tiling the autotuner searches, timed over one 26-step graph replay
    # on a copy of the state, then the autotuner's own choice
    per_tiling = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for r, pers, fuse in ((1, False, False), (2, False, False), (4, False, False), (1, True, False),
                          (2, True, False), (2, False, True)):
        bs.set_persistent(False)
        bs.set_rows(r)
        bs.set_persistent(pers)
        bs.set_stage_fusion(fuse)
        w = q.clone()
        bs.step(w, 26)
        torch.cuda.synchronize()
        e0.record()
        bs.step(w, 26)
        e1.record()
        torch.cuda.synchronize()
        name = "rows2_two_stages_per_launch" if fuse else f"rows{r}_{'persistent' if pers else 'per_tile'}"
        per_tiling[name] = 4.0 * cells * 26 / (e0.elapsed_time(e1) * 1e-3)
        del w
    bs.set_persistent(False)
    rows = bs.autotune(q)
    tiling = bs.tiling()
    bs.step(q, warmup)
    torch.cuda.synchronize()
    e0.record()
    bs.step(q, steps)
    e1.record()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    d = bs.mass_energy(q)
    bs.close()
    solvers = [sgn.Solver.from_problem(p, prec="f32") for p in probs]
    states = [s.init_aux(s.state(p.q0)) for s, p in zip(solvers, probs)]
    for s, st, p in zip(solvers, states, probs):
        s.step(st, p.dt, warmup)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(loop_steps):
        for s, st, p in zip(solvers, states, probs):
            s.step(st, p.dt, 1)
    e1.record()
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1)
    for s in solvers:
        s.close()
    rate_b = 4.0 * cells * steps / (ms_batch * 1e-3)
    rate_l = 4.0 * cells * loop_steps / (ms_loop * 1e-3)
    fused = bool(tiling.get("fused")) and not tiling.get("persistent")
    bpcs = BYTES_PER_CELL_STAGE["f32" if fused else "f32_unfused"]
    hbm = bpcs * rate_b / 1e9
    peak, kind = _peaks()
    return {"workload": "256 instances N~U{128,192,256,384,512}, half periodic/half reflecting, FP32",
            "cells": cells, "steps": steps, "value": rate_b, "unit": UNIT, "wall_ms": ms_batch,
            "per_instance_loop": rate_l, "loop_steps": loop_steps, "speedup_vs_loop": rate_b / rate_l,
            "rows": rows, "tiling": tiling, "per_tiling_rate": per_tiling,
            "hbm_gbs": hbm, "hbm_frac": hbm / peak, "hbm_peak_kind": kind,
            "algorithmic_bytes_per_cell_stage": bpcs,
            "single_stage_hbm_roof": _single_stage_roof(rate_b, peak),
            "mass_finite": bool(np.all(np.isfinite(d)))}


def _single_stage_roof(rate: float, hbm_peak: float) -> dict:
    """The FP32 rate against the HBM roof of one launch per stage (the 74 B
    per cell-stage that scheme must move): the highest rate any single-stage
    FP32 kernel could reach at the measured copy bandwidth."""
    bpcs = BYTES_PER_CELL_STAGE["f32_unfused"]
    roof = hbm_peak * 1e9 / bpcs
    return {"bytes_per_cell_stage": bpcs, "roof_rate": roof, "value_over_roof": rate / roof}


def _adjoint(torch, nsteps: int = 0) -> dict:
    """Inversion workload: 512^2 reflecting, 2000 RK4 steps, 16 gauges read
    every 10 steps, checkpoints every 100 steps; time of the forward rollout
    (with checkpoints; the last segment keeps its stage states) and of the
    backward pass (recomputation of the other segments with stage stashes +
    adjoint steps): with the tapes of the stage RHS evaluations recorded by
    the recomputation (the default), without them (the adjoint evaluates
    each stage's tape), and with every stage state kept (no recomputation,
    no tape)."""
    from paper_2601_02540_b300 import adjoint, sgn
    p = inputs.workload4()
    if nsteps > 0:
        p.nsteps = nsteps
    s = sgn.Solver.from_problem(p, prec="f64")
    gauges = torch.as_tensor(p.extra["gauges"], device="cuda")
    b = torch.as_tensor(p.b, device="cuda").requires_grad_(True)
    h0 = torch.as_tensor(p.q0[0], device="cuda").requires_grad_(True)
    obs = torch.zeros((p.nsteps // p.extra["every"], gauges.numel()), dtype=torch.float64, device="cuda")
    # warm-up with the same operations (loads every kernel module once)
    for tape in (True, False):
        out = adjoint.gauge_rollout(b, h0, s, p.dt, 20, p.extra["every"], gauges, 10, tape)
        torch.sum((out - obs[: out.shape[0]]) ** 2).backward()
        b.grad = None
        h0.grad = None
    res = {"workload": f"reflecting 512x512, {p.nsteps} RK4 steps, 16 gauges every 10 steps, FP64"}
    TP = 4 * sgn.TAPE_PLANES
    for name, K, tape in (("checkpoint_K100", 100, True), ("checkpoint_K100_no_tape", 100, False),
                          ("all_stages_kept", 0, False)):
        b.grad = None
        h0.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = adjoint.gauge_rollout(b, h0, s, p.dt, p.nsteps, p.extra["every"], gauges, K, tape)
        loss = torch.sum((out - obs) ** 2)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        fwd, bwd = t1 - t0, t2 - t1
        res[name] = {"forward_s": fwd, "backward_s": bwd, "backward_over_forward": bwd / fwd,
                     "total_over_forward": (fwd + bwd) / fwd,
                     # K > 0: two K-step stashes (the recomputation of the next segment
                     # overlaps the walk of the current one)
                     "stash_gb": ((2 * min(K, p.nsteps)) if K > 0 else p.nsteps) * 20 * p.nx * p.ny * 8 / 1e9,
                     "tape_gb": (2 * min(K, p.nsteps) * TP * p.nx * p.ny * 8 / 1e9) if tape else 0.0}
        del out, loss
        torch.cuda.empty_cache()
    s.close()
    return res


RHS_PER_ATTEMPT = {"p5s3": 5, "bs3": 3}


def _adaptive(torch, size: int, rk4_ms_per_step: float) -> dict:
    """The paper's time path (Sec. 6): adaptive third-order FSAL integration,
    rtol = atol = 1e-6, on the benchmark workload (FP64), over the job's time
    span (500 fixed CFL steps), first step the CFL step; with the five-stage
    pair (the kind the paper uses) and, for comparison, Bogacki-Shampine 3(2).
    Wall-clock time of the whole call (the host reads the error norm after
    every attempt); one RHS evaluation per node and stage counts as one
    cell-stage.  The fixed-step RK4 job time over the same span is given for
    comparison."""
    from paper_2601_02540_b300 import sgn
    p = inputs.workload3(size, size)
    s = sgn.Solver.from_problem(p, prec="f64")
    q0 = s.state(p.q0)
    s.init_aux(q0)
    q = q0.clone()
    T = p.nsteps * p.dt
    cells = p.nx * p.ny
    out = {"workload": f"periodic {p.nx}x{p.ny}, t in [0, {p.nsteps} dt_cfl], rtol = atol = 1e-6, FP64",
           "rk4_fixed_step_job_s": rk4_ms_per_step * p.nsteps / 1e3}
    for pair in ("p5s3", "bs3"):
        s.step_adaptive(q, 0.0, 2 * p.dt, p.dt, want_history=False, pair=pair)   # warm-up (loads the kernels)
        q.copy_(q0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, hist = s.step_adaptive(q, 0.0, T, p.dt, pair=pair)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        rhs_evals = RHS_PER_ATTEMPT[pair] * st["attempts"] + 1
        out[pair] = {"accepted": st["accepted"], "rejected": st["rejected"], "rhs_evaluations": rhs_evals,
                     "mean_accepted_dt_over_cfl": float(np.mean([h[0] for h in hist if h[2] == 1.0]) / p.dt),
                     "wall_s": wall, "value": rhs_evals * cells / wall, "unit": "cell-stages/s",
                     "ms_per_rhs": wall / rhs_evals * 1e3}
    s.close()
    return out


def _relaxed(torch, size: int, rk4_ms_per_step: float, nsteps: int = 20) -> dict:
    """Relaxation RK4 (energy-conserving) on the benchmark workload, FP64:
    ms per step (4 fused stages + the energy-change reduction, a host read of
    its sums, Newton for gamma, the relaxed update) against plain RK4, and the
    energy drift of both over the same steps."""
    from paper_2601_02540_b300 import sgn
    p = inputs.workload3(size, size)
    s = sgn.Solver.from_problem(p, prec="f64")
    q0 = s.state(p.q0)
    s.init_aux(q0)
    q = q0.clone()
    dt = 4.0 * p.dt                              # CFL number 0.8: RK4's energy error shows in 20 steps
    s.step_relaxed(q, dt, 2)                     # warm-up (loads the kernels, allocates)
    q.copy_(q0)
    e0 = s.mass_energy(q)["energy_shifted"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gam, t = s.step_relaxed(q, dt, nsteps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    er = abs(s.mass_energy(q)["energy_shifted"] - e0) / abs(e0)
    q.copy_(q0)
    s.step(q, dt, nsteps)
    e4 = abs(s.mass_energy(q)["energy_shifted"] - e0) / abs(e0)
    s.close()
    return {"workload": f"periodic {p.nx}x{p.ny}, {nsteps} relaxed RK4 steps of 4 dt_cfl, FP64",
            "ms_per_step": wall / nsteps * 1e3, "rk4_ms_per_step": rk4_ms_per_step,
            "overhead": wall / nsteps * 1e3 / rk4_ms_per_step - 1.0,
            "gamma_minus_1_max": float(np.max(np.abs(np.array(gam) - 1.0))),
            "energy_drift_relaxed": er, "energy_drift_rk4": e4}


def _small_grids(torch) -> dict:
    """The launch-bound workloads at their stated lengths, FP64 RK4: the
    periodic 64^2 hump (200 steps) and the reflecting 1024x512 workload (2000
    steps).  sgn_step replays 50-step CUDA graphs on grids of at most 2^21
    nodes; the same steps issued one call per step take the direct launches.
    Both timed with CUDA events over the whole run, after a warm-up run."""
    from paper_2601_02540_b300 import sgn
    out = {"unit": UNIT}
    for name, p in (("workload1_64x64_200", inputs.workload1()), ("workload2_1024x512_2000", inputs.workload2())):
        s = sgn.Solver.from_problem(p, prec="f64")
        q0 = s.state(p.q0)
        s.init_aux(q0)
        row = {"steps": p.nsteps, "cells": p.nx * p.ny}
        for mode in ("graph", "direct"):
            q = q0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for rep in range(2):                 # the first run is the warm-up (and captures the graph)
                q.copy_(q0)
                torch.cuda.synchronize()
                e0.record()
                if mode == "graph":
                    s.step(q, p.dt, p.nsteps)
                else:
                    for _ in range(p.nsteps):
                        s.step(q, p.dt, 1)
                e1.record()
                torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row[mode] = {"ms": ms, "value": 4.0 * p.nx * p.ny * p.nsteps / (ms * 1e-3)}
            if mode == "graph":
                qg = q.clone()
            else:
                row["equal_bitwise"] = bool(torch.equal(q, qg))
        row["graph_speedup"] = row["direct"]["ms"] / row["graph"]["ms"]
        out[name] = row
        s.close()
    return out


def _reflecting(torch, steps: int = 20, warmup: int = 3) -> dict:
    """Reflecting walls (SATs and one-sided boundary rows): the workload-2
    recipe (reflecting [0,200]x[0,100], bumpy bathymetry, one hump) at its own
    size 1024x512 and scaled to 8192x4096 nodes, RK4 in each precision, timed
    like the periodic line."""
    from paper_2601_02540_b300 import sgn
    out = {}
    for nx, ny in ((1024, 512), (8192, 4096)):
        p = inputs.workload2(nx, ny)
        row = {"workload": f"reflecting {nx}x{ny} (workload-2 recipe), RK4"}
        for prec in ("f64", "f32", "f32_f64acc", "df64"):
            s = sgn.Solver.from_problem(p, prec=prec)
            q = s.state(p.q0)
            s.init_aux(q)
            ms, _ = _time_steps(torch, s, q, p.dt, steps, warmup)
            row[prec] = 4.0 * nx * ny * steps / (ms * 1e-3)
            del q
            s.close()
        out[f"{nx}x{ny}"] = row
    torch.cuda.empty_cache()
    return {"unit": UNIT, **out}


def _gaussian_obstacle(torch, prec: str = "f64", pair: str = "p5s3") -> dict:
    """The paper's headline GPU run shape (solitary wave over a Gaussian
    obstacle, 1600 x 800 periodic, to t = 12) with its time path: an adaptive
    third-order FSAL pair at rtol = atol = 1e-6 from the CFL step (the
    five-stage pair, the kind of integrator the paper names; its coefficients
    are this library's, so the step sequence is not the paper's).  Wall-clock
    time to solution, inputs already on the device.  The paper's H200 figure
    (12.7 s, FP64) is for its whole experiment including analysis, with the
    hyperbolic traveling wave as initial data: context, not the same
    measurement."""
    from paper_2601_02540_b300 import sgn
    p = inputs.gaussian_obstacle()
    s = sgn.Solver.from_problem(p, prec=prec)
    q0 = s.state(p.q0)
    s.init_aux(q0)
    q = q0.clone()
    s.step_adaptive(q, 0.0, 20 * p.dt, p.dt, want_history=False, pair=pair)      # warm-up
    q.copy_(q0)
    T = p.extra["t_end"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, hist = s.step_adaptive(q, 0.0, T, p.dt, max_attempts=1000000, pair=pair)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    d = s.mass_energy(q)
    d0 = s.mass_energy(q0)
    s.close()
    rhs = RHS_PER_ATTEMPT[pair] * st["attempts"] + 1
    return {"workload": f"gaussian obstacle {p.nx}x{p.ny} periodic, t in [0, {T}], adaptive tol 1e-6, "
                        f"{prec}, pair {pair}",
            "wall_s": wall, "t_reached": st["t"], "accepted": st["accepted"], "rejected": st["rejected"],
            "rhs_evaluations": rhs, "ms_per_rhs": wall / rhs * 1e3,
            "mean_dt": T / max(st["accepted"], 1), "dt_cfl": p.dt,
            "mass_drift": abs(d["mass"] - d0["mass"]) / abs(d0["mass"]),
            "paper_h200_s": 12.7}


def _manufactured(torch) -> dict:
    """The paper's convergence study (Sec. 6.1.2) on the GPU: the manufactured
    solution on [-1,1]^2, lambda = 500, to t = 1, RK4 with the source terms
    fused into the stages, N = 32..256; errors in the discrete L2 norm of the
    mass matrix and in the max norm, and the observed orders."""
    from paper_2601_02540_b300 import sgn
    out = {"workload": "manufactured solution (Sec. 6.1.2), [-1,1]^2, lambda = 500, t = 1, FP64"}
    for bc, name in ((inputs.PERIODIC, "periodic"), (inputs.REFLECTING, "reflecting")):
        l2s, mxs, sizes = [], [], (32, 64, 128, 256)
        for n in sizes:
            s = sgn.Solver(n, n, -1.0, 1.0, -1.0, 1.0, bc, torch.zeros((n, n), dtype=torch.float64, device="cuda"),
                           9.81, 500.0)
            q, b = s.mms_exact(0.0, with_b=True)
            s.set_bathymetry(b)
            dx = 2.0 / n if bc == inputs.PERIODIC else 2.0 / (n - 1)
            c = 0.3 + np.sqrt(9.81 * 2.7 + 500.0 / 3.0)
            nsteps = int(np.ceil(1.0 / (0.3 * dx / c)))
            s.step_mms(q, 0.0, 1.0 / nsteps, nsteps)
            e = (q - s.mms_exact(1.0)).cpu().numpy()
            s.close()
            w = np.ones(n)
            if bc == inputs.REFLECTING:
                w[0] = w[-1] = 0.5
            M = np.outer(w, w)
            l2s.append(np.sqrt(np.sum(M * e * e, axis=(1, 2)) / np.sum(M)))
            mxs.append(np.max(np.abs(e), axis=(1, 2)))
        l2s, mxs = np.array(l2s), np.array(mxs)
        out[name] = {"n": list(sizes),
                     "l2_error_h_u_v_w_eta": l2s.tolist(),
                     "l2_order_last": np.log2(l2s[-2] / l2s[-1]).tolist(),
                     "max_order_last": np.log2(mxs[-2] / mxs[-1]).tolist()}
    return out


def _e2e(torch, s, p, q_init_dev, steps: int) -> dict:
    """Same metric through the library's host-memory entry point
    (sgn_step_host, one C-ABI call): the library copies the state in from
    pinned host memory, runs the steps with the mass, energy and shifted
    energy of every new state reduced in the fused fourth stage, reads those
    per-step results back, and copies the final state back over the host
    buffer, all inside the timed region."""
    host = q_init_dev.cpu().pin_memory()
    warm = host.clone()
    s.step_host(warm, p.dt, steps)     # device state and monitor buffer allocated outside the timing
    del warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    diag = s.step_host(host, p.dt, steps)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    assert len(diag) == steps
    nbytes = host.numel() * host.element_size()
    return {"value": 4.0 * p.nx * p.ny * steps / sec, "unit": UNIT,
            "h2d_bytes_per_step": nbytes / steps, "d2h_bytes_per_step": (nbytes + 24 * steps) / steps,
            "how": f"sgn_step_host over {steps} steps: one copy of the state each way (amortized per step "
                   "above) and the 24-byte monitor of every step"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as orc
    p = inputs.workload3(256, 256)
    g = orc.Grid(p.nx, p.ny, p.xmin, p.xmax, p.ymin, p.ymax, p.bc, p.g, p.lam)
    q = orc.init_aux(g, p.b, p.q0)
    for _ in range(args.warmup):
        q = orc.rk4(g, p.b, q, p.dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q = orc.rk4(g, p.b, q, p.dt, 1)
    sec = time.perf_counter() - t0
    value = 4.0 * p.nx * p.ny * args.steps / sec
    sample = "periodic workload recipe at 256x256 (dx = 0.1), one RK4 step per bench step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "periodic 8192x8192 SGN split-form SBP, RK4 (4 fused stages/step)",
                   "sampled_as": "256x256"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-drift", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the ensemble and adjoint legs")
    ap.add_argument("--size", type=int, default=8192,
                    help="grid side (8192 = the workload; smaller sizes only for profiling)")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="NSTEPS",
                    help="run only the adjoint leg with NSTEPS RK4 steps and print its JSON (profiling)")
    ap.add_argument("--ensemble-only", type=int, default=0, metavar="NSTEPS",
                    help="run only the ensemble leg, timing NSTEPS steps, and print its JSON (profiling)")
    ap.add_argument("--adaptive-only", type=int, default=0, metavar="SIZE",
                    help="run only the adaptive leg on a SIZE x SIZE grid and print its JSON (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.adjoint_only > 0:
        import torch
        print(json.dumps({"adjoint": _adjoint(torch, args.adjoint_only)}))
        return
    if args.adaptive_only > 0:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"adaptive": _adaptive(torch, args.adaptive_only, float("nan"))}))
        return
    if args.ensemble_only > 0:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"ensemble": _ensemble(torch, args.ensemble_only, 5, loop_steps=5)}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
