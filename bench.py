"""Benchmark: zone-updates per second per IMEX stage of the resistive relativistic
MHD step (arXiv 2110.03732) on one GB300, FP64.

Workload: the 2-D resistive relativistic Orszag-Tang vortex, periodic [0, 2 pi]^2,
512 x 512 cells, Gamma = 4/3, eta = 1e-4, synthetic initial data from
paper_2110_03732_gb300.problems.  One timed step = one full IMEX-SSP2(2,2,2) step:
two stages, each an implicit E + velocity solve and the explicit MC/HLL/UCT/CT
operator, with the final combination folded into the last stage.  The time step is
fixed for a fixed metric and is computed once before timing.

value = interior cells x stages per step / seconds per step, whole job (N ranks each
advance an independent replica: weak scaling, no data-path collective).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "zone-updates/s per IMEX stage (FP64 vs mixed, 1 GB300, % HBM roofline); p50/p99 run latency"
UNIT = "zone-updates/s"
N_OT = 512
STAGES = 2

# Algorithmic HBM bytes per zone-stage of one IMEX stage (FP64, flat metric, uniform
# eta): each datum once; stage 1 reads q^n (11 doubles) and writes its increments
# (11 + 3), stage 2 reads q^n, the increments and writes q^{n+1} (37 doubles): mean
# 31.5 doubles = 252 B per zone-stage (uniform eta saves the 8 B per-cell field).
ALG_BYTES_PER_ZONE_STAGE = 252.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--n", type=int, default=N_OT, help=argparse.SUPPRESS)
    ap.add_argument("--case", choices=["star", "star_mixed", "clean", "ot", "ot_mixed"], default=None,
                    help="run one workload alone (for profiling) and print its timings: the 3-D star (FP64 or mixed) with "
                         "--case-n cells a side, the multigrid cleaning of the --case-n^2 Orszag-Tang problem, "
                         "or the --case-n^2 Orszag-Tang step in FP64 or mixed precision")
    ap.add_argument("--case-n", type=int, default=96)
    return ap.parse_args()


def run_case(args, grmhd, P, dev):
    """One secondary workload alone, `--warmup` untimed then `--steps` timed
    repetitions (CUDA events on the current stream)."""
    import torch
    n = args.case_n
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if args.case in ("star", "star_mixed", "ot", "ot_mixed"):
        if args.case.startswith("star"):
            prec = "mixed" if args.case == "star_mixed" else "fp64"
            S = grmhd.Solver.from_problem(P.star(n), device=dev, precision=prec)
            name = f"star_3d_{n}^3_{prec}"
        else:
            prec = "mixed" if args.case == "ot_mixed" else "fp64"
            S = grmhd.Solver.from_problem(P.orszag_tang(n), device=dev, precision=prec)
            name = f"orszag_tang_2d_{n}^2_{prec}"
        dt = S.compute_dt()
        for _ in range(args.warmup):
            S.step(dt)
        torch.cuda.synchronize()
        S.set_timing(True)
        S.kernel_times()
        e0.record()
        for _ in range(args.steps):
            S.step(dt)
        e1.record()
        e1.synchronize()
        kt = S.kernel_times()
        return {"case": name, "ms_per_step": e0.elapsed_time(e1) / args.steps,
                "us_per_launch": {k: 1e3 * v[0] / max(v[1], 1) for k, v in kt.items()},
                "newton_failures": S.diagnostics()[2]}
    S = grmhd.Solver.from_problem(P.orszag_tang(n), device=dev)
    S.step(S.compute_dt())
    out = {"case": f"multigrid_clean_orszag_tang_{n}^2"}
    for cyc in (1, 4):
        for _ in range(args.warmup):
            S.clean_divb(cyc)
        e0.record()
        for _ in range(args.steps):
            S.clean_divb(cyc)
        e1.record()
        e1.synchronize()
        out[f"{cyc}_cycles_ms"] = e0.elapsed_time(e1) / args.steps
    out["divb_max_after"] = S.diagnostics()[0][2]
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device):
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Algorithmic bytes per 512^2 launch of the mixed-precision kernels (each datum once,
# flat 2-D grid).  The stencil launch (the fluxes of both directions and the edge EMFs
# in one kernel) reads per cell the 10 FP32 values each face state needs (8 primitives
# and the 2 transverse cell q_B) once per direction (80 B), writes 16 FP32 fluxes and
# the 2 degenerate FP64 edge EMFs the flux tasks own (80 B), and for the z-edges reads
# E_z (FP32) and the two face q_B (FP64) and writes the FP64 EMF (28 B): 188 B.  The
# update reads the 16 FP32 fluxes and the FP32 primitives its sources use (u^1..3,
# E^1..2: 21 floats, 84 B) and, in doubles, q^n or the running sum (11), R (3) and the
# edge EMFs (3), and writes the later-stage base and the running sum (22, stage 0) or
# q^{n+1} (11, stage 1): 84 B + 33.5 doubles on average.
MIXED_ALG_BYTES_PER_CELL = {"stencil": 188.0, "update": 84.0 + 33.5 * 8}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: begin the timed region once it samples
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(n_sample, steps):
    """The CPU oracle as it stands (single thread) on a bounded sample of the same
    workload: `steps` IMEX steps of the Orszag-Tang problem at n_sample^2 cells."""
    import oracle
    from paper_2110_03732_gb300 import problems as P
    pr = P.orszag_tang(n_sample)
    st = oracle.from_problem(pr)
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    t0 = time.perf_counter()
    for _ in range(steps):
        st.step(dt)
    el = time.perf_counter() - t0
    return n_sample * n_sample * STAGES * steps / el, el


def _oracle_worker(n_sample, warmup, steps, barrier, out):
    """One host core: the oracle as it stands on its own copy of the sampled workload;
    waits for every worker before timing so that all cores run together."""
    import oracle
    from paper_2110_03732_gb300 import problems as P
    pr = P.orszag_tang(n_sample)
    st = oracle.from_problem(pr)
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    for _ in range(warmup):
        st.step(dt)
    barrier.wait()
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        st.step(dt)
        times.append(time.perf_counter() - t0)
    out.put(times)


def oracle_all_cores(n_sample, warmup, steps, procs=None):
    """The oracle on every host core at once (one process per core, started with
    spawn, each on its own n_sample^2 copy): aggregate zone-updates/s per stage =
    the work of all processes / the slowest process's time.  Returns (value,
    ms per step of the slowest process, processes)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    out = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(n_sample, warmup, steps, barrier, out)) for _ in range(procs)]
    for p_ in ps:
        p_.start()
    res = [out.get() for _ in range(procs)]
    for p_ in ps:
        p_.join()
    slow = max(sum(r) for r in res)
    value = procs * n_sample * n_sample * STAGES * steps / slow
    return value, 1e3 * slow / steps, procs


def run_reference(args):
    """--impl reference: the oracle on the host cores, same metric and workload family,
    each step a bounded sample (one IMEX step at 256^2 of the same initial data)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n_s = 256
    value, ms, procs = oracle_all_cores(n_s, args.warmup, args.steps)
    sample = (f"orszag_tang_2d {n_s}x{n_s} (quarter-size sample of the 512^2 workload) on each of {procs} host "
              f"cores at once, one IMEX-SSP2 step per timed step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"orszag_tang_2d_{N_OT}x{N_OT}_fp64", "cells": N_OT * N_OT,
                       "stages_per_step": STAGES, "sample_cells": n_s * n_s},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2110_03732_gb300 import build as _b
    from paper_2110_03732_gb300 import grmhd
    from paper_2110_03732_gb300 import problems as P
    _b.build()
    if args.case:
        print(json.dumps(run_case(args, grmhd, P, dev)), flush=True)
        return

    n = args.n
    pr = P.orszag_tang(n)
    S = grmhd.Solver.from_problem(pr, device=dev)
    dt = S.compute_dt()
    cells = S.cells
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    for _ in range(max(args.warmup, 3)):
        S.step(dt)
    torch.cuda.synchronize()
    ck = S.checkpoint()   # the kernel-timing pass below replays the same steps from here
    launches0 = S.launch_count()

    clocks = ClockSampler(torch.cuda.current_device())
    if rank == 0:
        clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        S.step(dt)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if rank == 0 else None
    launches = S.launch_count() - launches0

    # per-kernel device times: CUDA events on the launching stream around every launch,
    # over a second timed pass that replays the same steps from the same state (events
    # between the launches serialise them, so the pass above runs without them); the
    # replay must end bitwise where the timed pass ended
    end_state = S.state.clone()
    S.restore(ck)
    S.set_timing(True)
    S.kernel_times()
    kpass_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        S.step(dt)
        e1.record(stream)
        e1.synchronize()
        kpass_ms.append(e0.elapsed_time(e1))
        ktimes = S.kernel_times()   # fold this step's per-kernel events
    ktimes = {k: v for k, v in S.kernel_times().items() if v[1] > 0}   # no EMF kind: fused into the stencil
    S.set_timing(False)
    torch.cuda.synchronize()
    replay_bitwise = bool(torch.equal(S.state, end_state))
    del end_state, ck

    total_s = max_over_ranks(sum(step_ms) / 1e3, dev)
    ms_per_step = 1e3 * total_s / args.steps
    value = ws * cells * STAGES * args.steps / total_s

    # end to end: the same step through the public API with the state in pinned host
    # memory, host->device copy of the inputs and device->host copy of the result
    # inside the timed region
    host_state = S.state.detach().cpu().pin_memory()      # q (8) and the face fields (3)
    h2d = host_state.numel() * host_state.element_size()
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.state.copy_(host_state, non_blocking=True)
        S.step(dt)
        host_state.copy_(S.state, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = ws * cells * STAGES / (float(np.mean(e2e_ms)) / 1e3)

    divb, tot, nfail = S.diagnostics()

    # elliptic cleaning (Sec. 3.3) of the same state: multigrid V-cycles on the 512^2
    # field, timed alone (the paper applies one cleaning after every step)
    clean = {}
    for cyc in (1, 4):
        S.clean_divb(cyc)
        torch.cuda.synchronize()
        cl_ms = []
        for _ in range(min(20, max(3, args.steps))):
            flush.zero_()
            e0.record(stream)
            S.clean_divb(cyc)
            e1.record(stream)
            e1.synchronize()
            cl_ms.append(e0.elapsed_time(e1))
        clean[f"{cyc}_cycles_ms"] = float(np.median(cl_ms))
    clean["divb_max_after"] = S.diagnostics()[0][2]

    def kernel_pass(Sv, steps):
        """Per-kernel CUDA-event times over `steps` further steps (launches serialised)."""
        Sv.set_timing(True)
        Sv.kernel_times()
        for _ in range(steps):
            flush.zero_()
            Sv.step(dt)
            kt = Sv.kernel_times()
        kt = Sv.kernel_times()
        Sv.set_timing(False)
        torch.cuda.synchronize()
        return kt

    def time_variant(**kw):
        """The same workload and timing rules with another solver configuration."""
        Sv = grmhd.Solver.from_problem(pr, device=dev, **kw)
        for _ in range(max(args.warmup, 3)):
            Sv.step(dt)
        torch.cuda.synchronize()
        ms_l = []
        for _ in range(args.steps):
            flush.zero_()
            e0.record(stream)
            Sv.step(dt)
            e1.record(stream)
            e1.synchronize()
            ms_l.append(e0.elapsed_time(e1))
        total = max_over_ranks(sum(ms_l) / 1e3, dev)
        out = {"value": ws * cells * STAGES * args.steps / total, "unit": UNIT,
               "ms_per_step": 1e3 * total / args.steps, "p50_ms_per_step": float(np.percentile(ms_l, 50)),
               "p99_ms_per_step": float(np.percentile(ms_l, 99))}
        return out, Sv

    # mixed precision (FP32 reconstruction, HLL, edge EMF and sources; FP64 implicit
    # solve, CT and stage combination)
    mixed, Sm = time_variant(precision="mixed")
    mixed["dtype"] = ("f32 reconstruction/HLL/edge EMF/sources, double-word flux divergence, f64 implicit "
                      "solve/CT/stage combination")
    mixed_kt = kernel_pass(Sm, args.steps)
    del Sm
    # GLM hyperbolic cleaning (Sec. 3.1, cell-centred B, kappa_B = 1) instead of CT
    glm, Sg = time_variant(divb="glm", kappa=1.0)
    glm.update({"dtype": "f64", "kappa_b": 1.0, "divb_cell_central_max": Sg.diagnostics()[0][2],
                "scheme": "GLM hyperbolic cleaning with cell-centred B instead of staggered CT"})
    del Sg
    # PPM reconstruction (Sec. 5) and the ideal-limit edge EMF (App. A)
    ppm, _ = time_variant(rec="ppm")
    ppm.update({"dtype": "f64", "scheme": "PPM reconstruction of every face and edge state instead of MC"})
    ppm_mixed, _ = time_variant(rec="ppm", precision="mixed")
    ppm_mixed.update({"dtype": "f32 PPM reconstruction/HLL/edge EMF/sources, f64 implicit solve/CT",
                      "scheme": "PPM on the mixed-precision path"})
    ideal, _ = time_variant(emf="ideal")
    ideal.update({"dtype": "f64", "scheme": "ideal-limit HLL UCT (App. A) instead of the resistive edge EMF"})

    # the 3-D magnetised star on its fixed conformally flat metric (256^3, outflow,
    # atmosphere): the metric kernels at 17M cells; inputs far exceed L2
    Ss = grmhd.Solver.from_problem(P.star(256), device=dev)
    dts = Ss.compute_dt()
    for _ in range(3):
        Ss.step(dts)
    torch.cuda.synchronize()
    star_ms = []
    for _ in range(10):
        e0.record(stream)
        Ss.step(dts)
        e1.record(stream)
        e1.synchronize()
        star_ms.append(e0.elapsed_time(e1))
    star_total = max_over_ranks(sum(star_ms) / 1e3, dev)
    star = {"workload": "star_3d_256^3_fp64 (fixed conformally flat metric, outflow, atmosphere)",
            "value": ws * Ss.cells * STAGES * 10 / star_total, "unit": UNIT, "ms_per_step": 1e3 * star_total / 10,
            "steps": 10, "newton_failures": Ss.diagnostics()[2]}
    del Ss
    # the same star on the mixed-precision path
    Ss = grmhd.Solver.from_problem(P.star(256), device=dev, precision="mixed")
    for _ in range(3):
        Ss.step(dts)
    torch.cuda.synchronize()
    sm_ms = []
    for _ in range(10):
        e0.record(stream)
        Ss.step(dts)
        e1.record(stream)
        e1.synchronize()
        sm_ms.append(e0.elapsed_time(e1))
    sm_total = max_over_ranks(sum(sm_ms) / 1e3, dev)
    star_mixed = {"workload": "star_3d_256^3_mixed (FP32 reconstruction/HLL/edge EMF)",
                  "value": ws * Ss.cells * STAGES * 10 / sm_total, "unit": UNIT, "ms_per_step": 1e3 * sm_total / 10,
                  "steps": 10, "newton_failures": Ss.diagnostics()[2]}
    del Ss
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    pk, pk_src = peaks()
    from paper_2110_03732_gb300 import roofline as RL
    counts = RL.load_counts()
    probe = grmhd.fp64_fma_rate()
    # dominant kernel by measured time inside the timed region
    kname = max(ktimes, key=lambda k: ktimes[k][0])
    kms, kn = ktimes[kname]
    k_avg_ms = kms / max(kn, 1)
    tot_kernel_ms = sum(v[0] for v in ktimes.values())
    roof = RL.alu_entry(counts, "fp64", kname, k_avg_ms, probe)
    roof["inst_issue_frac"] = RL.issue_entry(counts, "fp64", kname, k_avg_ms).get("frac")
    # mixed precision: the dominant kernel, and the FP32 stencil kernels against HBM
    mixed_kt = {k: v for k, v in mixed_kt.items() if v[1] > 0}   # kinds that launched (no EMF kind: fused)
    mk = max(mixed_kt, key=lambda k: mixed_kt[k][0])
    avg = {k: v[0] / v[1] for k, v in mixed_kt.items()}
    mixed["kernel_ms_per_step"] = {k: v[0] / args.steps for k, v in mixed_kt.items()}
    # the mixed kernels spread their work over the FP32, integer and FP64 pipes: the
    # dominant one is measured against the instruction issue rate (its FP64 figures
    # beside it), and every kind's issue fraction is listed
    mixed["roofline"] = RL.issue_entry(counts, "mixed", mk, avg[mk])
    mixed["issue_frac"] = {k: RL.issue_entry(counts, "mixed", k, avg[k]).get("frac") for k in avg}
    # the one stencil launch of the mixed path is timed (and counted) as the flux kind
    mixed["stencil_hbm"] = {k: RL.hbm_entry(counts, "mixed", kk, avg[kk], MIXED_ALG_BYTES_PER_CELL[k] * cells,
                                            pk["hbm_gbs"]) for k, kk in (("stencil", "flux"), ("update", "update"))}
    mixed["stencil_hbm_note"] = ("the 512^2 working set (~0.2 GB) stays in the 129 MB L2 between kernels only in "
                                 "part; traffic is DRAM bytes per launch from the stored ncu counts")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"orszag_tang_2d_{n}x{n}_fp64", "cells": cells, "stages_per_step": STAGES,
                   "eta": pr.eta_u, "gamma": pr.gamma, "cfl": pr.cfl, "dt": dt,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"},
        "p50_ms_per_step": float(np.percentile(step_ms, 50)), "p99_ms_per_step": float(np.percentile(step_ms, 99)),
        "kernel_timing": "CUDA events around every launch over a replay of the timed steps from a checkpoint",
        "kernel_pass_replays_bitwise": replay_bitwise,
        "ms_per_step_with_kernel_events": float(np.mean(kpass_ms)),
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in ktimes.items()},
        "kernel_share": {k: v[0] / tot_kernel_ms for k, v in ktimes.items()},
        "roofline": roof,
        "fp64_fma_probe_tflops": probe,
        "hbm_fraction_of_step": ALG_BYTES_PER_ZONE_STAGE * cells * STAGES / (ms_per_step / 1e3) / (pk["hbm_gbs"] * 1e9),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d},
        "gpu_launches": launches,
        "clocks": clk,
        "divb_max": divb[2], "newton_failures": nfail,
        "mixed": mixed,
        "elliptic_clean": dict(clean, scheme="multigrid V(2,2), staggered projection of q_B, 512^2"),
        "glm": glm,
        "ppm": ppm,
        "ppm_mixed": ppm_mixed,
        "ideal_emf": ideal,
        "star": star,
        "star_mixed": star_mixed,
    }
    line["tube_run"] = bench_tube(grmhd, P, dev)
    line["star_mixed_error"] = star_mixed_error(grmhd, P, dev)
    if not args.no_batched:
        line["batched"] = bench_batched(grmhd, P, dev, args)
        line["serving"] = bench_serving(dev, args)
    if not args.no_cpu_baseline:
        rate, el = cpu_oracle_rate(256, 2)
        allv, all_ms, procs = oracle_all_cores(256, 0, 2)
        line["cpu_baseline"] = {"value": allv, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"orszag_tang_2d 256x256, 2 IMEX-SSP2 steps on each of {procs} host cores "
                                          f"at once ({all_ms:.0f} ms per step on the slowest)",
                                "single_core": {"value": rate, "cores": 1,
                                                "sample": f"the same, one thread ({el:.1f} s)"}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def bench_batched(grmhd, P, dev, args):
    """256 independent Orszag-Tang boxes (sides drawn from 64..512, eta log-uniform in
    [1e-6, 1], seeded phases) advanced by one batched, autotuned, graph-captured step
    (mixed precision).  Inputs (~20 GB) exceed L2, so no flush is needed."""
    import torch
    probs = P.ot_batch(0, 256)
    solvers = [grmhd.Solver.from_problem(pr, device=dev, precision="mixed") for pr in probs]
    cells = sum(s.cells for s in solvers)
    B = grmhd.Batch(solvers)
    B.set_dt([s.compute_dt() for s in solvers])
    cfg = B.autotune(reps=2)
    for _ in range(3):
        B.step()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            B.step(stream=side)
    torch.cuda.current_stream().wait_stream(side)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = max(5, min(args.steps, 20))
    times = []
    for _ in range(k):
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    # the same boxes through the persistent launch: k steps in one cooperative launch
    B.step_persistent(1)
    torch.cuda.synchronize()
    e0.record()
    B.step_persistent(k, synchronize=False)
    e1.record()
    e1.synchronize()
    assert B.persistent_status() == 0
    ms_p = e0.elapsed_time(e1) / k
    nfail = sum(s.diagnostics()[2] for s in solvers[:8])
    out = {"workload": "256 Orszag-Tang boxes, sides U{64,128,256,512}, eta 10^U[-6,0], seed 0",
           "boxes": len(probs), "cells": cells, "precision": "mixed", "value": cells * STAGES / (ms / 1e3),
           "unit": UNIT, "ms_per_step": ms, "steps": k, "graph_captured": True,
           "launch_config": {kk: list(vv) for kk, vv in cfg.items()}, "newton_failures_first8": nfail,
           "persistent": {"value": cells * STAGES / (ms_p / 1e3), "ms_per_step": ms_p,
                          "launch": f"{k} steps in one cooperative launch (phases separated by grid barriers)"}}
    del graph, B, solvers
    torch.cuda.synchronize()
    out["small_problems"] = bench_small_batch(grmhd, P, dev)
    return out


def bench_small_batch(grmhd, P, dev, n_tubes=32, steps=200):
    """Many small problems, where launches dominate: 32 1-D shock tubes of 400-4096
    cells (seeded) in mixed precision, `steps` steps by the per-kind batched kernels
    (replayed from a CUDA graph of one step) and by the persistent launch (all steps in
    one cooperative launch)."""
    import torch
    rng = np.random.default_rng(5)
    probs = [P.shock_tube(int(n), eta=10.0 ** rng.uniform(-6, 0)) for n in rng.integers(400, 4097, n_tubes)]
    out = {"workload": f"{n_tubes} shock tubes of 400-4096 cells, eta 10^U[-6,0], seed 5, mixed precision",
           "cells": int(sum(p.cells for p in probs)), "steps": steps}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for mode in ("per_kind_graph", "persistent"):
        solvers = [grmhd.Solver.from_problem(pr, device=dev, precision="mixed") for pr in probs]
        B = grmhd.Batch(solvers)
        B.set_dt([s.compute_dt() for s in solvers])
        B.step()
        torch.cuda.synchronize()
        if mode == "per_kind_graph":
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                with torch.cuda.graph(graph, stream=side):
                    B.step(stream=side)
            torch.cuda.current_stream().wait_stream(side)
            e0.record()
            for _ in range(steps):
                graph.replay()
            e1.record()
        else:
            e0.record()
            B.step_persistent(steps, synchronize=False)
            e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[mode] = {"ms_per_step": ms, "value": out["cells"] * STAGES / (ms / 1e3),
                     "newton_failures": sum(s.diagnostics()[2] for s in solvers)}
        del B, solvers
    out["unit"] = UNIT
    return out


def _pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(p / 100.0 * (len(xs) - 1)))))
    return xs[k]


def _latency_groups(results, reqs):
    """p50/p99 time to solution per eta decade and per kind of run."""
    by_id = {r.rid: r for r in reqs}
    dec, kind = {}, {}
    for res in results:
        info = by_id[res.rid].problem.info
        d = int(math.floor(math.log10(info["eta"]) + 1e-12))
        dec.setdefault(f"1e{d}..1e{d + 1}", []).append(res.time_to_solution)
        kind.setdefault(info["kind"], []).append(res.time_to_solution)
    f = lambda xs: {"n": len(xs), "p50_tts_s": _pct(xs, 50), "p99_tts_s": _pct(xs, 99)}
    return {k: f(v) for k, v in sorted(dec.items())}, {k: f(v) for k, v in sorted(kind.items())}


def bench_serving(dev, args):
    """The serving mix: 1-D shock tubes (400-4096 cells, to t = 0.4), 2-D Orszag-Tang
    vortices (128^2-512^2, 100 steps) and 3-D stars (64^3-128^3, 100 steps), eta
    log-uniform in [1e-6, 1], served by continuous batching under a 150 GB device-memory
    budget (mixed precision).
    - capacity: the mix admitted all at once (offline), runs per second;
    - the eta sweep at a sustainable load: a seeded Poisson stream at 80 % of that
      capacity, with p50/p99 time to solution overall, per eta decade and per kind;
    - overload: the stream at 200 requests/s, which queues (time to solution is then
      mostly waiting)."""
    from paper_2110_03732_gb300 import problems as P
    from paper_2110_03732_gb300.serve import Request, Server

    def make(seed, n, rate):
        return [Request(i, t, pr, steps, t_end=pr.t_end if pr.ndim == 1 else None)
                for i, (t, pr, steps) in enumerate(P.request_stream(seed, n, rate=rate))]

    def serve(reqs, realtime):
        srv = Server(budget_bytes=150e9, precision="mixed", device=dev)
        return srv.run(reqs, realtime=realtime)

    n = args.serve_requests
    off_reqs = make(0, n, 200.0)
    off_res, off = serve(off_reqs, realtime=False)
    capacity = len(off_res) / off["wall_s"]
    rate = 0.8 * capacity
    sus_reqs = make(1, int(1.25 * n), rate)
    sus_res, sus = serve(sus_reqs, realtime=True)
    dec, kinds = _latency_groups(sus_res, sus_reqs)
    ovl_reqs = make(0, n, 200.0)
    ovl_res, ovl = serve(ovl_reqs, realtime=True)
    out = dict(sus)
    out.update({"unit": UNIT, "workload": f"{len(sus_reqs)} requests, Poisson {rate:.2f}/s (80 % of capacity), seed 1",
                "arrival_rate_per_s": rate, "capacity_runs_per_s": capacity,
                "capacity_measure": f"{len(off_reqs)} requests of the same mix admitted at once (seed 0): "
                                    f"{off['wall_s']:.2f} s, {off['zone_updates_per_s']:.3g} zone-updates/s",
                "by_eta_decade": dec, "by_kind": kinds,
                "overload_200_per_s": {"requests": ovl["requests"], "wall_s": ovl["wall_s"],
                                       "p50_tts_s": ovl["p50_tts_s"], "p99_tts_s": ovl["p99_tts_s"],
                                       "zone_updates_per_s": ovl["zone_updates_per_s"],
                                       "note": "arrivals far above capacity: time to solution is queueing"}})
    return out


def bench_tube(grmhd, P, dev, runs=10):
    """The 1-D resistive shock tube (400 cells, eta = 1e-3, Gamma = 2, CFL 0.4) run to
    t = 0.4 (400 IMEX steps) in FP64, start to finish through the public API: problem
    set-up, time step, the steps and a final synchronisation, repeated `runs` times."""
    import torch
    pr = P.shock_tube(400)
    lat = []
    for _ in range(runs + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = grmhd.Solver.from_problem(pr, device=dev)
        dt = S.compute_dt()
        nsteps = int(math.ceil(pr.t_end / dt - 1e-9))
        t = 0.0
        for k in range(nsteps):
            d = dt if k < nsteps - 1 else pr.t_end - t
            S.step(d)
            t += d
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
    lat = lat[1:]   # the first run pays one-time set-up
    return {"workload": "shock_tube_1d_400 (eta 1e-3, Gamma 2) to t = 0.4, FP64", "steps": nsteps,
            "runs": runs, "p50_run_s": _pct(lat, 50), "p99_run_s": _pct(lat, 99),
            "ms_per_step_p50": 1e3 * _pct(lat, 50) / nsteps,
            "newton_failures": S.diagnostics()[2]}


def star_mixed_error(grmhd, P, dev, n=64, steps=100):
    """Mixed precision against FP64 on the 3-D star after `steps` steps: relative L1 of
    D and tau over the interior, and the div B maxima of both runs."""
    import torch
    pr = P.star(n)
    runs = {}
    for prec in ("fp64", "mixed"):
        S = grmhd.Solver.from_problem(pr, device=dev, precision=prec)
        dt = S.compute_dt()
        for _ in range(steps):
            S.step(dt)
        torch.cuda.synchronize()
        runs[prec] = (S, S.diagnostics())
    I = runs["fp64"][0].interior()
    out = {"workload": f"star_3d_{n}^3", "steps": steps}
    for v, name in ((0, "D"), (4, "tau")):
        a = runs["mixed"][0].q[v][I]
        b = runs["fp64"][0].q[v][I]
        out[f"rel_l1_{name}"] = float((a - b).abs().sum() / b.abs().sum())
    out["divb_max_mixed"] = runs["mixed"][1][0][2]
    out["divb_max_fp64"] = runs["fp64"][1][0][2]
    out["newton_failures"] = runs["mixed"][1][2] + runs["fp64"][1][2]
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
