"""Continuous-batching request loop for resistive-MHD runs on one GPU.

Requests (a problem plus a number of IMEX steps, arriving over time) are admitted
while their device memory fits an HBM budget, kept resident, and advanced together
in batched launches (grmhd_batch_step: one launch per kernel kind and stage for
all runs of a batch).  A request that arrives while others are running joins at
the next iteration; a finished run leaves and frees its memory for the next
admission.

Active runs are split into two lanes on two CUDA streams so that their work
overlaps on the device: a bulk lane (large grids) takes one step per iteration, and
a fast lane (small grids, typically many cheap steps) takes k steps per iteration,
with k adapted from the measured lane times so that both lanes take about as long.
When the resident large runs hold more cells than it takes to fill the GPU
(`bulk_cells`), the bulk lane advances those with the least remaining work
(cells x steps left) first -- shortest remaining work first -- and the others wait,
resident, for the next selection; this keeps the device saturated while short runs
finish early.
Every run keeps its own time step and runs the same batched kernels whatever lane
or batch it is in, so its result is bitwise the one it gets served alone.

The scheduler is host code; all arithmetic runs in libgrmhd's kernels.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import torch

from . import grmhd


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the loop starts
    problem: object         # problems.Problem
    steps: int              # IMEX steps to run
    t_end: float = None     # if set, the last step is clipped to land on it


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    cells: int
    state: list = field(default_factory=list)   # final q (8) + face B (3), on the host if kept

    @property
    def time_to_solution(self):
        return self.finished - self.arrival


def request_bytes(prob, precision="fp64"):
    """Device bytes of one run: state (11 arrays) + context scratch + metric/eta."""
    g = grmhd.make_grid(prob.ndim, prob.n, prob.lo, prob.hi, prob.bc)
    N = prob.N
    ncell = N[0] * N[1] * N[2]
    extra = 8 * ncell * ((2 if prob.alpha is not None else 0) + (1 if prob.eta is not None else 0))
    return 11 * 8 * ncell + grmhd.scratch_bytes(g, grmhd.ssp2()) + extra


class _Lane:
    """A set of runs advanced by one batch on one stream."""

    def __init__(self, stream):
        self.stream = stream
        self.runs = []
        self.batch = None
        self.dirty = True
        self.ms_per_step = None       # measured
        self.pending_timing = None    # (start event, end event, steps)

    def rebuild(self):
        if self.dirty:
            if self.batch is not None:
                # the old batch's descriptor table may still be read by kernels queued
                # on this stream: let them finish before its memory can be reused
                self.stream.synchronize()
            self.batch = grmhd.Batch([r["solver"] for r in self.runs]) if self.runs else None
            self.dirty = False

    def step(self, nsteps):
        """Advance every run of the lane by up to nsteps steps (fewer if one finishes
        earlier).  Returns the runs that finished."""
        self.rebuild()
        done = []
        if not self.runs:
            return done
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        taken = 0
        for _ in range(nsteps):
            dts = []
            for r in self.runs:
                dt = r["dt"]
                if r["req"].t_end is not None and r["left"] == 1:
                    dt = r["req"].t_end - r["t"]
                dts.append(dt)
            self.batch.set_dt(dts, stream=self.stream)
            self.batch.step(stream=self.stream)
            taken += 1
            finished = False
            for r, dt in zip(self.runs, dts):
                r["left"] -= 1
                r["t"] += dt
                if r["left"] == 0:
                    finished = True
            if finished:
                break
        e1.record(self.stream)
        self.pending_timing = (e0, e1, taken)
        for r in list(self.runs):
            if r["left"] == 0:
                r["event"] = e1
                done.append(r)
                self.runs.remove(r)
                self.dirty = True
        return done

    def poll_timing(self):
        if self.pending_timing and self.pending_timing[1].query():
            e0, e1, n = self.pending_timing
            ms = e0.elapsed_time(e1) / max(n, 1)
            self.ms_per_step = ms if self.ms_per_step is None else 0.7 * self.ms_per_step + 0.3 * ms
            self.pending_timing = None


class Server:
    """Admit, batch and retire runs under an HBM budget (bytes).  Runs of at most
    `small_cells` interior cells go to the fast lane."""

    def __init__(self, budget_bytes=150e9, precision="fp64", device="cuda", keep_results=False,
                 small_cells=65536, max_fast_steps=256, bulk_cells=8_000_000):
        self.budget = float(budget_bytes)
        self.precision = precision
        self.device = torch.device(device)
        self.keep = keep_results
        self.small_cells = int(small_cells)
        self.max_fast = int(max_fast_steps)
        self.bulk_cells = int(bulk_cells)

    def _select(self, bulk, waiting):
        """Shortest remaining work first among the large runs, up to bulk_cells."""
        pool = bulk.runs + waiting
        pool.sort(key=lambda r: r["cells"] * r["left"])
        chosen, total = [], 0
        for r in pool:
            if chosen and total + r["cells"] > self.bulk_cells:
                continue
            chosen.append(r)
            total += r["cells"]
        rest = [r for r in pool if r not in chosen]
        if [id(r) for r in chosen] != [id(r) for r in bulk.runs]:
            bulk.runs = chosen
            bulk.dirty = True
        return rest

    def run(self, requests, realtime=True):
        """Serve `requests` (list of Request).  realtime=True honours arrival times on
        the wall clock; False admits every request at once (offline batch).
        Returns (results, stats)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        bulk = _Lane(torch.cuda.Stream(device=self.device))
        fast = _Lane(torch.cuda.Stream(device=self.device))
        results = []
        used = 0.0
        peak = 0.0
        zone_stage_updates = 0
        iters = 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        finishing = []          # runs whose last step is submitted, waiting for their event
        waiting = []            # admitted large runs not in the current bulk selection
        reselect = False
        while pending or bulk.runs or fast.runs or finishing or waiting:
            # admit arrived requests that fit the budget (in arrival order)
            while pending and (not realtime or pending[0].arrival <= now()):
                r = pending[0]
                b = request_bytes(r.problem, self.precision)
                if used + b > self.budget and (bulk.runs or fast.runs or finishing or waiting):
                    break
                pending.pop(0)
                s = grmhd.Solver.from_problem(r.problem, device=self.device, precision=self.precision)
                run = {"req": r, "solver": s, "dt": s.compute_dt(), "left": r.steps, "t": 0.0,
                       "admitted": now(), "bytes": b, "cells": s.cells}
                lane = fast if s.cells <= self.small_cells else bulk
                # the new run's state must be initialised before the lane's stream reads it
                lane.stream.wait_stream(torch.cuda.current_stream(self.device))
                if lane is fast:
                    fast.runs.append(run)
                    fast.dirty = True
                else:
                    waiting.append(run)
                    reselect = True
                used += b
                peak = max(peak, used)
            # retire runs whose final step has completed
            for run in list(finishing):
                if run["event"].query():
                    fin = now()
                    r = run["req"]
                    st = [t.detach().cpu() for t in run["solver"].q + run["solver"].bf] if self.keep else []
                    nf = run["solver"].diagnostics()[2]
                    if nf:
                        raise grmhd.GrmhdError(f"request {r.rid}: {nf} Newton failures")
                    results.append(Result(r.rid, r.arrival, run["admitted"], fin, r.steps, run["cells"], st))
                    used -= run["bytes"]
                    finishing.remove(run)
            if reselect or (not bulk.runs and waiting):
                waiting = self._select(bulk, waiting)
                reselect = False
            if not (bulk.runs or fast.runs):
                if finishing:
                    time.sleep(1e-4)
                elif pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now(), 0.01)))
                continue
            bulk.poll_timing()
            fast.poll_timing()
            # fast-lane steps per iteration: balance against the bulk lane's step
            k = 1
            if bulk.runs and fast.ms_per_step and bulk.ms_per_step:
                k = int(min(self.max_fast, max(1, round(bulk.ms_per_step / fast.ms_per_step))))
            elif not bulk.runs:
                k = 16
            if fast.runs:
                k = min(k, min(r["left"] for r in fast.runs))
            for lane, n in ((bulk, 1), (fast, k)):
                before = sum(r["cells"] for r in lane.runs)
                done = lane.step(n)
                steps_taken = lane.pending_timing[2] if lane.pending_timing else 0
                zone_stage_updates += 2 * steps_taken * (before)
                finishing.extend(done)
                if done and lane is bulk:
                    reselect = True
            iters += 1
            # keep the host at most a couple of iterations ahead of the device
            if bulk.pending_timing and iters % 2 == 0:
                bulk.pending_timing[1].synchronize()
        torch.cuda.synchronize()
        wall = now()
        tts = sorted(r.time_to_solution for r in results)

        def pct(p):
            if not tts:
                return None
            k = min(len(tts) - 1, max(0, int(round(p / 100.0 * (len(tts) - 1)))))
            return tts[k]

        stats = {"requests": len(results), "wall_s": wall, "iterations": iters,
                 "zone_updates_per_s": zone_stage_updates / wall if wall > 0 else None,
                 "p50_tts_s": pct(50), "p99_tts_s": pct(99), "peak_bytes": peak, "budget_bytes": self.budget}
        return results, stats


def run_alone(req, precision="fp64", device="cuda"):
    """The same run served by itself (a batch holding only it), for the
    alone-vs-mix check."""
    s = grmhd.Solver.from_problem(req.problem, device=device, precision=precision)
    b = grmhd.Batch([s])
    dt = s.compute_dt()
    t = 0.0
    for k in range(req.steps):
        d = dt
        if req.t_end is not None and k == req.steps - 1:
            d = req.t_end - t
        b.set_dt([d])
        b.step()
        t += d
    torch.cuda.synchronize()
    return [x.detach().cpu() for x in s.q + s.bf]
