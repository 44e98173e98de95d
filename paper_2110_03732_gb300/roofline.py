"""Roofline inputs of the stage kernels: the FP64 work and DRAM traffic of one launch,
counted by ncu on the 512^2 Orszag-Tang workload and stamped with the kernel sources
they were counted on.

The counts live in ``profiles/roofline_counts.json``; ``bench.py`` divides them by the
live CUDA-event launch times.  A count taken on other kernel sources than the ones
built is reported as stale (``sources_digest`` differs), and its traffic is then not
reported.

Refresh (one GPU, the 512^2 case of bench.py; one capture per precision and kernel
kind, each of one kernel name pattern and two launches, taken after the three warm-up
steps have run the same kernels; OUT is any scratch folder):

    M=$(python -c "from paper_2110_03732_gb300 import roofline as R; print(','.join(R.METRICS))")
    python bench.py --case ot --case-n 512 --steps 1 --warmup 3 > $OUT/plain.log 2>&1 &&
    for k in k_implicit k_stencil k_update; do
      ncu --metrics $M --clock-control none --print-units base \
          -k "regex:^$k" -s 6 -c 2 --csv --log-file $OUT/counts_fp64_$k.csv \
          python bench.py --case ot --case-n 512 --steps 1 --warmup 3 || break
    done
    (the same with --case ot_mixed into counts_mixed_$k.csv)
    python -m paper_2110_03732_gb300.roofline --fp64 $OUT/counts_fp64_*.csv \
        --mixed $OUT/counts_mixed_*.csv > profiles/roofline_counts.json

k_stencil is the one launch per stage of the face fluxes of every direction and the
resistive edge EMFs; it is counted as the flux kind.  The three warm-up steps run 6
launches of each pattern (2 per step): the two captured are the two stages of the
next step.
"""
from __future__ import annotations

import csv
import glob
import hashlib
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
COUNTS = os.path.join(ROOT, "profiles", "roofline_counts.json")

METRICS = [
    "gpu__time_duration.sum",
    "smsp__sass_thread_inst_executed_op_dadd_pred_on.sum",
    "smsp__sass_thread_inst_executed_op_dfma_pred_on.sum",
    "smsp__sass_thread_inst_executed_op_dmul_pred_on.sum",
    "sm__inst_executed_pipe_fp64.sum",
    "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
    "dram__bytes_read.sum",
    "dram__bytes_write.sum",
    "smsp__inst_executed.sum",
]

# FP64 issue rate of GB300 from its unit counts and clock: 2 FP64 lanes per SM per
# cycle (ncu's peak of the DFMA counter), 152 SMs, 2.07 GHz.  A DFMA counts 2 flop,
# a DADD or DMUL 1, and each takes one issue slot.
FP64_LANES_PER_SM_CYCLE = 2
N_SM = 152
SM_GHZ = 2.07
FP64_INST_PEAK_PER_S = FP64_LANES_PER_SM_CYCLE * N_SM * SM_GHZ * 1e9        # 6.29e11
FP64_PEAK_TFLOPS = 2 * FP64_INST_PEAK_PER_S / 1e12                          # 1.26 (nominal 1.25)
# instruction issue rate: 4 schedulers per SM, each issuing one warp instruction (32
# thread instructions) per cycle, 152 SMs, 2.07 GHz -- the bound of a kernel whose
# instructions spread over the FP32, integer and FP64 pipes with none of them saturated
ISSUE_PEAK_TINST = 4 * 32 * N_SM * SM_GHZ * 1e9 / 1e12                     # 40.3 T thread inst/s


def sources_digest() -> str:
    """SHA-256 of the kernel sources and the C header (what the counts depend on)."""
    files = sorted(glob.glob(os.path.join(HERE, "csrc", "*")) + [os.path.join(ROOT, "include", "grmhd.h")])
    h = hashlib.sha256()
    for f in files:
        if os.path.isfile(f):
            h.update(os.path.basename(f).encode())
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def kind_of(kernel_name: str):
    for pre, kind in (("k_implicit", "implicit"), ("k_flux_march", "flux"), ("k_stencil", "flux"),
                      ("k_emf", "emf"), ("k_update", "update")):
        if kernel_name.startswith(pre) or kernel_name.startswith("void " + pre):
            return kind
    return None


_SCALE = {"": 1.0, "byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-3, "ns": 1e-3,
          "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3, "second": 1e6, "s": 1e6, "%": 1.0, "inst": 1.0,
          "cycle": 1.0}


def _num(x, unit=""):
    """A CSV value in base units (bytes, microseconds for durations)."""
    return float(str(x).replace(",", "")) * _SCALE.get(unit, 1.0)


def counts_from_ncu_csv(paths, cells: int):
    """Per kernel kind: launches, and per launch the mean duration, FP64 flop
    (2 DFMA + DADD + DMUL), FP64-pipe instructions (thread level), FP64-pipe busy
    fraction and DRAM bytes; per-kernel-name rows kept beside them.  ``paths``: one
    ncu CSV or a list of them (one capture per kernel kind)."""
    rows = {}
    for path in ([paths] if isinstance(paths, str) else list(paths)):
        with open(path) as fh:
            lines = [ln for ln in fh if ln.startswith('"')]
        for r in csv.DictReader(lines):
            key = (path, r["ID"], r["Kernel Name"])
            rows.setdefault(key, {})[r["Metric Name"]] = _num(r["Metric Value"], r.get("Metric Unit", ""))
    per_name = {}
    for (_, _, name), m in rows.items():
        kind = kind_of(name)
        if kind is None:
            continue
        flop = (2 * m["smsp__sass_thread_inst_executed_op_dfma_pred_on.sum"]
                + m["smsp__sass_thread_inst_executed_op_dadd_pred_on.sum"]
                + m["smsp__sass_thread_inst_executed_op_dmul_pred_on.sum"])
        e = per_name.setdefault(name, {"kind": kind, "launches": 0, "dur_us": 0.0, "fp64_flop": 0.0,
                                       "fp64_pipe_inst": 0.0, "fp64_pipe_busy": 0.0, "dram_bytes": 0.0,
                                       "inst": 0.0})
        e["launches"] += 1
        e["dur_us"] += m["gpu__time_duration.sum"]
        e["fp64_flop"] += flop
        e["fp64_pipe_inst"] += 32 * m["sm__inst_executed_pipe_fp64.sum"]
        e["fp64_pipe_busy"] += m["sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active"] / 100
        e["dram_bytes"] += m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"]
        e["inst"] += 32 * m.get("smsp__inst_executed.sum", 0.0)   # thread instructions (full warps)
    F = ("dur_us", "fp64_flop", "fp64_pipe_inst", "fp64_pipe_busy", "dram_bytes", "inst")
    for e in per_name.values():
        n = e["launches"]
        for k in F:
            e[k] /= n
    kinds = {}
    for name, e in per_name.items():
        k = kinds.setdefault(e["kind"], {"launches": 0, "kernels": []})
        k["kernels"].append(name)
        for f in F:
            k[f] = k.get(f, 0.0) + e[f] * e["launches"]
        k["launches"] += e["launches"]
    for k in kinds.values():
        n = k["launches"]
        for f in F:
            k[f] /= n
        k["inst_per_cell"] = k["inst"] / cells
        k["fp64_flop_per_cell"] = k["fp64_flop"] / cells
        k["fp64_pipe_inst_per_cell"] = k["fp64_pipe_inst"] / cells
        k["dram_bytes_per_cell"] = k["dram_bytes"] / cells
    return kinds, per_name


def _head():
    try:
        return subprocess.run(["git", "-C", ROOT, "rev-parse", "--short=12", "HEAD"], capture_output=True,
                              text=True, check=True).stdout.strip()
    except Exception:
        return None


def build_counts(fp64_csv, mixed_csv=None, n: int = 512):
    """The stored counts from the FP64 and mixed captures (a path or a list each)."""
    cells = n * n
    out = {"workload": f"orszag_tang_2d_{n}x{n}", "cells": cells, "sources_digest": sources_digest(),
           "head_when_counted": _head(), "metrics": METRICS,
           "units": "per launch (the 512^2 stage kernels); *_per_cell: divided by the interior cells"}
    for tag, path in (("fp64", fp64_csv), ("mixed", mixed_csv)):
        if path:
            kinds, names = counts_from_ncu_csv(path, cells)
            out[tag] = {"kinds": kinds, "kernels": names}
    return out


def load_counts(path: str = COUNTS):
    """The stored counts with ``stale`` set when the built sources differ."""
    try:
        with open(path) as fh:
            c = json.load(fh)
    except Exception:
        return None
    c["stale"] = c.get("sources_digest") != sources_digest()
    return c


def alu_entry(counts, prec: str, kind: str, avg_launch_ms: float, peak_probe_tflops=None):
    """Roofline entry of an FP64-bound kernel kind from the stored counts and its live
    mean launch time: achieved FP64 flop/s against the nominal FP64 rate, and the
    FP64-pipe issue fraction beside it (a DADD or DMUL takes an issue slot like a DFMA
    but counts one flop)."""
    if not counts or prec not in counts or kind not in counts[prec]["kinds"] or not avg_launch_ms > 0:
        return {"bound": "alu", "kernel": kind, "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "note": "no stored counts or no launches for this kernel"}
    k = counts[prec]["kinds"][kind]
    stale = counts["stale"]
    s = avg_launch_ms / 1e3
    ach = k["fp64_flop"] / s / 1e12
    return {"bound": "alu", "kernel": kind, "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None if stale else k["dram_bytes"],
            "avg_launch_ms": avg_launch_ms, "fp64_flop_per_cell": k["fp64_flop_per_cell"],
            "fp64_issue_frac": k["fp64_pipe_inst"] / s / FP64_INST_PEAK_PER_S,
            "peak_source": "nominal FP64 of GB300 from its unit counts and clock "
                           "(2 FP64 lanes/SM/cycle x 152 SMs x 2.07 GHz x 2 flop)",
            "peak_probe_tflops": peak_probe_tflops,
            "counts": {"head_when_counted": counts.get("head_when_counted"),
                       "sources_digest": counts.get("sources_digest"), "stale": stale}}


def issue_entry(counts, prec: str, kind: str, avg_launch_ms: float):
    """Roofline entry of a kernel bound by instruction issue (its instructions spread
    over the FP32, integer and FP64 pipes): executed thread instructions per launch
    over the live launch time, against the issue rate of the SMs; the FP64 figures of
    alu_entry beside it."""
    base = alu_entry(counts, prec, kind, avg_launch_ms)
    k = (counts or {}).get(prec, {}).get("kinds", {}).get(kind)
    if not k or not k.get("inst") or not avg_launch_ms > 0:
        return {"bound": "alu", "kernel": kind, "achieved": None, "peak": ISSUE_PEAK_TINST, "unit": "Tinst/s",
                "frac": None, "traffic": None, "note": "no stored instruction counts for this kernel"}
    s = avg_launch_ms / 1e3
    ach = k["inst"] / s / 1e12
    out = {"bound": "alu", "kernel": kind, "achieved": ach, "peak": ISSUE_PEAK_TINST, "unit": "Tinst/s",
           "frac": ach / ISSUE_PEAK_TINST, "traffic": base["traffic"], "avg_launch_ms": avg_launch_ms,
           "inst_per_cell": k["inst_per_cell"],
           "peak_source": "instruction issue of GB300 from its unit counts and clock (4 schedulers x 32 lanes "
                          "per SM per cycle x 152 SMs x 2.07 GHz)",
           "fp64_tflops": base["achieved"], "fp64_flop_frac": base["frac"],
           "fp64_issue_frac": base.get("fp64_issue_frac"), "counts": base.get("counts")}
    return out


def hbm_entry(counts, prec: str, kind: str, avg_launch_ms: float, alg_bytes_per_launch: float, hbm_gbs: float):
    """Roofline entry of a memory-side kernel: algorithmic bytes per launch over the
    live launch time, against the measured copy bandwidth; DRAM traffic from the
    stored counts."""
    s = avg_launch_ms / 1e3
    ach = alg_bytes_per_launch / s / 1e9
    k = (counts or {}).get(prec, {}).get("kinds", {}).get(kind)
    stale = True if not counts else counts["stale"]
    return {"bound": "hbm", "kernel": kind, "achieved": ach, "peak": hbm_gbs, "unit": "GB/s", "frac": ach / hbm_gbs,
            "traffic": None if (k is None or stale) else k["dram_bytes"], "avg_launch_ms": avg_launch_ms,
            "alg_bytes_per_launch": alg_bytes_per_launch,
            "counts": None if not counts else {"head_when_counted": counts.get("head_when_counted"),
                                                "sources_digest": counts.get("sources_digest"), "stale": stale}}


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="roofline counts from ncu captures (see the module docstring)")
    ap.add_argument("--fp64", nargs="+", required=True, help="ncu CSV captures of the FP64 512^2 step")
    ap.add_argument("--mixed", nargs="+", default=None, help="ncu CSV captures of the mixed 512^2 step")
    a = ap.parse_args()
    print(json.dumps(build_counts(a.fp64, a.mixed), indent=1))
