#!/usr/bin/env python
"""Benchmark: D3Q19 LES throughput (MLUPS) and HBM-roofline fraction on one B300.

Workload: the turbulent open-channel LES, 256 x 128 x 128 cells (periodic
x/z, bounce-back bottom, free-slip top, Smagorinsky C_s = 0.1, bulk-velocity
controller, seeded log-law + 5 % initial state), statistics accumulation on.
One step = one fused kernel over the whole grid (stream, canopy/driving
force, Smagorinsky collision, boundaries, plane statistics).  The populations
are resident in HBM; each step moves 152 B per cell (FP32 storage) or 76 B
(FP16/BF16 shifted storage), 637 MB / 319 MB per step, well above the 126 MB L2,
so no explicit L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica of the workload (the
path does not exchange data between independent domains); rank 0 prints one
JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 LES MLUPS & HBM-roofline fraction, fp32 vs fp16-store at stated error"
WORKLOAD = ("turbulent channel LES 256x128x128 (periodic x/z, bounce-back bottom, free-slip "
            "top, Cs=0.1, bulk-velocity controller, plane statistics on)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "f16s", "bf16s", "f32-aa", "f16s-aa", "bf16s-aa"],
                    default="f32")
    ap.add_argument("--no-half", action="store_true", help="skip the FP16/BF16 storage legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-box ensemble leg")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-correction leg")
    ap.add_argument("--no-canopy", action="store_true",
                    help="skip the 512x128x256 canopy leg (x-binned statistics)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--learned-window", default="1000,1000", metavar="SPINUP,AVERAGE",
                    help="coarse steps before and during averaging in the learned leg")
    ap.add_argument("--profile", metavar="NXxNYxNZ|canopy|ensemble|learned", default=None,
                    help="run a few steps of the channel workload at this size (or of the "
                         "64-box ensemble, or of a 256x64x128 canopy domain with the learned "
                         "correction) and exit: the cases the ncu summaries under profiles/ "
                         "capture")
    return ap.parse_args()


def code_tokens(text: str) -> str:
    """C/C++ source without its comments and with whitespace collapsed: what
    the compiler sees (string literals in this file hold no comment markers)."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


KERNEL_SOURCES = ("lbm_device.cuh", "lbm_aa.cuh", "lbm_kern.inc")


def kernel_source_hash(texts=None):
    """Hash of the step kernels' code (lbm_device.cuh: the pull kernel, its
    tile loop and collision; lbm_aa.cuh: the AA kernels; lbm_kern.inc: their
    instantiations and launch shapes; comments and layout do not count), to
    tell whether the profiles/ counters still apply."""
    import hashlib

    if texts is None:
        texts = []
        for name in KERNEL_SOURCES:
            with open(os.path.join(ROOT, "paper_2206_15454_b300", "csrc", name)) as fh:
                texts.append(fh.read())
    h = hashlib.sha256()
    for name, text in zip(KERNEL_SOURCES, texts):
        h.update(name.encode() + b"\0" + code_tokens(text).encode() + b"\0")
    return h.hexdigest()[:16]


def measured_traffic_rw(storage_name, cells, workload="channel"):
    """(read, write) DRAM bytes per launch of the step kernel from the committed
    ncu summary (the channel captures, or the canopy one), scaled from the
    captured case to `cells`; None if the kernel changed since.  The write
    count of a single captured launch misses what is still in L2 when the
    kernel ends, so read and write are reported apart."""
    try:
        with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    e = (t.get("storage", {}) if workload == "channel" else t.get(workload, {})).get(storage_name)
    if not e:
        return None
    return e["dram_read_bytes"] * cells / e["cells"], e["dram_write_bytes"] * cells / e["cells"]


def measured_traffic(storage_name, cells, workload="channel"):
    """Read plus write DRAM bytes per launch (see measured_traffic_rw), or None."""
    rw = measured_traffic_rw(storage_name, cells, workload)
    return None if rw is None else rw[0] + rw[1]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows
                                   if r[3].replace(".", "").isdigit()) if rows else None}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------- our arm ---

def time_storage(P, W, storage, steps, warmup, ws, with_stats=True, soak_s=0.0):
    """The channel in one storage: `warmup` steps, the timed region of `steps`
    launches, single launches between events, four more timed regions, then
    (soak_s > 0) more steps of the same loop until soak_s seconds have passed
    since the warm-up began, so a clock sampler running around this call sees
    the kernel's load for at least that long."""
    import torch

    t_start = time.perf_counter()
    case = W.channel_les()
    d = P.Domain(case, storage)
    d.mass0 = d.mass()  # FP64 global mass of the initial state (mass drift below)
    if with_stats:
        d.stats_reset(True)
    stream = d.stream
    d.step(warmup)
    d.sync()
    torch.cuda.synchronize()
    barrier(ws)
    # the timed region: `steps` launches back to back, events only around them
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    d.step(steps)
    t_end.record(stream)
    torch.cuda.synchronize()
    d.sync()
    total_ms = t_begin.elapsed_time(t_end)
    barrier(ws)
    # the step kernel's own duration: events around each launch of a second run
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(min(steps, 200))]
    for a, b in ev:
        a.record(stream)
        d.step(1)
        b.record(stream)
    torch.cuda.synchronize()
    d.sync()
    per_launch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    # four more timed regions of the same K steps: run-to-run spread (the
    # reported value stays the first region's)
    repeats = [total_ms]
    for _ in range(4):
        t_begin.record(stream)
        d.step(steps)
        t_end.record(stream)
        torch.cuda.synchronize()
        repeats.append(t_begin.elapsed_time(t_end))
    d.sync()
    d.repeats_ms = repeats
    while time.perf_counter() - t_start < soak_s:
        d.step(200)
        d.sync()
    return d, case, total_ms, per_launch_ms


def time_ensemble(P, W, steps, warmup, hbm):
    """The 64-box canopy ensemble (96..160 x 64 x 64 cells each, FP16-shifted):
    tuned at creation, then `steps` steps replayed as one CUDA graph."""
    import torch

    b = P.Batch(W.ensemble_boxes(), P.LBM_F16_SHIFTED, tune_steps=10)
    b.step(warmup)
    b.sync()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(b.stream)
    b.step(steps)
    t1.record(b.stream)
    torch.cuda.synchronize()
    b.sync()
    ms = t0.elapsed_time(t1) / steps
    cells = b.cells
    xt, blocks, tuned_ms = b.tuning()
    def width(nx):  # chunk width 0: each box its own (a single domain's size rule)
        return xt if xt else (64 if nx <= 64 else 128 if nx <= 128 else 256)
    padded = sum(c.ny * c.nz * ((c.nx + width(c.nx) - 1) // width(c.nx)) * width(c.nx) for c in b.cases)
    ach = P.BYTES_PER_LUP[P.LBM_F16_SHIFTED] * cells / (ms * 1e-3) / 1e9
    out = {"value": round(cells / ms / 1e3, 1), "unit": "MLUPS", "ms_per_step": ms,
           "steps": steps, "warmup": warmup, "boxes": len(b.cases), "cells": cells,
           "storage": "f16s", "timing": "one CUDA graph of all steps, CUDA events on its stream",
           "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(ach / hbm, 4), "traffic": None},
           "tuning": {"chunk_width": xt, "blocks_per_launch": blocks,
                      "fluid_fraction_of_tile_cells": round(cells / padded, 4),
                      "candidates": [{"chunk_width": c[0], "blocks": c[1], "ms_per_step": c[2]}
                                     for c in b.candidates()]}}
    b.close()
    return out


def time_canopy(P, W, steps, warmup, hbm):
    """The forest-canopy boundary layer on 512x128x256 cells (inflow/outflow,
    canopy over x in [128, 512), statistics per x-bin of 64 cells), FP32 and
    FP16-shifted storage."""
    import torch

    case = W.canopy_abl()
    out = {"workload": "canopy ABL 512x128x256 (h=10, a=0.2, C_D=0.15, inflow/outflow, "
                       "statistics per x-bin of 64)", "cells": case.cells, "steps": steps}
    for name, st in (("f32", P.LBM_F32), ("f16s", P.LBM_F16_SHIFTED)):
        d = P.Domain(case, st)
        d.stats_reset(True)
        d.step(warmup)
        d.sync()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(d.stream)
        d.step(steps)
        t1.record(d.stream)
        torch.cuda.synchronize()
        d.sync()
        d.close()
        ms = t0.elapsed_time(t1) / steps
        ach = P.BYTES_PER_LUP[st] * case.cells / (ms * 1e-3) / 1e9
        out[name] = {"value": round(case.cells / ms / 1e3, 1), "unit": "MLUPS", "ms_per_step": ms,
                     "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm,
                                  "unit": "GB/s", "frac": round(ach / hbm, 4),
                                  "traffic": measured_traffic(name, case.cells, "canopy")}}
    return out


def time_learned(P, W, steps, warmup, spinup=1000, average=1000):
    """The learned first-layer correction at its full size: the 1024x256x512
    canopy domain (h = 12, a = 0.25, C_D = 0.15, inflow/outflow, FP32) and the
    same set-up on the 2x finer 2048x512x1024 grid (1.07 G cells, FP32 in the
    in-place AA layout: 82 GB).  (1) Both plain runs for the same physical time
    (spinup + average coarse steps; the fine run takes twice as many), the
    network trained on the coarse run's column features against the fine run's
    first-cell deficits, and the gain: error of the coarse mean streamwise
    velocity against the coarsened fine run, plain and corrected (lowest 1, 6
    and 12 rows = first cell, half canopy, canopy layer); (2) throughput of the
    coarse domain with and without the correction in every step."""
    import torch

    from paper_2206_15454_b300 import learned as L

    case = W.canopy_abl(1024, 256, 512, h=12.0, a=0.25, cd=0.15, canopy_x0=256, xbin=16)
    fine_storage = P.LBM_F32 | P.LBM_STORAGE_AA
    t_ref = time.perf_counter()
    ref = L.reference_runs(case, spinup, average, sample_every=50, fine_storage=fine_storage)
    t_ref = time.perf_counter() - t_ref
    torch.cuda.empty_cache()
    t_train = time.perf_counter()
    net, l0, l1 = L.train_correction(ref, epochs=4, batch=4096)
    t_train = time.perf_counter() - t_train
    n_samples = int(ref.features.shape[0])
    t_corr = time.perf_counter()
    plain, corr = L.corrected_run(case, net, 0.01, spinup, average, plain=ref.coarse)
    t_corr = time.perf_counter() - t_corr
    gain = {f"rows_{r}": {"plain": round(L.profile_error(plain, ref.fine_coarsened, r), 4),
                          "corrected": round(L.profile_error(corr, ref.fine_coarsened, r), 4)}
            for r in (1, 6, 12)}
    del ref

    d = P.Domain(case, P.LBM_F32)
    out = {}
    for label, use in (("plain", False), ("corrected", True)):
        if use:
            d.set_correction(net, 0.01)
        d.step(warmup)
        d.sync()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(d.stream)
        d.step(steps)
        t1.record(d.stream)
        torch.cuda.synchronize()
        d.sync()
        ms = t0.elapsed_time(t1) / steps
        out[label] = {"value": round(case.cells / ms / 1e3, 1), "unit": "MLUPS", "ms_per_step": ms}
    d.close()
    net.close()
    torch.cuda.empty_cache()
    fine = L.refine(case)
    return {"workload": "canopy ABL 1024x256x512 (h=12, a=0.25, C_D=0.15, inflow/outflow), FP32",
            "cells": case.cells, "steps": steps, **out,
            "correction_share_of_step": round(1 - out["plain"]["ms_per_step"] /
                                              out["corrected"]["ms_per_step"], 4),
            "gain": {"workload": f"the same on {fine.nx}x{fine.ny}x{fine.nz} ({fine.cells} cells, "
                                 f"FP32 AA storage) coarsened; {spinup} + {average} coarse steps "
                                 f"({2 * spinup} + {2 * average} fine), lam = 0.01",
                     "training": {"samples": n_samples, "epochs": 4, "batch": 4096,
                                  "loss_first_last_epoch": [round(l0, 4), round(l1, 4)]},
                     "mean_u_rel_l2_vs_coarsened_fine": gain,
                     "seconds": {"plain_runs": round(t_ref, 1), "training": round(t_train, 1),
                                 "corrected_run": round(t_corr, 1)}}}


def e2e_run(P, d, steps):
    """Per step, through the public API: enqueue the step and the read-out of
    its result (the time-averaged plane statistics and health flags, one copy
    into pinned host memory), then wait for and take the previous step's
    read-out, so the host reads step k's result while step k+1 runs.  Every
    step's result crosses to the host inside the timed region."""
    import numpy as np

    out = np.zeros((9, d.case.stats_xbins, d.case.ny))
    t0 = time.perf_counter()
    d.step(1)
    d.stats_begin()
    for _ in range(steps - 1):
        d.step(1)
        d.stats_begin()
        d.stats_end(out)
    d.stats_end(out)
    dt = time.perf_counter() - t0
    d2h = out.nbytes + 32  # statistics + the device health flags (one 32-byte block; one pinned copy)
    return dt, d2h


def cpu_baseline_single_thread(seconds):
    """The same oracle sample in a child process with OMP_NUM_THREADS=1."""
    import subprocess
    import sys

    code = ("import json, bench, workloads as W; "
            f"print(json.dumps(bench.cpu_baseline(W.channel_les, {seconds!r})))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": out["value"], "unit": out["unit"], "cores": 1, "sample": out["sample"]}


def cpu_baseline(case_factory, seconds):
    """The FP64 oracle, as it stands, on this host's cores: a bounded sample of
    the same workload (whole time steps of the full grid)."""
    import oracle

    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    case = case_factory()
    o = oracle.Oracle(case)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    n = max(1, min(50, int(seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return {"value": case.cells * n / dt / 1e6, "unit": "MLUPS", "cores": threads,
            "kind": "oracle", "sample": f"{n} full time steps of the {case.nx}x{case.ny}x{case.nz}"
            f" channel (FP64, OpenMP over z planes, {threads} threads)"}


CANOPY_ERR = dict(nx=128, ny=32, nz=32, h=8.0, canopy_x0=32, xbin=32)
CANOPY_ERR_STEPS = (1000, 2000)  # spin-up, statistics window


def cpu_baseline_leg(W):
    """The FP64 oracle as it stands, on this host's cores, on two bounded
    samples: 100 full time steps of the 256x128x128 channel (the reported
    MLUPS) and a statistics run of a 128x32x32 canopy boundary layer
    (1000 + 2000 steps).  Returns (the baseline record, the oracle's end states,
    which the GPU results state their errors against)."""
    import oracle

    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    case = W.channel_les()
    o = oracle.Oracle(case)
    t0 = time.perf_counter()
    o.step(100)
    dt = time.perf_counter() - t0
    f_channel = o.get_f()
    o.close()
    cc = W.canopy_abl(**CANOPY_ERR)
    oc = oracle.Oracle(cc)
    spin, window = CANOPY_ERR_STEPS
    t1 = time.perf_counter()
    oc.step(spin)
    oc.stats_reset(True)
    oc.step(window)
    dt2 = time.perf_counter() - t1
    s_canopy = oc.stats()[0]
    oc.close()
    rec = {"value": round(case.cells * 100 / dt / 1e6, 2), "unit": "MLUPS", "cores": threads,
           "kind": "oracle",
           "sample": f"100 full time steps of the 256x128x128 channel (FP64, OpenMP over z "
                     f"planes, {threads} threads, {dt:.1f} s)",
           "canopy_sample": {"value": round(cc.cells * (spin + window) / dt2 / 1e6, 2),
                             "unit": "MLUPS",
                             "sample": f"{spin} + {window} steps of a 128x32x32 canopy boundary "
                                       f"layer with statistics ({dt2:.1f} s)"}}
    return rec, {"channel_f_100": f_channel, "canopy_stats": s_canopy}


def population_error(P, W, storage, ref):
    """Populations after 100 steps of the channel against the FP64 oracle's:
    relative L2 and the largest single error over max |f - w|."""
    import numpy as np

    d = P.Domain(W.channel_les(), storage)
    d.step(100)
    f = d.get_f()
    d.close()
    fo = ref["channel_f_100"]
    w = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)[:, None, None, None]
    num = den = elem = scale = 0.0
    for q in range(19):
        e = f[q] - fo[q]
        num += float(np.sum(e * e))
        den += float(np.sum(fo[q] * fo[q]))
        elem = max(elem, float(np.abs(e).max()))
        scale = max(scale, float(np.abs(fo[q] - w[q]).max()))
    return {"rel_l2_f_after_100_steps": float(np.sqrt(num / den)),
            "max_element_error_over_max_f_minus_w": elem / scale,
            "case": "channel 256x128x128, 100 steps, same seed"}


def canopy_profile_errors(P, ref):
    """Mean-velocity and <u'v'> profiles (per x-bin) of the canopy sample on the
    GPU in each storage against the FP64 oracle's: largest deviation over the
    profiles relative to the largest magnitude."""
    import numpy as np
    import workloads as W

    so = ref["canopy_stats"]
    out = {"case": "canopy 128x32x32 (h=8, inflow/outflow, x-bins of 32), "
                   f"{CANOPY_ERR_STEPS[0]} + {CANOPY_ERR_STEPS[1]} steps"}
    for name in ("f32", "f16s", "bf16s"):
        d = P.Domain(W.canopy_abl(**CANOPY_ERR), P.STORAGE_NAMES[name])
        d.step(CANOPY_ERR_STEPS[0])
        d.stats_reset(True)
        d.step(CANOPY_ERR_STEPS[1])
        s, _ = d.stats()
        d.close()
        out[name] = {"mean_u": float(np.abs(s[0] - so[0]).max() / np.abs(so[0]).max()),
                     "uv": float(np.abs(s[6] - so[6]).max() / np.abs(so[6]).max())}
    return out


def time_aa(P, W, steps, warmup, hbm, ws):
    """The channel with AA-pattern in-place storage (one population set) in
    FP32 and FP16: MLUPS, roofline fraction and the workspace beside the
    two-set pull layout."""
    out = {"workload": "the same channel, AA-pattern in-place storage"}
    g = P._case_inputs(W.channel_les())[0]
    for name in ("f32", "f16s"):
        st = P.STORAGE_NAMES[name + "-aa"]
        d, case, tot, _ = time_storage(P, W, st, steps, warmup, ws)
        d.close()
        tot = max_over_ranks(ws, tot)
        ach = P.BYTES_PER_LUP[st] * case.cells / (tot / steps * 1e-3) / 1e9
        out[name] = {"value": round(case.cells * steps * ws / (tot * 1e-3) / 1e6, 1),
                     "unit": "MLUPS", "ms_per_step": tot / steps,
                     "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm,
                                  "unit": "GB/s", "frac": round(ach / hbm, 4),
                                  "traffic": measured_traffic(name + "-aa", case.cells),
                                  "traffic_read_write": measured_traffic_rw(name + "-aa", case.cells)},
                     "workspace_bytes": P.lbm_workspace_bytes(g, st, 1),
                     "workspace_bytes_pull": P.lbm_workspace_bytes(g, P.STORAGE_NAMES[name], 1)}
    return out


def run_ours(args):
    import torch

    import paper_2206_15454_b300 as P
    import workloads as W

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    storage = P.STORAGE_NAMES[args.storage]
    hbm, peak_kind = peaks()
    clocks = Clocks(local)
    clocks.start()
    d, case, total_ms, launch_ms = time_storage(P, W, storage, args.steps, args.warmup, ws,
                                                soak_s=1.5)
    clk = clocks.stop()
    if clk:
        clk["window"] = ("nvidia-smi every 50 ms from the start of the warm-up through the timed "
                         "regions and further steps of the same loop to 1.5 s")
    total_ms = max_over_ranks(ws, total_ms)
    cells = case.cells
    bpl = P.BYTES_PER_LUP[storage]
    value = cells * args.steps * ws / (total_ms * 1e-3) / 1e6
    # the timed region holds nothing but the step launches, back to back (each
    # overlaps its predecessor's tail): their average duration is total / K
    step_ms = total_ms / args.steps
    achieved = bpl * cells / (step_ms * 1e-3) / 1e9
    res = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16s": "f16-storage/f32-compute",
                  "bf16s": "bf16-storage/f32-compute"}[args.storage.split("-")[0]],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": cells, "storage": args.storage,
                   "bytes_per_lup": bpl, "l2": "inputs larger than L2 (no flush needed)",
                   "parallelism": f"{ws} independent replica(s)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4),
                     "traffic": measured_traffic(args.storage, cells),
                     "traffic_read_write": measured_traffic_rw(args.storage, cells),
                     "kernel": "step_kernel", "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bpl * cells,
                     "launch_ms": step_ms,
                     "isolated_launch_ms": launch_ms,
                     "launch_ms_note": "average over the timed region (CUDA events around the "
                                       "K back-to-back launches); isolated_launch_ms times "
                                       "single launches between events, which also "
                                       "serialises them"},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    d.repeats_ms = [max_over_ranks(ws, r) for r in d.repeats_ms]  # slowest rank per region
    reps = sorted(r / args.steps for r in d.repeats_ms)
    res["repeats"] = {"timed_regions": len(reps),
                      "ms_per_step": [round(r / args.steps, 5) for r in d.repeats_ms],
                      "best_value": round(cells * ws / (reps[0] * 1e-3) / 1e6, 1),
                      "median_value": round(cells * ws / (reps[len(reps) // 2] * 1e-3) / 1e6, 1)}
    m1 = d.mass()
    res["mass"] = {"initial": d.mass0, "after_steps": d.steps_done(), "final": m1,
                   "rel_drift": (m1 - d.mass0) / d.mass0}
    # end to end through the public API with host-side results every step
    e2e_steps = max(1000, min(args.steps, 2000))  # a floor of its own
    dt, d2h = e2e_run(P, d, e2e_steps)
    res["e2e"] = {"value": round(cells * e2e_steps * ws / dt / 1e6, 1), "unit": "MLUPS",
                  "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
                  "note": "per step: lbm_step, lbm_stats_begin (copy of the plane statistics and "
                          "health flags to pinned host memory), lbm_stats_end of the previous "
                          "step's read-out; the flow state stays resident, so a step has no "
                          "host input (no copy is declared for the input)",
                  "steps": e2e_steps}
    d.close()
    # the CPU baseline (rank 0): the FP64 oracle as it stands, timed on bounded
    # samples of the channel and of a small canopy domain; its end states are
    # also what the GPU results state their errors against
    ref = None
    if rank == 0 and not args.no_cpu:
        res["cpu_baseline"], ref = cpu_baseline_leg(W)
        res["cpu_baseline"]["single_thread"] = cpu_baseline_single_thread(args.cpu_seconds / 3)
        res["error_vs_fp64_oracle"] = {"f32": population_error(P, W, P.LBM_F32, ref)}
    # half-precision storage legs
    if not args.no_half:
        for name in ("f16s", "bf16s"):
            st = P.STORAGE_NAMES[name]
            dh, _, tot, lms = time_storage(P, W, st, args.steps, args.warmup, ws)
            mh = dh.mass()
            drift = {"after_steps": dh.steps_done(), "rel_drift": (mh - dh.mass0) / dh.mass0}
            dh.close()
            tot = max_over_ranks(ws, tot)
            ach = P.BYTES_PER_LUP[st] * cells / (tot / args.steps * 1e-3) / 1e9
            res[name] = {"value": round(cells * args.steps * ws / (tot * 1e-3) / 1e6, 1),
                         "unit": "MLUPS", "ms_per_step": tot / args.steps,
                         "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm,
                                      "unit": "GB/s", "frac": round(ach / hbm, 4),
                                      "traffic": measured_traffic(name, cells),
                                      "traffic_read_write": measured_traffic_rw(name, cells)},
                         "mass": drift}
            if ref is not None:
                res[name]["error_vs_fp64_oracle"] = population_error(P, W, st, ref)
    # AA-pattern in-place storage (one population set) beside the two-set pull scheme
    res["aa"] = time_aa(P, W, args.steps, args.warmup, hbm, ws)
    if not args.no_canopy:
        res["canopy"] = time_canopy(P, W, min(args.steps, 500), max(args.warmup, 3), hbm)
    if not args.no_ensemble:
        res["ensemble"] = time_ensemble(P, W, min(args.steps, 1000), max(args.warmup, 3), hbm)
    if not args.no_learned:
        spin, avg = (int(v) for v in args.learned_window.split(","))
        res["learned"] = time_learned(P, W, min(args.steps, 100), max(min(args.warmup, 10), 3),
                                      spin, avg)
    if ref is not None and not args.no_canopy:
        res["canopy"]["profile_error_vs_fp64_oracle"] = canopy_profile_errors(P, ref)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm ---

def run_reference(args):
    """The FP64 CPU oracle timed on the host cores (rank 0 only)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workloads as W

    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # a z-slab of the channel: at least one z-plane per thread (the oracle runs
    # its OpenMP loop over z-planes), and as wide as warmup + steps allow in
    # about two minutes
    nz_min = min(128, max(8, threads))
    probe = oracle.Oracle(W.channel_les(256, 128, nz_min))
    probe.step(2)  # first touch
    t0 = time.perf_counter()
    probe.step(6)  # steady steps
    per_cell = (time.perf_counter() - t0) / (6 * 256 * 128 * nz_min)
    probe.close()
    budget = 120.0 / max(1, args.steps + args.warmup)
    nz = int(max(nz_min, min(128, budget / (per_cell * 256 * 128))))
    case = W.channel_les(256, 128, nz)
    o = oracle.Oracle(case)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = case.cells * args.steps / dt / 1e6
    sample = (f"{args.steps} time steps of a 256x128x{nz} z-slab of the channel workload "
              f"(FP64 oracle, {threads} OpenMP threads)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": case.cells, "sample_nz": nz},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_profile_case(args):
    """A few steps of the channel workload at a chosen size (ncu capture target)."""
    import torch

    import paper_2206_15454_b300 as P
    import workloads as W

    torch.cuda.set_device(0)
    if args.profile == "ensemble":
        b = P.Batch(W.ensemble_boxes(), P.LBM_F16_SHIFTED)
        b.step(6)
        b.sync()
        b.close()
        print("profile case: 64-box ensemble, FP16-shifted: 6 steps done")
        return
    if args.profile == "canopy":
        d = P.Domain(W.canopy_abl(512, 128, 128), P.STORAGE_NAMES[args.storage])
        d.stats_reset(True)
        d.step(6)
        d.sync()
        d.close()
        print(f"profile case: canopy 512x128x128 {args.storage} with x-binned statistics: 6 steps")
        return
    if args.profile == "learned":
        d = P.Domain(W.canopy_abl(256, 64, 128, h=12.0, a=0.25, cd=0.15, canopy_x0=64, xbin=16))
        net = P.CorrectionNet(seed=1)
        d.set_correction(net, 0.01)
        d.step(6)
        d.sync()
        d.close()
        net.close()
        print("profile case: canopy 256x64x128 with the learned correction: 6 steps done")
        return
    nx, ny, nz = (int(v) for v in args.profile.lower().split("x"))
    d = P.Domain(W.channel_les(nx, ny, nz), P.STORAGE_NAMES[args.storage])
    d.stats_reset(True)
    d.step(6)
    d.sync()
    d.close()
    print(f"profile case {nx}x{ny}x{nz} {args.storage}: 6 steps done")


if __name__ == "__main__":
    a = parse()
    if a.profile:
        run_profile_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
