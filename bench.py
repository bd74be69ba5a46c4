"""Benchmark of the XCSR transpose on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload heterogeneous]
                    [--impl mgt|reference]

One step = one full transpose (bucket counts, scans, stable bucket scatter,
per-bucket sort, outputs and value-run copy) of the heterogeneous
high-cardinality workload, the largest single-GPU configuration:
8,388,608 x 8,388,608, cells/row LogNormal (mean 20, capped at 4,096),
Zipf(1.1) columns without repeats per row, geometric run lengths (mean 5,
at most 64) of 32-byte values, 256 unequal row blocks, int64 offsets
(~168M cells, ~838M values; ~57.8 GB minimal bytes).  Inputs are resident in
HBM and far larger than L2, so no L2 flush is needed between steps.  The
balanced multigraph (4,194,304 x 4,194,304, 32 cells per row, 4 int64 values
per cell, 64 row blocks) is timed after it in the same run and reported under
the "balanced" key.  Prints one JSON line (rank 0).

``--impl reference`` times the CPU oracle (the plain counting transpose in
oracle/) on the host, on a bounded sample of the same workload, and prints
the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "transpose GB/s (frac of HBM peak), cells/s; batched vs per-matrix; p50/p99 ms"
UNIT = "GB/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_spec(name: str, seed: int, rank: int):
    import synth
    s = seed + 1000003 * rank
    if name == "balanced":
        return synth.balanced(seed=s)
    if name == "heterogeneous":
        return synth.heterogeneous(seed=s)
    if name == "tiny":
        return synth.tiny(seed=s)
    if name == "paper_balanced":
        return synth.paper_balanced(seed=s)
    if name in ("paper_heterogeneous", "chain"):
        return synth.paper_heterogeneous(seed=s)
    raise SystemExit(f"unknown workload {name}")


def sample_spec(name: str, spec, rows: int):
    """The same distributions at a bounded size for the CPU oracle: fewer rows
    (and columns, for the square workloads); the rectangular paper-shaped
    matrix keeps its columns and takes a few of its rows."""
    if spec.n_rows != spec.n_cols:
        spec.n_rows = min(spec.n_rows, 2)
        return spec
    spec.n_rows = spec.n_cols = min(rows, spec.n_rows)
    return spec


def spec_config(name: str, spec) -> dict:
    """The workload's config without generating it (the reference arm times a
    sample): sizes that the distributions fix exactly are included."""
    import synth
    cfg = {"workload": name, "n_rows": spec.n_rows, "n_cols": spec.n_cols, "n_cells": None,
           "n_values": None, "payload_stride": spec.stride, "offset_bytes": spec.offset_bytes,
           "partitions": spec.n_parts, "minimal_bytes": None,
           "l2": "inputs larger than L2 (no flush)", "seed": 0}
    if spec.row_dist == synth.ROW_EXACT and spec.len_dist == synth.LEN_EXACT:
        C = spec.n_rows * int(spec.row_a)
        V = C * int(spec.len_a)
        o = spec.offset_bytes
        side = 4 * C + (C + 1) * o + V * spec.stride
        cfg.update(n_cells=C, n_values=V,
                   minimal_bytes=(spec.n_rows + 1) * o + side + (spec.n_cols + 1) * o + side)
        cfg["l2"] = l2_note(cfg["minimal_bytes"])
    return cfg


L2_BYTES = 129 * 10**6


def l2_note(minimal_bytes) -> str:
    if minimal_bytes is not None and minimal_bytes < L2_BYTES:
        return "fits in L2, no flush (a latency case, not a bandwidth claim)"
    return "inputs larger than L2 (no flush)"


def workload_config(name: str, x) -> dict:
    return {"workload": name, "n_rows": x.n_rows, "n_cols": x.n_cols, "n_cells": x.n_cells,
            "n_values": x.n_values, "payload_stride": x.stride, "offset_bytes": x.offset_bytes,
            "partitions": x.n_parts, "minimal_bytes": x.minimal_bytes(),
            "l2": l2_note(x.minimal_bytes()), "seed": 0}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ multi-rank
def reduce_over_ranks(times_ms, units, device="cpu"):
    """Whole-job timing over the ranks of the current process group (one
    independent replica per rank): each time is the MAX over ranks, the units
    (bytes, cells) the SUM.  Without a process group, the local values."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in times_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(v) for v in units], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.cpu()], [float(v) for v in u.cpu()]


# ------------------------------------------------------------- CPU baseline
def time_oracle(name: str, seed: int, target_s: float = 15.0):
    """Times the CPU oracle (one thread) on a bounded sample of the workload:
    the same distributions with fewer rows.  Returns (GB/s, cells/s, sample)."""
    import oracle
    import synth
    rows = {"tiny": 1000, "paper_balanced": 1 << 15}.get(name, 1 << 19)
    spec = sample_spec(name, workload_spec(name, seed, 0), rows)
    x = synth.generate(spec)
    t_total, n = 0.0, 0
    while t_total < target_s or n == 0:
        t0 = time.perf_counter()
        oracle.transpose(x)
        t_total += time.perf_counter() - t0
        n += 1
        if n >= 50:
            break
    per = t_total / n
    sample = (f"{name} distributions at {x.n_rows:,} x {x.n_cols:,} ({x.n_cells:,} cells, "
              f"{x.n_values:,} values), {n} runs of the oracle")
    return x.minimal_bytes() / per / 1e9, x.n_cells / per, sample, per


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import synth
    spec = workload_spec(args.workload, args.seed, 0)
    config = spec_config(args.workload, spec)
    full_rows = spec.n_rows
    rows = {"paper_balanced": 1 << 15}.get(args.workload, 1 << 18)
    spec = sample_spec(args.workload, spec, rows)
    x = synth.generate(spec)
    if spec.n_rows == full_rows:  # the whole matrix when it is smaller than the sample
        config = workload_config(args.workload, x)
    # config names the workload whose rate this is; each timed step transposes
    # this smaller matrix of the same distributions (ms_per_step is its time)
    config["timed_sample"] = {"n_rows": x.n_rows, "n_cols": x.n_cols, "n_cells": x.n_cells,
                              "n_values": x.n_values, "minimal_bytes": x.minimal_bytes()}
    for _ in range(args.warmup):
        oracle.transpose(x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.transpose(x)
        times.append(time.perf_counter() - t0)
    per = sum(times) / len(times)
    gbs = x.minimal_bytes() / per / 1e9
    sample = (f"{args.workload} distributions at {x.n_rows:,} x {x.n_cols:,} rows/cols "
              f"({x.n_cells:,} cells, {x.n_values:,} values) per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": config,
        "cells_per_s": round(x.n_cells / per, 1),
        "p50_ms": round(float(np.percentile(times, 50)) * 1e3, 3),
        "p99_ms": round(float(np.percentile(times, 99)) * 1e3, 3),
        "cpu_baseline": {"value": round(gbs, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host_cores": os.cpu_count()},
        "e2e": {"value": round(gbs, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0



def time_extra(args, name, torch, mgt, barrier, stream, world):
    """Times one more workload (default plan, device-resident inputs) after
    the headline one, for the line's extra key: ms per transpose (max over
    ranks), GB/s of minimal bytes (summed over ranks), phase times."""
    import synth
    spec = workload_spec(name, args.seed, int(os.environ.get("RANK", "0")))
    x = synth.generate(spec)
    d = mgt.to_device(x)
    plan = mgt.plan_for(d)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    out = mgt.alloc_output(d, parts=True)
    mgt.transpose(plan, d.arrays(), out, ws, stream)
    if mgt.read_status(ws, stream) != 0:
        raise SystemExit(f"device status error on the {name} workload")
    for _ in range(args.warmup):
        mgt.transpose(plan, d.arrays(), out, ws, stream)
    steps = max(1, min(args.steps, 20))
    phases = plan.phases
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)] for _ in range(steps)]
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        mgt.transpose_profiled(plan, d.arrays(), out, ws, ev[k], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    if mgt.read_status(ws, stream) != 0:
        raise SystemExit(f"device status error on the {name} workload after timing")
    (tot,), (job_bytes, job_cells) = reduce_over_ranks([e0.elapsed_time(e1)], [plan.minimal_bytes(), x.n_cells],
                                                       device="cuda")
    ms = tot / steps
    phase_ms = {ph: round(statistics.mean(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(steps)), 4)
                for i, ph in enumerate(phases)}
    peak, _ = _peaks()
    gbs = job_bytes / (ms * 1e-3) / 1e9
    copy_alg = algorithmic_bytes("copy", x, plan)
    res = {"config": workload_config(name, x), "steps": steps, "ms_per_step": round(ms, 4),
           "value": round(gbs, 3), "unit": UNIT, "frac_of_hbm_peak": round(gbs / world / peak, 4),
           "cells_per_s": round(job_cells / (ms * 1e-3), 1), "phase_ms": phase_ms,
           "copy_roofline_frac": round(copy_alg / (phase_ms["copy"] * 1e-3) / 1e9 / peak, 4),
           "tiles": plan.config}
    del d, ws, out, x
    torch.cuda.empty_cache()
    return res

# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import synth
    from paper_2012_06012_gb300 import mgt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    l2f = apply_l2_fetch(args)

    def barrier():
        if world > 1:
            dist.barrier()

    spec = workload_spec(args.workload, args.seed, rank)
    if args.rows:
        spec.n_rows = spec.n_cols = args.rows
    # host inputs in pinned memory (also used by the end-to-end leg)
    pinned = []

    def alloc(n):
        t = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        pinned.append(t)
        return t.numpy()

    t_gen = time.perf_counter()
    x = synth.generate(spec, alloc=alloc)
    t_gen = time.perf_counter() - t_gen
    d = mgt.DeviceXCSR(x.n_rows, x.n_cols, x.offset_bytes, x.stride,
                       *[torch.from_numpy(a).cuda() for a in (x.row_ptr, x.col_idx, x.cell_ptr, x.values)],
                       x.part_off)
    out = mgt.alloc_output(d, parts=True)
    tiles_source = "explicit (--tiles)" if args.tiles else "default plan"
    cfg = json.loads(args.tiles) if args.tiles else None
    if cfg is None and args.autotune:
        # the library's autotuner (mgt_autotune), before and outside the timed
        # region: it times the candidate tile shapes on this matrix once
        cfg, _ = mgt.autotune(d, reps=2, out=out)
        torch.cuda.empty_cache()
        tiles_source = "mgt_autotune on this matrix, before the timed region"
    plan = mgt.plan_for(d, cfg)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    stream = torch.cuda.current_stream()
    phases = plan.phases
    nph = len(phases)
    minimal = plan.minimal_bytes()

    # correctness gate before timing
    mgt.transpose(plan, d.arrays(), out, ws, stream)
    st = mgt.read_status(ws, stream)
    if st != 0:
        raise SystemExit(f"device status {st} ({mgt.strerror(st)})")

    for _ in range(args.warmup):
        mgt.transpose(plan, d.arrays(), out, ws, stream)
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nph + 1)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        mgt.transpose_profiled(plan, d.arrays(), out, ws, ev[k], stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    st = mgt.read_status(ws, stream)
    if st != 0:
        raise SystemExit(f"device status {st} after timing ({mgt.strerror(st)})")
    total_ms = t_start.elapsed_time(t_end)
    step_ms = [ev[k][0].elapsed_time(ev[k][nph]) for k in range(args.steps)]
    phase_ms = {ph: statistics.mean(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps))
                for i, ph in enumerate(phases)}

    # values-only re-transposes on the same structure (mgt_transpose_values)
    v0 = torch.cuda.Event(enable_timing=True)
    v1 = torch.cuda.Event(enable_timing=True)
    mgt.transpose_values(plan, d.arrays(), out, ws, stream)
    v0.record(stream)
    for _ in range(args.steps):
        mgt.transpose_values(plan, d.arrays(), out, ws, stream)
    v1.record(stream)
    torch.cuda.synchronize()
    values_ms = v0.elapsed_time(v1) / args.steps

    # end-to-end leg through mgt_transpose_host: every step uploads its inputs
    # from pinned host memory, transposes and downloads the output arrays into
    # pinned host memory.  Inside a step the value upload overlaps the
    # structure phases and the structure download overlaps the value copy (a
    # second stream per lane); lanes (own device buffers and streams) take the
    # steps in turn, so one step's downloads overlap the next one's uploads.
    h_in = pinned[:4]  # row_ptr, col_idx, cell_ptr, values bytes, in generation order
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = sum(t.numel() * t.element_size() for t in out[:4])
    e2e_steps = max(1, args.e2e_steps)
    lanes = [(d, out, ws, stream, torch.cuda.Stream())]
    n_lanes = min(args.e2e_lanes, e2e_steps)
    lane_bytes = h2d + d2h + plan.workspace_bytes
    while n_lanes > 1 and (n_lanes - 1) * lane_bytes > 0.5 * torch.cuda.mem_get_info()[0]:
        n_lanes -= 1  # extra lanes only where their buffers fit comfortably
    for _ in range(n_lanes - 1):
        d1 = mgt.DeviceXCSR(x.n_rows, x.n_cols, x.offset_bytes, x.stride,
                            *[torch.empty_like(t) for t in d.arrays()], x.part_off)
        lanes.append((d1, mgt.alloc_output(d1, parts=True), mgt.alloc_workspace(plan.workspace_bytes),
                      torch.cuda.Stream(), torch.cuda.Stream()))
    h_outs = [[torch.empty(t.numel() * t.element_size(), dtype=torch.uint8, pin_memory=True)
               for t in lane[1][:4]] for lane in lanes]

    def e2e_step(k):
        dd, oo, ww, ss, cs = lanes[k % len(lanes)]
        mgt.transpose_host(plan, h_in, h_outs[k % len(lanes)], dd.arrays(), oo, ww, stream=ss,
                           copy_stream=cs)

    for k in range(len(lanes)):  # warm both lanes
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for lane in lanes[1:]:
        lane[3].wait_event(e0)
    for k in range(e2e_steps):
        e2e_step(k)
    for lane in lanes[1:]:
        ev = torch.cuda.Event()
        ev.record(lane[3])
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    st = mgt.read_status(lanes[-1][2], lanes[-1][3])
    if st != 0:
        raise SystemExit(f"device status {st} in the end-to-end leg ({mgt.strerror(st)})")

    extra = None
    n_lanes_used = len(lanes)
    if args.workload == "heterogeneous" and not args.no_extra and not args.rows:
        del lanes, h_outs, d, ws, out
        torch.cuda.empty_cache()
        extra = time_extra(args, "balanced", torch, mgt, barrier, stream, world)

    # max of the times over ranks, sum of the work
    (total_ms, e2e_ms), (job_bytes, job_cells) = reduce_over_ranks(
        [total_ms, e2e_ms], [minimal, x.n_cells], device="cuda")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    ms = total_ms / args.steps
    gbs = job_bytes / (ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    # roofline of the dominant kernel: the per-bucket sort + value copy (place)
    dom = max(phases, key=lambda p: phase_ms[p])
    dom_ms = phase_ms[dom]
    alg = algorithmic_bytes(dom, x, plan)
    achieved = alg / (dom_ms * 1e-3) / 1e9 if alg else None
    alg_meta = algorithmic_bytes(dom, x, plan, metadata=True)
    achieved_meta = alg_meta / (dom_ms * 1e-3) / 1e9 if alg_meta else None
    cpu = None
    if not args.no_cpu_baseline:
        cgbs, ccells, sample, per = time_oracle(args.workload, args.seed, args.cpu_seconds)
        cpu = {"value": round(cgbs, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": sample, "cells_per_s": round(ccells, 1), "host_cores": os.cpu_count()}
    line = {
        "metric": METRIC, "value": round(gbs, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": dict(workload_config(args.workload, x), l2_fetch_bytes=l2f),
        "frac_of_hbm_peak": round(gbs / world / peak, 4), "hbm_peak_gbs": peak,
        "hbm_peak_kind": peak_kind,
        "cells_per_s": round(job_cells / (ms * 1e-3), 1),
        "p50_ms": round(float(np.percentile(step_ms, 50)), 4),
        "p99_ms": round(float(np.percentile(step_ms, 99)), 4),
        "phase_ms": {k: round(v, 4) for k, v in phase_ms.items()},
        "tiles": plan.config, "tiles_source": tiles_source,
        "roofline": {"bound": "hbm", "kernel": dom,
                     "achieved": round(achieved, 2) if achieved else None, "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
                     "traffic": traffic_for(dom, args.workload), "algorithmic_bytes": alg,
                     "peak_kind": peak_kind,
                     "with_metadata": {"algorithmic_bytes": alg_meta,
                                       "achieved": round(achieved_meta, 2) if achieved_meta else None,
                                       "frac": round(achieved_meta / peak, 4) if achieved_meta else None}},
        "cpu_baseline": cpu,
        "e2e": {"value": round(job_bytes / (e2e_ms * 1e-3) / 1e9, 3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_ms, 3), "steps": e2e_steps, "lanes": n_lanes_used},
        "values_only": {"ms_per_step": round(values_ms, 4),
                        "note": "re-transpose of new payloads on an unchanged structure (value copy only)"},
        "gpu_launches": plan.kernel_launches * args.steps,
        "clocks": clk,
        "gen_s": round(t_gen, 2),
    }
    if extra is not None:
        line["balanced"] = extra
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------- batched (config 4)
def _device_matrix(x, torch, mgt):
    return mgt.DeviceXCSR(x.n_rows, x.n_cols, x.offset_bytes, x.stride,
                          *[torch.from_numpy(np.ascontiguousarray(a)).cuda()
                            for a in (x.row_ptr, x.col_idx, x.cell_ptr, x.values)], x.part_off)


def run_batched(args):
    """512 independent square matrices (rows log-uniform in [1e3, 2e6],
    lognormal cells/row of mean 16, geometric run lengths of mean 4, 16-byte
    payload), in waves that fit HBM.  Per wave, the same members with the
    same autotuned plans are timed two ways: one mgt_transpose per matrix
    (one launch sequence each), and the batch (one launch per phase for the
    whole wave) replayed as a CUDA graph.  value = batched GB/s over all
    waves; per_matrix = the other arm."""
    import torch
    import synth
    from paper_2012_06012_gb300 import mgt
    torch.cuda.set_device(0)
    l2f = apply_l2_fetch(args)
    stream = torch.cuda.current_stream()
    tune = mgt.TuneCache(reps=1)
    members = list(range(args.members))
    wave_bytes = int(args.wave_gb * 1e9)
    tot_bytes = tot_cells = 0
    t_batched = t_single = 0.0
    waves, launches_b, launches_s, gen_s = 0, 0, 0, 0.0
    i = 0
    clocks = ClockSampler(0)
    clocks.start()
    while i < len(members):
        # build one wave: generate and upload members until the payload budget
        devs, xs_bytes, wave_min = [], 0, 0
        t0 = time.perf_counter()
        while i < len(members) and (not devs or xs_bytes < wave_bytes):
            x = synth.generate(synth.batched_member(seed=args.seed, m=members[i]))
            devs.append((x.minimal_bytes(), x.n_cells, _device_matrix(x, torch, mgt)))
            xs_bytes += x.minimal_bytes()
            del x
            i += 1
        gen_s += time.perf_counter() - t0
        plans = [mgt.plan_for(d, tune.cfg_for(d)) for _, _, d in devs]
        outs = [mgt.alloc_output(d) for _, _, d in devs]
        wss = [mgt.alloc_workspace(p.workspace_bytes) for p in plans]
        bws = mgt.alloc_workspace(mgt.batched_workspace(plans))
        batch = mgt.Batch(plans, [d.arrays() for _, _, d in devs], outs, bws)
        # correctness gate: every member's status after one batched run
        batch.launch(stream)
        assert batch.status(stream) == [0] * len(devs)
        for k in range(args.warmup):
            batch.launch(stream)
            for p, (_, _, d), o, w in zip(plans, devs, outs, wss):
                mgt.transpose(p, d.arrays(), o, w, stream)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        for _ in range(args.steps):
            for p, (_, _, d), o, w in zip(plans, devs, outs, wss):
                mgt.transpose(p, d.arrays(), o, w, stream)
        e[1].record(stream)
        e[2].record(stream)
        for _ in range(args.steps):
            batch.launch(stream)
        e[3].record(stream)
        torch.cuda.synchronize()
        t_single += e[0].elapsed_time(e[1]) / args.steps
        t_batched += e[2].elapsed_time(e[3]) / args.steps
        tot_bytes += sum(b for b, _, _ in devs)
        tot_cells += sum(c for _, c, _ in devs)
        launches_b += batch.kernel_launches
        launches_s += sum(p.kernel_launches for p in plans)
        waves += 1
        batch.close()
        del batch, bws, wss, outs, plans, devs
        torch.cuda.empty_cache()
    clk = clocks.stop()
    peak, peak_kind = _peaks()
    gbs_b = tot_bytes / (t_batched * 1e-3) / 1e9
    gbs_s = tot_bytes / (t_single * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(gbs_b, 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_batched, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "batched", "members": len(members), "waves": waves, "l2_fetch_bytes": l2f,
                   "wave_payload_gb": args.wave_gb, "minimal_bytes": tot_bytes,
                   "n_cells": tot_cells, "payload_stride": 16, "offset_bytes": 4,
                   "l2": "inputs larger than L2 (no flush)", "seed": args.seed,
                   "tiles": "autotuned per size class"},
        "frac_of_hbm_peak": round(gbs_b / peak, 4), "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind,
        "cells_per_s": round(tot_cells / (t_batched * 1e-3), 1),
        "per_matrix": {"value": round(gbs_s, 3), "unit": UNIT, "ms_per_step": round(t_single, 3),
                       "gpu_launches_per_step": launches_s},
        "batched_over_per_matrix": round(t_single / t_batched, 4),
        "gpu_launches": launches_b * args.steps,
        "clocks": clk, "gen_s": round(gen_s, 1),
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- serving (config 5)
def run_serving(args):
    """Poisson arrivals (mean args.rate req/s) for args.duration seconds: 95 %
    drawn from a device-resident pool of config-4 members, 5 % large
    requests (4,194,304 rows, heterogeneous distributions), through the
    serving loop with an HBM admission budget.  Reports p50/p99 latency
    (submission -> completion), achieved and offered GB/s."""
    import torch
    import synth
    from paper_2012_06012_gb300 import mgt
    torch.cuda.set_device(0)
    l2f = apply_l2_fetch(args)
    rng = np.random.default_rng(args.seed)
    t0 = time.perf_counter()
    small = []
    for m in range(args.pool_small):
        x = synth.generate(synth.batched_member(seed=args.seed + 1, m=m))
        d = _device_matrix(x, torch, mgt)
        small.append((d, mgt.plan_for(d), mgt.alloc_output(d), x.minimal_bytes()))
        del x
    large = []
    for m in range(args.pool_large):
        x = synth.generate(synth.large_member(seed=args.seed + 2, m=m, n=args.large_rows))
        d = _device_matrix(x, torch, mgt)
        large.append((d, mgt.plan_for(d), mgt.alloc_output(d), x.minimal_bytes()))
        del x
    gen_s = time.perf_counter() - t0
    srv = mgt.Server(hbm_budget_bytes=int(args.budget_gb * 1e9), max_slots=args.slots,
                     n_streams=args.streams, max_queue=1 << 20, batch_max=args.batch_max,
                     fuse_max_cells=1 << 22)
    # warm-up: every pool entry once
    tk = [srv.submit(p, d.arrays(), o) for d, p, o, _ in small + large]
    srv.drain()
    for t in tk:
        assert srv.poll(t)[:2] == (True, 0)
    srv.reset_stats()
    n_req = int(args.rate * args.duration)
    gaps = rng.exponential(1.0 / args.rate, size=n_req)
    kinds = rng.random(n_req) < args.large_frac
    picks = rng.integers(0, 1 << 30, size=n_req)
    offered = 0
    tickets = []
    clocks = ClockSampler(0)
    clocks.start()
    start = time.perf_counter()
    t_next = start
    for k in range(n_req):
        t_next += gaps[k]
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        pool = large if (kinds[k] and large) else small
        d, p, o, mb = pool[picks[k] % len(pool)]
        tickets.append(srv.submit(p, d.arrays(), o))
        offered += mb
    t_sub = time.perf_counter() - start
    s_mid = srv.stats()  # backlog when the last request arrived
    srv.drain()
    t_all = time.perf_counter() - start
    clk = clocks.stop()
    for t in tickets:
        done, st, _ = srv.poll(t)
        assert done and st == 0
    s = srv.stats()
    srv.close()
    # the baseline the server is compared with: the SAME requests, in the same
    # order, one mgt_transpose each, back to back on one stream (no arrival
    # times: the GPU is never idle)
    n_seq = n_req if args.seq_requests <= 0 else min(n_req, args.seq_requests)
    ws_seq = mgt.alloc_workspace(max(p.workspace_bytes for _, p, _, _ in small + large))
    st = torch.cuda.current_stream()
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    seq_bytes = 0
    torch.cuda.synchronize()
    q0.record(st)
    for k in range(n_seq):
        pool = large if (kinds[k] and large) else small
        d, p, o, mb = pool[picks[k] % len(pool)]
        mgt.transpose(p, d.arrays(), o, ws_seq, st)
        seq_bytes += mb
    q1.record(st)
    torch.cuda.synchronize()
    if mgt.read_status(ws_seq) != 0:
        raise SystemExit("device status error in the sequential baseline")
    seq_gbs = seq_bytes / (q0.elapsed_time(q1) * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    gbs = s["bytes"] / t_all / 1e9
    line = {
        "metric": METRIC, "value": round(gbs, 3), "unit": UNIT, "n_gpus": 1,
        "steps": n_req, "warmup": len(tk), "ms_per_step": round(t_all * 1e3 / max(1, n_req), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+int64",
        "data": "synthetic",
        "config": {"workload": "serving", "rate_req_s": args.rate, "duration_s": args.duration,
                   "l2_fetch_bytes": l2f,
                   "large_frac": args.large_frac, "pool_small": args.pool_small,
                   "pool_large": args.pool_large, "large_rows": args.large_rows,
                   "budget_gb": args.budget_gb, "slots": args.slots, "streams": args.streams,
                   "batch_max": args.batch_max, "l2": "inputs larger than L2 (no flush)",
                   "seed": args.seed},
        "frac_of_hbm_peak": round(gbs / peak, 4), "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind,
        "p50_ms": round(s["p50_ms"], 3), "p99_ms": round(s["p99_ms"], 3),
        "mean_ms": round(s["mean_ms"], 3),
        "offered_gbs": round(offered / t_sub / 1e9, 3), "achieved_gbs": round(gbs, 3),
        "requests": n_req, "completed": s["completed"], "launches": s["launches"],
        "fused_requests": s["fused_requests"], "peak_inflight_gb": round(s["peak_inflight_bytes"] / 1e9, 2),
        "submit_s": round(t_sub, 3), "wall_s": round(t_all, 3),
        "sequential": {"gbs": round(seq_gbs, 3), "requests": n_seq,
                       "s": round(q0.elapsed_time(q1) * 1e-3, 3),
                       "note": ("the same requests in the same order, one mgt_transpose each, back to "
                                "back on one stream" if n_seq == n_req else
                                f"the first {n_seq} requests of the same stream, one mgt_transpose each")},
        "backlog_at_last_arrival": {"queued": int(s_mid["queued"]),
                                    "inflight_gb": round(s_mid["inflight_bytes"] / 1e9, 2),
                                    "drain_s": round(t_all - t_sub, 3)},
        "sustained": bool(t_all - t_sub < 0.05 * t_sub),
        # a server cannot deliver more than is offered: the ratio means
        # something only when the offered load exceeds the sequential rate
        # equal work both ways: the served run's wall time (first arrival to last
        # completion) against the back-to-back time of the same requests; above
        # 1 only when arrivals keep the GPU busy (offered load above capacity)
        "served_vs_sequential": (round(q0.elapsed_time(q1) * 1e-3 / t_all, 3) if n_seq == n_req else None),
        "clocks": clk, "gen_s": round(gen_s, 1),
    }
    print(json.dumps(line), flush=True)
    return 0


def apply_l2_fetch(args):
    """--l2-fetch: the context's L2 fetch granularity hint for every launch of
    this process (mgt_l2_fetch_granularity); returns the value in force."""
    from paper_2012_06012_gb300 import mgt
    if args.l2_fetch is None or args.l2_fetch < 0:
        return None  # the context's default (reported as 64, behaves as 128)
    mgt.l2_fetch_granularity(args.l2_fetch)
    return mgt.l2_fetch_granularity()


def run_probe(args):
    """Raw rates of the two orders in which the value copy can walk the run
    permutation (mgt_probe_runs): output order (gather: random reads,
    sequential writes), input order (scatter: sequential reads, random
    writes), the scatter's one random 4-byte offset write per run, and a
    sequential copy, for runs of 32 to 256 bytes over buffers far larger
    than L2 (args.probe_gb each)."""
    import torch
    from paper_2012_06012_gb300 import mgt
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream()
    nbytes = int(args.probe_gb * 2**30) // 256 * 256
    src = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    src.random_(0, 256)
    peak, peak_kind = _peaks()
    l2f = apply_l2_fetch(args)
    names = {0: "gather", 1: "scatter", 2: "offset_writes", 3: "sequential", 4: "gather_staged",
             5: "gather_tma_bulk"}
    res = []
    clocks = ClockSampler(0)
    clocks.start()
    for rb in (32, 64, 96, 128, 160, 256):
        n = nbytes // rb
        perm = torch.randperm(n, device="cuda", dtype=torch.int32)
        for mode in (3, 0, 4, 5, 1, 2):
            for _ in range(max(1, args.warmup)):
                mgt.probe_runs(mode, src, dst, perm, n, rb, st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(args.steps):
                mgt.probe_runs(mode, src, dst, perm, n, rb, st)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            moved = n * 4 if mode == 2 else 2 * n * rb
            res.append({"run_bytes": rb, "mode": names[mode], "ms": round(ms, 4),
                        "gbs": round(moved / (ms * 1e-3) / 1e9, 1),
                        "g_runs_per_s": round(n / (ms * 1e-3) / 1e9, 2),
                        "frac": round(moved / (ms * 1e-3) / 1e9 / peak, 4)})
        del perm
    clk = clocks.stop()
    if mgt.probe_errors():
        raise RuntimeError("probe mode 5: a bulk-copy wait ran out of polls")
    line = {"metric": "probe: raw GB/s of run permutations (gather vs scatter)", "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "hbm_peak_gbs": peak,
            "hbm_peak_kind": peak_kind, "buffer_gb": round(nbytes / 1e9, 2),
            "config": {"workload": "probe", "l2": "buffers larger than L2 (no flush)",
                       "l2_fetch_bytes": l2f},
            "results": res, "gpu_launches": len(res) * (args.steps + max(1, args.warmup)),
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_var(args):
    """Variable-width values (the paper's heterogeneous-datatype variant,
    Sec. 2, MPI_Alltoallw): the heterogeneous workload's cells and run
    lengths, each value a type of its own width drawn uniformly from
    synth.TYPE_SIZES (4 to 64 bytes), through mgt_transpose_var.  Minimal
    bytes count the value offsets and bytes on both sides."""
    import torch
    import synth
    from paper_2012_06012_gb300 import mgt
    torch.cuda.set_device(0)
    l2f = apply_l2_fetch(args)
    spec = workload_spec("heterogeneous", args.seed, 0)
    if args.rows:
        spec.n_rows = spec.n_cols = args.rows
    t0 = time.perf_counter()
    x = synth.generate_var(spec)
    gen_s = time.perf_counter() - t0
    d = mgt.to_device_var(x)
    plan = mgt.plan_for_var(d)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    out, ovo = mgt.alloc_output_var(d, parts=True)
    st = torch.cuda.current_stream()
    mgt.transpose_var(plan, d.arrays(), d.val_off, out, ovo, ws, st)
    if mgt.read_status(ws, st) != 0:
        raise SystemExit("device status error (variable-width workload)")
    for _ in range(args.warmup):
        mgt.transpose_var(plan, d.arrays(), d.val_off, out, ovo, ws, st)
    phases = plan.phases
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)] for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(args.steps):
        mgt.transpose_var(plan, d.arrays(), d.val_off, out, ovo, ws, st, events=ev[k])
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if mgt.read_status(ws, st) != 0:
        raise SystemExit("device status error after timing (variable-width workload)")
    ms = e0.elapsed_time(e1) / args.steps
    phase_ms = {ph: round(statistics.mean(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)), 4)
                for i, ph in enumerate(phases)}
    peak, peak_kind = _peaks()
    minimal = x.minimal_bytes()
    gbs = minimal / (ms * 1e-3) / 1e9
    copy_alg = 2 * x.n_bytes
    copy_meta = copy_alg + 2 * 8 * (x.n_values + 1) + (x.n_cells + 1) * x.offset_bytes + x.n_cells * 4
    line = {
        "metric": METRIC, "value": round(gbs, 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "var_width", "n_rows": x.n_rows, "n_cols": x.n_cols, "l2_fetch_bytes": l2f,
                   "n_cells": x.n_cells, "n_values": x.n_values, "n_bytes": x.n_bytes,
                   "value_widths": list(synth.TYPE_SIZES), "offset_bytes": x.offset_bytes,
                   "partitions": x.n_parts, "minimal_bytes": minimal,
                   "l2": l2_note(minimal), "seed": args.seed},
        "frac_of_hbm_peak": round(gbs / peak, 4), "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind,
        "cells_per_s": round(x.n_cells / (ms * 1e-3), 1), "phase_ms": phase_ms,
        "copy_roofline": {"bound": "hbm", "algorithmic_bytes": copy_alg,
                          "achieved": round(copy_alg / (phase_ms["copy"] * 1e-3) / 1e9, 2),
                          "frac": round(copy_alg / (phase_ms["copy"] * 1e-3) / 1e9 / peak, 4),
                          "with_metadata_frac": round(copy_meta / (phase_ms["copy"] * 1e-3) / 1e9 / peak, 4)},
        "tiles": plan.config, "gpu_launches": plan.kernel_launches * args.steps, "clocks": clk,
        "gen_s": round(gen_s, 2),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_chain(args):
    """The paper's repeated-transpose benchmark (Sec. 5): a composition of 12
    transposes of its imbalanced matrix shape (64 rows of 300 thousand to
    1 million uniform columns, 128-byte values, 5 per cell on average), M ->
    M^T -> M ... on the device, timed per transpose; after the even chain the
    matrix must equal the input bit for bit (involution, Sec. 3)."""
    import torch
    import synth
    from paper_2012_06012_gb300 import mgt
    torch.cuda.set_device(0)
    l2f = apply_l2_fetch(args)
    t0 = time.perf_counter()
    x = synth.generate(workload_spec("chain", args.seed, 0))
    gen_s = time.perf_counter() - t0
    d = mgt.to_device(x)
    mt = mgt.DeviceXCSR(x.n_cols, x.n_rows, x.offset_bytes, x.stride,
                        *mgt.alloc_output(d, parts=False)[:4], np.array([0, x.n_cols], np.int64))
    back = mgt.DeviceXCSR(x.n_rows, x.n_cols, x.offset_bytes, x.stride,
                          *mgt.alloc_output(mt, parts=False)[:4], x.part_off)
    fwd, rev = mgt.plan_for(d), mgt.plan_for(mt)
    ws = mgt.alloc_workspace(max(fwd.workspace_bytes, rev.workspace_bytes))
    st = torch.cuda.current_stream()
    nul = (None, None)
    # M -> M^T -> M once untimed (the chain then ping-pongs between mt and back;
    # d keeps the input for the final comparison), plus warm-up pairs
    mgt.transpose(fwd, d.arrays(), mt.arrays() + nul, ws, st)
    mgt.transpose(rev, mt.arrays(), back.arrays() + nul, ws, st)
    for _ in range(max(0, args.warmup - 2) // 2):
        mgt.transpose(fwd, back.arrays(), mt.arrays() + nul, ws, st)
        mgt.transpose(rev, mt.arrays(), back.arrays() + nul, ws, st)
    if mgt.read_status(ws, st) != 0:
        raise SystemExit("device status error before the chain")
    n = 12
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    ev[0].record(st)
    for k in range(n):
        if k % 2 == 0:
            mgt.transpose(fwd, back.arrays(), mt.arrays() + nul, ws, st)
        else:
            mgt.transpose(rev, mt.arrays(), back.arrays() + nul, ws, st)
        ev[k + 1].record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if mgt.read_status(ws, st) != 0:
        raise SystemExit("device status error in the chain")
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(n)]
    exact = all(torch.equal(a, b) for a, b in zip(back.arrays(), d.arrays()))
    minimal = fwd.minimal_bytes()
    total_ms = sum(ms)
    peak, peak_kind = _peaks()
    gbs = n * minimal / (total_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(gbs, 3), "unit": UNIT, "n_gpus": 1, "steps": n,
        "warmup": args.warmup, "ms_per_step": round(total_ms / n, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(workload_config("chain", x), transposes=n, l2_fetch_bytes=l2f),
        "frac_of_hbm_peak": round(gbs / peak, 4), "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind,
        "cells_per_s": round(n * x.n_cells / (total_ms * 1e-3), 1),
        "ms_forward": round(statistics.mean(ms[0::2]), 4),
        "ms_reverse": round(statistics.mean(ms[1::2]), 4),
        "involution_exact": bool(exact),
        "tiles_forward": fwd.config, "tiles_reverse": rev.config,
        "gpu_launches": (fwd.kernel_launches + rev.kernel_launches) * n // 2,
        "clocks": clk, "gen_s": round(gen_s, 1),
    }
    print(json.dumps(line), flush=True)
    return 0 if exact else 1


def algorithmic_bytes(phase: str, x, plan, metadata: bool = False) -> int | None:
    """Bytes one launch of a phase must move at minimum (its inputs read once,
    its outputs written once), records included where the phase reads or
    writes them.  r = record bytes (12, or 16 when V >= 2^32), o = offset
    width, s = payload stride, q = bytes of a run's source offset (4 or 8).
    hist: col_idx.  scatter: col_idx, cell_ptr, row_ptr in; records out.
    scatter2: records in and out.  place: records in; col_idx', cell_ptr',
    row_ptr' and the run source offsets out.  copy: the values in and out
    (2 V s, the value-run step's own bytes); with ``metadata`` also the run
    source offsets and cell_ptr' it reads to find the runs."""
    o, C, V, s, N, R = x.offset_bytes, x.n_cells, x.n_values, x.stride, x.n_cols, x.n_rows
    wide = x.n_values >= (1 << 32)
    rec = 16 if wide else 12
    q = 8 if wide else 4
    if phase == "hist":
        return C * 4
    if phase == "scatter":
        return C * 4 + (C + 1) * o + (R + 1) * o + C * rec
    if phase == "scatter2":
        return 2 * C * rec
    if phase == "place":
        return C * rec + C * 4 + (C + 1) * o + (N + 1) * o + C * q
    if phase == "copy":
        return 2 * V * s + ((C * q + (C + 1) * o) if metadata else 0)
    if phase == "part_counts":
        return 4 * C + (C + 1) * o
    return None


def traffic_for(phase: str, workload: str):
    """DRAM bytes per launch from a committed ncu capture, if one matches the
    current kernel sources (profiles/traffic.json)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d.get(f"{workload}/{phase}")
        if not ent or ent.get("sources") != sources_hash():
            return None
        return ent.get("bytes_per_launch")
    except Exception:
        return None


def sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2012_06012_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mgt", choices=["mgt", "reference"])
    ap.add_argument("--workload", default="heterogeneous",
                    choices=["balanced", "heterogeneous", "tiny", "batched", "serving",
                             "paper_balanced", "paper_heterogeneous", "chain", "probe", "var_width"])
    ap.add_argument("--config", type=int, choices=[1, 2, 3, 4, 5], default=None,
                    help="workload by number: 1 tiny, 2 balanced, 3 heterogeneous, 4 batched, 5 serving")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tiles", default="", help='tile configuration as JSON, e.g. {"stage_values": 2}')
    ap.add_argument("--rows", type=int, default=0, help="override rows/cols (profiling cases)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-lanes", type=int, default=3,
                    help="buffer sets taking the end-to-end steps in turn")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the default plan instead of the autotuned one")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the balanced workload timed after the heterogeneous one")
    # batched
    ap.add_argument("--members", type=int, default=512)
    ap.add_argument("--wave-gb", type=float, default=40.0, help="minimal bytes per wave")
    # serving
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--large-frac", type=float, default=0.05)
    ap.add_argument("--large-rows", type=int, default=4_194_304)
    ap.add_argument("--pool-small", type=int, default=64)
    ap.add_argument("--pool-large", type=int, default=2)
    ap.add_argument("--budget-gb", type=float, default=180.0)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--batch-max", type=int, default=16)
    ap.add_argument("--probe-gb", type=float, default=4.0, help="probe: GiB per buffer")
    ap.add_argument("--l2-fetch", type=int, default=32,
                    help="L2 fetch granularity hint in bytes (0-128) for this process's launches "
                         "(-1: leave the context's default)")
    ap.add_argument("--seq-requests", type=int, default=0,
                    help="serving: requests timed one transpose at a time as the baseline "
                         "(0: all of them, the same request set the server ran)")
    args = ap.parse_args()
    if args.config is not None:
        args.workload = ["tiny", "balanced", "heterogeneous", "batched", "serving"][args.config - 1]
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "chain":
        return run_chain(args)
    if args.workload == "probe":
        return run_probe(args)
    if args.workload == "var_width":
        return run_var(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
