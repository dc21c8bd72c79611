"""Benchmark of the parallel CPM copy-attempt sweep on GB300.

A step is one Monte Carlo step (MCS): one copy attempt per lattice site,
issued as P cycles x c^d colour sub-passes x k rounds of the checkerboard
scheme, all in the CUDA library's kernels.  The metric is copy attempts per
second (every attempt counts, early rejects included) and the fraction of
the HBM roofline of the round kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the scheme needs no data exchange between replicas); the value is
the attempts of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cpm_workloads as cw  # noqa: E402

METRIC = "copy attempts/s"
UNIT = "attempts/s"

# Workloads: (factory, algorithmic bytes per site per MCS, description)
# bytes: int32 lattice read + write (8 B); with Act the uint8 stamp read + write (2 B).
WORKLOADS = {
    "cpm2d_200": (lambda: cw.point_cells_2d(seed=1), 8,
                  "2D 200x200 Moore-8, 100 one-pixel cells, V_t=100, J(c,c)=20, J(c,m)=10, lambda_V=50, T=20; "
                  "a=4, c=2, P=1"),
    "cpm3d_256": (lambda: cw.cube_cells_3d(seed=1, n=256, a=4, c=2, P=8), 8,
                  "3D 256^3 Moore-26, ~17,576 cells, V_t=500, A_t=400, lambda_V=25, lambda_P=0.5, "
                  "J(c,c)=20, J(c,m)=12, T=20 (x2 integer scale); a=4, c=2, P=8"),
    # the same model on a lattice larger than L2, for DRAM counters
    "cpm3d_512": (lambda: cw.cube_cells_3d(seed=1, n=512, a=4, c=2, P=8), 8,
                  "3D 512^3, otherwise as cpm3d_256"),
    "cpm3d_tissue_1024": (lambda: cw.fibre_tissue_3d(seed=1, n=1024, device="cuda", **cw.TISSUE_SCHEDULE), 10,
                          "3D tissue 1024^3 Moore-26 with a Voronoi-edge fibre mask (15% frozen), ~0.9M motile "
                          "cells, V_t=800, A_t=4639, Act lambda=200 Max=30, J(c,c)=20, J(c,m)=10, "
                          "J(c,fibre)=40, lambda_V=25, lambda_P=0.2, T=20 (x5 integer scale); "
                          "a={a}, c={c}, P={P} (the schedule that matches the serial chain within 2 percent)"
                          .format(**cw.TISSUE_SCHEDULE)),
    "cpm3d_tissue_512": (lambda: cw.fibre_tissue_3d(seed=1, n=512, device="cuda", **cw.TISSUE_SCHEDULE), 10,
                         "3D tissue 512^3, otherwise as cpm3d_tissue_1024"),
    # smaller areas: faster, but biased against the serial chain (the paper's 4^3, and 8^3)
    "cpm3d_tissue_1024_a4": (lambda: cw.fibre_tissue_3d(seed=1, n=1024, a=4, c=2, P=8, device="cuda"), 10,
                             "as cpm3d_tissue_1024 with a=4, c=2, P=8"),
    "cpm3d_tissue_1024_a8": (lambda: cw.fibre_tissue_3d(seed=1, n=1024, a=8, c=2, P=64, device="cuda"), 10,
                             "as cpm3d_tissue_1024 with a=8, c=2, P=64"),
    # the tissue workload under the tiled schedule (tiles of edge 16, one tile cycle per MCS)
    "cpm3d_tissue_1024_tiled": (lambda: cw.fibre_tissue_3d(seed=1, n=1024, a=4, c=2, P=8, device="cuda")
                                .replace(tile=16, tile_cycles=1), 10,
                                "as cpm3d_tissue_1024, tiled schedule: tiles of edge 16, 1 tile cycle per MCS"),
    "cpm3d_tissue_1024_tiled2": (lambda: cw.fibre_tissue_3d(seed=1, n=1024, a=4, c=2, P=8, device="cuda")
                                 .replace(tile=16, tile_cycles=2), 10,
                                 "as cpm3d_tissue_1024, tiled schedule: tiles of edge 16, 2 tile cycles per MCS"),
    "cpm3d_tissue_1024_t32p8": (lambda: cw.fibre_tissue_3d(seed=1, n=1024, a=4, c=2, P=8, device="cuda")
                                .replace(tile=32, tile_cycles=8), 10,
                                "as cpm3d_tissue_1024, tiled schedule: tiles of edge 32, 8 tile cycles per MCS"),
    "cpm3d_tissue_512_t32p8": (lambda: cw.fibre_tissue_3d(seed=1, n=512, a=4, c=2, P=8, device="cuda")
                               .replace(tile=32, tile_cycles=8), 10,
                               "3D tissue 512^3, tiled schedule: tiles of edge 32, 8 tile cycles per MCS"),
    "cpm3d_tissue_512_tiled": (lambda: cw.fibre_tissue_3d(seed=1, n=512, a=4, c=2, P=8, device="cuda")
                               .replace(tile=16, tile_cycles=1), 10,
                               "3D tissue 512^3, tiled schedule: tiles of edge 16"),
}
# Ensembles for parameter sweeps: many independent lattices of uneven sizes advanced
# together; a step is one MCS of every member.
ENSEMBLES = {
    "cpm_ensemble_512": (lambda: cw.ensemble(512, seed=1),
                         "512 lattices (2D 64^2..512^2, 3D 64^3..128^3, log-uniform), 10..2,000 cells each, "
                         "J(c,c), J(c,m), lambda_V, lambda_P, lambda_act, Max_act, T from a Latin hypercube "
                         "(x10 integer scale); a=4, c=2, one round per colour visit; 2D and 3D members in two "
                         "batches on one stream"),
}

# The emulator of the parameter sweep: sweep points answered at <= 5% error on the summary
# statistics, emulator + CPM fallback against the CPM alone.
EMULATOR = {
    "emulator_sweep": "MLP-ensemble emulator (5 x 7-256x4-16, GELU, bf16/fp32) of 16 summary statistics of 2D "
                      "64x64 runs with 16 cells (V_t=128), J(c,c), J(c,m), lambda_V, lambda_P, lambda_act, "
                      "Max_act, T from a Latin hypercube (x10 integer scale); 200 MCS burn-in + 800 MCS observed "
                      "every 10 MCS; trained on batched-CPM runs (80/20 split); fallback when the ensemble std "
                      "exceeds 3x the validation RMSE",
}
SWEEP_METRIC = "sweep points/s at <=5% stat error"

# Burn-in MCS before the warm-up steps: cells start as small seeds and grow
# to their target volumes; the timed window is the tissue after growth (the
# per-MCS cost settles after ~60 MCS on the 1024^3 tissue).
BURN_IN = {"cpm2d_200": 50, "cpm3d_256": 50, "cpm3d_512": 50, "cpm3d_tissue_1024": cw.TISSUE_BURN_IN,
           "cpm3d_tissue_512": cw.TISSUE_BURN_IN}

DEFAULT_WORKLOAD = "cpm3d_tissue_1024"

# DRAM bytes per round-kernel launch from the last ncu capture, valid only for
# the kernel source and launch shapes it was taken on (sha1 of csrc/cpm_kernels.cu
# followed by csrc/cpm_internal.h, first 12 hex).  A single-pass capture
# (dram__bytes_read/write.sum) of one launch at full size, after the growth
# burn-in and the warm-up.
NCU_TRAFFIC = {
    ("cpm3d_tissue_1024", "e0e74b368ce0"): 131.31e6 + 7.67e6,
}


def kernel_hash() -> str:
    h = hashlib.sha1()
    for f in ("cpm_kernels.cu", "cpm_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2312_09317_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def peaks_bf16():
    """Dense bf16 tensor peak (TFLOP/s): the measured cuBLAS burst figure, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples: a file the caller names (--clocks-csv), else a temporary one
        self.path = path or os.path.join(tempfile.gettempdir(), "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("CPM_BENCH_BACKEND") != "gloo" else "gloo")
        return ws, rank, local, dist
    return 1, 0, 0, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------
# CPU oracle timing (the --impl reference arm and the cpu_baseline object)
# ----------------------------------------------------------------------------

def crop(w, edge: int = 128):
    """A bounded sample of a large 3D workload: its first edge^3 voxels (a
    multiple of a), cells renumbered, same parameters."""
    if w.dim != 3 or w.nx <= edge:
        return w
    lat = np.ascontiguousarray(w.lattice[:edge, :edge, :edge])
    ids = np.unique(lat[lat > 0])
    remap = np.zeros(w.n_cells + 1, dtype=np.int32)
    remap[ids] = np.arange(1, len(ids) + 1, dtype=np.int32)
    lat = np.where(lat > 0, remap[np.maximum(lat, 0)], lat).astype(np.int32)
    ct = np.concatenate([[0], w.cell_type[ids]]).astype(np.uint8)
    act = None if w.act is None else np.ascontiguousarray(w.act[:edge, :edge, :edge])
    return w.replace(nx=edge, ny=edge, nz=edge, lattice=lat, cell_type=ct, act=act)


def oracle_sample(w, budget_s: float):
    """Time oracle (a), the serial CPM, single-threaded on this host over whole
    MCS of a 128^3 crop of the workload (the whole workload when smaller)
    until about budget_s seconds; returns attempts/s."""
    import oracle
    w = crop(w)
    st = oracle.State(w)
    n_mcs, t_used = 0, 0.0
    while t_used < budget_s:
        t0 = time.perf_counter()
        st.serial_run(1)
        t_used += time.perf_counter() - t0
        n_mcs += 1
    return n_mcs * w.n_sites / t_used, n_mcs, t_used


def run_reference(args):
    ws, rank, local, dist = dist_init()
    if rank != 0:
        return 0
    if args.workload in EMULATOR:
        return run_reference_sweep(args, ws)
    if args.workload in ENSEMBLES:
        w_full = ENSEMBLES[args.workload][0]()[0]
    else:
        w_full = WORKLOADS[args.workload][0]()
    w = crop(w_full)
    import oracle
    st = oracle.State(w)
    for _ in range(args.warmup):
        st.serial_run(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st.serial_run(1)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    value = args.steps * w.n_sites / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": args.workload, "sites": w.n_sites, "cells": w.n_cells},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "serial CPM oracle (a), one thread, %d whole MCS after %d warm-up MCS of %s"
                                   % (args.steps, args.warmup, "a %d^3 crop of the workload" % w.nx
                                      if w is not w_full else "the whole workload")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference_sweep(args, ws):
    """The sweep answered by the serial CPM oracle alone: each step runs one
    emulator-geometry run (64x64, 16 cells) for a bounded number of MCS and
    extrapolates to the full 1,000 MCS of a sweep run; one run per point, so
    the figure is an upper bound on the CPU's sweep points/s at any error."""
    import oracle
    mcs = 20
    times = []
    X = cw.sweep_points(args.warmup + args.steps, 5)
    for k in range(args.warmup + args.steps):
        st = oracle.State(cw.emulator_run(X[k], 9000 + k))
        t0 = time.perf_counter()
        st.serial_run(mcs)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_run = sum(times) / len(times) * (1000.0 / mcs)
    value = 1.0 / per_run
    line = {
        "impl": "reference", "metric": SWEEP_METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_run, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (serial CPM)", "data": "synthetic",
        "config": {"workload": args.workload, "description": EMULATOR[args.workload]},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": "serial CPM oracle (a), one thread: %d MCS of each of %d emulator runs, "
                                   "extrapolated to 1,000 MCS per run, one run per sweep point" % (mcs, args.steps)},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_gpu(args):
    import torch
    from paper_2312_09317_gb300 import build as B
    from paper_2312_09317_gb300 import cpm

    ws, rank, local, dist = dist_init()
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    barrier(dist)
    factory, bytes_per_site, desc = WORKLOADS[args.workload]
    w = factory()
    w = w.replace(seed=w.seed + 1000 * rank)  # independent replicas
    stream = torch.cuda.Stream()
    sim = cpm.Sim(w, stream=stream)
    n = w.n_sites
    per_mcs = w.P * w.c ** w.dim
    rounds = per_mcs * (((w.a // w.c) ** w.dim) // w.P)
    if w.tile:
        per_mcs = w.tile_cycles * 2 ** w.dim   # epochs per MCS
        rounds = per_mcs                       # one launch per epoch
    lattice_bytes = 4 * n
    flush_l2 = lattice_bytes * 2 < 256 * 2 ** 20
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.int32, device="cuda") if flush_l2 else None

    burn = BURN_IN.get(args.workload, 60 if "tissue" in args.workload else 0)
    sim.step(burn)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = sim.launches()
    clocks = ClockSampler(local, args.clocks_csv)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("bench_timed")  # names the timed launches for profilers
    for k in range(args.steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(k)
        with torch.cuda.stream(stream):
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(dist)
    clk = clocks.stop()
    launches = sim.launches() - l0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1e3
    t_max = max_over_ranks(dist, t_local)
    attempts_all = sum_over_ranks(dist, float(args.steps * n))
    value = attempts_all / t_max

    # per-launch duration of the round kernel: sub-passes (k = 1: one round each) timed alone
    sub = []
    with torch.cuda.stream(stream):
        for k in range(min(64, per_mcs * 4)):
            if flush is not None:
                flush.fill_(k)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step_subpasses(1)
            b.record(stream)
            sub.append((a, b))
    torch.cuda.synchronize()
    k_rounds = 1 if w.tile else ((w.a // w.c) ** w.dim) // w.P
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in sub) / k_rounds
    peak, peak_kind = peaks()
    alg_bytes_launch = bytes_per_site * n / rounds
    achieved = alg_bytes_launch / (launch_ms / 1e3) / 1e9
    khash = kernel_hash()
    traffic = NCU_TRAFFIC.get((args.workload, khash))

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    host = torch.empty((w.nz, w.ny, w.nx), dtype=torch.int32, pin_memory=True).numpy()
    sim.read_lattice(host)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.load_lattice(host)      # H2D of the step's input + tally recount
        sim.step(1)
        sim.read_lattice(host)      # D2H of the step's result (synchronises)
    e2e_local = time.perf_counter() - t0
    e2e_t = max_over_ranks(dist, e2e_local)
    e2e_value = sum_over_ranks(dist, float(e2e_steps * n)) / e2e_t

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, n_mcs, t_used = oracle_sample(w, args.cpu_budget)
        cw_ = crop(w)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "serial CPM oracle (a), one thread, the first %d MCS from the initial state of %s "
                         "(%.1f s)" % (n_mcs, "a %d^3 crop of the workload" % cw_.nx if cw_ is not w
                                       else "the whole workload", t_used)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "sites": n, "cells": w.n_cells,
                       "rounds_per_mcs": rounds, "burn_in_mcs": burn,
                       "l2": "flushed between timed steps (512 MiB write)"
                       if flush_l2 else "inputs larger than L2", "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": "of %s" % peak_kind,
                         "kernel": "tile_epoch_kernel" if w.tile else "round_kernel", "launch_ms": launch_ms,
                         "alg_bytes_per_launch": alg_bytes_launch},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": lattice_bytes,
                    "d2h_bytes_per_step": lattice_bytes, "steps": e2e_steps},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
    sim.close()
    if rank == 0 and ws == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_sweep:
        # the second half of the headline metric: sweep points/s at <= 5% error (emulator + CPM
        # fallback against the CPM alone), measured as `--workload emulator_sweep` does
        try:
            import argparse as _ap
            sa = _ap.Namespace(**vars(args))
            # a quarter-million-point block per step keeps the default run within minutes
            sa.workload, sa.steps, sa.warmup, sa.emu_block = "emulator_sweep", 2, 1, 1 << 18
            torch.cuda.empty_cache()
            sl = emulator_sweep_measure(sa, 0, 1, None)
            line["sweep"] = {"metric": sl["metric"], "value": sl["value"], "unit": sl["unit"],
                             "config": sl["config"], **sl["sweep"], "roofline": sl["roofline"]}
        except Exception as exc:  # reported, not fatal: the sweep is the second half of the line
            line["sweep"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if rank == 0 and ws == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_ensemble:
        # the batched ensemble of the parameter sweep (512 lattices of uneven sizes), measured as
        # `--workload cpm_ensemble_512` does, without its CPU baseline
        try:
            import argparse as _ap
            ea = _ap.Namespace(**vars(args))
            ea.workload, ea.steps, ea.warmup, ea.no_cpu_baseline = "cpm_ensemble_512", 5, 3, True
            torch.cuda.empty_cache()
            el = ensemble_measure(ea, 1, 0, local, None)
            line["ensemble"] = {k: el[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup",
                                                   "config", "roofline", "e2e", "gpu_launches", "clocks")}
        except Exception as exc:  # reported, not fatal
            line["ensemble"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _oracle_replica(job):
    """One CPU replica of the ensemble baseline: whole serial MCS of the given
    members, in turn, until the time budget is spent; (attempts, seconds)."""
    ws, budget = job
    import oracle
    att, used = 0, 0.0
    states = [oracle.State(w) for w in ws]
    while used < budget and states:
        for w, st in zip(ws, states):
            if used >= budget:
                break
            t0 = time.perf_counter()
            st.serial_run(1)
            used += time.perf_counter() - t0
            att += w.n_sites
    return att, used


def run_gpu_batch(args):
    import torch
    from paper_2312_09317_gb300 import build as B

    ws_, rank, local, dist = dist_init()
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    barrier(dist)
    line = ensemble_measure(args, ws_, rank, local, dist)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def ensemble_measure(args, ws_, rank, local, dist):
    """One ensemble workload's line (rank 0; None on the other ranks)."""
    import torch
    from paper_2312_09317_gb300 import cpm
    factory, desc = ENSEMBLES[args.workload]
    members = [w.replace(seed=w.seed + 1000003 * rank) for w in factory()]
    stream = torch.cuda.Stream()
    groups = [[w for w in members if w.dim == d] for d in (2, 3)]
    batches = [cpm.Batch(g, stream=stream) for g in groups if g]
    n = sum(w.n_sites for w in members)
    alg_bytes = sum((10 if w.act_on else 8) * w.n_sites for w in members)
    rounds = sum(max((w.a // w.c) ** w.dim * w.c ** w.dim for w in g) for g in groups if g)
    # the autotuner times its CTA shapes on the batches themselves (untimed; it only changes the split)
    choices = [b.autotune(2) for b in batches]
    if args.loop == "persistent":
        for b in batches:
            b.set_persistent(True)
    for _ in range(args.warmup):
        for b in batches:
            b.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = sum(b.launches() for b in batches)
    clocks = ClockSampler(local, args.clocks_csv)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("bench_timed")
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            ev[k][0].record(stream)
            for b in batches:
                b.step(1)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(dist)
    clk = clocks.stop()
    launches = sum(b.launches() for b in batches) - l0
    t_local = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    t_max = max_over_ranks(dist, t_local)
    value = sum_over_ranks(dist, float(args.steps * n)) / t_max
    step_s = t_local / args.steps
    launch_ms = 1e3 * step_s / max(1, launches // args.steps)
    peak, peak_kind = peaks()
    achieved = alg_bytes / step_s / 1e9

    # end to end: every member's lattice in from pinned host memory, one MCS, every lattice out
    hosts = []
    for b in batches:
        for k, w in enumerate(b.ws):
            h = torch.empty((w.nz, w.ny, w.nx), dtype=torch.int32, pin_memory=True).numpy()
            b.read_lattice(k, h)
            hosts.append((b, k, h))
    e2e_steps = max(2, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for b, k, h in hosts:
            b.load_lattice(k, h)
        for b in batches:
            b.step(1)
        for b, k, h in hosts:
            b.read_lattice(k, h)
    e2e_t = max_over_ranks(dist, time.perf_counter() - t0)
    e2e_value = sum_over_ranks(dist, float(e2e_steps * n)) / e2e_t

    cpu = None
    if rank == 0 and ws_ == 1 and not args.no_cpu_baseline:
        # the serial oracle as independent replicas, one process per host core (spawned), each running
        # whole MCS of its own ensemble members for a bounded time; aggregate attempts / wall time
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        cores = os.cpu_count() or 1
        jobs = [([members[k] for k in range(c, min(len(members), 2 * cores), cores)], args.cpu_budget)
                for c in range(cores)]
        t0 = time.perf_counter()
        with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_oracle_replica, jobs))
        wall = time.perf_counter() - t0
        att = sum(r[0] for r in res)
        busy = max(r[1] for r in res)
        cpu = {"value": att / busy, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "serial CPM oracle (a), %d independent processes (one per host core), whole MCS of "
                         "the first %d ensemble members from their initial states, %.0f s per process (%.1f s "
                         "wall); "
                         "aggregate attempts over the longest process time"
                         % (cores, min(len(members), 2 * cores), args.cpu_budget, wall)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "members": len(members), "sites": n,
                       "launches_per_step": launches // args.steps, "autotuned_shapes": choices,
                       "loop": args.loop,
                       "l2": "inputs larger than L2",
                       "parallelism": "replicas" if ws_ > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": "of %s" % peak_kind,
                         "kernel": "batch_round_kernel", "launch_ms": launch_ms,
                         "alg_bytes_per_launch": alg_bytes / max(1, launches // args.steps)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n,
                    "steps": e2e_steps},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
    for b in batches:
        b.close()
    return line if rank == 0 else None


def run_emulator_sweep(args):
    """Emulator sweep: train the emulator on batched-CPM runs, measure its error
    against replicate means of the CPM at held-out points, then time sweeps
    answered by emulator + CPM fallback against the CPM alone (batched, and
    one lattice at a time), both at <= 5% error on the same statistics."""
    import torch
    from paper_2312_09317_gb300 import build as B

    ws_, rank, local, dist = dist_init()
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    barrier(dist)
    line = emulator_sweep_measure(args, rank, ws_, dist)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def emulator_sweep_measure(args, rank=0, ws_=1, dist=None):
    """The emulator sweep measurement; returns its JSON line as a dict."""
    import torch
    from paper_2312_09317_gb300 import cpm
    from paper_2312_09317_gb300 import emulator as em

    cpm.load()
    burn, window, every = 200, 800, 10
    sim = dict(burn=burn, window=window, every=every)
    N = args.emu_runs
    seed0 = 1 + 7919 * rank
    # 1. training data on the batched CPM
    tm = {}
    t0 = time.perf_counter()
    X = cw.sweep_points(N, seed0)
    Y = em.simulate(X, np.arange(N) + 10 ** 6 * seed0, chunk=8192, timings=tm, **sim)
    data_s = time.perf_counter() - t0
    t_run_batched = data_s / N
    # 2. training
    emu = em.Emulator(init_seed=seed0, max_rows=65536)
    hist = emu.fit(X, Y, seed=seed0)
    # 3. error against the CPM at held-out points (truth = mean of R_truth replicates)
    Q, R = args.emu_eval, 64
    Xq = cw.sweep_points(Q, seed0 + 99)
    Yr = em.simulate(np.repeat(Xq, R, axis=0), np.arange(Q * R) + 5 * 10 ** 6 * seed0, chunk=8192, **sim)
    Yr = Yr.reshape(Q, R, -1)
    truth = np.nanmean(Yr, axis=1)
    den = np.nanmean(np.abs(truth), axis=0)
    loo = (np.nansum(Yr, axis=1, keepdims=True) - Yr) / (R - 1)
    e1 = np.nanmean(np.abs(Yr - loo), axis=(0, 1)) / den
    reps = np.ceil((e1 / 0.05) ** 2).astype(int)
    Yh, _, fb = emu.predict(Xq)
    emu_err = np.nanmean(np.abs(Yh - truth), axis=0) / den
    meets = emu_err <= 0.05
    r_star = int(max(1, reps[meets].max())) if meets.any() else int(reps.max())
    # 4. timed sweeps: blocks of fresh query points, answered end to end (host in, host out)
    block = args.emu_block
    lib_l0 = emu.net.launches()
    times, n_fb, pts = [], 0, 0
    tm_sweep = {}
    for k in range(args.warmup + args.steps):
        Xs = cw.sweep_points(block, seed0 + 1000 + k)
        torch.cuda.synchronize()
        if k == args.warmup:
            tm_sweep = {}
            lib_l0 = emu.net.launches()
        t0 = time.perf_counter()
        Ys, f = emu.sweep(Xs, seed=seed0 + 2000 + k, replicates=r_star, timings=tm_sweep, chunk=8192, **sim)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            n_fb += int(f.sum())
            pts += block
    sweep_s = sum(times)
    t_max = max_over_ranks(dist, sweep_s)
    value = sum_over_ranks(dist, float(pts)) / t_max
    launches = emu.net.launches() - lib_l0 + tm_sweep.get("launches", 0)
    # 5. inference throughput on 1M device-resident points (the emulator's dominant kernels)
    Xi = torch.from_numpy(emu._x(cw.sweep_points(1 << 20, seed0 + 3))).cuda()
    mean = torch.empty((Xi.shape[0], 16), dtype=torch.float32, device="cuda")
    sd = torch.empty_like(mean)
    fbi = torch.empty(Xi.shape[0], dtype=torch.uint8, device="cuda")
    lib = cpm.load()
    import ctypes
    for _ in range(2):
        lib.cpm_mlp_predict(emu.net.h, ctypes.c_void_p(Xi.data_ptr()), Xi.shape[0], ctypes.c_void_p(mean.data_ptr()),
                            ctypes.c_void_p(sd.data_ptr()), ctypes.c_void_p(fbi.data_ptr()))
    e0, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("emulator_inference")  # names the launches for profilers
    e0.record()
    for _ in range(5):
        lib.cpm_mlp_predict(emu.net.h, ctypes.c_void_p(Xi.data_ptr()), Xi.shape[0], ctypes.c_void_p(mean.data_ptr()),
                            ctypes.c_void_p(sd.data_ptr()), ctypes.c_void_p(fbi.data_ptr()))
    e1_.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    inf_s = e0.elapsed_time(e1_) / 1e3 / 5
    sizes = emu.sizes
    flop_pt = 2.0 * emu.net.n_members * sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
    tflops = flop_pt * Xi.shape[0] / inf_s / 1e12
    # 6. the CPM alone, one lattice at a time (a batch of one: same kernels, one lattice per launch)
    t0 = time.perf_counter()
    n_single = 4
    for i in range(n_single):
        em.simulate(Xq[i:i + 1], [7 * 10 ** 6 + i], chunk=1, **sim)
    torch.cuda.synchronize()
    t_run_single = (time.perf_counter() - t0) / n_single
    pk = peaks_bf16()
    line = None
    if rank == 0:
        line = {
            "metric": SWEEP_METRIC, "value": value, "unit": "points/s", "n_gpus": ws_, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16/fp32 (network), int32 (CPM)",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": EMULATOR[args.workload],
                       "training_runs": N, "query_block": block, "eval_points": Q, "truth_replicates": R,
                       "parallelism": "replicas" if ws_ > 1 else "1 GPU"},
            "sweep": {
                "statistics_at_5pct": [em.STATS[k] for k in range(16) if meets[k]],
                "replicates_for_5pct": int(r_star),
                "emulator_error": {em.STATS[k]: round(float(emu_err[k]), 4) for k in range(16)},
                "single_run_cpm_error": {em.STATS[k]: round(float(e1[k]), 4) for k in range(16)},
                "fallback_fraction": n_fb / max(1, pts),
                "fallback_fraction_eval": float(fb.mean()),
                "cpm_batched_points_per_s": 1.0 / (r_star * t_run_batched),
                "cpm_single_lattice_points_per_s": 1.0 / (r_star * t_run_single),
                "gain_vs_single_lattice": value / (1.0 / (r_star * t_run_single)),
                "gain_vs_batched": value / (1.0 / (r_star * t_run_batched)),
                "cpm_run_s": {"batched": t_run_batched, "single_lattice": t_run_single},
                "data_s": data_s, "data_cpm_attempts_per_s": tm["attempts"] / tm["cpm"],
                "train_s": hist["train_s"], "best_epoch": hist["best_epoch"],
                "val_rmse_std_units": [round(float(v), 4) for v in hist["val_rmse"]],
            },
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": pk[0], "unit": "TFLOP/s",
                         "frac": tflops / pk[0], "traffic": None, "peak_kind": "of %s" % pk[1],
                         "kernel": "gemm_tc_kernel (tcgen05, TMEM accumulators) over the 1M-point prediction: "
                                   "every forward layer, the gathers and the ensemble/fallback kernel",
                         "inference_points_per_s": Xi.shape[0] / inf_s},
            "cpu_baseline": None,
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": block * 7 * 4,
                    "d2h_bytes_per_step": block * 16 * 4,
                    "note": "every step is end to end: parameters in from the host, statistics out to the host"},
            "gpu_launches": int(launches),
        }
    emu.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + sorted(ENSEMBLES) + sorted(EMULATOR))
    ap.add_argument("--emu-runs", type=int, default=100000, help="training runs of the emulator")
    ap.add_argument("--emu-eval", type=int, default=256, help="held-out points with replicate truth")
    ap.add_argument("--emu-block", type=int, default=1 << 20, help="query points per sweep step (the full sweep: 1M)")
    ap.add_argument("--no-sweep", action="store_true", help="default workload: skip the embedded emulator sweep")
    ap.add_argument("--clocks-csv", default=None, help="where to keep the raw nvidia-smi clock samples of the timed "
                    "region (default: a temporary file)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--loop", default="graph", choices=["persistent", "graph"],
                    help="ensembles: one CUDA graph per MCS (faster on GB300), or one persistent cooperative "
                         "launch per step")
    ap.add_argument("--no-ensemble", action="store_true", help="default workload: skip the embedded ensemble line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ENSEMBLES:
        return run_gpu_batch(args)
    if args.workload in EMULATOR:
        return run_emulator_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
