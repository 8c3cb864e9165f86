#!/usr/bin/env python3
"""Time-to-spectrum benchmark of the TACAW hot path on one GB300.

One step = the whole path on the paper-scale workload (fcc 20x20x50 cells,
80 000 atoms, 512^2 grid, 101 slices of 2 A, 200 keV, 4096 snapshots at
5 fs): slice potentials and multislice for every snapshot, FP64 time mean,
temporal transform on the natural energy grid and |Phi|^2 / T^2.  The
metric is grid-point x slice x snapshot per second of that step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) the trajectory is sharded: each rank takes a
contiguous block of snapshots (potentials and multislice), the FP64 sums of
the exit waves are all-reduced, each rank accumulates its part of Phi(q, E)
on the natural energies with the split-BF16 tensor-core transform, and Phi is
reduce-scattered over q (NCCL); value = the whole trajectory's units / the
slowest rank's time ("scaling": "strong").  --shard runs that path at N = 1.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "multislice gridpt*slice*snapshot/s (time-to-spectrum)"
UNIT = "gridpt*slice*snapshot/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS_SUSTAINED = 1700.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="paper_scale")
    p.add_argument("--batch", default="auto",
                   help="snapshots per multislice call, or 'auto' (tuned per grid and GPU, cached in JSON)")
    p.add_argument("--precision", choices=["fft32", "bf16x3", "fp32"], default="fft32",
                   help="temporal transform: FP32 FFT over time (natural grid), split-BF16 tcgen05 GEMM, "
                        "or FP32 SIMT GEMM")
    p.add_argument("--snapshots", type=int, default=0, help="override T (testing only)")
    p.add_argument("--slices", type=int, default=0,
                   help="override the slice count, with as many cells along z as fill it (profiling only)")
    p.add_argument("--cpu-snapshots", type=int, default=1,
                   help="least snapshots per oracle sample (raised to the host's core count)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the further measurements (explicit grid, plain cuFFT slice step, batched "
                        "jobs, adjoint)")
    p.add_argument("--spectrum-only", default="",
                   help="T,NQ: time only the temporal transform on seeded synthetic exit waves [T][NQ] "
                        "(a kernel micro-benchmark; not the benchmark line)")
    p.add_argument("--ms-flags", choices=["auto", "0", "1", "2", "3", "4"], default="auto",
                   help="variants of the multislice passes (tacaw_multislice flags): tuned (auto), or 0-4 "
                        "(1: one warp per 512-point row, 2: one block per column block, 4: work queue)")
    p.add_argument("--no-c3", action="store_true",
                   help="skip the full batched configuration (64 uneven jobs, 512-4096 snapshots each)")
    p.add_argument("--c3-only", action="store_true",
                   help="time only the full batched configuration (one eager run, then a CUDA-graph replay)")
    p.add_argument("--shard", action="store_true",
                   help="run the sharded multi-GPU path even on one GPU (the default for N > 1)")
    p.add_argument("--seg", default="512,256",
                   help="snapshots per set and offset for the set-averaged spectrum timing ('' = skip)")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x, device):
    """The largest x over the ranks of the process group (the slowest rank's
    time); x itself without a group or with one rank."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, ms_step):
    """Whole-job throughput: the units of all ranks over the slowest rank's step time."""
    return units_per_rank * world / (ms_step * 1e-3)


def workload(args):
    import workloads as W
    w = W.WORKLOADS[args.workload]
    if args.snapshots:
        w = w.with_(n_t=args.snapshots)
    if args.slices:
        import dataclasses
        import math
        g = w.grid
        nz = max(1, math.ceil(args.slices * g.dz / w.a))
        w = w.with_(grid=dataclasses.replace(g, n_slices=args.slices), ncell=(w.ncell[0], w.ncell[1], nz),
                    n_lo=(w.n_lo[0], w.n_lo[1], -(nz // 2)), n_hi=(w.n_hi[0], w.n_hi[1], max(1, nz // 2)))
    return w


def workload_config(w, extra=None):
    g = w.grid
    cfg = {
        "workload": f"{w.name}: {w.lattice} {w.ncell[0]}x{w.ncell[1]}x{w.ncell[2]} cells a={w.a} A, "
                    f"{g.nx}x{g.ny} grid over {g.lx}x{g.ly} A, {g.n_slices} slices of {g.dz} A, "
                    f"{g.kev:g} keV plane wave, {w.n_t} snapshots at {w.dt_fs} fs, {w.n_modes} harmonic modes",
        "grid": [g.nx, g.ny], "slices": g.n_slices, "snapshots": w.n_t,
        "spectrum": "natural energy grid (n_omega = T)",
        "l2": "inputs larger than L2 (positions 3.9 GB, exit waves 8.6 GB per step)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ oracle leg
def oracle_sample(w, n_snap, processes):
    """Run the FP64 oracle (as it stands) on the first n_snap snapshots."""
    import numpy as np

    import oracle as O
    import workloads as W
    inp = W.build_inputs(w)
    pos = inp.positions(range(n_snap)).astype(np.float64)
    g = O.grid_from_spec(w.grid)
    t0 = time.perf_counter()
    psi = O.exit_waves(g, pos, inp.species, inp.amp_sigma.astype(np.float64), processes=processes)
    O.spectrum(psi.reshape(n_snap, -1), w.dt_fs)
    dt = time.perf_counter() - t0
    units = n_snap * w.grid.nx * w.grid.ny * w.grid.n_slices
    return units / dt, dt


def host_cores():
    """Cores this process may run on (all of the machine's, unless restricted)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample_size(args):
    """Snapshots per oracle sample: at least one per host core, so the pool
    keeps every core busy."""
    return max(args.cpu_snapshots, host_cores())


def cpu_baseline(w, n_snap):
    """The oracle on every host core (one process per core, n_snap >= cores
    snapshots), and on one core (one snapshot, one process)."""
    cores = host_cores()
    value, dt = oracle_sample(w, n_snap, cores)
    one, dt1 = oracle_sample(w, 1, 1)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "machine_cores": os.cpu_count(),
            "sample": f"first {n_snap} snapshots of {w.name} (FP64 potential + multislice per snapshot "
                      f"in a {cores}-process pool on all {cores} host cores, then the spectrum of those "
                      f"snapshots); {dt:.1f} s",
            "single_core": {"value": one, "unit": UNIT, "cores": 1,
                            "sample": f"first snapshot of {w.name}, one process; {dt1:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload(args)
    n_snap = oracle_sample_size(args)
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(w, n_snap, cores)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt = oracle_sample(w, n_snap, cores)
        vals.append(v)
        times.append(dt)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "machine_cores": os.cpu_count(),
                         "sample": f"each step: first {n_snap} snapshots of {w.name} in a {cores}-process pool "
                                   f"(one per host core)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU leg
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def load_peaks():
    """(HBM GB/s, sustained BF16 dense TFLOP/s, 'measured' | 'fallback')."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS_SUSTAINED, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("multislice.cu", "fft.cuh"):
        with open(os.path.join(ROOT, "paper_2401_15599_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def slice_step_bytes(g):
    """Algorithmic DRAM bytes per grid point and slice of the slice step.

    Row pass: v_s (4 B) plus the wave read and written (8 + 8 B) in the kept
    columns only (|k_x| <= K, the columns the band limit keeps); column pass:
    the wave read and written (8 + 8 B) in the column blocks that hold a kept
    column.  K uses the same FP64 expressions as the device set-up kernel.
    """
    d = g.lx / g.nx
    val = 1.0 / (g.nx * d)
    qmax = g.bandlimit * min(g.nx / (2.0 * g.lx), g.ny / (2.0 * g.ly))
    qmax2 = qmax * qmax
    K = -1
    for k in range(g.nx // 2 + 1):
        q = k * val
        if q * q <= qmax2:
            K = k
        else:
            break
    kept = [kx <= K or kx >= g.nx - K for kx in range(g.nx)]
    w = 8 if g.ny >= 1024 else (4 if g.ny >= 512 else 16)   # columns per column-pass block
    blocks = [any(kept[b:b + w]) for b in range(0, g.nx, w)]
    f_col = sum(kept) / g.nx
    f_blk = sum(blocks) / len(blocks)
    return 4.0 + 16.0 * f_col + 16.0 * f_blk


def profiled_traffic(units_per_launch):
    """DRAM bytes of one slice step (row + column pass) from the committed ncu
    summary, scaled to the launch size, or None if absent or stale."""
    path = os.path.join(ROOT, "profiles", "multislice_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d["dram_bytes_per_point_slice"] * units_per_launch


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2401_15599_gb300 import _lib
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    import workloads as W

    _lib.load()
    w = workload(args)
    g = w.grid

    cpu = None
    if rank == 0 and world >= 1 and args.gpus == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, oracle_sample_size(args))

    inp = W.build_inputs(w)
    pos_host = torch.from_numpy(inp.positions()).pin_memory()
    species = torch.from_numpy(inp.species).to(dev)
    pos = pos_host.to(dev, non_blocking=True)
    n_t, n_atoms = pos.shape[0], pos.shape[1]
    if args.precision == "fft32" and n_t not in _lib.TIME_FFT_SIZES:
        args.precision = "bf16x3"                 # no time-FFT plan for this T: the GEMM path
    tts = TimeToSpectrum(g, n_t, n_atoms, inp.amp_sigma, w.dt_fs, batch=args.batch, device=dev,
                         precision=args.precision)
    if args.ms_flags != "auto":
        tts.ms_flags = int(args.ms_flags)
    tuning = None
    if args.batch == "auto":
        from paper_2401_15599_gb300 import tuning as T
        tuning = T.load_cache().get(T.cache_key(g, torch.cuda.get_device_name(dev)))
    tts.prepare(None, None)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    events = {"potential": [], "multislice": [], "spectrum": []}
    from paper_2401_15599_gb300 import api

    def timed(name, record, fn):
        if not record:
            return fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        events[name].append((e0, e1))
        return out

    def step(record, precision=args.precision):
        tts.psi_sum.zero_()
        for t0 in range(0, n_t, tts.batch):
            t1 = min(n_t, t0 + tts.batch)
            v = tts.V[: t1 - t0]
            timed("potential", record, lambda: api.potential(
                g, pos[t0:t1], species, inp.amp_sigma, out=v, workspace=tts._ws.get("pot")))
            timed("multislice", record, lambda: api.multislice(
                g, v, out=tts.psi[t0:t1], psi_sum=tts.psi_sum, workspace=tts._ws.get("ms"),
                ms_flags=tts.ms_flags))
        tts.precision = precision
        return timed("spectrum", record, tts.spectrum)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        step(True)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = start.elapsed_time(end)
    ms_step = max_over_ranks(ms_total / args.steps, dev)
    units_step = g.nx * g.ny * g.n_slices * n_t
    value = aggregate_rate(units_step, world, ms_step)

    # end to end through one library call with host buffers (tacaw_time_to_spectrum_host): pinned
    # host positions in (copied batch by batch on the library's copy stream, overlapping the work
    # on the previous batch), host I(q, E) and I_el out; one untimed warm-up call first
    e2e = None
    if not args.no_e2e:
        i_host = torch.empty(tts.I.shape, dtype=torch.float32).pin_memory()
        el_host = torch.empty(tts.I_el.shape, dtype=torch.float64).pin_memory()
        host_ws = None

        def host_call():
            return api.time_to_spectrum_host(g, pos_host, species, inp.amp_sigma, w.dt_fs, tts.batch,
                                             ms_flags=tts.ms_flags, precision=args.precision, out=i_host,
                                             out_el=el_host, workspace=host_ws)

        host_ws = api.time_to_spectrum_host_workspace(g, n_t, n_atoms, tts.batch, args.precision, device=dev)
        host_call()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks_e2e = ClockSampler(local)
        clocks_e2e.start()
        s2 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        s2.record(stream)
        for _ in range(args.steps):
            host_call()
        e2.record(stream)
        torch.cuda.synchronize()
        clk_e2e = clocks_e2e.stop()
        e2e_ms = max_over_ranks(s2.elapsed_time(e2) / args.steps, dev)
        e2e = {"value": aggregate_rate(units_step, world, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(pos_host.numel() * 4),
               "d2h_bytes_per_step": int(i_host.numel() * 4 + el_host.numel() * 8),
               "ms_per_step": e2e_ms, "call": "tacaw_time_to_spectrum_host (one C-ABI call, host buffers)",
               "clocks": clk_e2e}
        del host_ws
        torch.cuda.empty_cache()

    def stage_ms(name):
        return [a.elapsed_time(b) for a, b in events[name]]

    # dominant kernel: the multislice slice step (row + column pass), timed per call
    ms_call = stage_ms("multislice")
    units_call = g.nx * g.ny * g.n_slices * tts.batch
    avg_call_ms = statistics.mean(ms_call)
    bytes_pt = slice_step_bytes(g)
    achieved = bytes_pt * units_call / (avg_call_ms * 1e-3) / 1e9
    peak, peak_tf, peak_kind = load_peaks()
    traffic = profiled_traffic(units_call)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "multislice slice step (row pass + column pass kernels, all slices of one "
                          f"{tts.batch}-snapshot batch per call)",
                "bytes_per_unit": round(bytes_pt, 3), "peak_kind": f"{peak_kind} hbm_gbs"}
    spec_ms = statistics.mean(stage_ms("spectrum"))
    nq = g.nx * g.ny
    stages = {k: sum(stage_ms(k)) / args.steps for k in events}

    # the other forms of the temporal transform on the same exit waves, for comparison
    spec_by_prec = {args.precision: spec_ms}
    for prec in ("fft32", "bf16x3", "fp32"):
        if prec == args.precision or (prec == "fft32" and n_t not in _lib.TIME_FFT_SIZES):
            continue
        events["spectrum"].clear()
        tts.precision = prec
        for _ in range(2):
            timed("spectrum", False, tts.spectrum)
        for _ in range(args.steps):
            timed("spectrum", True, tts.spectrum)
        torch.cuda.synchronize()
        spec_by_prec[prec] = statistics.mean(stage_ms("spectrum"))
    tts.precision = args.precision
    fp32_ms = spec_by_prec.get("fp32")

    def spectrum_roofline(prec):
        ms = spec_by_prec.get(prec)
        if ms is None:
            return None
        if prec == "fft32":
            # one read of psi (8 B) and one write of I (4 B) per q and snapshot
            gbs = 12.0 * nq * n_t / (ms * 1e-3) / 1e9
            return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                    "traffic": None, "kernel": "tacaw_spectrum FFT32 (time FFT + |Phi|^2, one kernel)",
                    "bytes_per_unit": "8 B read + 4 B written per q x snapshot",
                    "peak_kind": f"{peak_kind} hbm_gbs"}
        if prec == "bf16x3":
            tf = 3 * 8.0 * nq * n_t * n_t / (ms * 1e-3) / 1e12   # three BF16 products per complex flop
            return {"bound": "tensor", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": tf / peak_tf,
                    "traffic": None,
                    "kernel": "tacaw_spectrum BF16X3 (split, centre, tcgen05 GEMM + |Phi|^2 epilogue)",
                    "flop_per_unit": "3 x 8 real flop per q x snapshot x energy",
                    "peak_kind": f"{peak_kind} bf16_tflops_sustained"}
        return None

    roofline_spectrum = spectrum_roofline(args.precision)
    roofline_spectrum_gemm = spectrum_roofline("bf16x3") if args.precision != "bf16x3" else None

    # spectra averaged over sets of consecutive snapshots, on the same exit waves
    seg = None
    if args.seg:
        from paper_2401_15599_gb300 import api as A
        seg_len, hop = (int(x) for x in args.seg.split(","))
        if seg_len <= n_t:
            psi2 = tts.psi.reshape(n_t, -1)
            n_sets = (n_t - seg_len) // hop + 1
            for _ in range(2):
                A.spectrum_segments(psi2, w.dt_fs, seg_len, hop, precision=args.precision)
            torch.cuda.synchronize()
            times = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                A.spectrum_segments(psi2, w.dt_fs, seg_len, hop, precision=args.precision)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            seg_ms = statistics.mean(times)
            flop = 8.0 * g.nx * g.ny * seg_len * seg_len * n_sets * (3 if args.precision == "bf16x3" else 1)
            seg = {"seg_len": seg_len, "hop": hop, "n_sets": n_sets, "ms": seg_ms,
                   "precision": args.precision, "tflops": flop / (seg_ms * 1e-3) / 1e12}

    further = None
    if rank == 0 and not args.no_extras:
        further = {
            "explicit_grid_1024_bins": explicit_grid_comparison(tts, w, args.steps, stream),
            "plain_cufft_multislice_call": plain_cufft_slice_step(tts, g, args.steps, stream),
            "batched_jobs": batched_jobs_sample(args.steps, stream),
            "batched_queue_vs_launches": batched_queue_vs_launches(args.steps, stream),
            "adjoint": adjoint_sample(args.steps, stream),
        }
        torch.cuda.synchronize()
        if not args.no_c3:
            # the full batched configuration needs most of the device: free this run's buffers first
            tts.psi = tts.V = tts.I = tts.I_el = None
            tts._ws.clear()
            tts._pos_stage = None
            del pos
            torch.cuda.empty_cache()
            try:
                further["batched_jobs_full"] = full_batched_jobs(stream)
            except torch.OutOfMemoryError as exc:         # report, do not lose the benchmark line
                further["batched_jobs_full"] = {"error": f"out of device memory: {exc}"[:300]}
                torch.cuda.empty_cache()
            torch.cuda.synchronize()

    n_batches = (n_t + tts.batch - 1) // tts.batch
    # twiddles, FFT | split A, split B, GEMM | centre, table, GEMM
    spec_launches = {"fft32": 2, "bf16x3": 3, "fp32": 3}[args.precision]
    launches = n_batches * (2 + 1 + 2 * g.n_slices + 1) + spec_launches
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+bf16x3" if args.precision == "bf16x3" else "f32",
            "data": "synthetic",
            "tuning": tuning,
            "config": workload_config(w, {"batch": tts.batch, "ms_flags": tts.ms_flags,
                                          "spectrum_precision": args.precision,
                                          "parallelism": "replicas" if world > 1 else "single GPU"}),
            "time_to_spectrum_ms": ms_step,
            "stage_ms": stages,
            "plain_fp32_spectrum_ms": fp32_ms,
            "spectrum_ms_by_precision": spec_by_prec,
            "time_to_spectrum_plain_fp32_ms": (ms_step - stages["spectrum"] + fp32_ms) if fp32_ms else None,
            "roofline": roofline, "roofline_spectrum": roofline_spectrum,
            "roofline_spectrum_bf16x3_gemm": roofline_spectrum_gemm,
            "set_averaged_spectrum": seg,
            "further": further,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ further measurements
def _events_ms(fn, reps, stream):
    """Mean device time of fn() over reps calls (CUDA events on the stream)."""
    import torch
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.mean(times)


def explicit_grid_comparison(tts, w, reps, stream):
    """The explicit energy grid of 1024 bins over [-200, 200) meV on the benchmark's
    exit waves: two- and three-term split-BF16 tcgen05 GEMMs against the FP32 SIMT
    GEMM, times and relative L2 differences per 50 meV band (the FP64 comparison
    is a GPU test)."""
    import torch
    from paper_2401_15599_gb300 import api
    n_t = tts.n_t
    psi = tts.psi.reshape(n_t, -1)
    omega = torch.arange(1024, dtype=torch.float64, device=psi.device) * (400.0 / 1024) - 200.0
    out = {}
    res = {}
    for prec in ("bf16x3", "bf16x6", "fp32"):
        buf = torch.empty((psi.shape[1], 1024), dtype=torch.float32, device=psi.device)
        el = torch.empty(psi.shape[1], dtype=torch.float64, device=psi.device)
        call = lambda: api.spectrum(psi, w.dt_fs, omega_meV=omega, psi_sum=tts.psi_sum.reshape(-1),
                                    precision=prec, out=buf, i_el=el)
        call()
        out[prec + "_ms"] = _events_ms(call, reps, stream)
        res[prec] = buf
    bands = []
    e = omega.cpu().numpy()
    bands6 = []
    for lo in range(-200, 200, 50):
        sel = torch.from_numpy(((e >= lo) & (e < lo + 50))).to(psi.device)
        a, a6, b = res["bf16x3"][:, sel].double(), res["bf16x6"][:, sel].double(), res["fp32"][:, sel].double()
        bands.append(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)))
        bands6.append(float(torch.linalg.norm(a6 - b) / torch.linalg.norm(b)))
    out["band_rel_l2_bf16x3_vs_fp32"] = bands
    out["band_rel_l2_bf16x6_vs_fp32"] = bands6
    out["bands_meV"] = [[lo, lo + 50] for lo in range(-200, 200, 50)]
    return out


def plain_cufft_slice_step(tts, g, reps, stream):
    """The unfused form of one multislice call for timing: transmission,
    cuFFT 2-D transforms (torch.fft) and the band-limited propagator as separate
    elementwise launches, on the benchmark's last batch of potentials."""
    import numpy as np
    import torch
    from paper_2401_15599_gb300 import _lib as L
    import ctypes
    lib = L.load()
    lam, sig = ctypes.c_double(0), ctypes.c_double(0)
    L.check("tacaw_beam_constants", lib.tacaw_beam_constants(float(g.kev), ctypes.byref(lam), ctypes.byref(sig)))
    qx = np.fft.fftfreq(g.nx, d=g.lx / g.nx)
    qy = np.fft.fftfreq(g.ny, d=g.ly / g.ny)
    q2 = qx[None, :] ** 2 + qy[:, None] ** 2
    qmax = g.bandlimit * min(g.nx / (2 * g.lx), g.ny / (2 * g.ly))
    prop = np.exp(-1j * np.pi * lam.value * g.dz * q2) * (q2 <= qmax * qmax)
    prop = torch.from_numpy(prop.astype(np.complex64)).to(tts.V.device)
    V = tts.V
    sigma = float(sig.value)

    def run():
        psi = torch.ones((V.shape[0], g.ny, g.nx), dtype=torch.complex64, device=V.device)
        for s in range(g.n_slices):
            psi = psi * torch.polar(torch.ones_like(V[:, s]), sigma * V[:, s])
            psi = torch.fft.fft2(psi, norm="forward") * prop
            if s + 1 < g.n_slices:
                psi = torch.fft.ifft2(psi, norm="forward")
        return psi

    ref = run()
    ours = torch.empty_like(ref)
    from paper_2401_15599_gb300 import api
    api.multislice(g, V, out=ours, ms_flags=tts.ms_flags)
    diff = float(torch.linalg.norm(ours - ref) / torch.linalg.norm(ref))
    ms = _events_ms(run, reps, stream)
    ours_ms = _events_ms(lambda: api.multislice(g, V, out=ours, ms_flags=tts.ms_flags), reps, stream)
    return {"snapshots": int(V.shape[0]), "plain_cufft_ms": ms, "ours_ms": ours_ms,
            "speedup": ms / ours_ms, "rel_l2_difference": diff}


def batched_queue_vs_launches(reps, stream, n_jobs=16, snapshots=24):
    """The multislice of uneven jobs (the first `n_jobs` of the 64 seeded batched
    jobs: grids 128-768, 10-150 slices; `snapshots` snapshots each, random slice
    potentials) through tacaw_multislice_batch (two launches per slice and grid
    size) and through tacaw_multislice_queue (one persistent launch per grid
    size over the device work queue, items of 32 rows or columns as the batched
    driver uses), on the same buffers; the exit waves must agree bit for bit."""
    import torch
    import workloads as W
    from paper_2401_15599_gb300 import api
    gen = torch.Generator(device="cuda").manual_seed(0)
    jobs, units, sizes = [], 0, []
    for wj in W.batching_jobs(n_jobs=n_jobs):
        g = wj.grid
        V = torch.rand((snapshots, g.n_slices, g.ny, g.nx), generator=gen, device="cuda") * 30.0
        jobs.append({"grid": g, "V": V, "out": torch.empty((snapshots, g.ny, g.nx), dtype=torch.complex64,
                                                           device="cuda")})
        units += g.nx * g.ny * g.n_slices * snapshots
        sizes.append(g.nx)
    api.multislice_batch(jobs)                           # warm-up (workspace, kernel attributes)
    launches_ms = _events_ms(lambda: api.multislice_batch(jobs), reps, stream)
    ref = [j["out"].clone() for j in jobs]
    api.multislice_batch(jobs, queue=True, span=32)
    queue_ms = _events_ms(lambda: api.multislice_batch(jobs, queue=True, span=32), reps, stream)
    api.status()
    same = all(torch.equal(j["out"], r) for j, r in zip(jobs, ref))
    del jobs, ref
    torch.cuda.empty_cache()
    return {"jobs": n_jobs, "snapshots_per_job": snapshots, "grids": sorted(set(sizes)), "units": units,
            "per_slice_launches_ms": launches_ms, "queue_ms": queue_ms,
            "value_per_slice_launches": units / (launches_ms * 1e-3), "value_queue": units / (queue_ms * 1e-3),
            "unit": UNIT, "bit_identical": same}


def batched_jobs_sample(reps, stream, n_jobs=64, snapshots=64):
    """The 64 uneven seeded jobs (grids 128-768, 10-150 slices, 1-3 species), each
    cut to its first `snapshots` snapshots, through the batched path: eager run and
    CUDA-graph replay, in grid point * slice * snapshot per second."""
    import torch
    import workloads as W
    from paper_2401_15599_gb300.batch import BatchTimeToSpectrum, Job
    jobs, units = [], 0
    for wj in W.batching_jobs(n_jobs=n_jobs):
        inp = W.build_inputs(wj)
        n = min(snapshots, wj.n_t)
        pos = torch.from_numpy(inp.positions(snapshots=list(range(n)))).cuda()
        jobs.append(Job(wj.grid, pos, torch.from_numpy(inp.species).cuda(), inp.amp_sigma, wj.dt_fs))
        units += wj.grid.nx * wj.grid.ny * wj.grid.n_slices * n
    run = BatchTimeToSpectrum(jobs, window=8, precision="fft32")
    run.capture()
    eager_ms = _events_ms(run.run, reps, stream)
    graph_ms = _events_ms(run.replay, reps, stream)
    return {"jobs": n_jobs, "snapshots_per_job": snapshots, "window": 8, "units": units,
            "eager_ms": eager_ms, "graph_ms": graph_ms,
            "value_graph": units / (graph_ms * 1e-3), "unit": UNIT}


def full_batched_jobs(stream, graph=True, max_jobs=64, max_snapshots=None, v_budget=120e9, max_window=512,
                      queue="auto"):
    """The batched configuration as stated: the 64 seeded uneven jobs (seeds
    1000-1063; grids 128-768, 10-150 slices, 512-4096 snapshots, 1-3 species)
    through the time-chunked batched driver, one group per grid size (so one
    launch covers many snapshots of like jobs): per window of snapshots the
    positions are synthesised on the device (the inputs of all jobs together
    would take 94 GB), then slice potentials, one batched multislice call for the
    group's jobs, and each job's Phi(q, E) accumulated on 1024 bins over
    [-200, 200) meV in split BF16 (three terms); each job's I(q, E) is finished
    at the end.  A group's window holds `v_budget` bytes of potentials.  Each
    group runs once eagerly (untimed), is captured in a CUDA graph and replayed
    (timed, CUDA events); the groups run one after another and their times add
    up.  The synthesis of the positions is inside the timed region."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2401_15599_gb300.batch import BatchTimeToSpectrum, Job
    omega = np.arange(1024) * (400.0 / 1024) - 200.0
    specs = W.batching_jobs(n_jobs=max_jobs)
    if max_snapshots:
        specs = [wj.with_(n_t=min(wj.n_t, max_snapshots)) for wj in specs]
    sizes = sorted({wj.grid.nx for wj in specs})
    groups, total_ms, units_all = [], 0.0, 0
    for n in sizes:
        members = [wj for wj in specs if wj.grid.nx == n]
        per_snapshot = sum(4.0 * wj.grid.n_slices * wj.grid.nx * wj.grid.ny for wj in members)
        window = int(max(8, min(max_window, v_budget // per_snapshot)))
        jobs, units = [], 0
        for wj in members:
            inp = W.build_inputs(wj)
            jobs.append(Job(wj.grid, None, torch.from_numpy(inp.species).cuda(), inp.amp_sigma, wj.dt_fs,
                            omega_meV=omega, n_t=wj.n_t, positions=inp.synth("cuda")))
            units += wj.grid.nx * wj.grid.ny * wj.grid.n_slices * wj.n_t
        run = BatchTimeToSpectrum(jobs, window=window, precision="bf16x6", chunked=True, queue=queue)
        if graph:
            run.capture()                                    # one eager run, then the recording
            ms = _events_ms(run.replay, 1, stream)
        else:
            run.prepare()
            run.run()
            torch.cuda.synchronize()
            ms = _events_ms(run.run, 1, stream)
        groups.append({"grid": n, "jobs": len(jobs), "window": window, "units": units, "ms": ms,
                       "value": units / (ms * 1e-3)})
        total_ms += ms
        units_all += units
        del run, jobs
        torch.cuda.empty_cache()
    return {"jobs": len(specs), "snapshots": int(sum(wj.n_t for wj in specs)), "units": units_all,
            "ms": total_ms, "value": units_all / (total_ms * 1e-3), "unit": UNIT, "graph": graph,
            "groups": groups, "spectrum": "1024 bins over [-200, 200) meV, BF16X6, time-chunked"}


def adjoint_sample(reps, stream, snapshots=64):
    """Forward and backward of the spectrum-mismatch loss on the differentiation
    workload (256^2, 50 slices, fcc 10x10x25), first `snapshots` snapshots:
    gradients with respect to the per-species (amp, sigma)."""
    import torch
    import workloads as W
    from paper_2401_15599_gb300.autograd import spectrum_from_atoms
    w = W.WORKLOADS["differentiation"]
    inp = W.build_inputs(w)
    pos = torch.from_numpy(inp.positions(snapshots=list(range(snapshots)))).cuda()
    species = torch.from_numpy(inp.species).cuda()
    amp = torch.tensor(inp.amp_sigma, dtype=torch.float64, device="cuda")
    target = spectrum_from_atoms(amp * torch.tensor([1.05, 1.0], device="cuda", dtype=torch.float64), pos,
                                 species, w.grid, w.dt_fs).detach()

    def fwd():
        a = amp.clone().requires_grad_(True)
        inten = spectrum_from_atoms(a, pos, species, w.grid, w.dt_fs)
        return a, ((inten - target) ** 2).sum() / (target ** 2).sum()

    def fwd_bwd():
        a, loss = fwd()
        loss.backward()

    fwd_bwd()
    f_ms = _events_ms(lambda: fwd(), reps, stream)
    fb_ms = _events_ms(fwd_bwd, reps, stream)
    g = w.grid
    units = g.nx * g.ny * g.n_slices * snapshots
    return {"workload": "differentiation, first %d snapshots" % snapshots, "forward_ms": f_ms,
            "forward_backward_ms": fb_ms, "backward_over_forward": (fb_ms - f_ms) / f_ms,
            "value_forward_backward": units / (fb_ms * 1e-3), "unit": UNIT}


def run_spectrum_only(args):
    """Temporal transform alone on seeded synthetic exit waves, through the
    public spectrum call: prints one JSON line with the mean time and the
    achieved bandwidth of one read of psi and one write of I."""
    import torch
    from paper_2401_15599_gb300 import api
    n_t, nq = (int(x) for x in args.spectrum_only.split(","))
    gen = torch.Generator(device="cuda").manual_seed(1)
    psi = 1 + 0.05 * torch.randn(n_t, nq, dtype=torch.complex64, device="cuda", generator=gen)
    out, el = api.spectrum(psi, 5.0, precision=args.precision)
    for _ in range(max(args.warmup - 1, 0)):
        api.spectrum(psi, 5.0, precision=args.precision, out=out, i_el=el)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        api.spectrum(psi, 5.0, precision=args.precision, out=out, i_el=el)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"spectrum_only": {"T": n_t, "nq": nq, "precision": args.precision, "ms": ms,
                                        "gbs_psi_read_I_write": 12.0 * n_t * nq / (ms * 1e-3) / 1e9}}))
    return 0


def natural_energies_meV(n_t, dt_fs):
    """E_k = h (k - T/2) / (T dt), k = 0 .. T-1 (the natural grid, ascending)."""
    import numpy as np
    h = 6.62607015e-34 / 1.602176634e-19 * 1e3 * 1e15          # meV fs
    return (np.arange(n_t) - n_t // 2) * (h / (n_t * dt_fs))


def run_sharded(args):
    """One trajectory over N GPUs (snapshot shards, all-reduce of the FP64 sums,
    reduce-scatter of Phi over q); strong scaling."""
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2401_15599_gb300 import _lib, api
    from paper_2401_15599_gb300.sharded import ShardedTimeToSpectrum, shard_bounds
    from paper_2401_15599_gb300.tuning import best_multislice_config
    import workloads as W

    _lib.load()
    w = workload(args)
    g = w.grid
    inp = W.build_inputs(w)
    n_t = w.n_t
    t_lo, t_hi = shard_bounds(n_t, world, rank)
    batch, ms_flags = best_multislice_config(g, device=dev) if args.batch == "auto" else (int(args.batch), 0)
    if args.ms_flags != "auto":
        ms_flags = int(args.ms_flags)
    batch = max(1, min(batch, t_hi - t_lo))
    omega = natural_energies_meV(n_t, w.dt_fs)
    sh = ShardedTimeToSpectrum(g, n_t, inp.crystal.n_atoms, inp.amp_sigma, w.dt_fs, omega, batch=batch,
                               precision="bf16x6", device=dev, ms_flags=ms_flags)
    pos_host = torch.from_numpy(inp.positions(list(range(t_lo, t_hi)))).pin_memory()
    pos = pos_host.to(dev, non_blocking=True)
    species = torch.from_numpy(inp.species).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        sh.run(pos, species)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        inten, iel = sh.run(pos, species)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    units = g.nx * g.ny * g.n_slices * n_t
    value = units / (ms_step * 1e-3)
    e2e = None
    if not args.no_e2e:
        out_host = torch.empty(tuple(inten.shape), dtype=torch.float32).pin_memory()
        el_host = torch.empty(tuple(iel.shape), dtype=torch.float64).pin_memory()
        s2 = torch.cuda.Event(enable_timing=True)
        t2 = torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        s2.record(stream)
        for _ in range(args.steps):
            pos.copy_(pos_host, non_blocking=True)
            a, b = sh.run(pos, species)
            out_host.copy_(a, non_blocking=True)
            el_host.copy_(b, non_blocking=True)
        t2.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(s2.elapsed_time(t2) / args.steps, dev)
        e2e = {"value": units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(pos_host.numel() * 4),
               "d2h_bytes_per_step": int(out_host.numel() * 4 + el_host.numel() * 8), "ms_per_step": e2e_ms,
               "call": "ShardedTimeToSpectrum.run with host copies of this rank's positions and I rows"}
    # dominant kernel: one multislice call of `batch` snapshots of this rank
    V = torch.empty((batch, g.n_slices, g.ny, g.nx), dtype=torch.float32, device=dev)
    api.potential(g, pos[:batch], species, inp.amp_sigma, out=V)
    out = torch.empty((batch, g.ny, g.nx), dtype=torch.complex64, device=dev)
    api.multislice(g, V, out=out, ms_flags=ms_flags)
    call_ms = _events_ms(lambda: api.multislice(g, V, out=out, ms_flags=ms_flags), 3, stream)
    peak, _, peak_kind = load_peaks()
    bytes_pt = slice_step_bytes(g)
    achieved = bytes_pt * g.nx * g.ny * g.n_slices * batch / (call_ms * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32+bf16x6", "data": "synthetic",
            "config": workload_config(w, {"batch": batch, "ms_flags": ms_flags, "spectrum_precision": "bf16x6",
                                          "spectrum": "natural energies as an explicit grid (n_omega = T)",
                                          "parallelism": f"{world} snapshot shards; all-reduce of the FP64 sums; "
                                                         f"reduce-scatter of Phi over q"}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": f"multislice slice step, one {batch}-snapshot call on rank 0",
                         "bytes_per_unit": round(bytes_pt, 3), "peak_kind": f"{peak_kind} hbm_gbs"},
            "cpu_baseline": None, "e2e": e2e,
            # per rank and step: binning + potential and set-up + 2 passes per slice + sum per batch;
            # mean; split A, split B, tensor-core transform; constant transform + finish
            "gpu_launches": args.steps * world * (-(-(t_hi - t_lo) // batch) * (4 + 2 * g.n_slices) + 1 + 3 + 2),
            "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.spectrum_only:
        return run_spectrum_only(args)
    if args.c3_only:
        import torch
        torch.cuda.set_device(0)
        from paper_2401_15599_gb300 import _lib
        _lib.load()
        print(json.dumps({"batched_jobs_full": full_batched_jobs(torch.cuda.current_stream())}))
        return 0
    if args.shard or dist_env()[1] > 1:
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
