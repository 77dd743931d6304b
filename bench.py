#!/usr/bin/env python
"""Throughput of the ICM time step (arXiv:1212.6427, Sec. III.C) on GB300.

One "step" is one pass of the whole hot path: midpoint predictor, fused
noise/viscous/advection right-hand side, spreading, three FFT Helmholtz/projection
round trips (two of them for the inertial correction), gathers and the blob
updates, for one synthetic simulation resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large|bulk|plain]
                  [--precision 32|64] [--impl ours|reference]

Default workload "large": 256^3 MAC grid, 20000 blobs (min spacing 2h), Peskin
4-point kernel, excess masses U[-0.5, 2] rho h^3, F = (1e-4, 0, 0), kT = 1e-3,
dt = 0.01, FP32 fields with FP64 blob state and momentum bookkeeping.  Every face
field (201 MB) is larger than the 126 MB L2, so no L2 flush is needed between steps.

Under torchrun (N > 1) every rank advances an independent replica (seed offset by
rank): the method does not shard within one simulation, so scaling is weak and no
collective is on the data path; the max over ranks of the timed region is used.

--impl reference times the FP64 numpy oracle (the CPU statement of the method) on
the host cores on the same workload and prints the same JSON line.
"""
import argparse
import faulthandler
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import icm_workloads as wl  # noqa: E402

METRIC = "cell-updates/s"
faulthandler.enable()


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def max_over_ranks(x, dist):
    """The largest x over the ranks of the process group (x itself without one): the
    timed region of a multi-rank run is its slowest rank's."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="large", choices=["large", "bulk", "plain", "batch", "served"])
    ap.add_argument("--jobs", type=int, default=120, help="served workload: number of Poisson-arriving jobs")
    ap.add_argument("--precision", type=int, default=None, choices=[32, 64])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, cuFFT and CPU comparison legs")
    ap.add_argument("--no-autotune", action="store_true", help="time the default plan instead of the tuned one")
    ap.add_argument("--grouped", type=int, default=None, choices=[0, 1, 2, 3],
                    help="batch workload: this batch mode (icm_batch_set_grouped) instead of the tuned one")
    ap.add_argument("--cpu-budget", type=float, default=150.0, help="seconds of oracle time for the CPU legs")
    return ap.parse_args()


def workload_config(w, precision, world):
    nx, ny, nz = w["grid"]
    return {"workload": "icm-%s-%dx%dx%d-%dblobs-k%d-fp%d" % (w["name"], nx, ny, nz, len(w["q"]), w["kernel"], precision),
            "grid": [nx, ny, nz], "blobs": int(len(w["q"])), "kernel": w["kernel"], "kT": w["kT"], "dt": w["dt"],
            "excess_mass": "U[-0.5,2] rho h^3" if w["me_range"] else "0",
            "force": [float(x) for x in np.asarray(w["force"]).reshape(-1, 3)[0]] if len(w["q"]) else [0.0, 0.0, 0.0], "replicas": world, "parallelism": "replicas only (independent per rank)",
            "l2": "inputs larger than L2 (one face field %.0f MB > 126 MB)" % (3 * nx * ny * nz * precision / 8 / 1e6)
            if 3 * nx * ny * nz * precision / 8 > 126e6 else "inputs smaller than L2 (no flush)"}


def load_workload(name, rank=0):
    w = wl.workload(name)
    if rank:
        w = wl.workload(name, seed=w["seed"] + rank, place_seed=w["place_seed"] + rank)
    w["name"] = name
    return w


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1212_6427_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it is current."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            t = json.load(fh)
        if t.get("source_sha") != source_hash():
            return None
        return t["kernels"].get(kernel)
    except Exception:
        return None


def kernel_of(stage):
    return stage.split(".", 1)[1] if "." in stage else stage


def fft_flops_per_step(grid, inertial):
    """Floating-point operations of the FFT passes of one step by the 5 n log2 n model of
    a complex n-point transform: per solve, forward and inverse lines along x (two real
    rows packed as one complex line), y and z (Nx/2+1 wave numbers) of 3 components;
    three solves when any blob has excess mass, else one."""
    nx, ny, nz = grid
    kx = nx // 2 + 1

    def line(n):
        return 5.0 * n * np.log2(n)
    per_solve = 2 * 3 * ((ny * nz / 2) * line(nx) + kx * nz * line(ny) + kx * ny * line(nz))
    return per_solve * (3 if inertial else 1)


def oracle_step_rate(w, budget_s, max_steps):
    """Time the FP64 numpy oracle on the workload: (seconds per step, steps timed)."""
    from oracle import icm as oracle
    prm = oracle.Params(w["grid"], h=w["h"], rho=w["rho"], eta=w["eta"], kT=w["kT"], dt=w["dt"],
                        kernel=w["kernel"], seed=w["seed"])
    st = oracle.State(np.zeros((3,) + prm.shape), w["q"], w["u"], w["me"], w["force"])
    times = []
    t_all = time.perf_counter()
    while len(times) < max(1, max_steps):
        t0 = time.perf_counter()
        st = oracle.icm_step(st, prm)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget_s:
            break
    return float(np.mean(times)), len(times)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload in ("batch", "served"):
        # the oracle on the first replica / job of the set: one bounded sample of the same workload
        w = (wl.batch_replicas(1) if args.workload == "batch" else wl.served_jobs(1))[0]
        w["name"] = args.workload
    else:
        w = load_workload(args.workload)
    prec = args.precision or w["precision"]
    ncell = int(np.prod(w["grid"]))
    sec, n = oracle_step_rate(w, args.cpu_budget, args.steps)
    val = ncell / sec
    cfg = workload_config(w, prec, 1)
    line = {"metric": METRIC, "value": val, "unit": "cell-updates/s", "n_gpus": world, "steps": n,
            "warmup": 0, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg, "impl": "reference",
            "blob_steps_per_s": len(w["q"]) / sec,
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "%d full oracle step(s) of the %s workload (numpy FP64, single thread)"
                                       % (n, args.workload)},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, dist):
    import torch
    import paper_1212_6427_gb300 as icm
    from paper_1212_6427_gb300 import build
    if rank == 0:
        build.build_library()
    if dist is not None:
        dist.barrier()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    log("[bench] rank %d: generating workload %s" % (rank, args.workload))
    w = load_workload(args.workload, rank)
    prec = args.precision or w["precision"]
    grid = w["grid"]
    ncell = int(np.prod(grid))
    nb = len(w["q"])
    sim = icm.Simulation(grid, w["h"], w["rho"], w["eta"], w["kT"], w["dt"], w["kernel"], w["seed"], prec)
    sim.add_blobs(w["q"], w["u"], w["me"])
    sim.set_forces(w["force"])
    stream = sim.stream

    def barrier():
        if dist is not None:
            dist.barrier()

    log("[bench] simulation created (%.0f MB on device); warming up" % (icm.icm_device_bytes(sim.handle) / 1e6))
    # warm-up (graph capture happens on the first step), then the autotuner picks the
    # plan on this state (which it restores) and the plan's graph is warmed up
    sim.step(max(args.warmup, 3))
    sim.sync()
    plan = None
    if not args.no_autotune:
        plan, plan_ms = icm.icm_autotune(sim.handle, 3)
        log("[bench] autotuned plan %s (%.4f ms/step)" % (plan, plan_ms))
        sim.step(max(args.warmup, 3))
    sim.sync()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    sim.sync()   # raises on a CFL / non-finite error raised during the timed steps
    ms = max_over_ranks(ms, dist)
    ms_step = ms / args.steps
    value = ncell * args.steps * world / (ms / 1e3)

    log("[bench] timed region: %.3f ms/step" % (ms / args.steps))
    # end to end through the public API: host forces in (pinned), blob state out (pinned)
    f_host = torch.empty((nb, 3), dtype=torch.float64, pin_memory=True).numpy()
    f_host[:] = w["force"]
    barrier()
    torch.cuda.synchronize()
    # (1) queued reads: the read of step n is queued behind it and collected after step
    # n+1 is queued, so the host's copy-out overlaps the GPU's next step
    t0 = time.perf_counter()
    sim.set_forces(f_host)
    sim.step(1)
    sim.read_begin()
    for _ in range(args.steps - 1):
        sim.set_forces(f_host)
        sim.step(1)
        sim.read_begin()
        sim.read_finish()
    sim.read_finish()
    e2e_s = time.perf_counter() - t0
    # (2) the synchronous loop: forces in, one step, wait for and read its state
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.set_forces(f_host)
        sim.step(1)
        sim.read()
    e2e_sync_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    e2e_sync_s = max_over_ranks(e2e_sync_s, dist)
    e2e = {"value": ncell * args.steps * world / e2e_s, "unit": "cell-updates/s",
           "h2d_bytes_per_step": nb * 3 * 8, "d2h_bytes_per_step": nb * 6 * 8 + 3 * 8 + 8 + 4,
           "calls_per_step": "icm_set_blob_forces + icm_step(1) + icm_read_begin (pos, vel, momentum, step); "
                             "icm_read_finish of the previous step (its copy-out overlaps this step)",
           "synchronous": {"value": ncell * args.steps * world / e2e_sync_s, "unit": "cell-updates/s",
                           "calls_per_step": "icm_set_blob_forces + icm_step(1) + icm_read_state(pos, vel, momentum)"}}

    log("[bench] e2e done; profiling launches")
    # per-kernel durations: every launch bracketed by CUDA events on the simulation stream
    nprof = min(args.steps, 10)
    prof = sim.profile(nprof)
    # kernels per stage: memsets are not kernels; the bin build is three (count, scan, fill)
    launches_per_step = sum({"zero": 0, "bins": 3, "wca": 4}.get(kernel_of(name), 1) for name, _, _ in prof)
    per_kernel = {}
    for name, ms_tot, by in prof:
        k = kernel_of(name)
        d = per_kernel.setdefault(k, {"ms": 0.0, "bytes": 0.0, "launches": 0})
        d["ms"] += ms_tot / nprof
        d["bytes"] += by
        d["launches"] += 1
    total = sum(d["ms"] for d in per_kernel.values())
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    d = per_kernel[dom]
    peak, peak_kind = measured_peaks()
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    traffic = ncu_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": traffic, "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                "avg_launch_ms": d["ms"] / d["launches"], "launches_per_step": d["launches"],
                "share_of_step": d["ms"] / total}
    step_bytes = sum(by for _, _, by in prof)
    kernels = {k: {"ms_per_step": round(v["ms"], 4), "launches": v["launches"],
                   "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None,
                   "share": round(v["ms"] / total, 4)} for k, v in sorted(per_kernel.items(), key=lambda kv: -kv[1]["ms"])}

    line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == 32 else "f64", "data": "synthetic",
            "config": dict(workload_config(w, prec, world), plan=plan or "default"),
            "blob_steps_per_s": nb * args.steps * world / (ms / 1e3),
            "step_hbm": {"algorithmic_bytes_per_step": step_bytes,
                         "achieved_GBps": step_bytes / (ms_step / 1e3) / 1e9,
                         "frac": step_bytes / (ms_step / 1e3) / 1e9 / peak, "peak_kind": peak_kind},
            "roofline": roofline, "kernels": kernels, "clocks": clk, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "launches_per_step": launches_per_step,
            "stage_ms": {"%02d.%s" % (i, name): round(ms_tot / nprof, 4) for i, (name, ms_tot, _) in enumerate(prof)}}

    if rank == 0 and world == 1 and not args.no_extras:
        extras(args, w, prec, sim, line, torch, icm, per_kernel)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def extras(args, w, prec, sim, line, torch, icm, per_kernel):
    grid = w["grid"]
    ncell = int(np.prod(grid))
    # the plain FP64 GPU path on the same workload
    log("[bench] extras: FP64 GPU path")
    if prec == 32:
        s64 = icm.Simulation(grid, w["h"], w["rho"], w["eta"], w["kT"], w["dt"], w["kernel"], w["seed"], 64)
        s64.add_blobs(w["q"], w["u"], w["me"])
        s64.set_forces(w["force"])
        s64.step(3)
        s64.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n64 = max(3, min(args.steps, 10))
        e0.record(s64.stream)
        s64.step(n64)
        e1.record(s64.stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1) / n64
        s64.close()
        peak64 = icm.icm_peak_fma(64, s64.stream.cuda_stream if hasattr(s64.stream, "cuda_stream") else None)
        flops = fft_flops_per_step(grid, any(np.asarray(w["me"]) != 0.0))
        step_bytes64 = 2.0 * line["step_hbm"]["algorithmic_bytes_per_step"]
        hbm_peak, hbm_kind = measured_peaks()
        line["fp64_gpu"] = {"ms_per_step": ms64, "value": ncell / (ms64 / 1e3), "unit": "cell-updates/s",
                            "speedup_fp32_over_fp64": ms64 / line["ms_per_step"],
                            "roofline": {"bound": "fp64", "kernel": "whole FP64 step",
                                         "achieved": flops / (ms64 / 1e3) / 1e12, "peak": peak64 / 1e12,
                                         "unit": "TFLOP/s", "frac": flops / (ms64 / 1e3) / peak64,
                                         "peak_kind": "measured (icm_peak_fma: FP64 FMA chains, CUDA events)",
                                         "flops_per_step": flops,
                                         "flop_model": "5 n log2 n per complex n-point FFT line, forward and "
                                                       "inverse along x, y and z for each solve; nothing else "
                                                       "counted"},
                            "hbm": {"algorithmic_bytes_per_step": step_bytes64,
                                    "achieved_GBps": step_bytes64 / (ms64 / 1e3) / 1e9,
                                    "frac": step_bytes64 / (ms64 / 1e3) / 1e9 / hbm_peak, "peak_kind": hbm_kind}}
        line["fp32_fma_peak_tflops"] = icm.icm_peak_fma(32) / 1e12
    log("[bench] extras: cuFFT round trip")
    # cuFFT (through torch.fft) R2C + C2R round trip of the three components, against ours
    x = torch.randn((3,) + tuple(reversed(grid)), device="cuda",
                    dtype=torch.float32 if prec == 32 else torch.float64)
    for _ in range(3):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=x.shape[1:], dim=(1, 2, 3))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=x.shape[1:], dim=(1, 2, 3))
    e1.record()
    e1.synchronize()
    del y
    cufft_ms = e0.elapsed_time(e1) / 10
    ours_rt = sum(per_kernel[k]["ms"] for k in ("x_fwd", "y_fwd", "xy_fwd", "z_sym", "y_inv", "x_inv")
                  if k in per_kernel) / max(1, per_kernel["z_sym"]["launches"])
    line["fft_roundtrip"] = {"ours_ms": ours_rt, "cufft_ms": cufft_ms,
                             "note": "ours includes the fused Helmholtz/projection symbol; cuFFT is R2C+C2R only"}
    log("[bench] extras: batched replicas")
    b = measure_batch(args, 0, 1, None, min(args.steps, 20))
    line["batch"] = {"workload": b["config"]["workload"], "ms_per_step": b["ms_per_step"], "value": b["value"],
                     "unit": "cell-updates/s", "blob_steps_per_s": b["blob_steps_per_s"],
                     "launches_per_step": b["launches_per_step"], "grouped": b["config"]["grouped"],
                     "step_hbm_frac": b["roofline"]["frac"], "speedup_over_unbatched": b["speedup_over_unbatched"],
                     "steps": b["steps"], "clocks": b["clocks"]}
    log("[bench] extras: served stream")
    v = measure_served(args, 0, 1, args.jobs)
    line["served"] = {"workload": v["config"]["workload"], "value": v["value"], "unit": "cell-updates/s",
                      "blob_steps_per_s": v["blob_steps_per_s"], "jobs_per_s": v["jobs_per_s"],
                      "latency_p50_s": v["latency_p50_s"], "latency_p99_s": v["latency_p99_s"],
                      "peak_device_bytes": v["peak_device_bytes"], "wall_s": v["wall_s"], "clocks": v["clocks"]}
    log("[bench] extras: oracle on the host")
    # the FP64 numpy oracle on the host cores, one bounded sample of the same workload
    sec, n = oracle_step_rate(w, min(args.cpu_budget, 60.0), 1)
    line["cpu_baseline"] = {"value": ncell / sec, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                            "sample": "%d full oracle step(s) of this workload (numpy FP64, single thread), %.1f s"
                                      % (n, sec * n)}


def run_batch(args, rank, world, dist):
    """64 replicas (sides {32,48,64,96}, 1-500 blobs, kernel 3 or 4, FP32), one graph launch per step."""
    import torch
    import paper_1212_6427_gb300 as icm
    from paper_1212_6427_gb300 import build
    if rank == 0:
        build.build_library()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    line = measure_batch(args, rank, world, dist, args.steps)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_batch(args, rank, world, dist, steps):
    """The batch workload's JSON line (the members stepped `steps` batch steps)."""
    import torch
    import paper_1212_6427_gb300 as icm
    icm.use_torch_allocator()
    reps = wl.batch_replicas(64, seed0=1 + 64 * rank)
    sims = []
    for r in reps:
        s = icm.Simulation(r["grid"], r["h"], r["rho"], r["eta"], r["kT"], r["dt"], r["kernel"], r["seed"], 32)
        s.add_blobs(r["q"], r["u"], r["me"])
        sims.append(s)
    cells = sum(int(np.prod(r["grid"])) for r in reps)
    blobs = sum(len(r["q"]) for r in reps)
    b = icm.icm_batch_create()
    icm.icm_batch_set(b, [s.handle for s in sims])
    plans = "default"
    if not args.no_autotune:
        icm.icm_batch_autotune(b, 3)
        plans = sorted({str(icm.icm_get_plan(s.handle)) for s in sims})
    if getattr(args, "grouped", None) is not None:
        icm.icm_batch_set_grouped(b, args.grouped)
    grouped = icm.icm_batch_get_grouped(b)
    # algorithmic bytes of one step of every member, with the plans the batch runs
    step_bytes = 0.0
    for s in sims:
        step_bytes += sum(by for _, _, by in s.profile(1))
    icm.icm_batch_step(b, max(args.warmup, 3))
    icm.icm_batch_sync(b)
    launches = icm.icm_batch_kernels_per_step(b)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    icm.icm_batch_step(b, steps)
    icm.icm_batch_sync(b)
    sec = time.perf_counter() - t0
    clk = clocks.stop()
    # the same replicas stepped one after another without batching
    t1 = time.perf_counter()
    for _ in range(max(3, steps // 10)):
        for s in sims:
            s.step(1)
    for s in sims:
        s.sync()
    seq = (time.perf_counter() - t1) / max(3, steps // 10)
    sec = max_over_ranks(sec, dist)
    ms_step = sec / steps * 1e3
    peak, peak_kind = measured_peaks()
    achieved = step_bytes / (ms_step / 1e3) / 1e9
    line = {"metric": METRIC, "value": cells * steps * world / sec, "unit": "cell-updates/s", "n_gpus": world,
            "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "icm-batch-64-replicas-sides-32-48-64-96-fp32", "replicas": 64 * world,
                       "plans": plans, "grouped": grouped,
                       "cells_per_replica_set": cells, "blobs": blobs, "parallelism": "replicas only",
                       "l2": "replica set of %.0f MB per field: timed on host clock around whole batch steps"
                             % (3 * cells * 4 / 1e6)},
            "blob_steps_per_s": blobs * steps * world / sec,
            "roofline": {"bound": "hbm", "kernel": "whole batched step", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None},
            "unbatched_ms_per_step": seq * 1e3, "speedup_over_unbatched": seq * 1e3 / ms_step,
            "clocks": clk, "gpu_launches": launches * steps, "launches_per_step": launches,
            "e2e": {"value": cells * steps * world / sec, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0, "note": "device-resident batch; no per-step host I/O"}}
    icm.icm_batch_destroy(b)
    for s in sims:
        s.close()
    return line


def run_served(args, rank, world, dist):
    """Poisson-arriving jobs (mean 50/s) admitted by a 150 GB HBM budget, continuously batched."""
    import torch
    import paper_1212_6427_gb300 as icm
    from paper_1212_6427_gb300 import build
    if rank == 0:
        build.build_library()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    line = measure_served(args, rank, world, args.jobs)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_served(args, rank, world, njobs):
    """The served workload's JSON line (njobs Poisson-arriving jobs)."""
    import paper_1212_6427_gb300 as icm
    icm.use_torch_allocator()
    jobs = wl.served_jobs(njobs, rate=50.0, seed=5 + rank)
    sv = icm.icm_server_create(150 * 10 ** 9, 256)
    ids = {}
    pending = list(jobs)
    done = 0
    peak_bytes = 0
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    t0 = time.perf_counter()
    while done < len(jobs):
        now = time.perf_counter() - t0
        while pending and pending[0]["arrival"] <= now:
            j = pending.pop(0)
            ids[icm.icm_server_submit(sv, j["grid"], j["h"], j["rho"], j["eta"], j["kT"], j["dt"], j["kernel"],
                                      j["seed"], 32, 0, j["q"], j["u"], j["me"], None, j["steps"])] = j
        a, w, f = icm.icm_server_pump(sv, 4)
        done += f
        peak_bytes = max(peak_bytes, icm.icm_server_bytes_in_use(sv))
        if a == 0 and w == 0 and pending:
            time.sleep(max(0.0, pending[0]["arrival"] - (time.perf_counter() - t0)))
        else:
            time.sleep(0.0005)   # let the enqueued steps run; polling, not waiting on the GPU
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    lat = []
    cell_steps = 0
    blob_steps = 0
    for jid, j in ids.items():
        r = icm.icm_server_result(sv, jid, len(j["q"]))
        assert r["state"] == 2, r["state"]
        lat.append(r["latency_s"])
        cell_steps += int(np.prod(j["grid"])) * j["steps"]
        blob_steps += len(j["q"]) * j["steps"]
    icm.icm_server_destroy(sv)
    lat = np.array(lat)
    line = {"metric": METRIC, "value": cell_steps / wall, "unit": "cell-updates/s", "n_gpus": world,
            "steps": int(sum(j["steps"] for j in jobs)), "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "icm-served-poisson-50ps-%djobs-sides-32-128-fp32" % len(jobs),
                       "hbm_budget_bytes": 150 * 10 ** 9, "max_active": 256, "steps_per_pump": 4,
                       "parallelism": "replicas only"},
            "blob_steps_per_s": blob_steps / wall, "jobs_per_s": len(jobs) / wall,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_mean_s": float(lat.mean()), "peak_device_bytes": peak_bytes, "wall_s": wall, "clocks": clk,
            "e2e": {"value": cell_steps / wall, "unit": "cell-updates/s", "note": "host submit to host result"}}
    return line


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch":
        run_batch(args, rank, world, dist)
    elif args.workload == "served":
        run_served(args, rank, world, dist)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
