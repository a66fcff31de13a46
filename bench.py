#!/usr/bin/env python3
"""Benchmark of the PW advection hot path (su, sv, sw) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one pw_advect call (all three source terms, every level) over the
512 x 512 x 64 workload (16.8M points, smooth 8-mode winds with a 5 m/s mean
wind and 1 % noise, dx = dy = 50 m, dz growing from 10 m by 3 % per level),
FP64 inputs and outputs, inputs resident in HBM. The headline path is the
FP64-accurate paired-FP32 kernel (results within 1e-13 of the FP64 oracle);
the native-FP64 kernel and the FP32 mean+perturbation kernel are measured
beside it, and all three again on the 1024 x 1024 x 128 (134M-point)
workload, with their errors against the FP64 oracle.

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method has no exchange step inside one evaluation): value = all ranks'
points / the slowest rank's time. ``--impl reference`` times the plain FP64
C oracle on the host cores instead (rank 0 only).

Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2107_13500_gb300 import synth  # noqa: E402

WORKLOAD = ("pw_advect su,sv,sw 512x512x64 (16.8M points), FP64 in/out, smooth 8-mode winds "
            "+1% noise, 5 m/s mean wind, dx=dy=50 m, stretched dz=10 m*1.03^(k-2)")
METRIC = "GPoints/s of su,sv,sw (FP64-accurate, <=1e-13 of the FP64 oracle) and % HBM roofline"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# Translation unit of each mode's forward kernel: a stored ncu traffic figure
# is used only while the hash of that file and of every local header it
# includes (transitively) matches the one it was captured with.
KERNEL_FILES = {"paired": "pw_paired.cu", "split": "pw_split.cu", "f64": "pw_kernels.cu"}
SOURCE_DIRS = (os.path.join(ROOT, "paper_2107_13500_gb300", "csrc"), os.path.join(ROOT, "include"))
# Paired-FP32 algorithm, FP32/INT lane operations per point as written: 31 pair
# sums x 8 + 28 pair products x 4 + 3 double->pair splits x 15 + 3 pair->double
# joins x 15 (halo re-splits and address/loop work excluded).
PAIRED_ALG_OPS_PER_POINT = 31 * 8 + 28 * 4 + 3 * 15 + 3 * 15
# FP32/INT issue peak: 152 SMs x 128 lanes x 2.07 GHz (maximum SM clock).
ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--mode", choices=["paired", "f64", "split"], default="paired",
                   help="arithmetic of the headline path")
    p.add_argument("--no-extras", action="store_true", help="skip the 134M-point comparison and the CPU baseline")
    return p.parse_args()


# ----------------------------------------------------------------------------- helpers

def kernel_sources(mode):
    """Paths of the kernel's translation unit and of every local header
    (#include "...") it reaches, sorted by file name."""
    found, todo = {}, [KERNEL_FILES[mode]]
    while todo:
        name = todo.pop()
        if name in found:
            continue
        path = next((os.path.join(d, name) for d in SOURCE_DIRS if os.path.exists(os.path.join(d, name))), None)
        if path is None:
            continue  # a system header
        found[name] = path
        with open(path) as fh:
            todo += re.findall(r'^\s*#\s*include\s+"([^"]+)"', fh.read(), flags=re.M)
    return [found[k] for k in sorted(found)]


def kernel_source_hash(mode):
    h = hashlib.sha256()
    for path in kernel_sources(mode):
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def time_launches(torch, fn, steps, warmup, nsets):
    """Mean ms per call of fn(set_index), CUDA events on the current stream."""
    for n in range(warmup):
        fn(n % nsets)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for n in range(steps):
        fn(n % nsets)
    end.record()
    torch.cuda.synchronize()
    return start.elapsed_time(end) / steps


def replica_throughput(local_ms, points_per_rank, dist=None, device="cpu"):
    """(max_ms, GPoints/s) of a replicas-only run: every rank evaluated
    points_per_rank points in local_ms; the job's time is the slowest rank's,
    its throughput all ranks' points over that time. Without a process group
    this is the single-GPU figure."""
    import torch
    world = 1
    ms = float(local_ms)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * points_per_rank / (ms * 1e-3) / 1e9


def error_stats(gpu_out, ref, ab, nx, ny):
    out = {}
    for name, g, o, a in zip(("su", "sv", "sw"), gpu_out, ref, ab):
        gi = g[:, 1:ny + 1, 1:nx + 1]
        oi = o[:, 1:ny + 1, 1:nx + 1]
        ai = a[:, 1:ny + 1, 1:nx + 1]
        err = np.abs(gi - oi)
        mo = float(np.max(np.abs(oi)))
        out[name] = {"max_err_over_A": float(np.max(err / np.maximum(ai, 1e-300))),
                     "max_rel": float(np.max(err)) / mo if mo else 0.0,
                     "rms_rel": float(np.sqrt(np.mean(err ** 2)) / max(np.sqrt(np.mean(oi ** 2)), 1e-300))}
    return out


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The plain FP64 C oracle on the host cores, on this arm's workload.

    Each step evaluates the full 512x512x64 domain when K + W such steps fit
    in about 100 s; otherwise each step evaluates a y-slab of the domain (all
    levels and columns, fewer rows) sized to that budget. GPoints/s counts
    the points actually evaluated.
    """
    if rank != 0:
        return
    import oracle
    oracle.build_oracle()
    cfg = synth.config_16m_modes()
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    u, v, w = cfg["fields"]()
    co = oracle.coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"])
    cores = os.cpu_count() or 1
    out = tuple(np.zeros_like(u) for _ in range(3))
    t0 = time.perf_counter()
    oracle.advect(u, v, w, co, nx, ny, nthreads=cores, out=out)
    t_full = time.perf_counter() - t0
    budget = 100.0 / max(args.steps + args.warmup, 1)
    rows = ny
    if t_full > budget:
        rows = max(4, min(ny, int(ny * budget / t_full)))
        u, v, w = (np.ascontiguousarray(f[:, : rows + 2, :]) for f in (u, v, w))
        out = tuple(np.zeros_like(u) for _ in range(3))
    for _ in range(max(args.warmup, 0)):
        oracle.advect(u, v, w, co, nx, rows, nthreads=cores, out=out)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.advect(u, v, w, co, nx, rows, nthreads=cores, out=out)
    dt = (time.perf_counter() - t0) / args.steps
    pts = nx * rows * nz
    val = pts / dt / 1e9
    sample = (f"{nx}x{rows}x{nz} {'(full domain)' if rows == ny else 'y-slab of the domain'} per step, "
              f"{args.steps} steps, OpenMP {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GPoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "nz": nz, "rows_per_step": rows},
        "cpu_baseline": {"value": val, "unit": "GPoints/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GPoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm

def cpu_model():
    """The host CPU's model name (lscpu), else the platform's processor string."""
    try:
        res = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in res.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(u, v, w, co, nx, ny, nz):
    """Oracle on the host cores: repeated full-domain calls for ~10-30 s on
    all cores, plus one single-thread evaluation."""
    import oracle
    cores = os.cpu_count() or 1
    out = tuple(np.zeros_like(u) for _ in range(3))
    t0 = time.perf_counter()
    oracle.advect(u, v, w, co, nx, ny, nthreads=cores, out=out)
    one = time.perf_counter() - t0
    reps = int(max(1, min(200, 12.0 / max(one, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.advect(u, v, w, co, nx, ny, nthreads=cores, out=out)
    dt = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    oracle.advect(u, v, w, co, nx, ny, nthreads=1, out=out)
    dt1 = time.perf_counter() - t0
    return {"value": nx * ny * nz / dt / 1e9, "unit": "GPoints/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} full {nx}x{ny}x{nz} evaluations ({reps * dt:.1f} s), OpenMP {cores} threads",
            "single_thread": {"value": nx * ny * nz / dt1 / 1e9, "sample": f"1 full evaluation ({dt1:.1f} s)"},
            "cpu_model": cpu_model()}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    from paper_2107_13500_gb300 import build, pw

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    build.build()
    pw.load_library()

    cfg = synth.config_16m_modes()
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    pts = nx * ny * nz
    u_np, v_np, w_np = cfg["fields"]()
    c = pw.make_coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"]).to_device()
    mode = args.mode
    tdt = torch.float32 if mode == "split" else torch.float64
    nsets = 2
    sets = []
    table = None
    for _ in range(nsets):
        fin = [pw.field_from_numpy(a, nx) for a in (u_np, v_np, w_np)]
        if mode == "split":
            fin, means = zip(*(pw.split_field(t, nx, ny) for t in fin))
            if table is None:
                table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
        fout = [pw.field_like(fin[0]) for _ in range(3)]
        sets.append((list(fin), fout))
    stream = torch.cuda.current_stream()

    def step(n):
        fi, fo = sets[n]
        pw.advect(*fi, c, nx, ny, mode=mode, out=tuple(fo), split_table=table, stream=stream)

    # warm-up + timed region (device time, inputs resident)
    sampler = ClockSampler(local)
    for n in range(args.warmup):
        step(n % nsets)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for n in range(args.steps):
        step(n % nsets)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    status = pw.device_status()
    if status != 0:
        raise SystemExit(f"kernel reported device status {status}")
    ms, value = replica_throughput(ms, pts, dist, device="cuda")
    # per-launch distribution (a separate loop, one event pair per launch;
    # the headline above is the K-step mean the contract asks for)
    nlaunch = 50
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nlaunch)]
    for n, (a0, a1) in enumerate(evs):
        a0.record(stream)
        step(n % nsets)
        a1.record(stream)
    torch.cuda.synchronize()
    per_launch = sorted(a0.elapsed_time(a1) for a0, a1 in evs)
    launch_stats = {"launches": nlaunch, "median_ms": statistics.median(per_launch),
                    "p10_ms": per_launch[nlaunch // 10], "p90_ms": per_launch[(9 * nlaunch) // 10]}

    # end to end through the public API: pinned host inputs -> device ->
    # pw_advect -> host outputs, inside the timed region. Overlapped form:
    # pw_advect_host_chunked (slabs of levels: transfers on two streams
    # around the compute stream); serial form for comparison.
    e2e_mode = mode if mode != "split" else "paired"
    host_in = [pw.pinned_field(nx, ny, nz) for _ in range(3)]
    for h, a in zip(host_in, (u_np, v_np, w_np)):
        h.copy_(torch.from_numpy(a))
    host_out = tuple(pw.pinned_field(nx, ny, nz) for _ in range(3))
    pipe = pw.HostPipeline(nx, ny, nz)
    nchunks = 8

    def e2e_step(_):
        pw.advect_host(*host_in, c, nx, ny, mode=e2e_mode, out_host=host_out, pipeline=pipe, nchunks=nchunks,
                       wait=False)

    e2e_steps = max(5, min(args.steps // 10, 200))
    e2e_ms = time_launches(torch, e2e_step, e2e_steps, 3, 1)
    e2e_ms, e2e_value = replica_throughput(e2e_ms, pts, dist, device="cuda")
    dev_in, dev_out = pipe.dev[:3], pipe.dev[3:]

    def serial_step(_):
        for d, h in zip(dev_in, host_in):
            d.copy_(h, non_blocking=True)
        pw.advect(*dev_in, c, nx, ny, mode=e2e_mode, out=tuple(dev_out), stream=stream)
        for h, d in zip(host_out, dev_out):
            h.copy_(d, non_blocking=True)

    serial_ms = time_launches(torch, serial_step, e2e_steps, 3, 1)
    # bytes the chunked path moves: every field up to its last interior
    # element in, rows 1..ny of every level out
    es = host_in[0].element_size()
    sy, sz = host_in[0].stride(1), host_in[0].stride(0)
    h2d_bytes = 3 * ((nz - 1) * sz + (ny + 1) * sy + nx + 2) * es
    d2h_bytes = 3 * nz * ny * sy * es
    e2e = {"value": e2e_value, "unit": "GPoints/s",
           "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
           "ms_per_step": e2e_ms,
           "path": f"pinned host fields -> pw_advect_host_chunked({e2e_mode}, {nchunks} slabs of levels: H2D / "
                   "compute / D2H streams overlapped) -> pinned host outputs",
           "serial_ms_per_step": serial_ms, "serial_GPoints_s": pts / (serial_ms * 1e-3) / 1e9}

    peak, peak_kind = measured_peaks()
    bpp = pw.BYTES_PER_POINT[mode]
    achieved = bpp * pts / (ms * 1e-3) / 1e9
    traffic = None
    if os.path.exists(PROFILE_TRAFFIC):
        with open(PROFILE_TRAFFIC) as fh:
            prof = json.load(fh)
        ent = prof.get(mode)
        if ent and ent.get("source_hash") == kernel_source_hash(mode):
            traffic = ent.get("bytes_per_launch")
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bpp * pts,
           "kernel": f"pw_advect[{mode}] (one launch per step)"}
    if mode == "paired":
        tops = PAIRED_ALG_OPS_PER_POINT * pts / (ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": tops, "peak": ALU_PEAK_TOPS, "unit": "TOP/s",
                    "frac": tops / ALU_PEAK_TOPS, "traffic": traffic,
                    "peak_kind": "derived: 152 SMs x 128 FP32/INT lanes x 2.07 GHz",
                    "algorithmic_ops_per_point": PAIRED_ALG_OPS_PER_POINT,
                    "kernel": "pw_advect[paired] (one launch per step)", "hbm": hbm}
    else:
        roofline = hbm

    line = {
        "metric": METRIC, "value": value, "unit": "GPoints/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"paired": "f32x2", "f64": "f64", "split": "f32"}[mode],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "nz": nz, "points_per_gpu": pts,
                   "mode": mode, "io_dtype": "f64" if mode != "split" else "f32+f64 level means",
                   "l2": "per-step working set 3x135 MB in + 3x135 MB out > 129 MB L2; 2 buffer sets rotate",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "hbm_roofline_frac": achieved / peak,
        "launch_ms": launch_stats,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }

    if rank == 0 and world == 1 and not args.no_extras:
        import oracle
        oracle.build_oracle()
        co = oracle.coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"])
        ref, ab = oracle.advect(u_np, v_np, w_np, co, nx, ny, want_abs=True, nthreads=os.cpu_count() or 1)
        # errors of this run's outputs (last timed step) against the oracle
        last = sets[(args.steps - 1) % nsets][1]
        gout = [t.double().cpu().numpy() for t in last]
        line["error_vs_oracle"] = error_stats(gout, ref, ab, nx, ny)
        line["cpu_baseline"] = cpu_baseline(u_np, v_np, w_np, co, nx, ny, nz)
        line["modes"] = extra_modes(torch, pw, oracle, args, sets, c, cfg, ref, ab, peak)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def extra_modes(torch, pw, oracle, args, sets16, c16, cfg16, ref16, ab16, peak):
    """The other arithmetic modes at 16.8M points, and all three at 134M
    points (FP32 vs FP64 on the same GPU), each with its error against the
    FP64 oracle."""
    res = {}
    steps = max(10, min(args.steps // 10, 300))
    nx, ny, nz = cfg16["nx"], cfg16["ny"], cfg16["nz"]
    fin16 = [sets16[0][0][n].double() if sets16[0][0][n].dtype != torch.float64 else sets16[0][0][n]
             for n in range(3)]

    def measure(label, fin, c, nx, ny, nz, mode, table, ref, ab):
        fout = [pw.field_like(fin[0]) for _ in range(3)]
        ms = time_launches(torch, lambda _: pw.advect(*fin, c, nx, ny, mode=mode, out=tuple(fout),
                                                       split_table=table), steps, 3, 1)
        pts = nx * ny * nz
        bpp = pw.BYTES_PER_POINT[mode]
        g = [t.double().cpu().numpy() for t in fout]
        res[label] = {"GPoints_s": pts / (ms * 1e-3) / 1e9, "ms": ms, "GB_s": bpp * pts / (ms * 1e-3) / 1e9,
                      "hbm_frac": bpp * pts / (ms * 1e-3) / 1e9 / peak, "bytes_per_point": bpp,
                      "error_vs_oracle": error_stats(g, ref, ab, nx, ny)}

    if sets16[0][0][0].dtype == torch.float64:
        # boundary helpers, timed apart from the headline: the periodic halo
        # fill and the mean/perturbation split (12 B/pt: read 8, write 4)
        t = fin16[0]
        fp_buf = pw.empty_field(nx, ny, nz, torch.float32)
        mean_buf = torch.empty(nz, dtype=torch.float64, device=t.device)
        halo_ms = time_launches(torch, lambda _: pw.fill_periodic_halo(t, nx, ny), steps, 3, 1)
        split_ms = time_launches(torch, lambda _: pw.split_field(t, nx, ny, out=fp_buf, mean=mean_buf), steps, 3, 1)
        res["16m_helpers_per_field"] = {
            "fill_periodic_halo_us": halo_ms * 1e3,
            "split_field_us": split_ms * 1e3,
            "split_field_GB_s": 12 * nx * ny * nz / (split_ms * 1e-3) / 1e9}
        for mode in ("f64", "paired", "split"):
            if mode == "split":
                fp, means = zip(*(pw.split_field(t, nx, ny) for t in fin16))
                table = torch.from_numpy(pw.make_split_table(c16, *(m.cpu().numpy() for m in means))).cuda()
                measure("16m_split", list(fp), c16, nx, ny, nz, "split", table, ref16, ab16)
            else:
                measure(f"16m_{mode}", fin16, c16, nx, ny, nz, mode, None, ref16, ab16)
    # 1024 x 1024 x 128 with i.i.d. winds and uniform 20 m levels
    cfg = synth.config_134m_iid()
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    u, v, w = cfg["fields"]()
    co = oracle.coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"])
    ref, ab = oracle.advect(u, v, w, co, nx, ny, want_abs=True, nthreads=os.cpu_count() or 1)
    c = pw.make_coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"]).to_device()
    fin = [pw.field_from_numpy(a, nx) for a in (u, v, w)]
    del u, v, w
    for mode in ("f64", "paired"):
        measure(f"134m_{mode}", fin, c, nx, ny, nz, mode, None, ref, ab)
    fp, means = zip(*(pw.split_field(t, nx, ny) for t in fin))
    table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
    del fin
    measure("134m_split", list(fp), c, nx, ny, nz, "split", table, ref, ab)
    r = res
    r["fp32_split_speedup_over_paired_134m"] = r["134m_split"]["GPoints_s"] / r["134m_paired"]["GPoints_s"]
    r["fp32_split_speedup_over_f64_134m"] = r["134m_split"]["GPoints_s"] / r["134m_f64"]["GPoints_s"]
    del fp, table
    torch.cuda.empty_cache()
    res["batched_96"] = batched_extra(torch, pw)
    res["adjoint_256"] = adjoint_extra(torch, pw)
    res["c1_64cubed_graph"] = c1_extra(torch, pw, oracle)
    return res


def c1_extra(torch, pw, oracle):
    """64 x 64 x 64 i.i.d. winds, uniform 20 m levels (the correctness
    configuration; its ~13 MB working set stays in L2), each mode timed as
    a CUDA graph of 100 launches, with errors against the FP64 oracle."""
    cfg = synth.config_small_iid()
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    u, v, w = cfg["fields"]()
    co = oracle.coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"])
    ref, ab = oracle.advect(u, v, w, co, nx, ny, want_abs=True, nthreads=os.cpu_count() or 1)
    c = pw.make_coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"]).to_device()
    fin = [pw.field_from_numpy(a, nx) for a in (u, v, w)]
    pts = nx * ny * nz
    out = {"working_set": "L2-resident (no flush between launches)", "launches_per_graph": 100}
    for mode in ("f64", "paired", "split"):
        table = None
        f = fin
        if mode == "split":
            fp, means = zip(*(pw.split_field(t, nx, ny) for t in fin))
            table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
            f = list(fp)
        fout = tuple(pw.field_like(f[0]) for _ in range(3))
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            pw.advect(*f, c, nx, ny, mode=mode, out=fout, split_table=table, stream=s)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                for _ in range(100):
                    pw.advect(*f, c, nx, ny, mode=mode, out=fout, split_table=table, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (5 * 100)
        gout = [t.double().cpu().numpy() for t in fout]
        out[mode] = {"us_per_launch": ms * 1e3, "GPoints_s": pts / (ms * 1e-3) / 1e9,
                     "error_vs_oracle": error_stats(gout, ref, ab, nx, ny)}
        del g
    return out


def batched_extra(torch, pw):
    """96 independent domains (x, y in 32..384, z in 32..128, seed 4,
    stretched grids) in one persistent launch per evaluation: autotuned
    variant, and a CUDA graph of 50 evaluations."""
    from paper_2107_13500_gb300 import autotune
    sizes = synth.batched_domain_sizes(96, seed=4)
    pts = sum(a * b * c for a, b, c in sizes)
    out = {"domains": 96, "points": pts}
    for mode in ("f32", "paired"):
        dt = torch.float64 if mode == "paired" else torch.float32
        gen = torch.Generator(device="cuda").manual_seed(4)
        doms = []
        for nx, ny, nz in sizes:
            c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_stretched(nz)).to_device()
            f = [pw.empty_field(nx, ny, nz, dt) for _ in range(3)]
            for t in f:
                t.uniform_(-10, 10, generator=gen)
            doms.append(dict(u=f[0], v=f[1], w=f[2], nx=nx, ny=ny, coeffs=c))
        variant, rec = autotune.tune(doms, mode, cache_path=os.path.join(tempfile.gettempdir(), "pw_bench_tune.json"),
                                     reps=10, force=True)
        b = pw.Batch(doms, mode, variant)
        ms = autotune.time_batch(b, reps=50, warmup=5)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            b.run(stream=s)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                for _ in range(50):
                    b.run(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_ms = e0.elapsed_time(e1) / (3 * 50)
        bpp = pw.BYTES_PER_POINT[mode]
        out[mode] = {"variant": variant, "variant_ms": rec["ms"], "ms": ms, "GPoints_s": pts / (ms * 1e-3) / 1e9,
                     "hbm_frac": bpp * pts / (ms * 1e-3) / 1e9 / measured_peaks()[0],
                     "graph50_ms_per_eval": graph_ms, "graph50_GPoints_s": pts / (graph_ms * 1e-3) / 1e9}
        del doms, b, g
        torch.cuda.empty_cache()
    return out


def adjoint_extra(torch, pw):
    """256 x 256 x 64 with the small configuration's winds: adjoint kernel
    time (native FP64, paired FP32, FP32) and a 20-step forward-Euler
    rollout (dt = 0.5 s) differentiated with checkpoints every 5 steps
    (native FP64 and paired forward/adjoint)."""
    from paper_2107_13500_gb300 import autograd as pa
    nx, ny, nz = 256, 256, 64
    pts = nx * ny * nz
    u, v, w = synth.fields_iid(nx, ny, nz, seed=1)
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    out = {"points": pts}
    for mode, dt in (("f64", torch.float64), ("paired", torch.float64), ("f32", torch.float32)):
        x = [pw.field_from_numpy(a, nx, dt) for a in (u, v, w)]
        g = [pw.field_like(x[0]).uniform_(-1, 1) for _ in range(3)]
        res = tuple(pw.field_like(x[0]) for _ in range(3))
        ms = time_launches(torch, lambda _: pw.advect_adjoint(*x, c, nx, ny, *g, mode=mode, out=res), 50, 3, 1)
        out[f"adjoint_{mode}"] = {"ms": ms, "GPoints_s": pts / (ms * 1e-3) / 1e9}
    x0 = [pw.field_from_numpy(a, nx, torch.float64) for a in (u, v, w)]
    y = [pw.field_like(x0[0]).uniform_(-1, 1) for _ in range(3)]
    inner = (slice(None), slice(1, ny + 1), slice(1, nx + 1))

    def one(mode):
        xs = [t.clone().requires_grad_() for t in x0]
        fin = pa.rollout(*xs, c, nx, ny, 0.5, 20, mode=mode, checkpoint_every=5)
        loss = sum((o[inner] * yy[inner]).sum() for o, yy in zip(fin, y))
        return torch.autograd.grad(loss, xs)

    for mode in ("f64", "paired"):
        one(mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one(mode)
        torch.cuda.synchronize()
        out[f"rollout20_ckpt5_{mode}_s"] = time.perf_counter() - t0
    return out


if __name__ == "__main__":
    main()
