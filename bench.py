#!/usr/bin/env python3
"""Benchmark of the PW advection hot path (su, sv, sw) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --only forward|adjoint|batched|split_field --mode M [--shape NX,NY,NZ] ...

One step = one pw_advect call (all three source terms, every level) over the
512 x 512 x 64 workload (16.8M points, smooth 8-mode winds with a 5 m/s mean
wind and 1 % noise, dx = dy = 50 m, dz growing from 10 m by 3 % per level),
FP64 inputs and outputs, inputs resident in HBM. The headline path computes
in native FP64 arithmetic (results within 1e-13 of the FP64 oracle). The
other arithmetic paths are measured beside it and reported as top-level
keys with their errors against the oracle: paired FP32 (FP64 in and out,
about 48-bit "double-float" arithmetic), plain FP32 and the FP32
mean + perturbation split, at 16.8M and at 134M (1024 x 1024 x 128) points,
plus the 96-domain batch, the adjoint and each path's FP64 energy budget.

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method has no exchange step inside one evaluation): value = all ranks'
points / the slowest rank's time. ``--impl reference`` times the plain FP64
C oracle on the host cores instead (rank 0 only). ``--only`` times one
library call on its own (for profiler runs) and prints one summary line.

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
METRIC = "GPoints/s of su,sv,sw and % HBM roofline, FP32 vs FP64 on the same GB300 at stated error"
CONFIG = {"workload": WORKLOAD, "nx": 512, "ny": 512, "nz": 64, "points_per_gpu": 512 * 512 * 64,
          "l2": "per-step working set 3x135 MB in + 3x135 MB out > 129 MB L2; 2 buffer sets rotate"}
DTYPES = {"f64": "f64", "paired": "f32x2", "split": "f32", "f32": "f32"}
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# Translation unit of each mode's forward kernel: a stored ncu traffic figure
# is used only while the hash of that file and of every local header it
# includes (transitively) matches the one it was captured with.
KERNEL_FILES = {"paired": "pw_paired.cu", "split": "pw_split.cu", "f64": "pw_f64.cu", "f32": "pw_split.cu"}
KERNEL_NAMES = {"paired": "fwd_paired_kernel", "split": "fwd_split_kernel", "f64": "fwd_f64_kernel",
                "f32": "fwd_split_kernel"}
SOURCE_DIRS = (os.path.join(ROOT, "paper_2107_13500_gb300", "csrc"), os.path.join(ROOT, "include"))
# FP64 lane operations per point of the native kernel's scheme on its 32 x 16
# tile: scaling tcx u and tcy v over the cells the faces read ((17*34 + 18*33)
# / 512), the six horizontal face-sum types ((3*16*33 + 3*17*32) / 512), three
# vertical face sums, 18 face products, and the vertical coefficient products:
# three (one per output, shared by the level's two vertical face terms) when
# every level's two vertical coefficients are equal, as on the benchmark's
# grid (no density stratification), else six.
F64_OPS_PER_POINT_DENSITY = (17 * 34 + 18 * 33) / 512 + (3 * 16 * 33 + 3 * 17 * 32) / 512 + 3 + 18 + 6
F64_OPS_PER_POINT = F64_OPS_PER_POINT_DENSITY - 3
# FP64 pipe: GB300 retires 2 FP64 lane operations per clock per SM (an FMA
# counted once): 152 SMs x 2 x 2.07 GHz (maximum SM clock).
FP64_PIPE_PEAK_GOPS = 152 * 2 * 2.07e9 / 1e9
# Adjoint algorithmic bytes per cell: read u, v, w and three cotangents,
# write three gradients (FP64 8 B, FP32 4 B each).
ADJOINT_BYTES = {"f64": 72, "paired": 72, "f32": 36}


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--mode", choices=["f64", "paired", "split", "f32"], default="f64",
                   help="arithmetic of the headline path (default: native FP64)")
    p.add_argument("--no-extras", action="store_true", help="skip the other paths, the oracle and the CPU baseline")
    p.add_argument("--only", choices=["forward", "adjoint", "batched", "split_field"],
                   help="time one library call on its own (profiler runs) and print one summary line")
    p.add_argument("--shape", default="512,512,64", help="--only: NX,NY,NZ of the single domain")
    p.add_argument("--variant", type=int, default=0, help="--only batched: tile/pipeline variant")
    p.add_argument("--domains", type=int, default=96, help="--only batched: number of domains")
    p.add_argument("--reps", type=int, default=50, help="--only: timed calls")
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


def stored_traffic(mode):
    """DRAM bytes per launch of the mode's forward kernel from the committed
    ncu capture, or None when the kernel's sources changed since."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    with open(PROFILE_TRAFFIC) as fh:
        prof = json.load(fh)
    ent = prof.get(mode)
    if ent and ent.get("source_hash") == kernel_source_hash(mode):
        return ent.get("bytes_per_launch")
    return None


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


def time_launches(torch, fn, steps, warmup, nsets, drain=None):
    """Mean ms per call of fn(set_index), CUDA events on the current stream;
    drain() (if given) orders the current stream after work fn left on other
    streams before the closing event."""
    for n in range(warmup):
        fn(n % nsets)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for n in range(steps):
        fn(n % nsets)
    if drain is not None:
        drain()
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


def error_stats(gpu_out, ref, strict, nx, ny, mono=None):
    """Per field: max err / strict scale A, max err / monomial scale M (if
    given), and the max and RMS errors relative to the oracle's max and RMS."""
    out = {}
    for n, (name, g, o, a) in enumerate(zip(("su", "sv", "sw"), gpu_out, ref, strict)):
        gi = g[:, 1:ny + 1, 1:nx + 1]
        oi = o[:, 1:ny + 1, 1:nx + 1]
        ai = a[:, 1:ny + 1, 1:nx + 1]
        err = np.abs(gi - oi)
        mo = float(np.max(np.abs(oi)))
        d = {"max_err_over_A": float(np.max(err / np.maximum(ai, 1e-300))),
             "max_rel": float(np.max(err)) / mo if mo else 0.0,
             "rms_rel": float(np.sqrt(np.mean(err ** 2)) / max(np.sqrt(np.mean(oi ** 2)), 1e-300))}
        if mono is not None:
            mi = mono[n][:, 1:ny + 1, 1:nx + 1]
            d["max_err_over_M"] = float(np.max(err / np.maximum(mi, 1e-300)))
        out[name] = d
    return out


def worst(stats, key):
    return max(v[key] for v in stats.values())


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
        "config": dict(CONFIG, parallelism=f"replicas x{world}"),
        "reference_sample_rows_per_step": rows,
        "cpu_baseline": {"value": val, "unit": "GPoints/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GPoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- one call on its own

def run_only(args):
    """Time one library call on seeded synthetic inputs (for profiler runs).

    Single domains have i.i.d. U[-10, 10] winds (seed 1) on a uniform 20 m
    grid with dx = dy = 50 m; split domains take float perturbations about
    the level means with their table; the adjoint's cotangents are U[-1, 1].
    The batch is --domains domains with x, y in 32..384 and z in 32..128
    (seed 4), stretched grids and U[-10, 10] winds, in one persistent launch
    of tile variant --variant. The call runs 3 times, then --reps times
    between two CUDA events on the current stream; inputs stay resident (no
    L2 flush): the figures this run prints are not bench values.
    """
    import torch
    from paper_2107_13500_gb300 import build, pw
    build.build()
    mode = args.mode
    if args.only == "batched":
        dt = torch.float32 if mode in ("f32", "split") else torch.float64
        gen = torch.Generator(device="cuda").manual_seed(4)
        doms = []
        for bx, by, bz in synth.batched_domain_sizes(args.domains, seed=4):
            c = pw.make_coeffs(bz, 50.0, 50.0, synth.dz_stretched(bz)).to_device()
            f = [pw.empty_field(bx, by, bz, dt) for _ in range(3)]
            for t in f:
                t.uniform_(-10, 10, generator=gen)
            d = dict(u=f[0], v=f[1], w=f[2], nx=bx, ny=by, coeffs=c)
            if mode == "split":
                d["split_table"] = torch.from_numpy(pw.make_split_table(c, *([np.zeros(bz)] * 3))).cuda()
            doms.append(d)
        batch = pw.Batch(doms, mode, args.variant)
        pts = sum(d["nx"] * d["ny"] * d["u"].shape[0] for d in doms)
        _only_timed(args, batch.run, pts, f"{args.domains} domains, {pts} points, variant {args.variant}")
        return
    nx, ny, nz = (int(x) for x in args.shape.split(","))
    label = f"{nx}x{ny}x{nz}"
    if args.only == "split_field":
        f = pw.field_from_numpy(synth.fields_iid(nx, ny, nz, seed=1)[0], nx, torch.float64)
        pert = pw.empty_field(nx, ny, nz, torch.float32)
        mean = torch.empty(nz, dtype=torch.float64, device="cuda")
        _only_timed(args, lambda: pw.split_field(f, nx, ny, out=pert, mean=mean), nx * ny * nz, label)
        return
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    x64 = [pw.field_from_numpy(a, nx) for a in synth.fields_iid(nx, ny, nz, seed=1)]
    if args.only == "adjoint":
        if mode == "split":
            raise SystemExit("the mean+perturbation form has no adjoint")
        dt = torch.float32 if mode == "f32" else torch.float64
        # the layout of the bench's adjoint figures: i = 1 on a 16-byte boundary
        x = [pw.field_from_numpy(a, nx, dt) for a in synth.fields_iid(nx, ny, nz, seed=1)]
        gen = torch.Generator(device="cuda").manual_seed(2)
        g = [pw.field_like(x[0]).uniform_(-1, 1, generator=gen) for _ in range(3)]
        out = tuple(pw.field_like(x[0]) for _ in range(3))
        _only_timed(args, lambda: pw.advect_adjoint(*x, c, nx, ny, *g, mode=mode, out=out), nx * ny * nz, label)
        return
    table = None
    if mode == "split":
        x, means = zip(*(pw.split_field(t, nx, ny) for t in x64))
        table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
    elif mode == "f32":
        x = [pw.empty_field(nx, ny, nz, torch.float32).copy_(t) for t in x64]
    else:
        x = x64
    out = tuple(pw.field_like(x[0]) for _ in range(3))
    _only_timed(args, lambda: pw.advect(*x, c, nx, ny, mode=mode, out=out, split_table=table), nx * ny * nz, label)


def _only_timed(args, call, pts, label):
    import torch
    from paper_2107_13500_gb300 import pw
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    print(f"{args.only} {args.mode} {label}: {ms * 1e3:.1f} us per call, {pts / ms / 1e6:.2f} GPoints/s, "
          f"device status {pw.device_status()}")


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


def make_inputs(torch, pw, mode, fields64, c, nx, ny):
    """Device inputs of one mode from the FP64 numpy winds: (fields, table)."""
    if mode in ("f64", "paired"):
        return [pw.field_from_numpy(a, nx) for a in fields64], None
    if mode == "f32":
        return [pw.field_from_numpy(a, nx, torch.float32) for a in fields64], None
    dev = [pw.field_from_numpy(a, nx) for a in fields64]
    fp, means = zip(*(pw.split_field(t, nx, ny) for t in dev))
    table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
    return list(fp), table


def main():
    args = parse_args()
    if args.only:
        run_only(args)
        return
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
    nsets = 2
    sets = []
    table = None
    for _ in range(nsets):
        fin, table = make_inputs(torch, pw, mode, (u_np, v_np, w_np), c, nx, ny)
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

    e2e = e2e_leg(torch, pw, mode, args, (u_np, v_np, w_np), c, nx, ny, nz, dist, table)

    peak, peak_kind = measured_peaks()
    bpp = pw.BYTES_PER_POINT[mode]
    achieved = bpp * pts / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": stored_traffic(mode), "peak_kind": ("measured copy bandwidth (MEASURED_PEAKS.json)" if peak_kind == "measured" else
                                         "fallback copy bandwidth (6.8 TB/s; MEASURED_PEAKS.json absent)"),
                "algorithmic_bytes_per_launch": bpp * pts,
                "kernel": f"{KERNEL_NAMES[mode]} (pw_advect[{mode}], one launch per step)"}
    if mode == "f64":
        gops = F64_OPS_PER_POINT * pts / (ms * 1e-3) / 1e9
        roofline["fp64_pipe"] = {
            "ops_per_point": F64_OPS_PER_POINT, "achieved_gops": gops, "peak_gops": FP64_PIPE_PEAK_GOPS,
            "frac": gops / FP64_PIPE_PEAK_GOPS,
            "peak_kind": "derived: 152 SMs x 2 FP64 lane ops/clk x 2.07 GHz (an FMA counted once)"}

    line = {
        "metric": METRIC, "value": value, "unit": "GPoints/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[mode], "data": "synthetic",
        "config": dict(CONFIG, parallelism=f"replicas x{world}"),
        "path": {"f64": "native FP64 arithmetic, FP64 in/out",
                 "paired": "paired-FP32 (double-float, ~48 significant bits) arithmetic, FP64 in/out",
                 "split": "FP32 arithmetic on float perturbations about FP64 level means",
                 "f32": "FP32 arithmetic on float winds"}[mode],
        "roofline": roofline,
        "launch_ms": launch_stats,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }

    if rank == 0 and world == 1 and not args.no_extras:
        extras(torch, pw, args, line, sets, c, cfg, (u_np, v_np, w_np), peak)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def e2e_leg(torch, pw, mode, args, fields64, c, nx, ny, nz, dist, table):
    """The same metric through the public API from pinned host buffers:
    pw_advect_host_chunked (slabs of levels: H2D, compute and D2H on three
    streams, overlapped) inside the timed region; the serial form (H2D ->
    pw_advect -> D2H on one stream) beside it. The split path's host inputs
    are its float perturbations (its level table already on the device)."""
    pts = nx * ny * nz
    dt = torch.float64 if mode in ("f64", "paired") else torch.float32
    if mode == "split":
        dev = [pw.field_from_numpy(a, nx) for a in fields64]
        fp, means = zip(*(pw.split_field(t, nx, ny) for t in dev))
        table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
        host_src = [t.cpu() for t in fp]
    else:
        host_src = [torch.from_numpy(a).to(dt) for a in fields64]
    host_in = [pw.pinned_field(nx, ny, nz, dt) for _ in range(3)]
    for h, a in zip(host_in, host_src):
        h[:, :, : nx + 2].copy_(a[:, :, : nx + 2])
    host_out = tuple(pw.pinned_field(nx, ny, nz, dt) for _ in range(3))
    pipe = pw.HostPipeline(nx, ny, nz, dt, depth=2)
    nchunks = 4
    stream = torch.cuda.current_stream()

    def e2e_step(_):
        pw.advect_host(*host_in, c, nx, ny, mode=mode, out_host=host_out, pipeline=pipe, nchunks=nchunks,
                       split_table=table, wait=False)

    e2e_steps = max(5, min(args.steps // 10, 200))
    # consecutive calls overlap on the pipeline's two staging sets; the
    # closing event follows the last call's outputs into host memory
    e2e_ms = time_launches(torch, e2e_step, e2e_steps, 3, 1, drain=pipe.wait)
    e2e_ms, e2e_value = replica_throughput(e2e_ms, pts, dist, device="cuda")
    dev_in, dev_out = pipe.dev[:3], pipe.dev[3:]

    def serial_step(_):
        for d, h in zip(dev_in, host_in):
            d.copy_(h, non_blocking=True)
        pw.advect(*dev_in, c, nx, ny, mode=mode, out=tuple(dev_out), split_table=table, stream=stream)
        for h, d in zip(host_out, dev_out):
            h.copy_(d, non_blocking=True)

    serial_ms = time_launches(torch, serial_step, e2e_steps, 3, 1)
    # bytes the chunked path moves: every field up to its last interior
    # element in, rows 1..ny of every level out
    es = host_in[0].element_size()
    sy, sz = host_in[0].stride(1), host_in[0].stride(0)
    h2d_bytes = 3 * ((nz - 1) * sz + (ny + 1) * sy + nx + 2) * es
    d2h_bytes = 3 * nz * ny * sy * es
    return {"value": e2e_value, "unit": "GPoints/s", "h2d_bytes_per_step": h2d_bytes,
            "d2h_bytes_per_step": d2h_bytes, "ms_per_step": e2e_ms,
            "path": f"pinned host fields -> pw_advect_host_chunked({mode}, {nchunks} slabs of levels: H2D / "
                    "compute / D2H streams overlapped, consecutive calls on two staging sets) -> pinned host outputs",
            "serial_ms_per_step": serial_ms, "serial_GPoints_s": pts / (serial_ms * 1e-3) / 1e9}


def measure_mode(torch, pw, mode, fin, table, c, nx, ny, nz, steps, peak):
    """(result dict, outputs) of one mode on resident inputs: mean time of
    `steps` launches after 3 warm-ups."""
    fout = [pw.field_like(fin[0]) for _ in range(3)]
    ms = time_launches(torch, lambda _: pw.advect(*fin, c, nx, ny, mode=mode, out=tuple(fout), split_table=table),
                       steps, 3, 1)
    pts = nx * ny * nz
    bpp = pw.BYTES_PER_POINT[mode]
    return {"GPoints_s": pts / (ms * 1e-3) / 1e9, "ms": ms, "GB_s": bpp * pts / (ms * 1e-3) / 1e9,
            "hbm_frac": bpp * pts / (ms * 1e-3) / 1e9 / peak, "bytes_per_point": bpp}, fout


def energy_residual(torch, pw, winds, outs, nx, ny, wu, ww):
    """max over u, v, w of |weighted energy tendency| / sum |summands|."""
    tot, _ = pw.energy_budget(*winds, *outs, nx, ny, wu, ww)
    t = tot.cpu().numpy()
    return max(abs(t[n]) / t[3 + n] for n in range(3) if t[3 + n] > 0)


def extras(torch, pw, args, line, sets, c16, cfg16, fields16, peak):
    """Every arithmetic path at 16.8M and 134M points with its error against
    the oracle, the helpers, the batch, the adjoint and the CPU baseline;
    the key figures become top-level keys of the line."""
    import oracle
    oracle.build_oracle()
    cores = os.cpu_count() or 1
    nx, ny, nz = cfg16["nx"], cfg16["ny"], cfg16["nz"]
    u_np, v_np, w_np = fields16
    co = oracle.coeffs(nz, cfg16["dx"], cfg16["dy"], cfg16["dz"])
    ref, ab = oracle.advect(u_np, v_np, w_np, co, nx, ny, want_abs=True, nthreads=cores)
    mono = oracle.monomial_scale(u_np, v_np, w_np, co, nx, ny, nthreads=cores)
    flat = {}
    # errors of this run's headline outputs (last timed step)
    last = sets[(args.steps - 1) % len(sets)][1]
    line["error_vs_oracle"] = error_stats([t.double().cpu().numpy() for t in last], ref, ab, nx, ny, mono)
    line["cpu_baseline"] = cpu_baseline(u_np, v_np, w_np, co, nx, ny, nz)
    steps = max(10, min(args.steps // 10, 300))
    wu_h, ww_h = pw.make_energy_weights(nz, cfg16["dz"])
    wu, ww = (torch.from_numpy(a).cuda() for a in (wu_h, ww_h))
    modes16 = {}
    for mode in ("f64", "paired", "f32", "split"):
        fin, table = make_inputs(torch, pw, mode, fields16, c16, nx, ny)
        res, fout = measure_mode(torch, pw, mode, fin, table, c16, nx, ny, nz, steps, peak)
        g = [t.double().cpu().numpy() for t in fout]
        res["error_vs_oracle"] = error_stats(g, ref, ab, nx, ny, mono)
        winds = fin if mode != "split" else [pw.field_from_numpy(a, nx) for a in fields16]
        res["energy_residual"] = energy_residual(torch, pw, winds, fout, nx, ny, wu, ww)
        modes16[mode] = res
        del fin, fout, winds
    # boundary helpers per field, timed apart: the periodic halo fill and
    # the mean/perturbation split (12 B/pt: read 8, write 4)
    t = pw.field_from_numpy(u_np, nx)
    fp_buf = pw.empty_field(nx, ny, nz, torch.float32)
    mean_buf = torch.empty(nz, dtype=torch.float64, device="cuda")
    halo_ms = time_launches(torch, lambda _: pw.fill_periodic_halo(t, nx, ny), steps, 3, 1)
    split_ms = time_launches(torch, lambda _: pw.split_field(t, nx, ny, out=fp_buf, mean=mean_buf), steps, 3, 1)
    helpers = {"fill_periodic_halo_us": halo_ms * 1e3, "split_field_us": split_ms * 1e3,
               "split_field_GB_s": 12 * nx * ny * nz / (split_ms * 1e-3) / 1e9,
               "split_field_hbm_frac": 12 * nx * ny * nz / (split_ms * 1e-3) / 1e9 / peak}
    del t, fp_buf
    line["modes_16m"] = modes16
    line["helpers_16m_per_field"] = helpers
    for mode, r in modes16.items():
        e = r["error_vs_oracle"]
        flat[f"{mode}_16m_GPoints_s"] = r["GPoints_s"]
        flat[f"{mode}_16m_hbm_frac"] = r["hbm_frac"]
        flat[f"{mode}_16m_max_rel_err"] = worst(e, "max_rel")
        flat[f"{mode}_16m_rms_rel_err"] = worst(e, "rms_rel")
        if mode in ("f64", "paired"):  # the FP64-output paths' per-point scales (strict A, monomial M)
            flat[f"{mode}_16m_max_err_over_A"] = worst(e, "max_err_over_A")
            flat[f"{mode}_16m_max_err_over_M"] = worst(e, "max_err_over_M")
        flat[f"{mode}_16m_energy_residual"] = r["energy_residual"]
    flat["split_field_16m_us_per_field"] = helpers["split_field_us"]
    flat["split_field_16m_hbm_frac"] = helpers["split_field_hbm_frac"]
    # 1024 x 1024 x 128 with i.i.d. winds and uniform 20 m levels
    cfg = synth.config_134m_iid()
    nx3, ny3, nz3 = cfg["nx"], cfg["ny"], cfg["nz"]
    f3 = cfg["fields"]()
    co3 = oracle.coeffs(nz3, cfg["dx"], cfg["dy"], cfg["dz"])
    ref3, ab3 = oracle.advect(*f3, co3, nx3, ny3, want_abs=True, nthreads=cores)
    mono3 = oracle.monomial_scale(*f3, co3, nx3, ny3, nthreads=cores)
    c3 = pw.make_coeffs(nz3, cfg["dx"], cfg["dy"], cfg["dz"]).to_device()
    modes134 = {}
    for mode in ("f64", "paired", "split"):
        fin, table = make_inputs(torch, pw, mode, f3, c3, nx3, ny3)
        res, fout = measure_mode(torch, pw, mode, fin, table, c3, nx3, ny3, nz3, max(5, steps // 4), peak)
        res["error_vs_oracle"] = error_stats([t.double().cpu().numpy() for t in fout], ref3, ab3, nx3, ny3, mono3)
        modes134[mode] = res
        del fin, fout
        torch.cuda.empty_cache()
    # the split path including the split of the three FP64 fields it needs
    pts3 = nx3 * ny3 * nz3
    d64 = [pw.field_from_numpy(a, nx3) for a in f3]
    fp3 = [pw.empty_field(nx3, ny3, nz3, torch.float32) for _ in range(3)]
    mean3 = [torch.empty(nz3, dtype=torch.float64, device="cuda") for _ in range(3)]
    split3_ms = time_launches(torch, lambda _: [pw.split_field(a, nx3, ny3, out=b, mean=m)
                                                for a, b, m in zip(d64, fp3, mean3)], max(5, steps // 4), 3, 1)
    del d64, fp3
    torch.cuda.empty_cache()
    with_split = modes134["split"]["ms"] + split3_ms
    line["modes_134m"] = modes134
    for mode, r in modes134.items():
        e = r["error_vs_oracle"]
        flat[f"{mode}_134m_GPoints_s"] = r["GPoints_s"]
        flat[f"{mode}_134m_hbm_frac"] = r["hbm_frac"]
        flat[f"{mode}_134m_max_rel_err"] = worst(e, "max_rel")
        flat[f"{mode}_134m_rms_rel_err"] = worst(e, "rms_rel")
        if mode in ("f64", "paired"):
            flat[f"{mode}_134m_max_err_over_A"] = worst(e, "max_err_over_A")
            flat[f"{mode}_134m_max_err_over_M"] = worst(e, "max_err_over_M")
    flat["split_134m_incl_split_field_GPoints_s"] = pts3 / (with_split * 1e-3) / 1e9
    flat["fp32_split_speedup_over_f64_134m"] = modes134["split"]["GPoints_s"] / modes134["f64"]["GPoints_s"]
    flat["fp32_split_incl_split_field_speedup_over_f64_134m"] = modes134["f64"]["ms"] / with_split
    flat["paired_speedup_over_f64_134m"] = modes134["paired"]["GPoints_s"] / modes134["f64"]["GPoints_s"]
    del f3, ref3, ab3, mono3
    line["batched_96"] = batched_extra(torch, pw, peak)
    for mode, r in line["batched_96"].items():
        if isinstance(r, dict):
            flat[f"batched96_{mode}_GPoints_s"] = r["GPoints_s"]
            flat[f"batched96_{mode}_hbm_frac"] = r["hbm_frac"]
    line["adjoint_256"] = adjoint_extra(torch, pw, peak)
    for mode in ("f64", "paired", "f32"):
        r = line["adjoint_256"][f"adjoint_{mode}"]
        flat[f"adjoint256_{mode}_GPoints_s"] = r["GPoints_s"]
        flat[f"adjoint256_{mode}_hbm_frac"] = r["hbm_frac"]
    line["c1_64cubed_graph"] = c1_extra(torch, pw, oracle)
    line.update(flat)


def c1_extra(torch, pw, oracle):
    """64 x 64 x 64 i.i.d. winds, uniform 20 m levels (the correctness
    configuration; its ~13 MB working set stays in L2), each mode timed as
    a CUDA graph of 100 launches, with errors against the FP64 oracle."""
    cfg = synth.config_small_iid()
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    fields = cfg["fields"]()
    co = oracle.coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"])
    ref, ab = oracle.advect(*fields, co, nx, ny, want_abs=True, nthreads=os.cpu_count() or 1)
    c = pw.make_coeffs(nz, cfg["dx"], cfg["dy"], cfg["dz"]).to_device()
    pts = nx * ny * nz
    out = {"working_set": "L2-resident (no flush between launches)", "launches_per_graph": 100}
    for mode in ("f64", "paired", "f32", "split"):
        f, table = make_inputs(torch, pw, mode, fields, c, nx, ny)
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


def batched_extra(torch, pw, peak):
    """96 independent domains (x, y in 32..384, z in 32..128, seed 4,
    stretched grids) in one persistent launch per evaluation: autotuned
    variant, and a CUDA graph of 50 evaluations, for every arithmetic."""
    from paper_2107_13500_gb300 import autotune
    sizes = synth.batched_domain_sizes(96, seed=4)
    pts = sum(a * b * c for a, b, c in sizes)
    out = {"domains": 96, "points": pts}
    for mode in ("f64", "paired", "f32", "split"):
        dt = torch.float64 if mode in ("f64", "paired") else torch.float32
        gen = torch.Generator(device="cuda").manual_seed(4)
        doms = []
        for nx, ny, nz in sizes:
            c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_stretched(nz)).to_device()
            f = [pw.empty_field(nx, ny, nz, dt) for _ in range(3)]
            for t in f:
                t.uniform_(-10, 10, generator=gen)
            d = dict(u=f[0], v=f[1], w=f[2], nx=nx, ny=ny, coeffs=c)
            if mode == "split":
                d["split_table"] = torch.from_numpy(pw.make_split_table(c, *([np.zeros(nz)] * 3))).cuda()
            doms.append(d)
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
                     "hbm_frac": bpp * pts / (ms * 1e-3) / 1e9 / peak,
                     "graph50_ms_per_eval": graph_ms, "graph50_GPoints_s": pts / (graph_ms * 1e-3) / 1e9}
        del doms, b, g
        torch.cuda.empty_cache()
    return out


def adjoint_extra(torch, pw, peak):
    """256 x 256 x 64 with the small configuration's winds: adjoint kernel
    time and HBM fraction (native FP64, paired FP32, FP32; algorithmic bytes
    per cell: u, v, w and three cotangents read, three gradients written)
    and a 20-step forward-Euler rollout (dt = 0.5 s) differentiated with
    checkpoints every 5 steps (native FP64 and paired forward/adjoint)."""
    from paper_2107_13500_gb300 import autograd as pa
    nx, ny, nz = 256, 256, 64
    pts = nx * ny * nz
    u, v, w = synth.fields_iid(nx, ny, nz, seed=1)
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    out = {"points": pts, "bytes_per_cell": ADJOINT_BYTES}
    for mode, dt in (("f64", torch.float64), ("paired", torch.float64), ("f32", torch.float32)):
        x = [pw.field_from_numpy(a, nx, dt) for a in (u, v, w)]
        g = [pw.field_like(x[0]).uniform_(-1, 1) for _ in range(3)]
        res = tuple(pw.field_like(x[0]) for _ in range(3))
        ms = time_launches(torch, lambda _: pw.advect_adjoint(*x, c, nx, ny, *g, mode=mode, out=res), 50, 3, 1)
        gbs = ADJOINT_BYTES[mode] * pts / (ms * 1e-3) / 1e9
        out[f"adjoint_{mode}"] = {"ms": ms, "GPoints_s": pts / (ms * 1e-3) / 1e9, "GB_s": gbs, "hbm_frac": gbs / peak}
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
