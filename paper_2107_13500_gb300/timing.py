"""Time one library call on the GPU: the forward (`pw_advect`), the adjoint
(`pw_advect_adjoint`), the batched forward (`pw_advect_batched`) or the
mean+perturbation split of one field (`pw_split_field`) on seeded synthetic
inputs.

    python -m paper_2107_13500_gb300.timing forward paired 512 512 64
    python -m paper_2107_13500_gb300.timing adjoint paired 256 256 64 --reps 5
    python -m paper_2107_13500_gb300.timing batched f32 --variant 3
    python -m paper_2107_13500_gb300.timing split_field f64 512 512 64

Single domains have i.i.d. U[-10, 10] winds (synth.fields_iid, seed 1) on a
uniform 20 m grid with dx = dy = 50 m; the adjoint's cotangents are U[-1, 1].
The batch is `--domains` (default 96) domains with x, y in 32..384 and z in
32..128 (synth.batched_domain_sizes, seed 4), stretched grids and U[-10, 10]
winds, run as one persistent launch of tile variant `--variant`. The call is
repeated `--warmup` times, then `--reps` times between two CUDA events on
the current stream; the line printed gives the mean time per call,
GPoints/s and the library's device status (0 = every bounded wait
completed). Inputs stay resident and are not flushed from L2 between calls:
use bench.py for the timing protocol of the reported figures.
"""
from __future__ import annotations

import argparse

from . import build, pw, synth


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("op", choices=["forward", "adjoint", "batched", "split_field"])
    p.add_argument("mode", choices=["f64", "paired", "f32", "split"])
    p.add_argument("nx", type=int, nargs="?")
    p.add_argument("ny", type=int, nargs="?")
    p.add_argument("nz", type=int, nargs="?")
    p.add_argument("--variant", type=int, default=0, help="batched: tile/pipeline variant")
    p.add_argument("--domains", type=int, default=96, help="batched: number of domains")
    p.add_argument("--reps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    args = p.parse_args(argv)
    import numpy as np
    import torch

    build.build()
    if args.op == "batched":
        if args.mode not in ("paired", "f32"):
            raise SystemExit("the batched launch takes paired or f32 domains")
        dt = torch.float64 if args.mode == "paired" else torch.float32
        gen = torch.Generator(device="cuda")
        gen.manual_seed(4)
        doms = []
        for bx, by, bz in synth.batched_domain_sizes(args.domains, seed=4):
            c = pw.make_coeffs(bz, 50.0, 50.0, synth.dz_stretched(bz)).to_device()
            f = [pw.empty_field(bx, by, bz, dt) for _ in range(3)]
            for t in f:
                t.uniform_(-10, 10, generator=gen)
            doms.append(dict(u=f[0], v=f[1], w=f[2], nx=bx, ny=by, coeffs=c))
        batch = pw.Batch(doms, args.mode, args.variant)
        pts = sum(d["nx"] * d["ny"] * d["u"].shape[0] for d in doms)
        label = f"{args.domains} domains, {pts} points, variant {args.variant}"
        _run(args, batch.run, pts, label)
        return
    if args.nz is None:
        raise SystemExit("nx ny nz are required")
    nx, ny, nz = args.nx, args.ny, args.nz
    label = f"{nx}x{ny}x{nz}"
    if args.op == "split_field":
        f = pw.field_from_numpy(synth.fields_iid(nx, ny, nz, seed=1)[0], nx, torch.float64)
        pert = pw.empty_field(nx, ny, nz, torch.float32)
        mean = torch.empty(nz, dtype=torch.float64, device="cuda")
        _run(args, lambda: pw.split_field(f, nx, ny, out=pert, mean=mean), nx * ny * nz, label)
        return
    if args.op == "adjoint" and args.mode == "split":
        raise SystemExit("the mean+perturbation form has no adjoint")
    dt = torch.float32 if args.mode in ("f32", "split") else torch.float64
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    x = [pw.field_from_numpy(a, nx, dt) for a in synth.fields_iid(nx, ny, nz, seed=1)]
    if args.op == "forward":
        table = None
        if args.mode in ("f32", "split"):
            table = torch.from_numpy(pw.make_split_table(c, *([np.zeros(nz)] * 3))).cuda()
        out = tuple(pw.field_like(x[0]) for _ in range(3))

        def call():
            pw.advect(*x, c, nx, ny, mode=args.mode, out=out, split_table=table)
    else:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(2)
        g = [pw.field_like(x[0]).uniform_(-1, 1, generator=gen) for _ in range(3)]
        out = tuple(pw.field_like(x[0]) for _ in range(3))

        def call():
            pw.advect_adjoint(*x, c, nx, ny, *g, mode=args.mode, out=out)

    _run(args, call, nx * ny * nz, label)


def _run(args, call, pts, label):
    import torch

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    print(f"{args.op} {args.mode} {label}: {ms * 1e3:.1f} us per call, {pts / ms / 1e6:.2f} GPoints/s, "
          f"device status {pw.device_status()}")


if __name__ == "__main__":
    main()
