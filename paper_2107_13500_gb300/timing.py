"""Time one library call on the GPU: the forward (`pw_advect`) or the adjoint
(`pw_advect_adjoint`) of one arithmetic mode on a seeded synthetic domain.

    python -m paper_2107_13500_gb300.timing forward paired 512 512 64
    python -m paper_2107_13500_gb300.timing adjoint paired 256 256 64 --reps 5

Inputs are i.i.d. U[-10, 10] winds (synth.fields_iid, seed 1) on a uniform
20 m grid with dx = dy = 50 m; the adjoint's cotangents are U[-1, 1]. The
call is repeated `--warmup` times, then `--reps` times between two CUDA
events on the current stream; the line printed gives the mean time per call,
GPoints/s and the library's device status (0 = every bounded wait completed).
Inputs stay resident and are not flushed from L2 between calls: use bench.py
for the timing protocol of the reported figures.
"""
from __future__ import annotations

import argparse

from . import build, pw, synth


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("op", choices=["forward", "adjoint"])
    p.add_argument("mode", choices=["f64", "paired", "f32", "split"])
    p.add_argument("nx", type=int)
    p.add_argument("ny", type=int)
    p.add_argument("nz", type=int)
    p.add_argument("--reps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    args = p.parse_args(argv)
    import numpy as np
    import torch

    build.build()
    nx, ny, nz = args.nx, args.ny, args.nz
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
    pts = nx * ny * nz
    print(f"{args.op} {args.mode} {nx}x{ny}x{nz}: {ms * 1e3:.1f} us per call, {pts / ms / 1e6:.2f} GPoints/s, "
          f"device status {pw.device_status()}")


if __name__ == "__main__":
    main()
