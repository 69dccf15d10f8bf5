"""Time the Lippmann-Schwinger operator passes (row FFT, column convolution,
inverse row FFT) on a synthetic batch, for kernel tuning and ncu captures.

    python -m paper_2604_15796_gb300.profile_op --grid 256 --rhs 256 --reps 3

Creates a context with ``rhs`` array elements at one frequency (so that one
operator application processes ``rhs`` right-hand sides), applies
A = I - K diag(m) ``reps`` times and prints the per-pass device times
measured with CUDA events (profiling mode) as JSON.
"""
import argparse
import json

import numpy as np


def main():
    import torch
    from paper_2604_15796_gb300 import libfwi, phantoms

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--depth", type=int, default=0, help="Nz (default: grid)")
    ap.add_argument("--rhs", type=int, default=256)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--freq", type=float, default=3e6)
    ap.add_argument("--fp64", action="store_true")
    args = ap.parse_args()
    nz = args.depth or args.grid
    shape = (nz, args.grid)
    h = 0.1e-3
    w = phantoms.tissue_phantom(shape, h, args.rhs, min(0.2e-3, args.grid * h / args.rhs),
                                np.array([args.freq]), 5, inclusions=[1520.0, 1580.0])
    prec = libfwi.FWI_FP64 if args.fp64 else libfwi.FWI_MIXED
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = libfwi.Context(w.shape, w.h, w.c0, w.elem, w.freqs, precision=prec,
                             stream=stream)
        m = ctx.contrast_from_sos(torch.from_numpy(np.ascontiguousarray(w.sos)).cuda())
        dt = torch.complex128 if args.fp64 else torch.complex64
        v = torch.from_numpy(phantoms.complex_normal((args.rhs,) + shape, 3)).to(
            device="cuda", dtype=dt)
        ctx.apply("A", v, 0, m)  # warm-up
        torch.cuda.synchronize()
        ctx.reset_stats()
        ctx.set_profiling(True)
        for _ in range(args.reps):
            ctx.apply("A", v, 0, m)
        torch.cuda.synchronize()
        _, ks = ctx.stats()
        ctx.set_profiling(False)
        ctx.close()
    out = {}
    for name, k in ks.items():
        if k["launches"]:
            ms = k["ms"] / k["launches"]
            out[name] = {"ms_per_launch": ms,
                         "gbs": k["bytes"] / k["launches"] / (ms * 1e6) if k["bytes"] else None}
    print(json.dumps({"grid": list(shape), "rhs": args.rhs, "passes": out}))


if __name__ == "__main__":
    main()
