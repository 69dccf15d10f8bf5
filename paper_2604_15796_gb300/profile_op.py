"""Time the Lippmann-Schwinger operator passes (row FFT, column convolution,
inverse row FFT) or the Jacobian contractions on a synthetic batch, for
kernel tuning and ncu captures.

    python -m paper_2604_15796_gb300.profile_op --grid 256 --rhs 256 --reps 3
    python -m paper_2604_15796_gb300.profile_op --jac --grid 256 --rhs 128 --nfreq 2
    python -m paper_2604_15796_gb300.profile_op --dim3 --grid 160 --depth 128 --rhs 32
    python -m paper_2604_15796_gb300.profile_op --solve --dim3 --grid 160 --depth 128 --rhs 16

Solve mode (--solve): ``reps`` forward solves of the ``rhs`` right-hand sides
(every BiCGSTAB pass mode: INIT, ITER, S, V, T).

Operator mode: a context with ``rhs`` array elements at one frequency (one
operator application processes ``rhs`` right-hand sides) applies
A = I - K diag(m) ``reps`` times.  Jacobian mode (--jac): ``rhs`` elements at
``nfreq`` frequencies; one forward solve, then ``reps`` products J a and
J^H b.  Prints the per-kernel-class device times measured with CUDA events
(profiling mode) as JSON.
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
    ap.add_argument("--jac", action="store_true")
    ap.add_argument("--solve", action="store_true",
                    help="time forward solves (every BiCGSTAB pass mode) instead of A v")
    ap.add_argument("--nfreq", type=int, default=2)
    ap.add_argument("--cuda-core-jacobian", action="store_true")
    ap.add_argument("--dim3", action="store_true",
                    help="3-D grid of depth x grid x grid voxels (0.2 mm)")
    ap.add_argument("--no-col-tma", action="store_true",
                    help="column passes with plain loads instead of TMA staging")
    ap.add_argument("--no-row-l2-prefetch", action="store_true",
                    help="row passes without the L2 prefetch of their next work item")
    ap.add_argument("--no-jac-tma", action="store_true",
                    help="tensor-core contractions load their operand tiles with cp.async")
    ap.add_argument("--no-col-pairs", action="store_true",
                    help="the convolution computes one column per thread instead of two")
    ap.add_argument("--no-row-stage", action="store_true",
                    help="the forward row pass loads its rows from global memory instead "
                         "of staging them in shared memory")
    args = ap.parse_args()
    nz = args.depth or args.grid
    shape = (nz, args.grid, args.grid) if args.dim3 else (nz, args.grid)
    h = 0.2e-3 if args.dim3 else 0.1e-3
    freqs = np.linspace(0.5e6, args.freq, args.nfreq) if args.jac else np.array([args.freq])
    w = phantoms.tissue_phantom(shape, h, args.rhs, min(0.2e-3, args.grid * h / args.rhs),
                                freqs, 5, inclusions=[1520.0, 1580.0])
    prec = libfwi.FWI_FP64 if args.fp64 else libfwi.FWI_MIXED
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = libfwi.Context(w.shape, w.h, w.c0, w.elem, w.freqs, precision=prec,
                             stream=stream)
        if args.no_col_tma:
            ctx.set_col_tma(False)
        if args.no_row_l2_prefetch:
            ctx.set_row_l2_prefetch(False)
        if args.no_row_stage:
            ctx.set_row_stage(False)
        if args.no_col_pairs:
            ctx.set_col_pairs(False)
        m = ctx.contrast_from_sos(torch.from_numpy(np.ascontiguousarray(w.sos)).cuda())
        if args.jac:
            if args.cuda_core_jacobian:
                ctx.set_jac_tensor_cores(False)
            if args.no_jac_tma:
                ctx.set_jac_tma(False)
            ctx.forward(m)
            a = torch.from_numpy(phantoms.complex_normal(shape, 3)).cuda()
            y = ctx.jac_forward(a)
            ctx.jac_adjoint(y)  # warm-up
            torch.cuda.synchronize()
            ctx.reset_stats()
            ctx.set_profiling(True)
            for _ in range(args.reps):
                y = ctx.jac_forward(a)
                ctx.jac_adjoint(y)
            torch.cuda.synchronize()
            _, ks = ctx.stats()
            ctx.set_profiling(False)
            ctx.close()
            report(shape, args.rhs * args.nfreq, ks)
            return
        if args.solve:
            ctx.forward(m)  # warm-up
            torch.cuda.synchronize()
            ctx.reset_stats()
            ctx.set_profiling(True)
            for _ in range(args.reps):
                ctx.forward(m)
            torch.cuda.synchronize()
            _, ks = ctx.stats()
            ctx.set_profiling(False)
            ctx.close()
            report(shape, args.rhs, ks)
            return
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
    report(shape, args.rhs, ks)


def report(shape, rhs, ks):
    out = {}
    for name, k in ks.items():
        if k["launches"]:
            ms = k["ms"] / k["launches"]
            out[name] = {"ms_per_launch": ms, "bytes_per_launch": k["bytes"] / k["launches"],
                         "gbs": k["bytes"] / k["launches"] / (ms * 1e6) if k["bytes"] else None,
                         "tflops": k["flops"] / k["launches"] / (ms * 1e9) if k["flops"] else None}
    print(json.dumps({"grid": list(shape), "rhs": rhs, "passes": out}))


if __name__ == "__main__":
    main()
