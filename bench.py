"""Benchmark of the FWI hot path on one GB300 (per process).

One step = one pass of the whole hot path over the batch of the workload:
fwi_gradient (forward BiCGSTAB solves for every transmit x frequency, data,
misfit, adjoint sources, adjoint solves, gradient assembly) followed by
fwi_admm_tv_step (Gauss-Newton CG with implicit Jacobian products, isotropic
shrink, dual update, SoS map).  Every step starts from the same iterate
(m_k, g_k, u_k) so that all steps do the same work.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload volume3d|thyroid256|large512|disc64|planewave2d|elev3d|serving]

The default workload is the largest single-GPU configuration, the 3-D
single-sided volume (160 x 160 x 128 voxels, 128 elements x 4 frequencies);
after its timed region the line also carries a short serving stream's
p50/p99 reconstruction latency (--serving-requests, 0 for none).

Prints one JSON line (rank 0).  Multi-GPU: independent replicas, one per
rank (the solves shard by right-hand side with no exchange step).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS solves/s & gradient evals/s at rel err <=1e-4; p50/p99 recon latency"
UNIT = "RHS solves/s"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name):
    from paper_2604_15796_gb300 import phantoms
    return {"thyroid256": phantoms.thyroid_256, "large512": phantoms.large_512,
            "volume3d": phantoms.volume_3d, "disc64": phantoms.disc_phantom,
            "planewave2d": phantoms.planewave_2d, "elev3d": phantoms.elevation_3d}[name]()


def describe(w):
    grid = "x".join(str(s) for s in reversed(w.shape))
    tx = w.meta.get("tx_angles")
    txs = "" if tx is None else (f", {len(tx)} plane-wave transmits synthesised from the "
                                 f"{w.n_elem} element solves")
    if w.meta.get("elem_length"):
        txs += f", line elements of {w.meta['elem_length'] * 1e3:.0f} mm elevation"
    return (f"{w.name}: {grid} grid, h={w.h * 1e3:.2f} mm, {w.n_elem} elements x "
            f"{w.n_freq} freqs ({w.n_rhs} RHS){txs}, per step 1 forward + 1 adjoint BiCGSTAB "
            f"solve per RHS + data + gradient + ADMM-TV step (n_cg=10)")


# the sources each kernel class is compiled from: the FFT operator passes
# (row_*, col_*) and the pixel contractions (everything else)
KERNEL_SOURCES = {"operator": ("fft_core.cuh", "lsop_kernels.cuh", "col_pair.cuh", "common.cuh",
                               "lsop_f32.cu", "tc.cuh"),
                  "contraction": ("common.cuh", "jac.cu", "jac_tc.cu", "tc.cuh")}


def kernel_source_hash(kernel="col_conv"):
    """Hash of the sources of ``kernel``'s class (a recorded ncu figure is
    used only while they are unchanged)."""
    cls = "operator" if kernel.startswith(("row_", "col_")) else "contraction"
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[cls]:
        with open(os.path.join(ROOT, "paper_2604_15796_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def recorded_traffic(kernel, wname, path=None):
    """(DRAM bytes, algorithmic bytes) of one ncu-captured launch of a kernel
    class on a workload, recorded in profiles/traffic.json, if the kernel's
    sources have not changed since the capture (hash match); else None."""
    path = path or TRAFFIC_PATH
    if not os.path.exists(path):
        return None
    with open(path) as f:
        recs = json.load(f).get("records", [])
    for r in recs:
        if r.get("kernel") == kernel and r.get("workload") == wname and \
                r.get("src") == kernel_source_hash(kernel):
            return float(r["dram_bytes"]), float(r["algorithmic_bytes"])
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=10)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def oracle_solves_per_s(w, budget_s=15.0, seed=0, keep=0):
    """FP64 oracle (numpy/scipy, all host cores) on a bounded sample of the
    workload: BiCGSTAB solves (tol 1e-10) of transmit/frequency pairs drawn
    from the workload at the benchmark's iterate m = 0.8 m_true, until the
    time budget is spent.  Only the solves are timed (the right-hand sides,
    like the device's incident fields, are setup).  The first ``keep``
    solutions and their data rows are returned for the accuracy check of
    the GPU result.  Line elements: the oracle's element quadrature takes
    about a minute per element at full size, so the solves take point-source
    right-hand sides (the same operator and iteration) and no solution is
    kept.  Returns (rate, solves, solve seconds, kept, line elements)."""
    import oracle
    from oracle import inverse, model, operator
    line = float(w.meta.get("elem_length", 0.0)) > 0.0
    extra = {"elem_length": 0.0 if line else float(w.meta.get("elem_length", 0.0))}
    if line:
        keep = 0
    prob = oracle.Problem(tuple(w.shape), w.h, w.c0, w.elem, np.asarray(w.freqs), dict(extra))
    m = 0.8 * model.contrast_from_sos(w.sos, w.c0)
    rng = np.random.default_rng(seed)
    tx = w.meta.get("tx_angles")
    specs = {}
    kept = []
    n, t0, t_solve = 0, time.perf_counter(), 0.0
    while True:
        l = int(rng.integers(0, w.n_freq))
        e = int(rng.integers(0, w.n_elem if tx is None else len(tx)))
        if l not in specs:
            specs[l] = operator.kernel_spectrum(prob, l)
        wrow = None
        if tx is None:
            sub = oracle.Problem(prob.shape, prob.h, prob.c0, prob.elem[[e]],
                                 np.asarray([w.freqs[l]]), dict(extra))
            b = operator.incident_fields(sub)[0, 0]
        else:
            # plane-wave transmit e, solved directly from its incident field
            sub = oracle.Problem(prob.shape, prob.h, prob.c0, prob.elem, np.asarray([w.freqs[l]]),
                                 dict(extra))
            wl = model.plane_wave_weights(sub, [tx[e]])
            b = operator.transmit_incident_fields(sub, wl)[0, 0]
            wrow = wl[0, 0]
        spec = specs[l]
        ts = time.perf_counter()
        x, _, _ = operator.bicgstab(lambda v: operator.apply_A(v.reshape(prob.shape), m, prob,
                                                              l, spec).ravel(), b.ravel(), 1e-10)
        t_solve += time.perf_counter() - ts
        if len(kept) < keep:
            subr = oracle.Problem(prob.shape, prob.h, prob.c0, prob.elem, np.asarray([w.freqs[l]]),
                                  dict(extra))
            row = inverse.forward_data(m, x.reshape((1, 1) + prob.shape), subr)[0, 0]
            kept.append((l, e, x.reshape(prob.shape), row, wrow))
        n += 1
        if time.perf_counter() - t0 > budget_s and n >= keep:
            break
    return n / t_solve, n, t_solve, kept, line


def run_reference(args, rank):
    """Reference arm: the FP64 oracle, timed on the host cores."""
    if rank != 0:
        return None
    w = workload(args.workload)
    per_step = []
    solves = 0
    for i in range(args.warmup + args.steps):
        rate, n, dt, _, _ = oracle_solves_per_s(w, budget_s=args.ref_step_s, seed=i)
        if i >= args.warmup:
            per_step.append(dt)
            solves += n
    total = sum(per_step)
    value = solves / total
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (FP64 oracle)",
            "data": "synthetic", "config": {"workload": describe(w)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{solves} FP64 BiCGSTAB solves (tol 1e-10) of random "
                                       f"transmit/frequency pairs of the workload, "
                                       f"~{args.ref_step_s:.0f} s per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    return line


def replicas_aggregate(ms_local, units_local, world, device):
    """Whole-job figures of N independent replicas (one process per GPU, no
    data exchange): the slowest rank's timed-region duration and the units
    (RHS solves) all ranks processed."""
    if world <= 1:
        return ms_local, units_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
def run_ours(args, rank, world, samples):
    import torch
    from paper_2604_15796_gb300 import libfwi

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    stream = torch.cuda.Stream()
    peaks, peak_kind = load_peaks()
    with torch.cuda.stream(stream):
        ctx = libfwi.Context(w.shape, w.h, w.c0, w.elem, w.freqs, tol=1e-6, stream=stream,
                             tx_angles=w.meta.get("tx_angles"),
                             elem_length=float(w.meta.get("elem_length", 0.0)),
                             max_batch=args.max_batch)
        if args.cuda_core_jacobian:
            ctx.set_jac_tensor_cores(False)
        if args.chains is not None:
            ctx.set_overlap(args.chains == 2)
        if args.no_col_tma:
            ctx.set_col_tma(False)
        if args.no_row_l2_prefetch:
            ctx.set_row_l2_prefetch(False)
        if args.no_spectrum_stage:
            ctx.set_col_spectrum_stage(False)
        if args.no_jac_tma:
            ctx.set_jac_tma(False)
        if args.no_row_stage:
            ctx.set_row_stage(False)
        if args.no_col_pairs:
            ctx.set_col_pairs(False)
        tuning = ctx.tuning()
        c128 = torch.complex128
        sos_true = torch.from_numpy(np.ascontiguousarray(w.sos)).cuda()
        m_true = ctx.contrast_from_sos(sos_true)
        m0 = (0.8 * m_true).contiguous()
        # observed data: forward data of the true model + 2% complex noise
        d_obs = ctx.empty_data()
        ctx.forward(m_true, data=d_obs)
        from paper_2604_15796_gb300 import phantoms
        noise = phantoms.complex_normal(tuple(d_obs.shape), 4242)
        dn = float(torch.linalg.vector_norm(d_obs).item())
        scale = 0.02 * dn / np.sqrt(2.0 * d_obs.numel())
        d_obs += torch.from_numpy(noise * scale).to(device="cuda", dtype=d_obs.dtype)
        # ADMM parameters scaled to ||J^H J|| (power iteration at m0)
        ctx.forward(m0)
        v = torch.from_numpy(phantoms.complex_normal(w.shape, 7)).cuda()
        nrm = 1.0
        for _ in range(4):
            v = v / torch.linalg.vector_norm(v)
            v = ctx.jac_adjoint(ctx.jac_forward(v))
            nrm = float(torch.linalg.vector_norm(v).item())
        params = dict(lam=1e-4 * nrm, rho=1e-2 * nrm, gamma=1e-5 * nrm, n_cg=10)
        g0, u0 = ctx.admm_init(m0)  # g0 = nabla m0, u0 = 0 (Algorithm 1)
        m0h = m0.cpu().numpy()
        m = torch.empty_like(m0)
        g = torch.empty_like(g0)
        u = torch.empty_like(u0)
        grad = torch.empty(w.shape, dtype=c128, device="cuda")
        sos = torch.empty(w.shape, dtype=torch.float64, device="cuda")
        reports = []

        def step():
            m.copy_(m0)
            g.copy_(g0)
            u.copy_(u0)
            mis, rf, ra = ctx.gradient(m, d_obs, grad)
            ctx.admm_tv_step(m, g, u, grad, sos=sos, **params)
            reports.append((mis, rf.max_iters, ra.max_iters, float(np.mean(rf.iters)),
                            float(np.mean(ra.iters))))

        for _ in range(args.warmup):
            step()
        reports.clear()
        launches0, _ = ctx.stats()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1)
        launches1, _ = ctx.stats()
        ms, solves = replicas_aggregate(ms, 2.0 * w.n_rhs * args.steps, world, "cuda")
        value = solves / (ms / 1e3)

        # ---- end to end through the C ABI with host buffers ----
        e2e = None
        if not args.no_e2e:
            m_h = torch.from_numpy(m0h).pin_memory()
            d_h = d_obs.cpu().pin_memory()
            g_h = g0.cpu().pin_memory()
            u_h = u0.cpu().pin_memory()
            sos_h = torch.empty(w.shape, dtype=torch.float64).pin_memory()
            mo_h = torch.empty_like(m_h).pin_memory()
            d_dev = torch.empty_like(d_obs)
            ke = max(3, min(args.steps, 20))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(ke):
                m.copy_(m_h, non_blocking=True)
                d_dev.copy_(d_h, non_blocking=True)
                g.copy_(g_h, non_blocking=True)
                u.copy_(u_h, non_blocking=True)
                ctx.gradient(m, d_dev, grad)
                ctx.admm_tv_step(m, g, u, grad, sos=sos, **params)
                sos_h.copy_(sos, non_blocking=True)
                mo_h.copy_(m, non_blocking=True)
                stream.synchronize()
            dt = time.perf_counter() - t0
            h2d = (m_h.numel() * 16 + d_h.numel() * d_h.element_size()
                   + (g_h.numel() + u_h.numel()) * 16)
            d2h = sos_h.numel() * 8 + mo_h.numel() * 16
            e2e = {"value": 2.0 * w.n_rhs * ke * world / dt, "unit": UNIT,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "steps": ke, "ms_per_step": 1e3 * dt / ke}

        # ---- comparator: plain unbatched per-RHS FP64 path (same kernels,
        # complex128 fields, one right-hand side per launch) on a subset of
        # the array (every 8th element, all frequencies) ----
        comp = None
        if not args.no_comparator:
            sub = np.ascontiguousarray(w.elem[::8])
            c64 = libfwi.Context(w.shape, w.h, w.c0, sub, w.freqs, precision=libfwi.FWI_FP64,
                                 tol=1e-6, max_batch=1, stream=stream)
            c64.forward(m0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = c64.forward(m0)
            torch.cuda.synchronize()
            dtc = time.perf_counter() - t0
            comp = {"value": c64.n_rhs / dtc, "unit": UNIT, "rhs": c64.n_rhs,
                    "kind": "FP64 fields, one RHS per launch (max_batch=1), same operator",
                    "mean_iters": float(np.mean(rep.iters))}
            comp["speedup_solves_per_s"] = value / comp["value"]
            c64.close()

        # ---- comparator: the same matvec through batched cuFFT (library
        # context for the three fused passes) ----
        cufft = None
        if not args.no_comparator:
            cufft = cufft_matvec_comparator(ctx, w, m0, stream)

        # ---- live per-kernel timing (CUDA events, profiling mode) ----
        ctx.reset_stats()
        ctx.set_profiling(True)
        step()
        ctx.set_profiling(False)
        _, kst = ctx.stats()
        torch.cuda.synchronize()

        # ---- sampled error against the FP64 oracle solutions of the CPU leg ----
        err = sampled_error(ctx, m0, samples) if samples else None

    tot_ms = sum(k["ms"] for k in kst.values())
    op_classes = [k for k in kst if k.startswith(("row_", "col_"))]
    dominant = max(kst, key=lambda k: kst[k]["ms"])
    tensor = bool(tuning.get("jac_tensor_cores"))
    roof = roofline(dominant, kst[dominant], peaks, peak_kind, w.name, tensor)
    rates = {k: kernel_rates(k, v, peaks, tensor) for k, v in kst.items() if v["launches"]}
    share = {k: round(v["ms"] / tot_ms, 4) for k, v in sorted(kst.items(),
                                                             key=lambda kv: -kv[1]["ms"])}
    op_ms = sum(kst[k]["ms"] for k in op_classes)
    op_bytes = sum(kst[k]["bytes"] for k in op_classes)
    its = np.array([r[1:] for r in reports])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 fields / FP64 Krylov scalars", "data": "synthetic",
        "config": {"workload": describe(w), "l2": "inputs larger than L2 (fields "
                   f"{w.n_rhs * w.n * 8 / 1e6:.0f} MB per array)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "krylov_tol": 1e-6, "admm": {k: v for k, v in params.items()},
                   "jacobian": "tensor cores (tcgen05, 3xTF32)" if tensor
                   else "CUDA cores (FP32 FMA)",
                   "krylov_chains": 2 if tuning.get("overlap_halves") else 1,
                   "tuning": {k: tuning.get(k) for k in ("row_fwd", "row_inv", "col", "col_y",
                                                         "col_tma", "col_spectrum_stage",
                                                         "jac_tma", "row_l2_prefetch",
                                                         "row_stage", "col_pairs")}},
        "gradient_evals_per_s": args.steps * world / (ms / 1e3),
        "bicgstab_iters": {"fwd_max": int(its[:, 0].max()), "adj_max": int(its[:, 1].max()),
                           "fwd_mean": float(its[:, 2].mean()),
                           "adj_mean": float(its[:, 3].mean())},
        "rel_err_vs_oracle": err,
        "roofline": roof,
        "operator_passes": {"ms": op_ms, "achieved_gbs": op_bytes / (op_ms * 1e6) if op_ms else None,
                            "frac_of_hbm": (op_bytes / (op_ms * 1e6)) / peaks["hbm_gbs"]
                            if op_ms else None},
        "kernel_time_share": share,
        "kernel_rates": rates,
        "gpu_launches": int(launches1 - launches0),
        "clocks": clk.summary(),
        "e2e": e2e,
        "comparator_fp64_unbatched": comp,
        "comparator_cufft_matvec": cufft,
    }
    ctx.close()
    return line


TENSOR_CLASSES = ("contract_pixels", "mix_jac_adjoint", "mix_adjoint_sources")


def cufft_matvec_comparator(ctx, w, m, stream, reps=5):
    """Time of one matvec A v = v - K(m v) over all N_E x N_F right-hand
    sides (Eq. 5-6, K by zero-padded FFT convolution): libfwi's three fused
    passes (fwi_apply_A per frequency) against the textbook batched route
    through cuFFT (torch.fft, C2C FP32: product with m, zero-pad to the 2^d N
    lattice, forward FFT, product with the kernel spectrum, inverse FFT,
    crop, subtract), both on the same vectors and stream.  The cuFFT route
    multiplies by a random spectrum (its time does not depend on the
    values), so only the times are compared."""
    import torch
    dim = len(w.shape)
    pshape = tuple(2 * s for s in w.shape)
    n_pad = int(np.prod(pshape))
    chunk = int(max(1, min(w.n_elem, (2 << 30) // (8 * n_pad))))  # <= 2 GB padded
    gen = torch.Generator(device="cuda").manual_seed(7)
    spec = torch.randn(pshape, dtype=torch.complex64, device="cuda", generator=gen)
    v = torch.randn((chunk,) + tuple(w.shape), dtype=torch.complex64, device="cuda",
                    generator=gen)
    m32 = m.to(torch.complex64)
    pad = torch.zeros((chunk,) + pshape, dtype=torch.complex64, device="cuda")
    crop = tuple(slice(0, s) for s in w.shape)
    axes = tuple(range(1, dim + 1))
    blocks = [(l, e0, min(chunk, w.n_elem - e0))
              for l in range(w.n_freq) for e0 in range(0, w.n_elem, chunk)]

    def ours():
        for l, _, nb in blocks:
            ctx.apply("A", v[:nb], l, m)

    def library():
        for _, _, nb in blocks:
            pad[:nb].zero_()
            pad[(slice(0, nb),) + crop].copy_(v[:nb] * m32)
            f = torch.fft.fftn(pad[:nb], dim=axes)
            f *= spec
            v[:nb] - torch.fft.ifftn(f, dim=axes)[(slice(None),) + crop]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    try:
        with torch.cuda.stream(stream):
            t_ours, t_lib = timed(ours), timed(library)
    except Exception as exc:  # e.g. a batch limit below the chunk
        return {"unavailable": str(exc).splitlines()[0]}
    finally:
        del pad
    return {"kind": "one A v over all RHS: fwi_apply_A (fused passes: 3 in 2-D, 5 in 3-D) vs torch.fft/cuFFT "
                    "C2C FP32 batched (pad, FFT, spectrum, IFFT, crop)",
            "rhs": w.n_rhs, "rhs_per_call": chunk, "libfwi_ms": t_ours, "cufft_ms": t_lib,
            "speedup": t_lib / t_ours}


def sm_count(default=152):
    """SMs of the current CUDA device (the nominal GB300 count without one)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device())
                       .multi_processor_count)
    except Exception:
        pass
    return default


def peak_table(peaks, peak_kind, sms=None):
    """Denominators: measured HBM copy bandwidth; FP32 FMA peak from the
    device's SM count and the clock; the TF32 tensor peak from the measured
    bf16 GEMM peak and the nominal tf32/bf16 ratio (1/2), divided by the
    three TF32 products of one FP32 product (3xTF32)."""
    mhz = peaks.get("sm_max_mhz", 2070.0)
    sms = sm_count() if sms is None else sms
    return {
        "hbm": (peaks["hbm_gbs"], "GB/s", f"{peak_kind} hbm_gbs"),
        "alu": (sms * 128 * 2 * mhz * 1e6 / 1e12, "TFLOP/s",
                f"{sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"),
        "tensor": (peaks["bf16_tflops"] * 0.5 / 3.0, "TFLOP/s",
                   f"{peak_kind} bf16_tflops {peaks['bf16_tflops']:.0f} x 1/2 (tf32/bf16 nominal)"
                   " / 3 (3xTF32 products per FP32 product)"),
    }


def bound_of(name, k, tensor):
    """The roofline a kernel class is measured against: the pixel
    contractions run on the tensor cores (or FP32 FMA without them); the
    FFT operator passes (row and column) and the vector kernels stream
    their algorithmic bytes through HBM (the column passes also report
    their nominal FFT flop rate)."""
    if name in TENSOR_CLASSES:
        return "tensor" if tensor else "alu"
    if k["bytes"] > 0:
        return "hbm"
    return "alu" if k["flops"] > 0 else None


def kernel_rates(name, k, peaks, tensor):
    tab = peak_table(peaks, "measured")
    avg_ms = k["ms"] / k["launches"]
    out = {"ms_per_launch": round(avg_ms, 4), "launches": k["launches"]}
    if k["bytes"] > 0:
        gbs = k["bytes"] / k["launches"] / (avg_ms * 1e6)
        out["gbs"] = round(gbs, 1)
        out["hbm_frac"] = round(gbs / tab["hbm"][0], 3)
    if k["flops"] > 0:
        tf = k["flops"] / k["launches"] / (avg_ms * 1e9)
        out["tflops"] = round(tf, 2)
        b = bound_of(name, k, tensor)
        if b in ("alu", "tensor"):
            out[b + "_frac"] = round(tf / tab[b][0], 3)
    return out


def roofline(name, k, peaks, peak_kind, wname, tensor):
    avg_ms = k["ms"] / k["launches"]
    rec = recorded_traffic(name, wname)
    bound = bound_of(name, k, tensor) or "hbm"
    peak, unit, src = peak_table(peaks, peak_kind)[bound]
    if bound == "hbm":
        achieved = k["bytes"] / k["launches"] / (avg_ms * 1e6)
    else:
        achieved = k["flops"] / k["launches"] / (avg_ms * 1e9)
    out = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
           "frac": achieved / peak, "peak_source": src}
    if bound != "hbm" and k["bytes"] > 0:
        gbs = k["bytes"] / k["launches"] / (avg_ms * 1e6)
        out["hbm_gbs_at_algorithmic_bytes"] = gbs
        out["hbm_frac"] = gbs / peaks["hbm_gbs"]
    if bound == "hbm" and k["flops"] > 0:
        alu = peak_table(peaks, peak_kind)["alu"][0]
        out["fft_tflops_nominal"] = k["flops"] / k["launches"] / (avg_ms * 1e9)
        out["alu_frac_nominal"] = out["fft_tflops_nominal"] / alu
    out.update({"kernel": name, "launches": k["launches"], "avg_launch_ms": avg_ms,
                "algorithmic_bytes_per_launch": k["bytes"] / k["launches"],
                "algorithmic_flops_per_launch": k["flops"] / k["launches"],
                "traffic": None})
    if rec is not None:
        # the captured launch's DRAM bytes, scaled to this run's average
        # launch by algorithmic bytes
        dram, alg = rec
        out["traffic"] = dram * (k["bytes"] / k["launches"]) / alg
        out["traffic_over_algorithmic"] = dram / alg
    return out


def sampled_error(ctx, m0, samples):
    """Relative L2 error of sampled forward fields and of their data rows
    against the FP64 oracle solutions (BiCGSTAB tol 1e-10) computed in the
    CPU-baseline leg, at full size.  For a plane-wave sample the device
    field is the superposition of the element fields with the oracle's
    weight row, and the data row is the transmit's row."""
    import torch
    fields = ctx.empty_fields()
    data = ctx.empty_data()
    ctx.forward(m0, fields=fields, data=data)
    torch.cuda.synchronize()
    errs_f, errs_d = [], []
    for l, e, ref, refd, wrow in samples:
        if wrow is None:
            got = fields[l, e].cpu().numpy()
        else:
            wt = torch.from_numpy(wrow).to(device="cuda")
            got = torch.einsum("e,en->n", wt, fields[l].reshape(ctx.n_elem, -1).to(
                torch.complex128)).reshape(ctx.shape).cpu().numpy()
        errs_f.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        gotd = data[l, e].cpu().numpy()
        errs_d.append(float(np.linalg.norm(gotd - refd) / np.linalg.norm(refd)))
    return {"fields_max": max(errs_f), "data_row_max": max(errs_d),
            "samples": len(samples), "tolerance": 1e-4}


def serving_fp64_comparator(work, results, rate, n_sample=2):
    """Latency of the plain unbatched FP64 path (complex128 fields, one RHS
    per Krylov launch, same tolerance and ADMM parameters) on the smallest
    requests of the stream (by N x RHS, which bounds its run time), each run
    alone; beside it the same request alone through the batched path and
    its latency in the mix.  A path whose service time exceeds the mean
    inter-arrival time cannot keep up with the stream at all."""
    from paper_2604_15796_gb300 import libfwi
    order = sorted(range(len(work)), key=lambda k: int(np.prod(work[k][0].shape)) * work[k][0].n_rhs)
    rows = []
    for k in order[:n_sample]:
        w, s0, d, prm = work[k]
        row = {"request": k, "grid": "x".join(map(str, reversed(w.shape))), "rhs": int(w.n_rhs),
               "in_mix_ms": results[k]["latency_ms"]}
        for name, kw in (("batched_alone_ms", {}),
                         ("fp64_unbatched_alone_ms", dict(precision=libfwi.FWI_FP64, max_batch=1))):
            one = libfwi.Server(max_active=1)
            _, r = one.wait(one.submit(w.shape, w.h, w.c0, w.elem, w.freqs, s0, d, **prm, **kw))
            one.close()
            row[name] = r["latency_ms"]
            row[name.replace("_ms", "_status")] = r["status"]
        row["factor_alone"] = row["fp64_unbatched_alone_ms"] / row["batched_alone_ms"]
        row["factor_vs_in_mix"] = row["fp64_unbatched_alone_ms"] / row["in_mix_ms"]
        rows.append(row)
        print(f"serving comparator: request {k} {row['grid']} FP64 unbatched "
              f"{row['fp64_unbatched_alone_ms'] / 1e3:.1f} s, batched alone "
              f"{row['batched_alone_ms'] / 1e3:.2f} s", file=sys.stderr, flush=True)
    return {"kind": "plain unbatched FP64 path (complex128 fields, max_batch 1), each request "
                    "alone, on the smallest requests of the stream",
            "requests": rows,
            "factor_alone_min": min(r["factor_alone"] for r in rows),
            "mean_interarrival_ms": 1e3 / rate}


def run_serving(args, n_requests=None, n_burst=4, n_comparator=2):
    """Serving stream: Poisson arrivals of whole reconstructions (5 ADMM-TV
    iterations each) over grids {128^2, 256^2, 384^2, 512^2, 96^3}, 64-192
    elements, 2-12 frequencies; continuous batching with admission by HBM
    footprint.  Arrival rate: 80 % of the capacity measured on a burst of
    ``n_burst`` requests."""
    import threading
    import torch
    from paper_2604_15796_gb300 import libfwi, phantoms
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n_requests = args.requests if n_requests is None else n_requests
    specs = phantoms.serving_requests(n_req=n_requests + n_burst, seed=1004, rate_hz=1.0)

    def build(sp):
        """Request inputs (untimed): observed data = forward data of the
        phantom (device solve) + 2 % noise; start = half the phantom's SoS
        perturbation; ADMM weights scaled to ||J^H J|| at the start."""
        w = phantoms.tissue_phantom(sp["shape"], sp["h"], sp["n_elem"], sp["pitch"],
                                    sp["freqs"], sp["seed"], inclusions=[1520.0, 1580.0])
        sos0 = w.c0 + 0.5 * (w.sos - w.c0)
        ctx = libfwi.Context(w.shape, w.h, w.c0, w.elem, w.freqs)
        d = ctx.empty_data()
        ctx.forward(ctx.contrast_from_sos(torch.from_numpy(np.ascontiguousarray(w.sos)).cuda()),
                    data=d)
        m0 = ctx.contrast_from_sos(torch.from_numpy(np.ascontiguousarray(sos0)).cuda())
        ctx.forward(m0)
        v = torch.from_numpy(phantoms.complex_normal(w.shape, 7)).cuda()
        nrm = 1.0
        for _ in range(3):
            v = v / torch.linalg.vector_norm(v)
            v = ctx.jac_adjoint(ctx.jac_forward(v))
            nrm = float(torch.linalg.vector_norm(v).item())
        dh = d.cpu().numpy()
        noise = phantoms.complex_normal(dh.shape, sp["seed"] + 1)
        dh = dh + 0.02 * np.linalg.norm(dh) / np.sqrt(2 * dh.size) * noise
        ctx.close()
        # standard scaled dual step (1): the literal u += rho (g - grad m) of
        # Algorithm 1 is unstable once rho >> 1, which the 3-D requests reach
        # (their ||J^H J|| is ~1e5 times that of the 2-D ones)
        prm = dict(n_iter=5, lam=1e-4 * nrm, rho=1e-2 * nrm, gamma=1e-3 * nrm, n_cg=10,
                   max_it=200, dual_step=1.0)
        return w, sos0, dh.astype(np.complex64), prm

    srv = libfwi.Server(max_active=args.max_active)
    # capacity on a burst of n_burst requests
    burst = [build(sp) for sp in specs[:n_burst]]
    print("serving: burst requests built", file=sys.stderr, flush=True)
    t0 = time.perf_counter()
    ids = [srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, s0, d, **prm)
           for w, s0, d, prm in burst]
    burst_solves = 0
    for i in ids:
        _, r = srv.wait(i)
        burst_solves += r["rhs_solves"]
    cap = len(ids) / (time.perf_counter() - t0)
    rate = 0.8 * cap
    rng = np.random.default_rng(77)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    print(f"serving: burst capacity {cap:.3f} req/s", file=sys.stderr, flush=True)
    work = [build(sp) for sp in specs[n_burst:n_burst + n_requests]]
    results = [None] * len(work)
    lock = threading.Lock()
    start = time.perf_counter()

    def waiter(k, rid):
        sos, r = srv.wait(rid)
        w = work[k][0]
        r = dict(r, grid="x".join(map(str, reversed(w.shape))), rhs=int(w.n_rhs))
        with lock:
            results[k] = r
        print(f"serving: request {k} {r['grid']} rhs={r['rhs']} status={r['status']} "
              f"latency {r['latency_ms'] / 1e3:.1f} s, BiCGSTAB iterations max "
              f"{r['krylov_iters_max']} (not converged: {r['not_converged']})",
              file=sys.stderr, flush=True)

    threads = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k, ((w, s0, d, prm), ta) in enumerate(zip(work, arrivals)):
            delay = start + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            rid = srv.submit(w.shape, w.h, w.c0, w.elem, w.freqs, s0, d, **prm)
            th = threading.Thread(target=waiter, args=(k, rid))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
    wall = time.perf_counter() - start
    srv.close()
    comp = None if args.no_comparator else serving_fp64_comparator(work, results, rate,
                                                                   n_sample=n_comparator)
    lat = np.array([r["latency_ms"] for r in results])
    bad = sum(1 for r in results if r["status"] != 0)
    solves = sum(r["rhs_solves"] for r in results)
    return {"metric": METRIC, "value": solves / wall, "unit": UNIT, "n_gpus": 1,
            "steps": len(work), "warmup": n_burst, "ms_per_step": 1e3 * wall / len(work),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 fields / FP64 Krylov scalars", "data": "synthetic",
            "config": {"workload": f"serving stream: {len(work)} reconstruction requests, "
                                   "Poisson arrivals at 80% of burst capacity, grids "
                                   "{128^2,256^2,384^2,512^2,96^3}, 64-192 elements, 2-12 "
                                   "frequencies in 0.3-min(5 MHz, c0/(3.85 h)), 5 ADMM-TV iterations each (scaled dual step 1)",
                       "max_active": args.max_active, "arrival_rate_hz": rate,
                       "burst_capacity_req_per_s": cap},
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "queue_ms_mean": float(np.mean([r["queue_ms"] for r in results])),
            "requests_per_s": len(work) / wall, "failed_requests": bad,
            "requests": [{k: r[k] for k in ("grid", "rhs", "status", "queue_ms", "run_ms",
                                              "latency_ms", "krylov_iters_max",
                                              "krylov_iters_mean", "not_converged")}
                         for r in results],
            "comparator_fp64_unbatched": comp,
            "clocks": clk.summary()}


def serving_brief(args):
    """Latency sub-record of the headline line, measured after its timed
    region: a short serving stream (``--serving-requests`` requests of the
    serving workload, Poisson arrivals at 80 % of the capacity of a
    two-request burst) with its p50/p99 reconstruction latency, and the
    plain unbatched FP64 path's latency on the smallest request of the
    stream, alone, against the batched path's."""
    r = run_serving(args, n_requests=args.serving_requests, n_burst=2, n_comparator=1)
    out = {"kind": "serving stream after the timed region (not in value)",
           "requests": r["steps"], "failed_requests": r["failed_requests"],
           "latency_ms": r["latency_ms"], "rhs_solves_per_s": r["value"],
           "arrival_rate_hz": r["config"]["arrival_rate_hz"],
           "grids": sorted({q["grid"] for q in r["requests"]})}
    comp = r.get("comparator_fp64_unbatched")
    if comp:
        # the FP64 path is timed on the stream's smallest request alone (its
        # full stream would not keep up with the arrivals); the factor is the
        # ratio of the two paths' service times for the same request
        row = comp["requests"][0]
        out["fp64_unbatched"] = {
            "request": f"{row['grid']} x {row['rhs']} RHS", "alone_ms": row[
                "fp64_unbatched_alone_ms"], "batched_alone_ms": row["batched_alone_ms"],
            "factor_alone": row["factor_alone"],
            "mean_interarrival_ms": comp["mean_interarrival_ms"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="volume3d",
                    choices=["thyroid256", "large512", "volume3d", "disc64", "planewave2d",
                             "elev3d", "serving"])
    ap.add_argument("--max-batch", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--chains", type=int, choices=[1, 2], default=None,
                    help="iterate each batch as one chain or as two halves on two streams "
                         "(default: two on 2-D lattices, one on 3-D)")
    ap.add_argument("--cuda-core-jacobian", action="store_true",
                    help="run the pixel contractions on CUDA cores instead of tensor cores")
    ap.add_argument("--no-col-tma", action="store_true",
                    help="column passes read their tiles with plain loads instead of TMA")
    ap.add_argument("--no-row-l2-prefetch", action="store_true",
                    help="row passes without the L2 prefetch of their next work item")
    ap.add_argument("--no-spectrum-stage", action="store_true",
                    help="the convolution reads the kernel spectrum from global memory")
    ap.add_argument("--no-jac-tma", action="store_true",
                    help="tensor-core contractions load their operand tiles with cp.async")
    ap.add_argument("--no-col-pairs", action="store_true",
                    help="the convolution computes one column per thread instead of two")
    ap.add_argument("--no-row-stage", action="store_true",
                    help="the forward row pass loads its rows from global memory instead "
                         "of staging them in shared memory")
    ap.add_argument("--requests", type=int, default=12)
    ap.add_argument("--max-active", type=int, default=4)
    ap.add_argument("--check-samples", type=int, default=2)
    ap.add_argument("--ref-step-s", type=float, default=2.0)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--serving-requests", type=int, default=6,
                    help="requests of the serving sub-record after the timed region "
                         "(0: none)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == "serving" and args.impl == "ours":
        if rank == 0:
            print(json.dumps(run_serving(args)), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group(
            "nccl", device_id=torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0"))))
    cpu = None
    samples = []
    if rank == 0 and world == 1 and not args.no_cpu:
        # oracle timed on the host cores before the GPU work starts
        w = workload(args.workload)
        rate, n, dt, samples, line = oracle_solves_per_s(w, budget_s=args.cpu_budget_s,
                                                         keep=args.check_samples)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} FP64 BiCGSTAB solves (tol 1e-10) of random transmit/frequency "
                         f"pairs of {w.name}, {dt:.1f} s of solves, scipy.fft over all host "
                         f"cores" + ("; point-source right-hand sides on the line-element "
                                     "workload's operator" if line else "")}
    line = run_ours(args, rank, world, samples)
    if rank == 0 and world == 1 and args.serving_requests > 0:
        line["serving"] = serving_brief(args)
    if rank == 0:
        line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
