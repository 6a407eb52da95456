"""Benchmark of the BAE hot path on GB300.

Workload (default): modified Helmholtz kappa^2 = 10 on the torus R = 0.5,
r = 0.2 in [-1,1]^3, N = 128 (h = 1/64), u = sin(2x) cos(y) exp(z), double
layer, GMRES tolerance 1e-10. One step = one full solve of Algorithm 1 for
that problem: classification from phi (the LGF spectrum per (N, kappa^2 h^2)
is cached by the context, as the numerical section reuses tables), the
particular solution, the GMRES solve with float32 convolutions inside float64
iterative refinement, and the volume reconstruction. Inputs are synthetic
and resident in device memory; the L2 cache is flushed between steps.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on
the host cores instead. Multi-GPU (torchrun): independent replicas, one
problem per rank, no collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BAE solves/s + p50/p99 latency at 1e-8 err; LGF-conv GB/s vs HBM peak"
UNIT = "solves/s"
TOL = 1e-10
N = 128
KAPPA2 = 10.0
WORKLOAD = "torus R=0.5 r=0.2, kappa^2=10, N=128 (h=1/64), double layer, GMRES tol 1e-10"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------ roofline arithmetic
def kernel_model(n, pb, n_gm, npl=None):
    """Algorithmic (bytes, flops) of one launch of each convolution pass for
    one right-hand side at grid size n, element precision pb bytes (complex
    = 2 pb), when the solve transforms npl of the n x-planes (the planes that
    hold sources or read-back nodes; all n if None). FFT flops use the
    5 L log2 L convention per complex transform of length L = 2n; the
    spectral multiply counts 2 flops per element."""
    npl = n if npl is None else npl
    c = 2 * pb
    L = 2 * n
    n1 = n + 1
    # N k-columns per (i, j): the real kk = N spectrum is packed into column 0
    A = npl * n * n * c            # k-spectra of the transformed planes
    B = 2 * npl * n * n * c        # after the j pass: 2n rows, n columns per plane
    F = 5.0 * L * math.log2(L)
    src = 8 * n_gm + 4 * (npl * n + 1)
    plane_f = (npl * n / 2) * F + npl * n * F
    return {
        "conv_kfwd": (A + src, (npl * n / 2) * F),
        "conv_jfwd": (A + B, npl * n * F),
        # i pass: reads and writes the rows of the transformed planes
        "conv_i": (2 * B + n1 ** 3 * pb, 2 * (2 * n * n) * F + 2.0 * (2 * n * n) * L),
        "conv_jinv": (A + B, npl * n * F),
        "conv_kinv": (A + npl * n * n * pb, (npl * n / 2) * F),
        # k and j fused per plane (one CTA, or a cluster): A stays on chip
        "conv_plane_fwd": (B + src, plane_f),
        "conv_plane_inv": (B + npl * n * n * pb, plane_f),
        "conv_cplane_fwd": (B + src, plane_f),
        "conv_cplane_inv": (B + npl * n * n * pb, plane_f),
    }


FP64_PEAK_TFLOPS = 1.25   # nominal FP64 rate of GB300 (a probe measured 1.20)
# double-float kernels run on the float32 pipes: a radix-2 butterfly (10
# float64-equivalent flops: one complex product, two complex sums) costs 70
# float32 instructions (a complex product as two fused a b + c d forms of 19,
# a sum 8), 7 per flop; the float32 instruction rate is half the measured
# 70.2 TFLOP/s FMA rate
DF64_OPS_PER_FLOP = 7.0
FP32_INST_PEAK_T = 35.1


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the default workload's convolution kernels, from one ncu capture of the
# current kernels (profiles/conv_i_traffic_torus_N128.md); a kernel changed
# since its capture must be dropped from this table (its traffic is then
# reported as null)
NCU_TRAFFIC_TORUS128 = {
    "conv_i.f32": 33.98e6,
}


def roofline_for(name, ms_total, launches, n_gm, hbm, hbm_kind, npl=None):
    base, _, prec = name.partition(".")
    model = kernel_model(N, 4 if prec == "f32" else 8, n_gm, npl)
    if base not in model:
        return None
    nbytes, flops = model[base]
    t = (ms_total / launches) / 1000.0
    if prec == "df64":
        a = flops * DF64_OPS_PER_FLOP / t / 1e12
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": FP32_INST_PEAK_T,
                "unit": "T float32 instructions/s", "frac": a / FP32_INST_PEAK_T, "traffic": None,
                "peak_kind": "measured float32 FMA probe / 2", "us_per_launch": t * 1e6,
                "algorithmic_flops_fp64_equiv": flops}
    if prec == "f64":
        a = flops / t / 1e12
        return {"kernel": name, "bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": a / FP64_PEAK_TFLOPS, "traffic": None, "peak_kind": "nominal FP64 (recipe table)",
                "us_per_launch": t * 1e6, "algorithmic_flops": flops}
    a = nbytes / t / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
            "traffic": NCU_TRAFFIC_TORUS128.get(name) if N == 128 else None,
            "peak_kind": hbm_kind + " HBM copy bandwidth", "us_per_launch": t * 1e6,
            "algorithmic_bytes": nbytes}


def aggregate_replicas(local_ms, steps, world, device):
    """Whole-job throughput of independent replicas: every rank solved
    `steps` problems in local_ms; the job took the slowest rank's time (a
    MAX all-reduce, the only collective: the solves exchange nothing)."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    return steps * world / (total_ms / 1000.0), total_ms


def _flush_l2(buf):
    buf.add_(1.0)


def _problem_inputs(P, torch, dev):
    phi = torch.from_numpy(P.phi).to(dev)
    f = torch.from_numpy(P.f()).to(dev)
    return phi, f


def run_ours(args, rank, world, dev):
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Context, Problem, launch_count, profile_start, profile_stop

    torch.cuda.set_device(dev)
    P = W.torus_helmholtz(N, kappa2=KAPPA2)
    ctx = Context(dev)
    phi, f = _problem_inputs(P, torch, dev)
    prob0 = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
    xs = prob0.boundary_points()
    g = torch.from_numpy(P.g_at(xs)).to(dev)
    n_gm = prob0.n_gm
    plo, phi_ = prob0.plane_range()
    npl = phi_ - plo
    prob0.close()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step(precision, use_graphs=False):
        pr = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
        q, u, st = pr.solve(f, g, tol=TOL, precision=precision, use_graphs=use_graphs)
        pr.close()
        return q, u, st

    torch.cuda.set_stream(ctx.stream)   # events, flushes and library work share one stream
    for _ in range(max(args.warmup, 0)):
        step(args.precision)
    torch.cuda.synchronize()

    # ---------------------------------------------------------- timed region
    clocks = ClockSampler(dev)
    clocks.start()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    stats = []
    for k in range(args.steps):
        _flush_l2(flush)
        e0[k].record()
        q, u, st = step(args.precision)
        e1[k].record()
        stats.append(st)
    torch.cuda.synchronize()
    l1 = launch_count()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = np.array([a.elapsed_time(b) for a, b in zip(e0, e1)])
    value, total_ms = aggregate_replicas(float(ms.sum()), args.steps, world, torch.device("cuda", dev))

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": float(ms.mean()), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 conv + f64 refinement" if args.precision == "mixed"
           else "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                          "min": float(ms.min()), "max": float(ms.max())},
           "solve": {"iterations": int(stats[-1]["iterations"]), "refinements": int(stats[-1]["refinements"]),
                     "applies_fp32": int(stats[-1]["applies_fp32"]), "applies_fp64": int(stats[-1]["applies_fp64"]),
                     "rel_residual": stats[-1]["rel_residual"], "n_gm": n_gm},
           "gpu_launches": int(l1 - l0), "clocks": clk}
    if rank != 0 or args.only_timed:
        ctx.close()
        return out if rank == 0 else None

    # per-kernel device times: the same steps again (launched kernel by
    # kernel, as in the timed region) with every launch bracketed by CUDA
    # events; kept out of the timed region, where the event records would
    # add host time to every step
    profile_start(60 * max(l1 - l0, 1) // max(args.steps, 1) + 5000)
    for k in range(min(args.steps, 5)):
        _flush_l2(flush)
        step(args.precision, use_graphs=False)
    torch.cuda.synchronize()
    prof = profile_stop()

    # ------------------------------------------------------ kernel roofline
    hbm, hbm_kind = _peaks()
    kt = sorted(prof.items(), key=lambda kv: -kv[1][0])
    tot = sum(v[0] for v in prof.values())
    out["kernels"] = [{"name": k, "ms_total": round(v[0], 3), "launches": v[1],
                       "share": round(v[0] / tot, 4) if tot else None} for k, v in kt[:14]]
    dom = next((k for k, _ in kt if k.startswith("conv_")), None)
    out["roofline"] = roofline_for(dom, prof[dom][0], prof[dom][1], n_gm, hbm, hbm_kind, npl) if dom else None
    # the float32 i-pass (forward FFT, ghat multiply, inverse FFT) inside the timed region
    if "conv_i.f32" in prof:
        out["conv_f32_roofline"] = roofline_for("conv_i.f32", *prof["conv_i.f32"], n_gm, hbm, hbm_kind, npl)
    # whole float32 apply: algorithmic bytes of the passes that ran / their
    # summed time per apply (either schedule the autotuner picked)
    if "conv_i.f32" in prof:
        napp = prof["conv_i.f32"][1]
        m = kernel_model(N, 4, n_gm, npl)
        names = [k for k in prof if k.startswith("conv_") and k.endswith(".f32")]
        nbytes = sum(m[k.split(".")[0]][0] * prof[k][1] / napp for k in names)
        t_apply = sum(prof[k][0] for k in names) / napp / 1000.0
        out["conv_f32_apply"] = {"us": t_apply * 1e6, "passes": sorted(k.split(".")[0] for k in names),
                                 "algorithmic_bytes": nbytes, "GBps": nbytes / t_apply / 1e9,
                                 "frac_hbm": nbytes / t_apply / 1e9 / hbm,
                                 "note": "N=128 buffers fit in the 129 MB L2, so this can exceed HBM peak"}

    # ------------------------------------- other arithmetics, for comparison
    interior = P.phi < 0   # M+, where Algorithm 1 defines the solution
    ud = u.cpu().numpy()
    others = {}
    for label, prec, res in (("fp64", "fp64", None), ("df64", "df64", None), ("mixed_fp64_residual", "mixed", "fp64")):
        def run():
            pr = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
            out_ = pr.solve(f, g, tol=TOL, precision=prec, residual_precision=res)
            pr.close()
            return out_
        run()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        qo, uo_, sto = run()
        t1.record()
        torch.cuda.synchronize()
        uu = uo_.cpu().numpy()
        others[label] = {"solves_per_s": 1000.0 / t0.elapsed_time(t1), "iterations": sto["iterations"],
                         "applies_fp64_accurate": sto["applies_fp64"], "applies_fp32": sto["applies_fp32"],
                         "u": uu}
    uf = others["fp64"]["u"]
    out["err_mixed_vs_fp64"] = float(np.max(np.abs(ud - uf)[interior]) / np.max(np.abs(uf[interior])))
    out["other_arithmetic"] = {k: {kk: vv for kk, vv in v.items() if kk != "u"} for k, v in others.items()}
    out["fp64_solve"] = out["other_arithmetic"]["fp64"]

    # --------------------------------------------------------- e2e (host)
    phi_h, f_h = P.phi, P.f()
    g_h = P.g_at(xs.cpu().numpy() if hasattr(xs, "cpu") else xs)
    e2e_ms = []
    for k in range(min(args.steps, 8) + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        pr = Problem(ctx, phi_h, P.grid.h, P.grid.origin, P.kappa2, "double")
        qh, uh, sth = pr.solve(f_h, g_h, tol=TOL, precision=args.precision)
        pr.close()
        dt = time.perf_counter() - t
        if k > 0:
            e2e_ms.append(dt * 1000.0)
    out["e2e"] = {"value": 1000.0 / float(np.mean(e2e_ms)), "unit": UNIT,
                  "h2d_bytes_per_step": int(phi_h.nbytes + f_h.nbytes + g_h.nbytes),
                  "d2h_bytes_per_step": int(qh.nbytes + uh.nbytes)}

    # --------------------------------------------------------- cpu baseline
    if world == 1 and not args.no_cpu:
        out["cpu_baseline"], uo = cpu_oracle_solve(P)
        m = interior
        out["err_vs_oracle"] = {"mixed": float(np.max(np.abs(ud[m] - uo[m])) / np.max(np.abs(uo[m]))),
                                "fp64": float(np.max(np.abs(uf[m] - uo[m])) / np.max(np.abs(uo[m]))),
                                "on": "M+ (interior nodes), max-norm relative"}
    ctx.close()
    return out


def cpu_oracle_solve(P):
    """The oracle (FFT route, float64 scipy.fft on every host core) solving
    the same problem once; the LGF table is built beforehand and not timed
    (the GPU side caches it too)."""
    from oracle import lgf as OL
    from oracle import potentials as OP
    from oracle import solve as OS
    cores = os.cpu_count() or 1
    s = P.kappa2 * P.grid.h ** 2
    t = time.perf_counter()
    table = OL.LGFTable(P.grid.N, s)
    spec = OP.lgf_spectrum(table)
    t_table = time.perf_counter() - t
    t = time.perf_counter()
    r = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, layer="double", tol=TOL,
                 potential="fft", spectrum=spec, workers=cores)
    dt = time.perf_counter() - t
    return ({"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"one full oracle solve of the workload (FFT route, {r.iterations} GMRES iterations, "
                       f"{dt:.1f} s); LGF table build ({t_table:.1f} s) excluded as cached"},
            r.u)


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample, one
    oracle boundary-operator apply (the unit of a GMRES iteration);
    solves/s = 1 / (mean apply time x applies per oracle solve), the apply
    count taken from one untimed full oracle solve of the same workload."""
    import workloads as W
    from oracle import grid as OG
    from oracle import lgf as OL
    from oracle import potentials as OP
    from oracle import solve as OS
    cores = os.cpu_count() or 1
    P = W.torus_helmholtz(N, kappa2=KAPPA2)
    s = P.kappa2 * P.grid.h ** 2
    spec = OP.lgf_spectrum(OL.LGFTable(N, s))
    full = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, layer="double", tol=TOL,
                    potential="fft", spectrum=spec, workers=cores)
    applies = full.iterations + 2
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    q = np.random.default_rng(0).standard_normal(cls.gm_idx.size)

    def apply_once():
        v = OP.fft_convolve(OP.source_density(cls, q, "double"), spectrum=spec, workers=cores).reshape(-1)
        return OS.closure_apply(cls, v)

    for _ in range(args.warmup):
        apply_once()
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        apply_once()
        ts.append(time.perf_counter() - t)
    per_solve = float(np.mean(ts)) * applies
    value = 1.0 / per_solve
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * per_solve, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle boundary applies (scipy.fft float64), scaled by "
                                       f"{applies} applies per oracle solve"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _timed(fn, torch):
    torch.cuda.synchronize()
    t = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t


def run_sphere32(args):
    """Poisson, sphere r=0.6, N=32, u=exp(x+y+z), double layer, float64."""
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Context, Problem
    P = W.sphere_exp(32)
    ctx = Context(0)
    torch.cuda.set_stream(ctx.stream)
    phi, f = _problem_inputs(P, torch, 0)
    pr0 = Problem(ctx, phi, P.grid.h, P.grid.origin, 0.0, "double")
    g = torch.from_numpy(P.g_at(pr0.boundary_points())).cuda()
    pr0.close()

    def step():
        pr = Problem(ctx, phi, P.grid.h, P.grid.origin, 0.0, "double")
        out = pr.solve(f, g, tol=TOL, precision="fp64")
        pr.close()
        return out
    for _ in range(args.warmup):
        step()
    ms = []
    for _ in range(args.steps):
        (q, u, st), dt = _timed(step, torch)
        ms.append(dt * 1e3)
    ms = np.array(ms)
    u = u.cpu().numpy()
    m = P.phi < 0
    ctx.close()
    return {"metric": METRIC, "value": 1e3 / ms.mean(), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms.mean(), "higher_is_better": True, "dtype": "f64",
            "config": {"workload": "sphere r=0.6, Poisson, N=32 (h=1/16), u=exp(x+y+z), double layer, fp64, tol 1e-10"},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "iterations": st["iterations"], "max_err_vs_exact": float(np.max(np.abs(u[m] - P.u_exact()[m])))}


def run_batched64(args):
    """64 right-hand sides u_k = exp(a_k . x) on the N=128 Poisson torus, one
    batched mixed-precision solve per step."""
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Context, Problem
    nrhs = args.nrhs
    dirs = W.torus_batch_dirs(64, seed=3)[:nrhs]
    probs = [W.torus_poisson_dir(128, a) for a in dirs]
    ctx = Context(0)
    torch.cuda.set_stream(ctx.stream)
    P0 = probs[0]
    phi = torch.from_numpy(P0.phi).cuda()
    pr0 = Problem(ctx, phi, P0.grid.h, P0.grid.origin, 0.0, "double")
    xs = pr0.boundary_points()
    pr0.close()
    f = torch.from_numpy(np.stack([P.f() for P in probs])).cuda()
    g = torch.from_numpy(np.stack([P.g_at(xs) for P in probs])).cuda()

    def step():
        pr = Problem(ctx, phi, P0.grid.h, P0.grid.origin, 0.0, "double")
        out = pr.solve_batched(f, g, tol=TOL, precision="mixed")
        pr.close()
        return out
    for _ in range(max(1, args.warmup)):
        step()
    ms = []
    for _ in range(args.steps):
        (q, u, st), dt = _timed(step, torch)
        ms.append(dt * 1e3)
    ms = np.array(ms)
    u = u.cpu().numpy()
    m = P0.phi < 0
    errs = [float(np.max(np.abs(u[k][m] - probs[k].u_exact()[m]))) for k in range(nrhs)]
    ctx.close()
    return {"metric": METRIC, "value": nrhs * 1e3 / ms.mean(), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms.mean(), "higher_is_better": True,
            "dtype": "f32 conv + df64 refinement",
            "config": {"workload": f"{nrhs} RHS exp(a_k.x), Poisson torus R=0.5 r=0.2, N=128, one batched solve per step"},
            "iterations_max": max(s_["iterations"] for s_ in st), "rel_residual_max": max(s_["rel_residual"] for s_ in st),
            "max_err_vs_exact": max(errs)}


def run_star256(args):
    """N=256 star, kappa^2 in {0, 1, 100}, double vs single layer: GMRES
    iterations and solves/s (mixed precision)."""
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Context, Problem
    ctx = Context(0)
    torch.cuda.set_stream(ctx.stream)
    rows = []
    for k2 in (0.0, 1.0, 100.0):
        for layer in ("double", "single"):
            P = W.star(256, kappa2=k2, layer=layer)
            phi, f = _problem_inputs(P, torch, 0)
            pr0 = Problem(ctx, phi, P.grid.h, P.grid.origin, k2, layer)
            g = torch.from_numpy(P.g_at(pr0.boundary_points())).cuda()
            n_gm = pr0.n_gm
            pr0.close()

            def step():
                pr = Problem(ctx, phi, P.grid.h, P.grid.origin, k2, layer)
                out = pr.solve(f, g, tol=TOL, precision="mixed", max_iter=2000, restart=400)
                pr.close()
                return out
            step()
            (q, u, st), dt = _timed(step, torch)
            uu = u.cpu().numpy()
            m = P.phi < 0
            rows.append({"kappa2": k2, "layer": layer, "iterations": st["iterations"], "solves_per_s": 1.0 / dt,
                         "rel_residual": st["rel_residual"], "n_gm": n_gm,
                         "max_err_vs_exact": float(np.max(np.abs(uu[m] - P.u_exact()[m])))})
    ctx.close()
    return {"metric": METRIC, "value": float(np.mean([r["solves_per_s"] for r in rows])), "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32 conv + df64 refinement",
            "config": {"workload": "star r=0.6+0.1 sin5t cos3p, N=256, kappa^2 in {0,1,100}, double vs single layer"},
            "table": rows}


def run_direct128(args):
    """The torus N=128 workload (kappa^2 = 10, tol 1e-10, mixed precision)
    with the direct formulation (unknown u on gamma = gamma- u gamma+,
    difference potentials), beside the double layer: solves/s, iterations,
    and the agreement of the two solutions on N+ (the same discrete problem)."""
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Context, Problem
    ctx = Context(0)
    torch.cuda.set_stream(ctx.stream)
    P = W.torus_helmholtz(128, kappa2=10.0)
    phi, f = _problem_inputs(P, torch, 0)
    rows, us = [], {}
    for layer in ("direct", "double"):
        pr0 = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, layer)
        g = torch.from_numpy(P.g_at(pr0.boundary_points())).cuda()
        n_unk = pr0.n_unknowns
        pr0.close()

        def step():
            pr = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, layer)
            out = pr.solve(f, g, tol=TOL, precision="mixed", max_iter=2000)
            pr.close()
            return out
        for _ in range(max(1, args.warmup)):
            step()
        times = []
        for _ in range(max(1, args.steps)):
            (q, u, st), dt = _timed(step, torch)
            times.append(dt)
        us[layer] = u.cpu().numpy()
        rows.append({"layer": layer, "unknowns": n_unk, "iterations": st["iterations"],
                     "refinements": st["refinements"], "solves_per_s": 1.0 / float(np.median(times)),
                     "ms_p50": 1e3 * float(np.median(times)), "rel_residual": st["rel_residual"]})
    m = P.phi < 0
    diff = float(np.max(np.abs(us["direct"] - us["double"])) / np.max(np.abs(us["double"][m])))
    ctx.close()
    return {"metric": METRIC, "value": rows[0]["solves_per_s"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32 conv + df64 refinement",
            "config": {"workload": "torus R=0.5 r=0.2, kappa^2=10, N=128, direct formulation (eq. direct_sys)"},
            "table": rows, "rel_diff_direct_vs_double_on_grid": diff}


def run_serving(args):
    """Serving trace: requests with N in {32,64,128,256}, kappa^2 in {0,10},
    random spheres/ellipsoids/tori, u = exp(a.x); Poisson arrivals at 0.8x
    the measured saturation throughput; p50/p99 latency and solves/s."""
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Server
    nreq = args.requests
    reqs = W.serving_trace(nreq, seed=5)
    probs = [W.trace_problem(r) for r in reqs]
    srv = Server(0, slots=args.slots, hbm_budget_bytes=int(args.hbm_gb * (1 << 30)))
    # warm the spectrum cache and the slots, then measure saturation throughput
    warm = [srv.submit(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, kappa2=P.kappa2) for P in probs[:32]]
    for t in warm:
        srv.poll(t)
        srv.release(t)
    t0 = time.perf_counter()
    sat = [srv.submit(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, kappa2=P.kappa2) for P in probs[32:96]]
    for t in sat:
        srv.poll(t)
        srv.release(t)
    sat_rate = len(sat) / (time.perf_counter() - t0)
    lam = 0.8 * sat_rate
    rng = np.random.default_rng(55)
    gaps = rng.exponential(1.0 / lam, size=nreq)
    tickets, arrive = [], []
    start = time.perf_counter()
    tnext = start
    for P, gap in zip(probs, gaps):
        tnext += gap
        d = tnext - time.perf_counter()
        if d > 0:
            time.sleep(d)
        arrive.append(srv.clock())
        tickets.append(srv.submit(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, kappa2=P.kappa2))
    res = [srv.poll(t) for t in tickets]
    wall = time.perf_counter() - start
    lat = np.array([(r["t_done"] - a) * 1e3 for r, a in zip(res, arrive)])
    ok = sum(1 for r in res if r["status"] == 0)
    srv.close()
    return {"metric": METRIC, "value": ok / wall, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32 conv + df64 refinement",
            "config": {"workload": f"serving trace, {nreq} Poisson-arrival requests, N in {{32,64,128,256}}, "
                                   f"kappa^2 in {{0,10}}, spheres/ellipsoids/tori", "slots": args.slots,
                       "arrival_rate_per_s": lam, "saturation_solves_per_s": sat_rate},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "completed": ok, "requests": nreq}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default="torus128",
                    choices=["torus128", "sphere32", "batched64", "star256", "serving", "direct128"])
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--nrhs", type=int, default=64, help="batched64: right-hand sides (at most 64)")
    ap.add_argument("--slots", type=int, default=6, help="serving: concurrent slots")
    ap.add_argument("--hbm-gb", type=float, default=96.0, help="serving: device-memory budget")
    ap.add_argument("--only-timed", action="store_true",
                    help="warm-up and timed steps only (no profile, fp64 comparison, e2e or CPU baseline)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    import torch
    extra = {"sphere32": run_sphere32, "batched64": run_batched64, "star256": run_star256,
             "serving": run_serving, "direct128": run_direct128}
    if args.workload in extra:
        if rank == 0:
            print(json.dumps(extra[args.workload](args)))
        return
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
