"""Benchmark of the BAE hot path on GB300.

Headline workload (default, `--workload batched64`): 64 right-hand sides
u_k = exp(a_k . x) (a_k seeded unit vectors) of the Poisson problem on the
torus R = 0.5, r = 0.2 in [-1,1]^3, N = 128 (h = 1/64), double layer, GMRES
tolerance 1e-10. One step = one batched solve of Algorithm 1 for the 64
right-hand sides: classification from phi (the LGF spectrum per
(N, kappa^2 h^2) is cached by the context, as the numerical section reuses
tables), the particular solutions, the batched GMRES with float32
convolutions inside iterative refinement whose residuals use the
double-float (about 48-bit) apply, float64 Gram-Schmidt and Givens, and the
volume reconstruction. Inputs are synthetic and resident in device memory
(1.1 GB of f, larger than the L2); the L2 is also flushed between steps.

Extra keys of the same line: the single right-hand side kappa^2 = 10 torus
(N = 128) and the N = 256 star table (kappa^2 in {0, 1, 100}, single and
double layer), each with its own timing and error against the exact
solution.

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on
the host cores instead. Multi-GPU (torchrun): independent replicas, one
batched problem per rank, no collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
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
NRHS = 64
WORKLOAD = ("64 right-hand sides u_k = exp(a_k.x) (a_k = normalised default_rng(3) normals), Poisson, "
            "torus R=0.5 r=0.2 in [-1,1]^3, N=128 (h=1/64), double layer, GMRES tol 1e-10, one batched solve "
            "per step")
DTYPE_MIXED = "f32 conv + double-float (~48-bit) residual applies + f64 Gram-Schmidt/Givens"
# nominal float32 lane rate from the unit counts and the clock: 152 SMs x
# 128 FP32 lanes x 2.07 GHz (an FMA is one lane operation)
FP32_LANE_PEAK_T = 152 * 128 * 2.07e9 / 1e12


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Arm CPU part numbers of /proc/cpuinfo that the GPU hosts may report
_ARM_PARTS = {"0xd4f": "Arm Neoverse-V2 (NVIDIA Grace)", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1",
              "0xd49": "Arm Neoverse-N2", "0xd8f": "Arm Neoverse-V3"}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key, _, val = line.partition(":")
                key = key.strip().lower()
                if key == "model name":
                    return val.strip()
                if key == "cpu part":
                    return _ARM_PARTS.get(val.strip(), "Arm CPU part " + val.strip())
    except Exception:
        pass
    return platform.processor() or platform.machine()


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
def kernel_model(n, pb, n_gm, npl=None, nb=1):
    """Algorithmic (bytes, flops) per right-hand side of one launch of each
    convolution pass at grid size n, element precision pb bytes (complex =
    2 pb), when the solve transforms npl of the n planes along the axis the
    convolution prunes (the planes that hold sources or read-back nodes, on
    the axis with the fewest of them; all n if None) and nb right-hand sides
    share the launch (the spectrum is read once per launch). FFT flops use
    the 5 L log2 L convention per complex transform of length L = 2n; the
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
        "conv_i": (2 * B + n1 ** 3 * pb / nb, 2 * (2 * n * n) * F + 2.0 * (2 * n * n) * L),
        "conv_jinv": (A + B, npl * n * F),
        "conv_kinv": (A + npl * n * n * pb, (npl * n / 2) * F),
        # k and j fused per plane (one CTA, or a cluster): A stays on chip
        "conv_plane_fwd": (B + src, plane_f),
        "conv_plane_inv": (B + npl * n * n * pb, plane_f),
        "conv_cplane_fwd": (B + src, plane_f),
        "conv_cplane_inv": (B + npl * n * n * pb, plane_f),
    }


def apply_bytes_min(n, pb, npl, nb=1):
    """The minimum a float32 (pb = 4) apply must move per right-hand side
    when the padded field cannot stay on chip: the 2 n^2 npl complex
    elements of the transformed planes after the xy stage are written once
    by it, read and written by the i stage and read by the xy^-1 stage
    (64 n^2 npl bytes); the spectrum octant is read once per launch (shared
    by the batch) and the float32 potential written on the transformed
    planes."""
    c = 2 * pb
    return 8 * c * n * n * npl + (n + 1) ** 3 * pb / nb + pb * n * n * npl


FP64_PEAK_TFLOPS = 1.25   # nominal FP64 rate of GB300 (a probe measured 1.20)
# double-float kernels run on the float32 pipes: a radix-2 butterfly (10
# float64-equivalent flops: one complex product, two complex sums) costs 70
# float32 instructions (a complex product as two fused a b + c d forms of 19,
# a sum 8), 7 per flop
DF64_OPS_PER_FLOP = 7.0


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum)
# of convolution kernels, from ncu captures of the current kernels and
# workloads (profiles/); a kernel or plane range changed since its capture
# is dropped from this table (its traffic is then reported as null). Keyed
# by (kernel, N, right-hand sides per launch).
NCU_TRAFFIC = {
    # conv_i_narrow_batched32_torus_N128.md: 494.8 MB per 32-right-hand-side
    # launch, scaled by 2 less one extra read of the 8.6 MB spectrum octant
    ("conv_i.f32", 128, 64): 2 * 494.8e6 - 8.59e6,
}


def roofline_for(name, ms_total, launches, n, n_gm, hbm, hbm_kind, npl=None, nb=1):
    base, _, prec = name.partition(".")
    model = kernel_model(n, 4 if prec == "f32" else 8, n_gm, npl, nb)
    if base not in model:
        return None
    nbytes, flops = model[base]
    nbytes *= nb
    flops *= nb
    t = (ms_total / launches) / 1000.0
    common = {"kernel": name, "us_per_launch": t * 1e6, "rhs_per_launch": nb}
    if prec == "df64":
        a = flops * DF64_OPS_PER_FLOP / t / 1e12
        return {**common, "bound": "alu", "achieved": a, "peak": FP32_LANE_PEAK_T,
                "unit": "T float32 lane-ops/s", "frac": a / FP32_LANE_PEAK_T, "traffic": None,
                "peak_kind": "nominal float32 lane rate (152 SMs x 128 lanes x 2.07 GHz)",
                "algorithmic_flops_fp64_equiv": flops}
    if prec == "f64":
        a = flops / t / 1e12
        return {**common, "bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": a / FP64_PEAK_TFLOPS, "traffic": None, "peak_kind": "nominal FP64 (recipe table)",
                "algorithmic_flops": flops}
    # float32: bound by whichever of HBM and the float32 pipes it is closer
    # to (the i pass, two length-2N transforms per element moved, is
    # ALU-bound once the convolution transforms few planes)
    a = nbytes / t / 1e9
    f_hbm = a / hbm
    a_alu = flops / t / 1e12
    f_alu = a_alu / (2 * FP32_LANE_PEAK_T)
    traffic = NCU_TRAFFIC.get((name, n, nb))
    both = {"algorithmic_bytes": nbytes, "GBps": a, "frac_hbm": f_hbm, "hbm_peak": hbm,
            "hbm_peak_kind": hbm_kind + " HBM copy bandwidth", "traffic_bytes": traffic,
            # ncu DRAM bytes over the same launch time
            "traffic_GBps": traffic / t / 1e9 if traffic else None,
            "traffic_frac_hbm": traffic / t / 1e9 / hbm if traffic else None,
            "fp32_flops_5LlogL": flops, "fp32_TFLOPs_5LlogL": a_alu, "frac_fp32": f_alu}
    if f_alu > f_hbm:
        return {**common, "bound": "alu", "achieved": a_alu, "peak": 2 * FP32_LANE_PEAK_T,
                "unit": "TFLOP/s (5 L log2 L per transform)", "frac": f_alu,
                "traffic": NCU_TRAFFIC.get((name, n, nb)),
                "peak_kind": "nominal float32 FMA rate (152 SMs x 128 lanes x 2.07 GHz x 2 flops)", **both}
    return {**common, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": f_hbm,
            "traffic": NCU_TRAFFIC.get((name, n, nb)), "peak_kind": hbm_kind + " HBM copy bandwidth", **both}


def kernel_table(prof, top=16):
    kt = sorted(prof.items(), key=lambda kv: -kv[1][0])
    tot = sum(v[0] for v in prof.values())
    return [{"name": k, "ms_total": round(v[0], 3), "launches": v[1],
             "us_per_launch": round(1000.0 * v[0] / max(v[1], 1), 2),
             "share": round(v[0] / tot, 4) if tot else None} for k, v in kt[:top]]


def apply_summary(prof, n, npl, nb, hbm, suffix=".f32"):
    """Whole float32 apply: the minimum bytes of apply_bytes_min over the
    summed time per apply of the passes that ran (either schedule)."""
    names = [k for k in prof if k.startswith("conv_") and k.endswith(suffix)]
    ikey = "conv_i" + suffix
    if ikey not in prof:
        return None
    napp = prof[ikey][1]
    t_apply = sum(prof[k][0] for k in names) / napp / 1000.0
    nbytes = apply_bytes_min(n, 4, npl, nb) * nb
    return {"us_per_apply": t_apply * 1e6, "rhs_per_apply": nb, "passes": sorted(k.split(".")[0] for k in names),
            "min_bytes": nbytes, "GBps": nbytes / t_apply / 1e9, "frac_hbm": nbytes / t_apply / 1e9 / hbm,
            "bytes_model": "per rhs 64 N^2 npl (xy out 16, i in+out 32, xy^-1 in 16 B per complex element) "
                           "+ 4 N^2 npl potential out + 4 (N+1)^3 / nb spectrum"}


def aggregate_replicas(local_ms, steps, world, device, units_per_step=1):
    """Whole-job throughput of independent replicas: every rank solved
    `steps` x `units_per_step` problems in local_ms; the job took the slowest
    rank's time (a MAX all-reduce, the only collective: the solves exchange
    nothing)."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    return steps * units_per_step * world / (total_ms / 1000.0), total_ms


def _flush_l2(buf):
    buf.add_(1.0)


def _timed_loop(step, steps, torch, flush, world=1):
    """Events around each step on the current stream, the L2 flushed before
    each; returns per-step ms and the last step's result."""
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    out = None
    torch.cuda.nvtx.range_push("timed")   # the launches ncu captures (--nvtx-include timed/)
    for k in range(steps):
        _flush_l2(flush)
        e0[k].record()
        out = step()
        e1[k].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    return np.array([a.elapsed_time(b) for a, b in zip(e0, e1)]), out


def _rel_err(u, ref, mask):
    return float(np.max(np.abs(u[mask] - ref[mask])) / np.max(np.abs(ref[mask])))


# ----------------------------------------------------- headline: batched64
def run_ours(args, rank, world, dev):
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Context, Problem, launch_count, profile_start, profile_stop

    torch.cuda.set_device(dev)
    nrhs = args.nrhs
    dirs = W.torus_batch_dirs(64, seed=3)[:nrhs]
    probs = [W.torus_poisson_dir(N, a) for a in dirs]
    P0 = probs[0]
    ctx = Context(dev)
    torch.cuda.set_stream(ctx.stream)   # events, flushes and library work share one stream
    phi = torch.from_numpy(P0.phi).to(dev)
    pr0 = Problem(ctx, phi, P0.grid.h, P0.grid.origin, 0.0, "double")
    xs = np.asarray(pr0.boundary_points())
    n_gm = pr0.n_gm
    conv_axis, plo, phi_ = pr0.conv_planes()
    npl = phi_ - plo
    pr0.close()
    f_h = np.stack([P.f() for P in probs])
    g_h = np.stack([P.g_at(xs) for P in probs])
    f = torch.from_numpy(f_h).to(dev)
    g = torch.from_numpy(g_h).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step(residual="df64"):
        pr = Problem(ctx, phi, P0.grid.h, P0.grid.origin, 0.0, "double")
        out = pr.solve_batched(f, g, tol=TOL, precision="mixed", residual_precision=residual)
        pr.close()
        return out

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    # ---------------------------------------------------------- timed region
    clocks = ClockSampler(dev)
    clocks.start()
    l0 = launch_count()
    ms, (q, u, st) = _timed_loop(step, args.steps, torch, flush, world)
    l1 = launch_count()
    clk = clocks.stop()
    value, total_ms = aggregate_replicas(float(ms.sum()), args.steps, world, torch.device("cuda", dev), nrhs)

    it = [s["iterations"] for s in st]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": float(ms.mean()), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_MIXED, "data": "synthetic",
           "config": {"workload": WORKLOAD, "rhs_per_step": nrhs, "precision": "mixed (residual double-float)",
                      "l2": "inputs (1.1 GB of f) larger than L2, and a 256 MB write between steps",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                          "min": float(ms.min()), "max": float(ms.max()),
                          "note": "per batched step; every right-hand side of a step completes with it"},
           "timed_region_s": float(ms.sum()) / 1000.0,
           "solve": {"iterations_max": max(it), "iterations_min": min(it),
                     "refinements_max": max(s["refinements"] for s in st),
                     "applies_fp32_max": max(s["applies_fp32"] for s in st),
                     "applies_fp64_accurate_max": max(s["applies_fp64"] for s in st),
                     "rel_residual_max": max(s["rel_residual"] for s in st), "n_gm": n_gm,
                     "planes_transformed": npl, "plane_axis": "xyz"[conv_axis]},
           "gpu_launches": int(l1 - l0), "clocks": clk}
    if rank != 0 or args.only_timed:
        ctx.close()
        return out if rank == 0 else None
    interior = P0.phi < 0   # M+, where Algorithm 1 defines the solution
    ud = u.cpu().numpy()
    out["max_err_vs_exact"] = max(_rel_err(ud[k], probs[k].u_exact(), interior) for k in range(nrhs))

    # the same steps with float64 residual applies, after their own warm-up
    # (the first float64 apply of this batch size times the schedules)
    for _ in range(max(args.warmup, 1)):
        step("fp64")
    ms64, (q64, u64, st64) = _timed_loop(lambda: step("fp64"), args.steps, torch, flush)
    out["mixed_fp64_residual"] = {"value": nrhs * 1000.0 / float(ms64.mean()), "unit": UNIT,
                                  "ms_per_step": float(ms64.mean()), "steps": args.steps,
                                  "iterations_max": max(s["iterations"] for s in st64),
                                  "dtype": "f32 conv + f64 residual applies + f64 Gram-Schmidt/Givens"}
    u64d = u64.cpu().numpy()

    # per-kernel device times: two more steps with every launch bracketed by
    # events (kept out of the timed region, where the event records would
    # add host time to every step)
    hbm, hbm_kind = _peaks()
    profile_start(60 * max(l1 - l0, 1) // max(args.steps, 1) + 5000)
    for _ in range(2):
        _flush_l2(flush)
        step()
    torch.cuda.synchronize()
    prof = profile_stop()
    out["kernels"] = kernel_table(prof)
    dom = next((k["name"] for k in out["kernels"] if k["name"].startswith("conv_")), None)
    out["roofline"] = roofline_for(dom, prof[dom][0], prof[dom][1], N, n_gm, hbm, hbm_kind, npl, nrhs) \
        if dom else None
    out["conv_f32_apply"] = apply_summary(prof, N, npl, nrhs, hbm)

    # the plain float64 GPU form (and double-float throughout) on 8 of the
    # right-hand sides: solves/s at the same tolerance
    others = {}
    for label, prec in (("fp64", "fp64"), ("df64", "df64")):
        k8 = min(8, nrhs)
        pr = Problem(ctx, phi, P0.grid.h, P0.grid.origin, 0.0, "double")
        pr.solve_batched(f[:k8].contiguous(), g[:k8].contiguous(), tol=TOL, precision=prec)
        torch.cuda.synchronize()
        t = time.perf_counter()
        qo, uo, sto = pr.solve_batched(f[:k8].contiguous(), g[:k8].contiguous(), tol=TOL, precision=prec)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        pr.close()
        uo = uo.cpu().numpy()
        others[label] = {"solves_per_s": k8 / dt, "rhs": k8, "iterations_max": max(s["iterations"] for s in sto),
                         "u": uo}
    uf = others["fp64"]["u"]
    k8 = uf.shape[0]
    out["err_mixed_vs_fp64_gpu"] = max(_rel_err(ud[k], uf[k], interior) for k in range(k8))
    out["other_arithmetic"] = {k: {kk: vv for kk, vv in v.items() if kk != "u"} for k, v in others.items()}

    # --------------------------------------------------------- e2e (host)
    # through the public API with host buffers: phi, f and g copied in and
    # u and the densities copied out by the library inside every step (the
    # library copies the box of f that holds M+, the only part a solve
    # reads, and the same box of u, writing the zeros around it on the host;
    # the bytes below are what it reports having copied)
    pinned = [torch.from_numpy(f_h).pin_memory(), torch.from_numpy(g_h).pin_memory(),
              torch.from_numpy(P0.phi).pin_memory(), torch.empty(f_h.shape, dtype=torch.float64).pin_memory(),
              torch.empty((nrhs, n_gm), dtype=torch.float64).pin_memory()]
    f_pin, g_pin, phi_pin, u_pin, q_pin = (t.numpy() for t in pinned)
    e2e_ms = []
    for k in range(min(args.steps, 5) + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        pr = Problem(ctx, phi_pin, P0.grid.h, P0.grid.origin, 0.0, "double")
        _, _, st_e = pr.solve_batched(f_pin, g_pin, tol=TOL, precision="mixed", density=q_pin, u=u_pin)
        pr.close()
        dt = time.perf_counter() - t
        if k > 0:
            e2e_ms.append(dt * 1000.0)
    h2d = int(phi_pin.nbytes + sum(s["h2d_bytes"] for s in st_e))
    d2h = int(sum(s["d2h_bytes"] for s in st_e))
    out["e2e"] = {"value": nrhs * 1000.0 / float(np.mean(e2e_ms)), "unit": UNIT,
                  "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": len(e2e_ms),
                  "host_buffers": "pinned",
                  "host_input_bytes": int(phi_pin.nbytes + f_pin.nbytes + g_pin.nbytes),
                  "note": "the library copies f and u only in the box of planes that holds N+ and writes u's "
                          "zeros around it on host threads (it reports the bytes it copied)"}

    # --------------------------------------------------- secondary configs
    if not args.no_extra:
        out["torus128_kappa10"] = run_torus128_extra(ctx, torch, flush, hbm, hbm_kind)
        out["star256"] = run_star256_table(ctx, torch)
        out["serving"] = serving_run(2000)

    # --------------------------------------------------------- cpu baseline
    if world == 1 and not args.no_cpu:
        out["cpu_baseline"], uo = cpu_oracle_solve(probs[0])
        out["err_vs_oracle"] = {"mixed": _rel_err(ud[0], uo, interior),
                                "mixed_fp64_residual": _rel_err(u64d[0], uo, interior),
                                "fp64_gpu": _rel_err(uf[0], uo, interior),
                                "on": "M+ (interior nodes), max-norm relative, right-hand side 0"}
    ctx.close()
    return out


def run_torus128_extra(ctx, torch, flush, hbm, hbm_kind, steps=50, warmup=3):
    """Single right-hand side: kappa^2 = 10 torus, N = 128, u = sin 2x cos y
    e^z (mixed precision): solves/s, p50/p99, per-kernel roofline."""
    import workloads as W
    from paper_2502_05507_gb300 import Problem, profile_start, profile_stop
    P = W.torus_helmholtz(N, kappa2=10.0)
    phi = torch.from_numpy(P.phi).cuda()
    f = torch.from_numpy(P.f()).cuda()
    pr0 = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
    g = torch.from_numpy(P.g_at(np.asarray(pr0.boundary_points()))).cuda()
    n_gm = pr0.n_gm
    conv_axis, plo, phi_ = pr0.conv_planes()
    pr0.close()

    def step():
        pr = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
        r = pr.solve(f, g, tol=TOL, precision="mixed")
        pr.close()
        return r
    for _ in range(warmup):
        step()
    ms, (q, u, st) = _timed_loop(step, steps, torch, flush)
    profile_start(20000)
    for _ in range(3):
        _flush_l2(flush)
        step()
    torch.cuda.synchronize()
    prof = profile_stop()
    m = P.phi < 0
    dom = next((k["name"] for k in kernel_table(prof) if k["name"].startswith("conv_")), None)
    return {"workload": "torus R=0.5 r=0.2, kappa^2=10, N=128, u=sin2x cos y e^z, double layer, tol 1e-10, "
                        "one right-hand side", "solves_per_s": 1000.0 / float(ms.mean()), "steps": steps,
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "iterations": st["iterations"], "rel_residual": st["rel_residual"],
            "max_err_vs_exact": _rel_err(u.cpu().numpy(), P.u_exact(), m),
            "kernels": kernel_table(prof, 8),
            "roofline": roofline_for(dom, prof[dom][0], prof[dom][1], N, n_gm, hbm, hbm_kind, phi_ - plo, 1)
            if dom else None,
            "conv_f32_apply": apply_summary(prof, N, phi_ - plo, 1, hbm),
            "note": "N=128 single right-hand side: every buffer of the apply (~45 MB) stays in the 129 MB L2"}


def run_star256_table(ctx, torch, reps=3):
    """N=256 star, kappa^2 in {0, 1, 100}, double vs single layer: GMRES
    iterations and solves/s (mixed precision), with the float32 apply's
    bytes per second at this size."""
    import workloads as W
    from paper_2502_05507_gb300 import Problem, profile_start, profile_stop
    hbm, _ = _peaks()
    rows = []
    for k2 in (0.0, 1.0, 100.0):
        for layer in ("double", "single"):
            P = W.star(256, kappa2=k2, layer=layer)
            phi = torch.from_numpy(P.phi).cuda()
            f = torch.from_numpy(P.f()).cuda()
            pr0 = Problem(ctx, phi, P.grid.h, P.grid.origin, k2, layer)
            g = torch.from_numpy(P.g_at(np.asarray(pr0.boundary_points()))).cuda()
            n_gm = pr0.n_gm
            conv_axis, plo, phi_ = pr0.conv_planes()
            pr0.close()

            def step():
                pr = Problem(ctx, phi, P.grid.h, P.grid.origin, k2, layer)
                r = pr.solve(f, g, tol=TOL, precision="mixed", max_iter=2000, restart=400)
                pr.close()
                return r
            step()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                t = time.perf_counter()
                q, u, st = step()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t)
            row = {"kappa2": k2, "layer": layer, "iterations": st["iterations"],
                   "solves_per_s": 1.0 / float(np.median(ts)), "ms_p50": 1e3 * float(np.median(ts)),
                   "rel_residual": st["rel_residual"], "n_gm": n_gm,
                   "max_err_vs_exact": _rel_err(u.cpu().numpy(), P.u_exact(), P.phi < 0)}
            if k2 == 0.0 and layer == "double":
                profile_start(20000)
                torch.cuda.nvtx.range_push("star256_profiled")   # ncu --nvtx-include star256_profiled/
                step()
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_pop()
                prof = profile_stop()
                row["kernels"] = kernel_table(prof, 10)
                row["conv_f32_apply"] = apply_summary(prof, 256, phi_ - plo, 1, hbm)
            rows.append(row)
    return {"workload": "star r=0.6+0.1 sin5t cos3p, N=256, kappa^2 in {0,1,100}, double vs single layer, "
                        "u = exp(a.x), tol 1e-10, mixed precision", "table": rows,
            "solves_per_s_mean": float(np.mean([r["solves_per_s"] for r in rows]))}


def cpu_oracle_solve(P):
    """The oracle (FFT route, float64 scipy.fft on every host core) solving
    one right-hand side of the workload once; the LGF table is built
    beforehand and not timed (the GPU side caches it too)."""
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
    return ({"value": 1.0 / dt, "unit": UNIT, "cores": cores, "cpu": _cpu_model(), "kind": "oracle",
             "sample": f"one full oracle solve of right-hand side 0 of the workload (FFT route, {r.iterations} "
                       f"GMRES iterations, {dt:.1f} s); LGF table build ({t_table:.1f} s) excluded as cached"},
            r.u)


def run_reference(args):
    """The oracle as the reference arm, on the headline workload: each step
    (warm-up or timed) is one full oracle solve (FFT route, float64
    scipy.fft on all host cores, unpreconditioned MGS GMRES) of one of the 64
    right-hand sides, in order; solves/s = timed steps / their total time.
    The LGF table is built once before the steps (cached on both sides)."""
    import workloads as W
    from oracle import lgf as OL
    from oracle import potentials as OP
    from oracle import solve as OS
    cores = os.cpu_count() or 1
    dirs = W.torus_batch_dirs(64, seed=3)
    spec = OP.lgf_spectrum(OL.LGFTable(N, 0.0))
    k = 0

    def one():
        nonlocal k
        P = W.torus_poisson_dir(N, dirs[k % len(dirs)])
        k += 1
        t = time.perf_counter()
        r = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, 0.0, layer="double", tol=TOL,
                     potential="fft", spectrum=spec, workers=cores)
        return time.perf_counter() - t, r.iterations

    for _ in range(args.warmup):
        one()
    ts, its = [], []
    for _ in range(args.steps):
        dt, itn = one()
        ts.append(dt)
        its.append(itn)
    total = float(np.sum(ts))
    value = len(ts) / total if ts else 0.0
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * total / max(len(ts), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": _cpu_model(), "kind": "oracle",
                             "sample": f"each step one full oracle solve of one of the 64 right-hand sides (FFT "
                                       f"route, {int(np.median(its)) if its else 0} GMRES iterations median)"},
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
    phi = torch.from_numpy(P.phi).cuda()
    f = torch.from_numpy(P.f()).cuda()
    pr0 = Problem(ctx, phi, P.grid.h, P.grid.origin, 0.0, "double")
    g = torch.from_numpy(P.g_at(np.asarray(pr0.boundary_points()))).cuda()
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


def run_torus128(args):
    """The single right-hand side kappa^2 = 10 torus (N = 128) alone, with
    the given steps and warm-up."""
    import torch
    from paper_2502_05507_gb300 import Context
    ctx = Context(0)
    torch.cuda.set_stream(ctx.stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    hbm, hbm_kind = _peaks()
    t = run_torus128_extra(ctx, torch, flush, hbm, hbm_kind, steps=args.steps, warmup=args.warmup)
    ctx.close()
    return {"metric": METRIC, "value": t["solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": DTYPE_MIXED,
            "config": {"workload": t["workload"]}, **{k: v for k, v in t.items() if k != "workload"}}


def run_star256(args):
    import torch
    from paper_2502_05507_gb300 import Context
    ctx = Context(0)
    torch.cuda.set_stream(ctx.stream)
    t = run_star256_table(ctx, torch)
    ctx.close()
    return {"metric": METRIC, "value": t["solves_per_s_mean"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": DTYPE_MIXED, "config": {"workload": t["workload"]}, "table": t["table"]}


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
    phi = torch.from_numpy(P.phi).cuda()
    f = torch.from_numpy(P.f()).cuda()
    rows, us = [], {}
    for layer in ("direct", "double"):
        pr0 = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, layer)
        g = torch.from_numpy(P.g_at(np.asarray(pr0.boundary_points()))).cuda()
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
            "higher_is_better": True, "dtype": DTYPE_MIXED,
            "config": {"workload": "torus R=0.5 r=0.2, kappa^2=10, N=128, direct formulation (eq. direct_sys)"},
            "table": rows, "rel_diff_direct_vs_double_on_grid": diff}


def serving_run(nreq, slots=6, hbm_gb=96.0, seed=5):
    """The serving trace through bae_server: requests with N in {32, 64,
    128, 256}, kappa^2 in {0, 10}, random spheres / ellipsoids / tori,
    u = exp(a.x). phi and f are made on the device (torch) and passed as
    device pointers, u is written to the device, g comes from a host
    callback at the boundary points. The saturation throughput of the mix
    is measured first (64 requests submitted at once), then the trace
    arrives as a Poisson process at 0.8 x that rate. Latency = completion
    minus arrival, split into admission wait and service."""
    import torch
    import workloads as W
    from paper_2502_05507_gb300 import Server
    reqs = W.serving_trace(nreq, seed=seed)
    srv = Server(0, slots=slots, hbm_budget_bytes=int(hbm_gb * (1 << 30)))

    def submit(r):
        phi, f = W.trace_tensors(r, "cuda")
        u = torch.empty_like(f)
        torch.cuda.synchronize()          # the server's streams read them
        a = np.asarray(r["a"], dtype=np.float64)
        t = srv.submit(phi, 2.0 / r["N"], -1.0 + 1.0 / r["N"], f, lambda xyz, a=a: np.exp(xyz @ a),
                       kappa2=r["kappa2"], u_out=u)
        return t, (phi, f, u)

    def drain(ts):
        out = []
        for t, keep in ts:
            out.append(srv.poll(t))
            srv.release(t)
        return out

    drain([submit(r) for r in W.serving_trace(32, seed=seed + 100)])      # warm: spectra and slots
    t0 = time.perf_counter()
    drain([submit(r) for r in W.serving_trace(64, seed=seed + 200)])
    sat_rate = 64 / (time.perf_counter() - t0)
    lam = 0.8 * sat_rate
    gaps = np.random.default_rng(seed + 50).exponential(1.0 / lam, size=nreq)
    live, arrive = [], []
    start = time.perf_counter()
    tnext = start
    for r, gap in zip(reqs, gaps):
        tnext += gap
        d = tnext - time.perf_counter()
        if d > 0:
            time.sleep(d)
        arrive.append(srv.clock())
        live.append(submit(r))
    res = drain(live)
    wall = time.perf_counter() - start
    srv.close()
    lat = np.array([(x["t_done"] - a) * 1e3 for x, a in zip(res, arrive)])
    wait = np.array([(x["t_admit"] - a) * 1e3 for x, a in zip(res, arrive)])
    serv = np.array([(x["t_done"] - x["t_admit"]) * 1e3 for x in res])
    ok = sum(1 for x in res if x["status"] == 0)
    by_n = {}
    for n in (32, 64, 128, 256):
        sel = np.array([r["N"] == n for r in reqs])
        if sel.any():
            by_n[str(n)] = {"requests": int(sel.sum()), "latency_p50_ms": float(np.percentile(lat[sel], 50)),
                            "latency_p99_ms": float(np.percentile(lat[sel], 99)),
                            "service_p50_ms": float(np.percentile(serv[sel], 50)),
                            "wait_p50_ms": float(np.percentile(wait[sel], 50))}
    return {"solves_per_s": ok / wall, "requests": nreq, "completed": ok, "slots": slots,
            "arrival_rate_per_s": lam, "saturation_solves_per_s": sat_rate,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "admission_wait_ms": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
            "service_ms": {"p50": float(np.percentile(serv, 50)), "p99": float(np.percentile(serv, 99))},
            "by_N": by_n,
            "workload": f"serving trace, {nreq} Poisson-arrival requests at 0.8x saturation, N in {{32,64,128,256}}, "
                        f"kappa^2 in {{0,10}}, spheres/ellipsoids/tori (seed {seed}), mixed precision, tol 1e-10"}


def run_serving(args):
    """The serving trace alone (config 5): p50/p99 latency and solves/s."""
    t = serving_run(args.requests, args.slots, args.hbm_gb)
    return {"metric": METRIC, "value": t["solves_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": DTYPE_MIXED, "config": {"workload": t["workload"], "slots": t["slots"]},
            **{k: v for k, v in t.items() if k not in ("workload", "solves_per_s")}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the N=128 single-RHS and N=256 star keys")
    ap.add_argument("--workload", default="batched64",
                    choices=["batched64", "torus128", "sphere32", "star256", "serving", "direct128"])
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--nrhs", type=int, default=NRHS, help="batched64: right-hand sides (at most 64)")
    ap.add_argument("--slots", type=int, default=6, help="serving: concurrent slots")
    ap.add_argument("--hbm-gb", type=float, default=96.0, help="serving: device-memory budget")
    ap.add_argument("--only-timed", action="store_true",
                    help="warm-up and timed steps only (no profile, comparisons, e2e or CPU baseline)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    import torch
    extra = {"torus128": run_torus128, "sphere32": run_sphere32, "star256": run_star256, "serving": run_serving, "direct128": run_direct128}
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
