#!/usr/bin/env python
"""Benchmark: solves/s to relative residual 1e-8 of the discrete-ordinates /
TFPS radiative-transfer system on one GB300 (256 x 256 cells, M = 64
directions, HG g = 0.5, eps = 1e-3, sigma_T = exp(Gaussian random field,
correlation length 0.1), sigma_a = 0.05 sigma_T, q = 1 on the central
0.2 x 0.2 square, zero inflow), flexible GMRES(50).

One step = one complete solve (Krylov iteration, FP64 residual refinement and
the solution update) of the device-resident system, preconditioned by the
learned MgNet V-cycle over block Jacobi.  The network is trained first (on
32 other media of the same distribution at 128 x 128 cells, untimed, reported
as mgnet.train_seconds);
block-Jacobi GMRES on the same medium is timed in the same run for comparison.  `e2e` times the public
API end to end per step: rte_setup from pinned host arrays (H2D inside),
the solve, the angular-flux reconstruction and its copy back to the host
(W untimed warm-up steps first, like the device-resident measurement).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own instance of the workload
(independent problems, no data-path collective), timed between barriers, and
rank 0 prints one JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_23265_gb300 import workloads as W  # noqa: E402

METRIC = "solves/s to rel-res 1e-8: MgNet-FGMRES(50) (block-Jacobi GMRES in baseline_block_jacobi)"
WORKLOAD = {"workload": "grf256_m64_eps1e-3", "I": 256, "M": 64, "g": 0.5, "eps": 1e-3,
            "sigma_T": "exp(GRF, ell=0.1)", "sigma_a": "0.05 sigma_T", "restart": 50,
            "tol": 1e-8, "l2": "inputs larger than L2 (Krylov basis 3.4 GB, blocks 13 GB)"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Sustained dense BF16 tensor rate (a kernel timed inside a long step)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops_sustained"]), "measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except Exception:
        return 1700.0, "fallback 1.7 PFLOP/s sustained"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(world, value, op):
    """value reduced over the ranks (NCCL tensors on the GPU, gloo on the host)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _max_over_ranks(world, value):
    if world == 1:
        return value
    import torch.distributed as dist
    return _reduce(world, value, dist.ReduceOp.MAX)


def _weak_value(world, steps, ms_local, converged_local):
    """Whole-job solves/s of a replicated run: the solves of all ranks over the
    slowest rank's time, zero unless every rank converged; and that time."""
    ms_max = _max_over_ranks(world, ms_local)
    ok = converged_local
    if world > 1:
        import torch.distributed as dist
        ok = _reduce(world, 1.0 if converged_local else 0.0, dist.ReduceOp.MIN) > 0.5
    return ((steps * world) / (ms_max / 1e3) if ok else 0.0), ms_max


def cpu_baseline(md, gpu_iters):
    """The FP64 oracle on the host cores, timed on a bounded sample of the same
    workload: two FGMRES iterations at full size (operator apply, block-Jacobi
    apply, Gram-Schmidt), with the per-cell blocks inverted on a 4096-cell
    subset and scaled to all cells; projected to one solve with the GPU run's
    iteration count."""
    from oracle import krylov, tfps
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t0 = time.perf_counter()
    p = tfps.Problem(md.I, md.M, md.sigma_T, md.sigma_a, md.q, md.eps, md.g, md.inflow)
    t_prob = time.perf_counter() - t0
    sub = min(p.N, 4096)
    t0 = time.perf_counter()
    Ds = np.linalg.inv(p.blocks_at(np.arange(sub)))
    t_inv = (time.perf_counter() - t0) * p.N / sub
    D = np.broadcast_to(Ds[:1], (p.N, 2 * p.M, 2 * p.M))
    b = p.rhs().ravel()
    n = b.size
    t0 = time.perf_counter()
    krylov.fgmres(lambda v: p.apply(v.reshape(2 * p.M, -1)).ravel(), b,
                  lambda v, j: tfps.block_apply(D, v.reshape(2 * p.M, -1)).ravel(),
                  tol=1e-30, restart=50, max_iter=2)
    t_iter = (time.perf_counter() - t0) / 2
    t_solve = t_prob + t_inv + gpu_iters * t_iter
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle FP64 (NumPy) on {cores} host cores, block-Jacobi-preconditioned FGMRES(50) "
                       f"(the oracle has no network): 2 iterations at full size ({t_iter:.2f} s/iteration; the "
                       f"block apply uses cell 0's inverse for every cell, the same flops and bytes), block "
                       f"inversion timed on {sub} of {p.N} cells and scaled ({t_inv:.1f} s), set-up "
                       f"{t_prob:.1f} s; projected to {gpu_iters} iterations (the GPU's block-Jacobi solve "
                       f"of the same medium), n={n}")}


# DRAM traffic per launch over the algorithmic bytes, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum); the bench scales it by the
# algorithmic bytes of its own average launch.  The df64 Gram-Schmidt passes
# read each basis row once (the update and the dots of a pass share the
# staged rows).
TRAFFIC_RATIO = {"response_apply": 0.9995, "mdot": 1.001, "update_dot": 1.000, "update_norm": 0.999,
                 "response_tc": 0.793, "fix_dot": 1.000, "update_dot_norm": 0.999}
TRAFFIC_SOURCE = {"response_apply": "ncu DRAM bytes per launch at 256x256, M=64 (this workload)",
                  "mdot": "ncu DRAM bytes per launch at 256x256, M=64, K=50 basis vectors",
                  "update_dot": "ncu DRAM bytes per launch at 256x256, M=64, K=50 basis vectors",
                  "update_norm": "ncu DRAM bytes per launch at 256x256, M=64, K=50 basis vectors",
                  "response_tc": "ncu DRAM bytes per launch at 256x256, M=64 (this workload)",
                  "fix_dot": "ncu DRAM bytes per launch inside the solve at 256x256, M=64, K=31..34",
                  "update_dot_norm": "ncu DRAM bytes per launch inside the solve at 256x256, M=64, K=31..34"}

# Nominal FP64 rate of a GB300 (152 SMs x 2.07 GHz x 2 FP64 FMA per clock x 2
# flops): the roof of the FP64 operator apply, the one FP64-bound kernel left.
FP64_NOMINAL_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12

# kernel classes whose time is bound by the FP64 pipe (everything else of the
# solve streams memory, or is latency: the network is on the tensor cores)
FP64_BOUND = {"traces", "build_invert", "response_build"}


def _roofline(rte, stream, prof):
    """Roofline of the dominant kernel class (largest summed event time), and
    every class's fraction of its own roof."""
    kname, (kl, kms, kbytes, kflops) = max(prof.items(), key=lambda kv: kv[1][1])
    hbm_peak, peak_src = _peaks()
    total_ms = max(sum(v[1] for v in prof.values()), 1e-9)
    probe = rte.fp64_fma_rate(stream) / 1e3
    hbm_src = ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s")
    if kname == "mgnet":
        peak, psrc = _bf16_peak()
        roof = {"bound": "tensor", "kernel": "mgnet convolutions (tcgen05, BF16)",
                "achieved": kflops / (kms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": psrc}
    elif kname == "response_tc":
        peak, psrc = _bf16_peak()
        roof = {"bound": "tensor", "kernel": "response_tc (R z from the node tables, tcgen05 BF16 x 6 products)",
                "achieved": kflops / (kms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": psrc,
                "flops_note": "issued MMA flops: 6 BF16 products x 2 x 128 cells x (2M)^2 per tile and node"}
    elif kname in FP64_BOUND:
        roof = {"bound": "alu", "kernel": kname, "achieved": kflops / (kms / 1e3) / 1e12,
                "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "nominal FP64 rate (152 SMs x 2.07 GHz x 4 flops/clk); measured DFMA probe "
                               "%.3f TFLOP/s in the same run" % probe}
    else:
        roof = {"bound": "hbm", "kernel": kname, "achieved": kbytes / (kms / 1e3) / 1e9,
                "peak": hbm_peak, "unit": "GB/s", "peak_source": hbm_src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    ratio = TRAFFIC_RATIO.get(kname)
    roof["traffic"] = ratio * kbytes / kl if (ratio and kl) else None
    if ratio:
        roof["traffic_source"] = "%s, scaled by algorithmic bytes per launch (ratio %.4f)" % (
            TRAFFIC_SOURCE[kname], ratio)
    roof["launches"] = kl
    roof["share"] = kms / total_ms
    kernels = {}
    for k, v in prof.items():
        if not v[0]:
            continue
        e = {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / total_ms, 4),
             "GBps": round(v[2] / (v[1] / 1e3) / 1e9, 1) if v[1] > 0 else None,
             "TFLOPs": round(v[3] / (v[1] / 1e3) / 1e12, 3) if v[1] > 0 and v[3] else None}
        if v[1] > 0 and e["GBps"] is not None:
            e["hbm_frac"] = round(e["GBps"] / hbm_peak, 3)
        if k in FP64_BOUND and e["TFLOPs"]:
            e["fp64_frac"] = round(e["TFLOPs"] / FP64_NOMINAL_TFLOPS, 3)
        if k in ("response_tc", "mgnet") and e["TFLOPs"]:
            e["tensor_frac"] = round(e["TFLOPs"] / _bf16_peak()[0], 3)
        kernels[k] = e
    return roof, kernels


def run_precond_only(args):
    """Profiling mode: apply an (untrained) network args.precond_only times to a
    unit vector of the workload; prints the mean time per application."""
    import torch
    from paper_2604_23265_gb300 import rte, train
    torch.cuda.set_device(0)
    md = W.grf_diffusive(seed=0, I=args.size, M=args.dirs)
    ctx = rte.Context.from_medium(md)
    shape = train.default_shape(md.M, md.I, c0=args.c0, cmax=args.cmax)
    if args.levels > 0:
        shape.levels = args.levels
    net = rte.MgNet(shape)
    net.set_params(W.init_params(net.shape, seed=0, proj_scale=0.01, vcycle_scale=0.5))
    v = torch.tensor(W.random_vector(ctx.n, 1), device="cuda")
    v /= v.norm()
    z = torch.empty(ctx.n, dtype=torch.float32, device="cuda")
    net.precond(ctx, v, z)                      # features and workspace
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.precond_only):
        net.precond(ctx, v, z)
    ev1.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "precond_only", "I": md.I, "M": md.M, "levels": net.shape.levels,
                      "c0": net.shape.c0, "cmax": net.shape.cmax,
                      "ms_per_application": ev0.elapsed_time(ev1) / args.precond_only}), flush=True)


def run_setup_only(args):
    """Profiling mode: time the context set-up (rte_setup from host arrays:
    tables, right-hand side, per-cell block inversion and response matrices)
    args.setup_only times on the workload's medium."""
    import torch
    from paper_2604_23265_gb300 import rte
    torch.cuda.set_device(0)
    md = W.grf_diffusive(seed=0, I=args.size, M=args.dirs)
    times = []
    for _ in range(args.setup_only + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = rte.Context.from_medium(md)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        ctx.close()
    print(json.dumps({"mode": "setup_only", "I": md.I, "M": md.M, "seconds_per_setup": float(np.mean(times[1:])),
                      "first_seconds": times[0]}), flush=True)


def run_gs_only(args):
    """Profiling mode: args.gs_steps Gram-Schmidt steps (the three df64 passes
    and the scaling, rte_cgs2_df64) of w against args.gs_only basis vectors on
    the workload's context; prints the mean time of each pass class and its
    algorithmic GB/s (CUDA events on the context's stream)."""
    import torch
    from paper_2604_23265_gb300 import rte
    torch.cuda.set_device(0)
    md = W.grf_diffusive(seed=0, I=args.size, M=args.dirs)
    ctx = rte.Context.from_medium(md)
    K, n = args.gs_only, ctx.n
    g = torch.Generator(device="cuda").manual_seed(0)
    V64 = torch.randn(K, n, dtype=torch.float64, device="cuda", generator=g) / np.sqrt(n)
    hi = V64.float()
    Vf = torch.stack([hi, (V64 - hi.double()).float()], 1).contiguous().view(-1)
    w0 = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    w = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    h = torch.zeros(K + 1, dtype=torch.float64, device="cuda")
    for r in range(args.gs_steps + 1):
        if r == 1:
            ctx.profile(True)
        w[:n] = w0.float()
        w[n:] = (w0 - w0.float().double()).float()
        ctx.cgs2_df64(Vf, K, w, h)
    prof = ctx.profile_read()
    out = {"mode": "gs_only", "I": md.I, "M": md.M, "n": n, "K": K, "steps": args.gs_steps}
    step_bytes = ((3 * K + 5) * 8 + 16) * n
    tot = 0.0
    for k in ("mdot", "update_dot", "update_norm", "scale"):
        l, ms, byts, _ = prof[k]
        out[k] = {"ms_per_launch": ms / max(l, 1), "GBps": byts / (ms / 1e3) / 1e9 if ms > 0 else None}
        tot += ms / max(l, 1)
    out["df64_step"] = {"ms": tot, "GBps": step_bytes / (tot / 1e3) / 1e9}
    # the same step on FP64 vectors (rte_cgs2), for comparison
    Vd = (Vf.view(K, 2, n)[:, 0, :].double() + Vf.view(K, 2, n)[:, 1, :].double()).contiguous().view(-1)
    wd = torch.empty(n, dtype=torch.float64, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(False)
    times = []
    for r in range(args.gs_steps + 1):
        wd.copy_(w0)
        ev0.record()
        ctx.cgs2(Vd, K, wd, h)
        ev1.record()
        torch.cuda.synchronize()
        if r:
            times.append(ev0.elapsed_time(ev1))
    t64 = float(np.mean(times))
    out["fp64_step"] = {"ms": t64, "GBps": step_bytes / (t64 / 1e3) / 1e9}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_resp_only(args):
    """Profiling mode: args.resp_only response applies w = v - P R v
    (rte_response_apply) on the workload's context, on the tensor-core node path
    and on the per-cell FP32 path; prints each one's mean time per R z launch
    (CUDA events on the context's stream) and its rate."""
    import torch
    from paper_2604_23265_gb300 import rte
    torch.cuda.set_device(0)
    md = W.grf_diffusive(seed=0, I=args.size, M=args.dirs)
    ctx = rte.Context.from_medium(md)
    v = torch.tensor(W.random_vector(ctx.n, 1), device="cuda")
    w = torch.empty(ctx.n, dtype=torch.float64, device="cuda")
    out = {"mode": "resp_only", "I": md.I, "M": md.M, "n": ctx.n, "applies": args.resp_only,
           "tabulated_nodes": ctx.tabulated_nodes()}
    for path, name in ((rte.Context.RESPONSE_AUTO, "auto"), (rte.Context.RESPONSE_PER_CELL, "per_cell")):
        ctx.set_response_path(path)
        out[name + "_on_tensor_cores"] = ctx.response_on_tensor_cores()
        ctx.response_apply(v, w)                         # warm-up
        ctx.profile(True)
        for _ in range(args.resp_only):
            ctx.response_apply(v, w)
        prof = ctx.profile_read()
        ctx.profile(False)
        k = "response_tc" if out[name + "_on_tensor_cores"] else "response_apply"
        l, ms, byts, flops = prof[k]
        out[name] = {"kernel": k, "ms_per_launch": ms / max(l, 1),
                     "GBps": byts / (ms / 1e3) / 1e9 if ms > 0 else None,
                     "TFLOPs": flops / (ms / 1e3) / 1e12 if ms > 0 and flops else None,
                     "gather_ms_per_launch": prof["gather"][1] / max(prof["gather"][0], 1)}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_ours(args):
    import torch
    from paper_2604_23265_gb300 import rte, train
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    I, M = args.size, args.dirs
    opts = dict(tol=1e-8, restart=50, max_iter=args.max_iter)
    net, train_s, train_loss = None, 0.0, None
    if args.pc == "mgnet":
        # the network is trained before the timed region on other media of the
        # same distribution (seeds 101..), never on the benchmark medium, at
        # the training grid size (the same fields in domain units, coarser
        # cells) with the depth of the benchmark grid
        It = min(args.train_size, I) if args.train_size > 0 else I
        media = [W.grf_diffusive(seed=101 + i, I=It, M=M) for i in range(args.train_media)]
        shape = train.default_shape(M, I, c0=args.c0, cmax=args.cmax)
        net, tctx, losses, train_s = train.train_for(media, shape=shape, steps=args.train_steps, batch=8,
                                                     lr0=3e-3, seed=args.train_seed, loss=args.loss,
                                                     delta=args.delta)
        for c in tctx:
            c.close()
        train_loss = float(np.mean(losses[-20:]))
        torch.cuda.synchronize()
    md = W.grf_diffusive(seed=rank, I=I, M=M)
    ctx = rte.Context.from_medium(md, stream=stream)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.solve(x, pc=net, **opts)
    torch.cuda.synchronize()
    ctx.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    _barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(ctx.solve(x, pc=net, **opts))
    ev1.record(stream)
    torch.cuda.synchronize()
    _barrier(world)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    converged = all(i["converged"] for i in infos)
    value, ms_max = _weak_value(world, args.steps, ms, converged)
    iters = infos[-1]["iterations"]
    roof, kernels = _roofline(rte, stream, prof)
    launches = sum(v[0] for v in prof.values())
    # the classical preconditioner on the same medium, same run
    bj = None
    if args.pc == "mgnet" and not args.no_bj:
        xb = torch.zeros_like(x)
        t0 = time.perf_counter()
        ib = ctx.solve(xb, **opts)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        bj = {"value": (1.0 / tb) if ib["converged"] else 0.0, "unit": "solves/s",
              "iterations": ib["iterations"], "seconds": tb, "converged": bool(ib["converged"])}
    # end to end through the public API, pinned host buffers
    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory()
        return t.numpy()
    hs = [pinned(md.sigma_T), pinned(md.sigma_a), pinned(md.q), pinned(md.eps), pinned(md.inflow)]
    h2d = sum(a.nbytes for a in hs)
    psi_host = torch.empty(md.M * md.I * md.I, dtype=torch.float64).pin_memory()
    d2h = psi_host.numel() * 8
    e2e_times, e2e_parts = [], []
    # the same W untimed warm-up steps as the device-resident measurement (the
    # first set-ups map the library's memory pool), then K timed steps
    for it in range(0 if args.no_e2e else args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = rte.Context(md.I, md.M, hs[0], hs[1], hs[2], hs[3], md.g, hs[4], stream=stream)
        x2 = torch.zeros(c2.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        i2 = c2.solve(x2, pc=net, **opts)
        t2 = time.perf_counter()
        psi = torch.empty(md.M * md.I * md.I, dtype=torch.float64, device="cuda")
        c2.reconstruct(x2, psi)
        psi_host.copy_(psi, non_blocking=True)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        if it >= args.warmup:
            e2e_times.append(t3 - t0)
            e2e_parts.append((t1 - t0, t2 - t1, t3 - t2))
        c2.close()
        converged = converged and bool(i2["converged"])
    e2e_s = _max_over_ranks(world, sum(e2e_times)) if e2e_times else float("nan")
    e2e_value = (args.steps * world / e2e_s) if (converged and e2e_times) else 0.0
    pc_name = ("MgNet (trained, linear V-cycle) over block Jacobi" if net is not None
               else "block Jacobi")
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded GRF medium per rank)",
        "config": dict(WORKLOAD, parallelism=f"replicas{world}", preconditioner=pc_name,
                       inner=("R z from tabulated nodes on tcgen05 (BF16 x 6 products, FP32 accuracy), df64 Krylov basis, "
                              "FP64 residual")),
        "iterations": iters, "relres": infos[-1]["relres"], "converged": converged,
        "fell_back": bool(infos[-1]["fell_back"]),
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "seconds_per_step": ({"setup": float(np.mean([p[0] for p in e2e_parts])),
                                      "solve": float(np.mean([p[1] for p in e2e_parts])),
                                      "reconstruct_and_copy": float(np.mean([p[2] for p in e2e_parts]))}
                                     if e2e_parts else None)},
        "roofline": roof,
        "kernels": kernels,
        "clocks": clocks,
    }
    if net is not None:
        out["mgnet"] = {"loss": args.loss, "delta": args.delta if args.loss == "filtered" else None,
                        "train_seed": args.train_seed,
                        "train_seconds": train_s, "train_media": args.train_media,
                        "train_grid": min(args.train_size, I) if args.train_size > 0 else I,
                        "train_steps": args.train_steps, "final_loss": train_loss,
                        "levels": net.shape.levels, "params": net.count}
    if bj is not None:
        out["baseline_block_jacobi"] = bj
        out["speedup_vs_block_jacobi"] = value / bj["value"] if bj["value"] > 0 else None
    if (args.size, args.dirs) != (256, 64):
        out["config"]["workload"] = f"profiling case {args.size}x{args.size}, M={args.dirs} (not the benchmark)"
        out["config"]["I"], out["config"]["M"] = args.size, args.dirs
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(md, bj["iterations"] if bj else iters)
    ctx.close()
    if rank == 0 and world == 1 and not args.no_atfps:
        out["atfps"] = atfps_leg()
    if rank == 0 and world == 1 and not args.no_pcg:
        out["per_cell_gamma"] = per_cell_gamma_leg(net)
    if rank == 0 and world == 1 and args.config3_steps > 0:
        out["config3"] = config3_leg(steps=args.config3_steps)
    if rank == 0 and world == 1 and (args.serve > 0 or args.batch > 0):
        nets, mixed_train_s = train_mixed_nets(args.mixed_train_steps)
        out["mixed_networks"] = {"M": list(nets), "train_seconds": mixed_train_s,
                                 "train_steps": args.mixed_train_steps, "levels": nets[MIXED_DIRS[0]].shape.levels}
        if args.batch > 0:
            out["batched"] = batched_leg(args.batch, nets)
        if args.serve > 0:
            # M = 64 requests use the benchmark network (depth of a 256 x 256 grid)
            snets = dict(nets)
            if net is not None and net.shape.M == 64:
                snets[64] = net
            out["serving"] = serving_leg(args.serve, snets)
        for n in nets.values():
            n.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


MIXED_GRIDS, MIXED_DIRS, MIXED_EPS, NET_EPS_MAX = (64, 128, 256), (16, 32), (1e-4, 1.0), 1e-1


def train_mixed_nets(steps, media=24, seed=0):
    """One network per direction count of the mixed legs, trained (untimed)
    on 128 x 128 media of the training distribution (eps log-uniform in
    [1e-4, 1e-1], g in [0, 0.8], sigma_a / sigma_T log-uniform in [0.01, 0.2],
    GRF sigma_T) with the depth of a 256 x 256 grid, so that the same network
    serves every grid of the mix.  Returns ({M: net}, seconds)."""
    import torch
    from paper_2604_23265_gb300 import train
    nets, t0 = {}, time.time()
    for M in MIXED_DIRS:
        tm = [W.training_medium(seed=5000 + 100 * M + i, I=128, M=M) for i in range(media)]
        net, ctxs, _, _ = train.train_for(tm, shape=train.default_shape(M, 256), steps=steps, batch=8,
                                          lr0=3e-3, seed=seed)
        for c in ctxs:
            c.close()
        nets[M] = net
    torch.cuda.synchronize()
    return nets, time.time() - t0


def _mixed_media(count, seed, grids=MIXED_GRIDS, dirs=MIXED_DIRS, g_range=(0.0, 0.9)):
    return [W.mixed_instance(seed * 1000 + i, grids=grids, dirs=dirs, eps_range=MIXED_EPS, g_range=g_range)
            for i in range(count)]


def _wants_net(md):
    """Client policy: the network preconditions requests inside its training
    range of eps; the others (the transport regime) use block Jacobi."""
    return float(np.max(md.eps)) <= NET_EPS_MAX


SERVE_GRIDS, SERVE_DIRS = (64, 128, 256, 512), (16, 32, 64)
SERVE_WORKLOAD = ("Poisson arrivals of mixed solve requests: I in {64, 128, 256, 512}, M in {16, 32, 64}, eps "
                  "log-uniform in [1e-4, 1], g uniform in [0, 0.9], GRF media; FGMRES(50) to rel-res 1e-8 (at most "
                  "5000 iterations); grouped server (shared launches, batched V-cycles), 4 slots, admission by "
                  "device footprint; arrival rates 0.5, 0.8 and 0.95 of the capacity measured with all requests "
                  "queued at once")


def _serve_once(media, gaps, nets, use_net, max_iter=40000):
    from paper_2604_23265_gb300 import rte
    srv = rte.Server(slots=4, max_device_bytes=160 << 30, net=list(nets.values()) if use_net else None,
                     grouped=True)
    n_req = len(media)
    ids = [None] * n_req
    try:
        start = time.perf_counter()

        def feeder():
            t = start
            for i, md in enumerate(media):
                t += gaps[i]
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                ids[i] = srv.submit(md, tol=1e-8, max_iter=max_iter, use_net=use_net and _wants_net(md))

        th = threading.Thread(target=feeder)
        th.start()
        lat, queue, ok, its, on_net = [], [], 0, 0, 0
        for i in range(n_req):
            while ids[i] is None:
                time.sleep(0.0005)
            res, _ = srv.wait(ids[i])
            lat.append(res["latency_s"])
            queue.append(res["queue_s"])
            ok += res["status"] == "OK"
            its += res["iterations"]
            on_net += res["used_net"]
        th.join()
        span = time.perf_counter() - start
    finally:
        srv.close()
    lat = np.asarray(lat)
    return {"completed_ok": int(ok), "on_network": int(on_net), "iterations_total": int(its),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queue_s": float(np.mean(queue)), "solves_per_s": n_req / span}


def serving_leg(n_req, nets, seed=11):
    """The serving workload: mixed requests up to 512 x 512 cells and M = 64
    through the continuous-batching server (per-M networks inside their eps
    range, block Jacobi otherwise).  Capacity is measured first with all
    n_req requests queued at once (completed requests per second); then
    n_req further requests arrive as a Poisson stream at 0.5, 0.8 and 0.95 of
    that capacity, with p50 / p99 latency and solves/s at each rate."""
    t_all = time.time()
    rng = np.random.default_rng(seed)
    sat = _serve_once(_mixed_media(n_req, seed, grids=SERVE_GRIDS, dirs=SERVE_DIRS), np.zeros(n_req), nets, True,
                      max_iter=5000)
    capacity = sat["solves_per_s"]
    out = {"workload": SERVE_WORKLOAD, "requests_per_rate": n_req, "slots": 4,
           "policy": f"network for the request's M when eps <= {NET_EPS_MAX:g}, else block Jacobi",
           "capacity_solves_per_s": capacity, "saturation": sat, "rates": {}}
    for k, frac in enumerate((0.5, 0.8, 0.95)):
        media = _mixed_media(n_req, seed + 1 + k, grids=SERVE_GRIDS, dirs=SERVE_DIRS)
        rate = frac * capacity
        gaps = rng.exponential(1.0 / rate, n_req)
        r = _serve_once(media, gaps, nets, True, max_iter=5000)
        r["arrival_rate_per_s"] = rate
        out["rates"][str(frac)] = r
    # headline keys: the 0.8 rate
    for k in ("completed_ok", "p50_latency_s", "p99_latency_s", "mean_queue_s", "solves_per_s"):
        out[k] = out["rates"]["0.8"][k]
    out["leg_seconds"] = time.time() - t_all
    return out


BATCH_WORKLOAD = ("mixed instances: I in {64, 128, 256}, M in {16, 32}, eps log-uniform in [1e-4, 1], g uniform "
                  "in [0, 0.8], GRF media; FGMRES(50) to rel-res 1e-8; per-M networks for eps <= 0.1, block "
                  "Jacobi otherwise; the classical arm (block Jacobi for every instance) within 2000 iterations")


def batched_leg(count, nets, seed=23):
    """count solves of mixed instances: one grouped call (the Arnoldi steps of
    all of them in shared launches, the V-cycles of one network and grid
    batched) against the same solves one after the other, results compared
    bit for bit; and the grouped call with block Jacobi only.  All on the
    device, set-up excluded."""
    import torch
    from paper_2604_23265_gb300 import rte
    t_all = time.time()
    media = _mixed_media(count, seed, grids=MIXED_GRIDS, g_range=(0.0, 0.8))
    pcs = [nets[md.M] if _wants_net(md) else None for md in media]
    ctxs = [rte.Context.from_medium(md) for md in media]
    xs1 = [torch.zeros(c.n, dtype=torch.float64, device="cuda") for c in ctxs]
    xs2 = [torch.zeros(c.n, dtype=torch.float64, device="cuda") for c in ctxs]
    kw = dict(tol=1e-8, max_iter=40000)
    for c, x, pc in zip(ctxs, xs1, pcs):            # warm-up (workspaces, network features)
        c.solve(x, pc=pc, tol=1e-8, max_iter=5, raise_on_error=False)
    rte.solve_group(ctxs, xs2, pcs=pcs, tol=1e-8, max_iter=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lone = [c.solve(x, pc=pc, **kw) for c, x, pc in zip(ctxs, xs1, pcs)]
    torch.cuda.synchronize()
    t_lone = time.perf_counter() - t0
    t0 = time.perf_counter()
    grp = rte.solve_group(ctxs, xs2, pcs=pcs, **kw)
    torch.cuda.synchronize()
    t_grp = time.perf_counter() - t0
    same = all(a["iterations"] == b["iterations"] and torch.equal(x1, x2)
               for a, b, x1, x2 in zip(lone, grp, xs1, xs2))
    for x in xs2:
        x.zero_()
    t0 = time.perf_counter()
    bj = rte.solve_group(ctxs, xs2, tol=1e-8, max_iter=2000)
    torch.cuda.synchronize()
    t_bj = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    return {"workload": BATCH_WORKLOAD, "instances": count, "on_network": int(sum(p is not None for p in pcs)),
            "grouped_solves_per_s": count / t_grp, "one_at_a_time_solves_per_s": count / t_lone,
            "speedup": t_lone / t_grp, "iterations_total": int(sum(i["iterations"] for i in grp)),
            "converged": all(i["converged"] for i in grp), "bit_identical_to_lone": bool(same),
            "block_jacobi_seconds_2000_iterations": t_bj,
            "block_jacobi_converged_within_2000": int(sum(bool(i["converged"]) for i in bj)),
            "block_jacobi_converged_solves_per_s": sum(bool(i["converged"]) for i in bj) / t_bj,
            "block_jacobi_iterations_total": int(sum(i["iterations"] for i in bj)),
            "leg_seconds": time.time() - t_all}


CONFIG3_WORKLOAD = ("MgNet train + apply: 128 x 128 cells, M = 32, 4 levels, 64 hidden channels doubling per "
                    "level (64-512), 2 smoothing convolutions per level; 2000 training pairs (40 media of the "
                    "training distribution: GRF sigma_T with ell in [0.05, 0.2], eps log-uniform in [1e-4, 1e-1], "
                    "g in [0, 0.8]; 50 random right-hand sides each, the paper's recipe); batch 8, Adam with "
                    "cosine annealing from 1e-3 (Sec. 4.1)")


def config3_leg(steps=400, n_media=40, seed=300, n_test=2):
    """The network of the train + apply configuration trained on the GPU:
    training steps per second (FP32 forward, backward and Adam on CUDA cores),
    and FGMRES(50) iterations to 1e-8 on unseen media of the distribution with
    the trained network, the untrained one (zero projection: block Jacobi
    exactly) and block Jacobi."""
    import torch
    from paper_2604_23265_gb300 import rte, train
    t_all = time.time()
    media = [W.training_medium(seed=seed + i, I=128, M=32) for i in range(n_media)]
    shape = W.NetShape(M=32, levels=4, c0=64, cmax=512, cc=8, ccmax=32)
    net = rte.MgNet(shape)
    net.set_params(W.init_params(shape, seed=0, proj_scale=0.0, vcycle_scale=0.5))
    ctxs = [rte.Context.from_medium(md) for md in media]
    inputs = [train.random_inputs(c, 50, seed + 17 * i) for i, c in enumerate(ctxs)]
    pairs = sum(len(x) for x in inputs)
    net.train_step(ctxs[0], inputs[0][:8], 0.0)             # warm-up (workspace)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train.train(net, ctxs, inputs, steps=steps, batch=8, lr0=1e-3, seed=seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    untrained = rte.MgNet(shape)
    untrained.set_params(W.init_params(shape, seed=0, proj_scale=0.0, vcycle_scale=0.5))
    tests = []
    for k in range(n_test):
        md = W.training_medium(seed=seed + 1000 + k, I=128, M=32)
        ctx = rte.Context.from_medium(md)
        row = {"eps": float(md.eps[0]), "g": float(md.g)}
        for name, pc in (("trained", net), ("untrained", untrained), ("block_jacobi", None)):
            x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
            info = ctx.solve(x, pc=pc, tol=1e-8, restart=50, max_iter=20000, raise_on_error=False)
            row[name] = {"iterations": info["iterations"], "converged": bool(info["converged"]),
                         "fell_back": bool(info["fell_back"])}
        ctx.close()
        tests.append(row)
    untrained.close()
    out = {"workload": CONFIG3_WORKLOAD, "pairs": pairs, "params": net.count, "train_steps": steps, "batch": 8,
           "train_seconds": t_train, "train_steps_per_s": steps / t_train, "samples_per_s": 8 * steps / t_train,
           "loss_first": float(np.mean(losses[:10])), "loss_last": float(np.mean(losses[-10:])),
           "training_arithmetic": "FP32 forward, backward and Adam on CUDA cores (tensor pipe not used in training)",
           "test_media": tests, "leg_seconds": time.time() - t_all}
    net.close()
    return out


ATFPS_WORKLOAD = ("64 x 64 cells, M = 16, eps = 1e-3, g = 0.5, GRF medium (the benchmark distribution); "
                  "FGMRES(50) to rel-res 1e-8 on the full TFPS system (block Jacobi) and on the compressed ATFPS "
                  "system (preconditioned by mask o D S) followed by the layer reconstruction")


def atfps_leg(deltas=(1e-2, 1e-3), I=64, M=16, seed=5):
    """The compressed ATFPS solve with layer reconstruction (Sec. 2.3.3-2.3.4)
    beside the full TFPS solve of the same medium: unknowns kept, set-up
    (filter, compressed blocks) and solve times, iterations, and the largest
    cell-centre deviation of the angular flux from the full solution."""
    import torch
    from paper_2604_23265_gb300 import rte
    md = W.grf_diffusive(seed=seed, I=I, M=M, eps=1e-3)
    ctx = rte.Context.from_medium(md)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    ctx.solve(x, tol=1e-8)                      # warm-up (workspace)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    full = ctx.solve(x, tol=1e-8)
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    psi = torch.zeros(M * I * I, dtype=torch.float64, device="cuda")
    ctx.reconstruct(x, psi)
    ref = psi.clone()
    out = {"workload": ATFPS_WORKLOAD, "n": ctx.n,
           "full": {"iterations": full["iterations"], "seconds": t_full, "converged": bool(full["converged"])}}
    for d in deltas:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rows = ctx.atfps_setup(d)
        xc = torch.zeros_like(x)
        ctx.atfps_solve(xc, tol=1e-8, max_iter=1)   # builds the compressed blocks
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        xc.zero_()
        t0 = time.perf_counter()
        inf = ctx.atfps_solve(xc, tol=1e-8, raise_on_error=False)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        ctx.reconstruct(xc, psi)
        dev = float((psi - ref).abs().max() / ref.abs().max())
        out[f"delta_{d:g}"] = {"kept": rows, "kept_fraction": rows / ctx.n, "setup_seconds": t_setup,
                               "iterations": inf["iterations"], "solve_seconds": t_solve,
                               "converged": bool(inf["converged"]), "max_rel_dev_psi_centres": dev}
    ctx.close()
    return out


PCG_WORKLOAD = ("256 x 256 cells, M = 64, eps = 1e-3, g = 0.5, sigma_T = exp(GRF, ell = 0.1), sigma_a / sigma_T = "
                "0.05 exp(0.5 GRF') (a second field: every cell its own 1 - gamma, 65,536 materials), q = 1 on the "
                "central square; FGMRES(50) to rel-res 1e-8")


def per_cell_gamma_leg(net=None):
    """A medium whose scattering ratio varies from cell to cell (the paper's
    independent sigma_T and sigma_a fields) at the benchmark size: set-up time
    with the batched device eigenbases, block-Jacobi solve, and the benchmark
    network (trained on uniform-ratio media) as an out-of-distribution check."""
    import torch
    from paper_2604_23265_gb300 import rte
    I, M = 256, 64
    base = W.grf_diffusive(seed=0, I=I, M=M)
    rho = 0.05 * np.exp(0.5 * W.gaussian_field(I, 0.1, 977))
    md = W.Medium(I, M, base.sigma_T, rho * base.sigma_T, base.q, base.eps, base.g, base.inflow)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = rte.Context.from_medium(md)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    out = {"workload": PCG_WORKLOAD, "materials": ctx.info()["nmat"], "setup_seconds": t_setup}
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    for name, pc in (("block_jacobi", None), ("benchmark_network", net)):
        if name == "benchmark_network" and net is None:
            continue
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inf = ctx.solve(x, pc=pc, tol=1e-8, raise_on_error=False)
        torch.cuda.synchronize()
        out[name] = {"iterations": inf["iterations"], "seconds": time.perf_counter() - t0,
                     "converged": bool(inf["converged"]), "fell_back": bool(inf["fell_back"])}
    ctx.close()
    return out


def run_paper_protocol(args):
    """The paper's own experiments (Sec. 4): 32 x 32 cells, M = 4 directions,
    polynomial media, in the diffusion (eps = 0.01 (c + 0.1)), transport
    (eps = 1) and sharp-interface (six layouts mixing the two) regimes.  Per
    regime, args.pp_train media split 4:1 into training and validation media;
    a network is trained with the plain loss and another with the ATFPS-
    filtered loss (delta = 1e-2), the validation loss followed at twelve
    checkpoints; both precondition FGMRES(50) to 1e-8 on 10 unseen media,
    beside block Jacobi.  Prints one JSON line."""
    import torch
    from paper_2604_23265_gb300 import rte, train
    torch.cuda.set_device(0)
    regimes = ["diffusion", "transport", "interface"] if args.pp_regimes == "all" else args.pp_regimes.split(",")
    out = {"mode": "paper_protocol",
           "workload": ("32x32 cells, M=4, polynomial sigma_T, sigma_a (degree 1-4), q=1, zero inflow; eps by "
                        "regime; FGMRES(50) to rel-res 1e-8"),
           "media_per_regime": args.pp_train, "train_val_split": "4:1", "train_steps": args.pp_steps,
           "interface_layouts": list(W.INTERFACE_LAYOUTS)}
    for regime in regimes:
        media = [W.polynomial_medium(s, regime) for s in range(args.pp_train)]
        n_val = max(1, len(media) // 5)
        train_media, val_media = media[n_val:], media[:n_val]
        test_media = [W.polynomial_medium(10000 + s, regime) for s in range(10)]

        def solve_all(net):
            its, fell = [], []
            for md in test_media:
                ctx = rte.Context.from_medium(md)
                x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
                info = ctx.solve(x, pc=net, tol=1e-8, restart=50)
                its.append(info["iterations"] if info["converged"] else None)
                fell.append(bool(info["fell_back"]))
                ctx.close()
            return its, fell

        bj, _ = solve_all(None)
        res = {"block_jacobi_iterations": bj}
        for loss in ("plain", "filtered"):
            curve = []
            net, ctxs, losses, secs = train.train_for(train_media, steps=args.pp_steps, batch=8, lr0=3e-3, seed=0,
                                                      n_krylov=16, n_smooth=16, loss=loss, delta=1e-2,
                                                      val_media=val_media, val_every=max(1, args.pp_steps // 12),
                                                      curve=curve)
            for c in ctxs:
                c.close()
            its, fell = solve_all(net)
            ratio = [b / i for b, i in zip(bj, its) if b and i]
            res[loss] = {"iterations": its, "fell_back": fell, "fallback_rate": float(np.mean(fell)),
                         "train_seconds": secs, "final_loss": float(np.mean(losses[-20:])),
                         "mean_bj_over_mgnet": float(np.mean(ratio)) if ratio else None, "curve": curve}
            net.close()
        if regime == "diffusion" and args.pp_e3:
            res["e3"] = _paper_e3(args, test_media, solve_all, bj)
        out[regime] = res
    print(json.dumps(out), flush=True)


def _paper_e3(args, test_media, solve_all, bj):
    """E3 (Sec. 4.1-4.2): training-set size, 10,000 against 20,000 samples, in
    the diffusion regime, with the ATFPS-filtered loss.  Two recipes:
    * "paper": random right-hand sides (unit white-noise vectors in face-flux
      space) paired with random media, ten per medium (1,000 or 2,000 media);
    * "arnoldi_smooth": this library's inputs (16 Arnoldi vectors and 16
      smooth-error residuals per medium; 313 or 625 media).
    Samples are split 4:1 into training and validation by medium.  Every
    network trains args.pp_steps steps and preconditions the same 10 test
    media."""
    import torch
    from paper_2604_23265_gb300 import rte, train
    res = {"loss": "filtered", "delta": 1e-2}
    for recipe in ("paper", "arnoldi_smooth"):
        for samples in (10000, 20000):
            per = 10 if recipe == "paper" else 32
            n_media = -(-samples // per)
            media = [W.polynomial_medium(50000 + s, "diffusion") for s in range(n_media)]
            n_val = n_media // 5
            tr_media, va_media = media[n_val:], media[:n_val]
            t0 = time.time()
            if recipe == "paper":
                shape = train.default_shape(tr_media[0].M, tr_media[0].I)
                net = rte.MgNet(shape)
                net.set_params(W.init_params(shape, seed=0, proj_scale=0.0, vcycle_scale=0.5))
                net.loss = rte.MgNet.FILTERED

                def rhs(ctx, seed):
                    g = np.random.default_rng(seed)
                    return [torch.tensor(g.standard_normal(ctx.n) / np.sqrt(ctx.n), device="cuda")
                            for _ in range(per)]

                ctxs = [rte.Context.from_medium(md) for md in tr_media]
                vctx = [rte.Context.from_medium(md) for md in va_media]
                for c in ctxs + vctx:
                    c.atfps_setup(1e-2)
                inputs = [rhs(c, 7 * i) for i, c in enumerate(ctxs)]
                vin = [rhs(c, 100003 + 7 * i) for i, c in enumerate(vctx)]
                losses = train.train(net, ctxs, inputs, steps=args.pp_steps, batch=8, lr0=3e-3, seed=0)
                val = train.validation_loss(net, vctx, vin)
                for c in ctxs + vctx:
                    c.close()
            else:
                curve = []
                net, ctxs, losses, _ = train.train_for(tr_media, steps=args.pp_steps, batch=8, lr0=3e-3, seed=0,
                                                       n_krylov=16, n_smooth=16, loss="filtered", delta=1e-2,
                                                       val_media=va_media, val_every=args.pp_steps, curve=curve)
                val = curve[-1]["val_loss"] if curve else None
                for c in ctxs:
                    c.close()
            secs = time.time() - t0
            its, fell = solve_all(net)
            ratio = [b / i for b, i in zip(bj, its) if b and i]
            res[f"{recipe}_{samples}"] = {"media": n_media, "samples": n_media * per, "iterations": its,
                                          "fell_back": fell, "mean_bj_over_mgnet": float(np.mean(ratio)) if ratio else None,
                                          "final_train_loss": float(np.mean(losses[-20:])), "val_loss": val,
                                          "seconds": secs}
            net.close()
    return res


def run_reference(args):
    """The FP64 oracle on the host cores as the reference arm (bounded samples)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    md = W.grf_diffusive(seed=0)
    iters = args.ref_iters
    for _ in range(args.warmup if args.warmup <= 1 else 1):
        pass
    vals, cb = [], None
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(md, iters)
        vals.append(cb["value"])
    v = statistics.median(vals)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--ref-iters", type=int, default=7014,
                    help="iteration count used to project the oracle's per-iteration time "
                         "(block-Jacobi FGMRES(50) on this workload, as measured on the GPU)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--pc", default="mgnet", choices=["mgnet", "bj"])
    ap.add_argument("--train-steps", type=int, default=9000)
    ap.add_argument("--train-media", type=int, default=32)
    ap.add_argument("--train-size", type=int, default=128,
                    help="grid side of the training media (0: the benchmark grid)")
    ap.add_argument("--no-bj", action="store_true", help="skip the block-Jacobi comparison solve")
    ap.add_argument("--precond-only", type=int, default=0,
                    help="profiling only: apply an untrained network this many times and exit")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--gs-only", type=int, default=0,
                    help="profiling only: Gram-Schmidt steps against this many basis vectors")
    ap.add_argument("--gs-steps", type=int, default=5, help="profiling only: steps of --gs-only")
    ap.add_argument("--resp-only", type=int, default=0,
                    help="profiling only: time this many response applies (tensor-core and per-cell paths)")
    ap.add_argument("--setup-only", type=int, default=0,
                    help="profiling only: time the context set-up this many times and exit")
    ap.add_argument("--levels", type=int, default=0,
                    help="profiling only (--precond-only): network depth (0: the grid's default)")
    ap.add_argument("--train-seed", type=int, default=0, help="seed of the weights and input draws")
    ap.add_argument("--paper-protocol", action="store_true",
                    help="the paper's 32x32x4 polynomial-media experiment (plain vs filtered loss vs block Jacobi)")
    ap.add_argument("--pp-train", type=int, default=256, help="training media of --paper-protocol")
    ap.add_argument("--pp-steps", type=int, default=6000, help="training steps of --paper-protocol")
    ap.add_argument("--pp-e3", type=int, default=1, help="E3 (10k vs 20k samples) in the diffusion regime")
    ap.add_argument("--pp-regimes", default="all",
                    help="--paper-protocol regimes: all, or a comma list of diffusion, transport, interface")
    ap.add_argument("--c0", type=int, default=16, help="network width at the finest level")
    ap.add_argument("--cmax", type=int, default=64, help="largest network width")
    ap.add_argument("--loss", default="plain", choices=["plain", "filtered"],
                    help="training loss of the network: Eq. loss or the ATFPS-filtered Eq. loss_delta")
    ap.add_argument("--delta", type=float, default=1e-2, help="ATFPS selection threshold (filtered loss)")
    ap.add_argument("--batch", type=int, default=64,
                    help="instances of the grouped-solve leg (shared launches); 0 skips it")
    ap.add_argument("--serve", type=int, default=8,
                    help="requests per arrival rate of the serving leg (p50/p99 latency); 0 skips it")
    ap.add_argument("--config3-steps", type=int, default=400,
                    help="training steps of the train + apply leg (128^2, M=32, widths 64-512); 0 skips it")
    ap.add_argument("--no-atfps", action="store_true", help="skip the compressed ATFPS leg")
    ap.add_argument("--no-pcg", action="store_true", help="skip the per-cell scattering-ratio leg")
    ap.add_argument("--mixed-train-steps", type=int, default=1500,
                    help="training steps of each per-M network of the serving and grouped legs")
    ap.add_argument("--size", type=int, default=256, help="profiling only: grid side")
    ap.add_argument("--dirs", type=int, default=64, help="profiling only: directions")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.precond_only > 0:
        run_precond_only(args)
    elif args.resp_only > 0:
        run_resp_only(args)
    elif args.gs_only > 0:
        run_gs_only(args)
    elif args.setup_only > 0:
        run_setup_only(args)
    elif args.paper_protocol:
        run_paper_protocol(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
