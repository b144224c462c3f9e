#!/usr/bin/env python
"""Benchmark of the projection-method hot path on GB300: PCG DOF*iterations/s and time to the homogenized
coefficient a*.

Default workload (the configuration the metric is quoted on): d = 2 lifted to n = 4,
P = [[1, sqrt2, 0, 0], [0, 0, 1, sqrt3]], A = (5 + sum_j cos theta_j) I, 16^4 = 65,536 Fourier modes per field,
both correctors (e_1, e_2) by Jacobi-PCG to a relative residual of 1e-10 in FP64, then the 2 x 2 a*.
One step = corrector right-hand sides -> PCG solves -> a* reduction -> a* on the host, with the coefficient
already on the device (time-to-a*). Inputs are synthetic (seeded); L2 is flushed before every timed step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload cfg0..cfg4]
For N > 1 launch with torch.distributed.run; every rank solves its own replica (independent units, no
collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import os

# The CPU baseline is the single-threaded oracle; pin numpy's helper libraries to one thread so the reported
# core count is what it used.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qp_workloads as W  # noqa: E402

WORKLOADS = {
    "cfg0": ("d=1 n=2 P=(1,sqrt2) a=3+cos th1+cos th2, 32^2 modes, 1 corrector, Jacobi-PCG to 1e-12", "fp64"),
    "cfg1": ("d=2 n=4 P=[[1,sqrt2,0,0],[0,0,1,sqrt3]] A=(5+sum cos th_j)I, 16^4 modes, 2 correctors, "
             "Jacobi-PCG to 1e-10", "fp64"),
    "cfg2": ("d=2 n=4 full SPD 2x2 grid coefficient (81-tap field, eigenvalues clamped to [0.5,5]), 32^4 modes, "
             "2 correctors, FP32 PCG in FP64 refinement to 1e-10", "refine"),
    "cfg3": ("64 instances in one batched solve: 32 with d=1 n=2 P=(1,alpha) N in {64..512}, 32 with d=2 n=4 "
             "N in {8..24}; scalar cosine coefficients; 96 correctors, FP32 PCG in FP64 refinement to 1e-10", "refine"),
    "cfg4": ("d=3 n=6 diag A, a_i=4+sum_j 0.5cos(th_j+phi_ij), 16^6 modes, 3 correctors, FP32 PCG in FP64 "
             "refinement to 1e-10", "refine"),
    "tab2": ("Sec. 5.1.1 example (alpha_1, u_1): d=1 n=2 P=2pi(1,sqrt2), alpha=6+cos th1+cos th2, "
             "u=sin th1+sin th2, f=-div(alpha grad u) exact, 128^2 modes, Jacobi-PCG to 1e-14, L2_QP error", "fp64"),
}
# The paper's own number for the tab2 workload (Table 2, C-PCG at N = 128: 19 iterations of 16,384 unknowns in
# 17.32 s of MATLAB CPU time on a laptop): 1.8e4 DOF*iter/s. Context, not the target.
PAPER_TAB2_DOF_ITER_PER_S = 19 * 16384 / 17.32
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 rate (CUDA cores); the FMA-loop probe measured 1.196


def instance(name, N=None):
    """The workload's instance (for the batched cfg3: its largest instance, used for samples and the apply)."""
    if name == "cfg3":
        return W.cfg3()[-1]
    if name == "tab2":
        return W.paper_elliptic_u1(N or 128)
    return getattr(W, name)() if N is None else getattr(W, name)(N=N)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


# ---------------------------------------------------------------------------------------------- roofline model

def apply_flops_per_dof(kind, d, ntaps, real, nrhs, stored=False):
    """Algorithmic flops of one stiffness apply per mode, taps backend: per tap and right-hand side the complex
    multiply-accumulate with h (4 flops real weight, 8 complex), and unless the plan stores its weights Q_ij
    (formed once at plan creation, then only read) per tap the weight lambda(k)^T C_t lambda(k -N m_t)
    (scalar: 2d, diag: 3d, sym: 3d^2; doubled for complex taps)."""
    w = 0 if stored else {"scalar": 2 * d, "diag": 3 * d, "sym": 3 * d * d}[kind] * (1 if real else 2)
    return ntaps * (w + nrhs * (4 if real else 8))


# ---------------------------------------------------------------------------------------------- ranks

def shard(n_units, rank, world):
    """The independent units (instances) of rank: round robin, every unit on exactly one rank."""
    return list(range(rank, n_units, world))


def reduce_over_ranks(x, world, device, op="max"):
    """max (time) or sum (work) of a host scalar over the ranks; the identity for one rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def update_flops_per_dof():
    """Flops of one PCG vector update per mode and right-hand side (Algorithm 2): U += alpha h, r -= alpha Q h
    (8), (r, M r) and |r|^2 (5), h = M r + beta h (6), rounded up to 20 with alpha/beta bookkeeping."""
    return 20


def fft_apply_bytes(d, ncomp, nrhs, D, es):
    """Algorithmic bytes of the FFT-backend apply on the three-pass schedule: per right-hand side read h and
    write w (2 es) and the d gradient fields written, read + written, read (4 d es) per mode; the coefficient
    samples (ncomp reals of es / 2 bytes) once."""
    return nrhs * D * es * (2 + 4 * d) + ncomp * D * (es // 2)


# Per-launch DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels below, from one ncu capture
# of the current kernel each (summaries and commands under profiles/); None where no capture of the current kernel
# exists.
TRAFFIC = {
    # cfg1: one solve (33 iterations, 2 correctors) in k_pcg_persistent; vectors and stored weights stay in L2
    ("k_pcg_persistent", "cfg1"): 9572352 + 236032,
    # cfg4: k_apply_plain_star (geometry compiled in) captured at N = 14 (7.53 M modes; h and w exceed L2), scaled
    # by 16^6 / 14^6
    ("k_apply_plain", "cfg4"): int((207640320 + 153260032) * (16 ** 6 / 14 ** 6)),
    # cfg2: the three fused passes of one FP32 apply (the gradient fields stay in L2 between passes)
    ("k_fft_group", "cfg2"): 16874752 + 9472 + 46255616 + 0 + 33646848 + 0,
}


def measured_traffic(kernel_key, workload):
    return TRAFFIC.get((kernel_key, workload))


def persistent_roofline(qp, plan, inst, pinfo, real, tol, stream, dev):
    """The persistent FP64 solve kernel (one launch per qp_pcg_solve when the automatic execution picks it):
    algorithmic flops of its applies and vector updates per launch / its event-timed duration. Returns None
    when this plan's solve is not a single persistent launch."""
    import torch
    nrhs = inst.d
    F = torch.zeros((nrhs, inst.D), dtype=torch.complex128, device=dev)
    qp.qp_corrector_rhs(plan, 0, nrhs, F)
    U = torch.zeros_like(F)
    torch.cuda.synchronize()
    l0 = qp.qp_launch_count()
    infos = qp.qp_pcg_solve(plan, F, U, tol=tol, maxit=2000)
    if qp.qp_launch_count() - l0 != 1:
        return None
    reps = 20
    ms = 0.0
    for _ in range(reps):
        U.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = qp.qp_pcg_solve(plan, F, U, tol=tol, maxit=2000)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    ms /= reps
    its = [i["iterations"] for i in infos]
    c = inst.coeff
    # every iteration applies Q to all right-hand sides; plus the warm-start apply and the final true residual
    applies = max(its) + 2
    stored = bool(pinfo.get("stored_weights"))
    flops = (applies * apply_flops_per_dof(c.kind, inst.d, pinfo["ntaps"], real, nrhs, stored) * inst.D
             + sum(its) * update_flops_per_dof() * inst.D)
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": round(achieved, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": None,
            "kernel": "k_pcg_persistent (whole FP64 PCG solve in one cooperative launch), timed alone on the bench "
                      "stream (the events also bracket two 4-byte memsets and the solver-state read-back)",
            "kernel_key": "k_pcg_persistent", "launch_us": round(ms * 1e3, 2), "flops_per_launch": flops,
            "iterations": its, "stored_weights": stored,
            "peak_source": "nominal FP64 1.25 TFLOP/s (FMA-loop probe on GB300: 1.196)"}


def apply_roofline(qp, plan, inst, pinfo, real, mode_name, stream, dev):
    """The stiffness apply in the precision of the workload's bulk iterations, timed alone."""
    import torch
    nrhs = inst.d
    prec = qp.QP_FP64 if mode_name == "fp64" else qp.QP_FP32
    dt = torch.complex128 if prec == qp.QP_FP64 else torch.complex64
    es = 16 if prec == qp.QP_FP64 else 8
    h = torch.randn((nrhs, inst.D), dtype=dt, device=dev)
    w = torch.empty_like(h)
    for _ in range(5):
        qp.qp_apply_stiffness(plan, h, w, prec)
    reps = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        qp.qp_apply_stiffness(plan, h, w, prec)
    e1.record(stream)
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / reps
    c = inst.coeff
    pk = peaks()
    if prec == qp.QP_FP64 and c.taps_k is not None:
        stored = bool(pinfo.get("stored_weights"))
        flops = apply_flops_per_dof(c.kind, inst.d, pinfo["ntaps"], real, nrhs, stored) * inst.D
        achieved = flops / (apply_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": round(achieved, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": None,
                "kernel": "k_apply_plain<double> (taps stencil, FP64 pipe), timed alone on the bench stream",
                "kernel_key": "k_apply_plain<double>", "apply_us": round(apply_ms * 1e3, 2), "flops_per_launch": flops,
                "peak_source": "nominal FP64 1.25 TFLOP/s (FMA-loop probe on GB300: 1.196)"}
    if c.taps_k is not None:
        bytes_ = 2 * nrhs * inst.D * es
        kernel, key = "k_apply_plain (taps stencil; read h, write w), timed alone", "k_apply_plain"
    else:
        from qp_workloads import ncomp
        bytes_ = fft_apply_bytes(inst.d, ncomp(c.kind, inst.d), nrhs, inst.D, es)
        kernel, key = ("FFT-backend apply (fused group passes), timed alone; bytes of the three-pass schedule",
                       "k_fft_group")
    achieved = bytes_ / (apply_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": None, "kernel": kernel, "kernel_key": key,
            "apply_us": round(apply_ms * 1e3, 2), "bytes_per_launch": bytes_,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" + (" (fallback)" if pk.get("_fallback") else "")}


# ---------------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region runs."""
    Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        # the raw samples (the JSON line carries their summary); QP_BENCH_CLOCKS_CSV chooses the file
        self.path = os.environ.get("QP_BENCH_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                          "qp_bench_clocks.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.bus_id and self.bus_id[-12:] not in parts[1].lower():
                continue
            rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2404_06841_gb300 as qp

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    name = args.workload
    desc, default_mode = WORKLOADS[name]
    mode_name = args.mode or default_mode
    mode = qp.QP_MODE_FP64 if mode_name == "fp64" else qp.QP_MODE_FP32_REFINE
    exec_mode = {"auto": qp.QP_EXEC_AUTO, "graph": qp.QP_EXEC_GRAPH, "direct": qp.QP_EXEC_DIRECT,
                 "persistent": qp.QP_EXEC_PERSISTENT}[args.exec]
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2 (129 MiB)
    if name == "cfg3":
        # independent instances: with several ranks each solves its share (no collective on the data path)
        all_insts = W.cfg3()
        insts = [all_insts[i] for i in shard(len(all_insts), rank, world)]
        tol = 1e-10
        plans = [qp.plan_from_instance(i, exec_mode=exec_mode) for i in insts]
        batch = qp.qp_batch_create(plans)
        unit_D = [i.D for i in insts for _ in range(i.d)]
        inst = insts[-1]
        plan = plans[-1]
        total_D = sum(unit_D)

        def step():
            As, infs = qp.qp_batch_homogenized(batch, tol=tol, mode=mode, maxit=2000)
            return As, infs

        def dof_iters(infs):
            return sum(D * (i["iterations"] + i["outer_iterations"]) for D, i in zip(unit_D, infs))
    elif name == "tab2":
        # the general elliptic solve with a user right-hand side: f is Q applied to the exact coefficients of u
        # (exact on K_N^n for N >= 8, no aliasing), then the L2_QP error of the computed solution
        inst = instance(name, args.N)
        tol = inst.tol
        plan = qp.plan_from_instance(inst, max_rhs=1, exec_mode=exec_mode)
        total_D = inst.D
        Uex = torch.from_numpy(W.modes_on_grid(inst.N, inst.meta["u_modes"], inst.meta["u_amps"])[None].copy()).to(dev)
        Fd = torch.empty_like(Uex)
        qp.qp_apply_stiffness(plan, Uex, Fd, qp.QP_FP64)
        Ud = torch.zeros_like(Fd)

        def step(m=mode):
            Ud.zero_()
            infs = qp.qp_pcg_solve(plan, Fd, Ud, tol=tol, maxit=2000, mode=m)
            return qp.qp_l2qp_error(plan, Ud, Uex), infs

        def dof_iters(infs):
            return sum(inst.D * (i["iterations"] + i["outer_iterations"]) for i in infs)
    else:
        inst = instance(name, args.N)
        tol = inst.tol
        plan = qp.plan_from_instance(inst, exec_mode=exec_mode)
        total_D = inst.D * inst.d

        def step():
            return qp.qp_homogenized(plan, tol=tol, mode=mode, maxit=2000)

        def dof_iters(infs):
            return sum(inst.D * (i["iterations"] + i["outer_iterations"]) for i in infs)
    pinfo = qp.qp_plan_query(plan)

    for _ in range(max(args.warmup, 3)):
        A, infos = step()
    dof_iters_step = dof_iters(infos)

    sampler = ClockSampler(None)
    sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = qp.qp_launch_count()
    wall0 = time.perf_counter()
    total_dof_iters = 0
    max_rel = 0.0
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        A, infos = step()
        ends[k].record(stream)
        total_dof_iters += dof_iters(infos)
        max_rel = max(max_rel, max(i["rel_residual"] for i in infos))
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    launches = qp.qp_launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    t_sec = reduce_over_ranks(ms / 1e3, world, dev, "max")
    value = reduce_over_ranks(total_dof_iters, world, dev, "sum") / t_sec

    # ---- roofline of the dominant kernel, timed with CUDA events on this stream
    c = inst.coeff
    real = bool(np.all(np.asarray(c.taps_val).imag == 0)) if c.taps_k is not None else False
    roof = None
    if mode_name == "fp64" and c.taps_k is not None and name != "cfg3":
        roof = persistent_roofline(qp, plan, inst, pinfo, real, tol, stream, dev)
    if roof is None:
        roof = apply_roofline(qp, plan, inst, pinfo, real, mode_name, stream, dev)
    roof["traffic"] = measured_traffic(roof["kernel_key"], name)

    # ---- end to end through the public API with host inputs: plan from host taps -> a* on the host
    e2e = None
    if name == "tab2":
        # plan from host taps, the right-hand side copied from pinned host memory, solve, e_N read back
        kk = np.ascontiguousarray(c.taps_k, dtype=np.int32)
        vv = np.ascontiguousarray(np.asarray(c.taps_val, dtype=np.complex128))
        Fh = Fd.cpu().pin_memory()
        h2d = kk.nbytes + vv.nbytes + inst.P.nbytes + 4 * inst.n + Fh.numel() * 16
        d2h = 8
        e2e_steps = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            p2 = qp.qp_plan_create(inst.d, inst.n, inst.P, inst.N, W.Coefficient(c.kind, kk, vv), max_rhs=1)
            F2 = Fh.to(dev, non_blocking=True)
            U2 = torch.zeros_like(F2)
            qp.qp_pcg_solve(p2, F2, U2, tol=tol, maxit=2000, mode=mode)
            qp.qp_l2qp_error(p2, U2, Uex)
            qp.qp_plan_destroy(p2)
        torch.cuda.synchronize()
        e2e_t = (time.perf_counter() - t0) / e2e_steps
        e2e = {"value": world * dof_iters_step / e2e_t, "unit": "DOF*iter/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_t * 1e3, 3),
               "what": "qp_plan_create(host taps) + f host->device + qp_pcg_solve + qp_l2qp_error + destroy"}
    elif name == "cfg3":
        # every step: the batch's plans from host taps, the batch, the batched solve, a* on the host, destroy
        hk = [(np.ascontiguousarray(i.coeff.taps_k, dtype=np.int32),
               np.ascontiguousarray(np.asarray(i.coeff.taps_val, dtype=np.complex128))) for i in insts]
        h2d = sum(k.nbytes + v.nbytes + i.P.nbytes + 4 * i.n for (k, v), i in zip(hk, insts))
        d2h = sum(16 * i.d * i.d for i in insts)
        e2e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ps = [qp.qp_plan_create(i.d, i.n, i.P, i.N, W.Coefficient(i.coeff.kind, k, v))
                  for (k, v), i in zip(hk, insts)]
            b2 = qp.qp_batch_create(ps)
            qp.qp_batch_homogenized(b2, tol=tol, mode=mode, maxit=2000)
            qp.qp_batch_destroy(b2)
            for p2 in ps:
                qp.qp_plan_destroy(p2)
        torch.cuda.synchronize()
        e2e_t = (time.perf_counter() - t0) / e2e_steps
        e2e = {"value": world * dof_iters_step / e2e_t, "unit": "DOF*iter/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_t * 1e3, 3),
               "what": "64 x qp_plan_create(host taps) + qp_batch_create + qp_batch_homogenized + destroy per step"}
    elif c.grid is not None:
        # every step: the coefficient samples copied from pinned host memory, plan, a* on the host, destroy
        gh = torch.from_numpy(np.ascontiguousarray(c.grid, dtype=np.float64)).pin_memory()
        h2d = gh.numel() * 8 + inst.P.nbytes + 4 * inst.n
        d2h = 16 * inst.d * inst.d
        e2e_steps = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            gd = gh.to(dev, non_blocking=True)
            p2 = qp.qp_plan_create(inst.d, inst.n, inst.P, inst.N, W.Coefficient(c.kind, grid=gd))
            qp.qp_homogenized(p2, tol=tol, mode=mode, maxit=2000)
            qp.qp_plan_destroy(p2)
        torch.cuda.synchronize()
        e2e_t = (time.perf_counter() - t0) / e2e_steps
        e2e = {"value": world * dof_iters_step / e2e_t, "unit": "DOF*iter/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_t * 1e3, 3),
               "what": "coefficient samples host->device + qp_plan_create(grid) + qp_homogenized + destroy per step"}
    elif c.taps_k is not None:
        kk = np.ascontiguousarray(c.taps_k, dtype=np.int32)
        vv = np.ascontiguousarray(np.asarray(c.taps_val, dtype=np.complex128))
        h2d = kk.nbytes + vv.nbytes + inst.P.nbytes + 4 * inst.n
        d2h = 16 * inst.d * inst.d
        e2e_steps = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            p2 = qp.qp_plan_create(inst.d, inst.n, inst.P, inst.N, W.Coefficient(c.kind, kk, vv))
            qp.qp_homogenized(p2, tol=tol, mode=mode, maxit=2000)
            qp.qp_plan_destroy(p2)
        torch.cuda.synchronize()
        e2e_t = (time.perf_counter() - t0) / e2e_steps
        e2e = {"value": world * dof_iters_step / e2e_t, "unit": "DOF*iter/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_t * 1e3, 3),
               "what": "qp_plan_create(host taps) + qp_homogenized + qp_plan_destroy per step"}

    # ---- the other precision mode on the same workload (time-to-a*), for the FP64-vs-refinement comparison
    variants = {}
    other = "refine" if mode_name == "fp64" else "fp64"
    if not args.no_variants and name == "tab2":
        om = qp.QP_MODE_FP32_REFINE if other == "refine" else qp.QP_MODE_FP64
        for _ in range(3):
            step(om)
        ts = []
        for _ in range(max(5, min(args.steps, 20))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2_, inf2 = step(om)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        variants[other] = {"time_to_solution_ms": round(statistics.median(ts), 4),
                           "iterations": [(i["iterations"], i["outer_iterations"]) for i in inf2],
                           "e_N": float(e2_[0])}
    elif not args.no_variants and name != "cfg3":
        om = qp.QP_MODE_FP32_REFINE if other == "refine" else qp.QP_MODE_FP64
        for _ in range(3):
            qp.qp_homogenized(plan, tol=tol, mode=om, maxit=2000)
        ts = []
        for _ in range(max(5, min(args.steps, 20))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            A2, inf2 = qp.qp_homogenized(plan, tol=tol, mode=om, maxit=2000)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        di = sum(inst.D * (i["iterations"] + i["outer_iterations"]) for i in inf2)
        variants[other] = {"time_to_astar_ms": round(statistics.median(ts), 4),
                           "dof_iter_per_s": di / (statistics.median(ts) / 1e3),
                           "iterations": [(i["iterations"], i["outer_iterations"]) for i in inf2],
                           "max_abs_astar_diff_vs_main": float(np.abs(A2 - A).max())}

    # ---- the paper's Frobenius-optimal diagonal (Sec. 4.3) against Jacobi on the same solve (iterations, time)
    if not args.no_variants and name not in ("cfg3", "tab2"):
        P_F = qp.QP_PRECOND_FROBENIUS
        qp.qp_homogenized(plan, tol=tol, mode=mode, maxit=4000, precond=P_F)        # builds the diagonal once
        ts = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            A3, inf3 = qp.qp_homogenized(plan, tol=tol, mode=mode, maxit=4000, precond=P_F)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        variants["frobenius"] = {"time_to_astar_ms": round(statistics.median(ts), 4),
                                 "iterations": [(i["iterations"], i["outer_iterations"]) for i in inf3],
                                 "jacobi_iterations": [(i["iterations"], i["outer_iterations"]) for i in infos],
                                 "max_abs_astar_diff_vs_main": float(np.abs(A3 - A).max())}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(name, max_seconds=args.cpu_seconds)

    out = {
        "metric": ("PCG DOF*iter/s (time-to-solution at 1e-14)" if name == "tab2"
                   else "PCG DOF*iter/s (time-to-a* at 1e-10)"),
        "value": value,
        "unit": "DOF*iter/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "strong" if name == "cfg3" else "weak",
        "vs_baseline": (value / PAPER_TAB2_DOF_ITER_PER_S) if name == "tab2" else None,
        "dtype": "f64" if mode_name == "fp64" else "f32+f64-refine",
        "data": "synthetic",
        "config": {"workload": name + ": " + desc, "D": total_D if name == "cfg3" else inst.D,
                   "correctors": len(infos), "mode": mode_name, "exec": args.exec,
                   "backend": pinfo["backend"], "tol": tol, "l2": "flushed before every step (256 MiB write)",
                   "parallelism": ("single GPU" if world == 1 else
                                   "instances sharded over %d ranks" % world if name == "cfg3" else
                                   "replicas on %d ranks" % world)},
        "time_to_astar_ms": ms / args.steps,
        "iterations_per_step": [(i["iterations"], i["outer_iterations"]) for i in infos],
        "max_rel_residual": max_rel,
        "astar": (None if name == "tab2" else np.round(A.real, 14).tolist() if name != "cfg3" else
                  [np.round(a, 12).tolist() for a in (A[:2] + A[-2:])]),
        "wall_s_timed_region": wall1 - wall0,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "variants": variants,
    }
    if name == "tab2":
        out["e_N"] = float(A[0])
        out["vs_baseline_note"] = ("value / 1.8e4 DOF*iter/s, the paper's Table 2 C-PCG run at N = 128 (MATLAB on a laptop "
                                   "CPU): context only")
        out["time_to_solution_ms"] = out.pop("time_to_astar_ms")
    if name == "cfg3":
        qp.qp_batch_destroy(batch)
        for p_ in plans:
            qp.qp_plan_destroy(p_)
    else:
        qp.qp_plan_destroy(plan)
    return out


def cpu_baseline(name, max_seconds=12.0):
    """The FP64 oracle (numpy, one thread) on a bounded sample of the same workload: Algorithm 2 on corrector 1
    for as many iterations as fit in about max_seconds."""
    from oracle import qp_oracle as O
    inst = instance(name)
    dof_iters, secs, iters = O.timed_pcg_sample(inst, max_seconds=max_seconds)
    return {"value": dof_iters / secs, "unit": "DOF*iter/s", "cores": 1, "kind": "oracle",
            "sample": "%s corrector e_1: %d oracle PCG iterations (incl. initial and final true-residual applies), "
                      "%.1f s, numpy FP64 single thread" % (name, iters, secs)}


# ---------------------------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle as it stands, on the host cores: each step is 2 oracle PCG iterations of corrector e_1 of the
    same workload (a bounded sample); value in the same unit."""
    from oracle import qp_oracle as O
    inst = instance(args.workload)
    op = O.Operator(inst)
    M = O.jacobi_inverse(op.P, op.N, op.Ahat)
    F = O.corrector_rhs(op.P, op.N, op.Ahat, 0)
    for _ in range(max(args.warmup, 1)):
        O.pcg(op, F, M, tol=0.0, maxit=1)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        _, info = O.pcg(op, F, M, tol=0.0, maxit=2)
        its += info["iterations"] + 2
    secs = time.perf_counter() - t0
    v = inst.D * its / secs
    desc = WORKLOADS[args.workload][0]
    return {"impl": "reference", "metric": "PCG DOF*iter/s (time-to-a* at 1e-10)", "value": v, "unit": "DOF*iter/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload + ": " + desc, "D": inst.D},
            "cpu_baseline": {"value": v, "unit": "DOF*iter/s", "cores": 1, "kind": "oracle",
                             "sample": "2 oracle PCG iterations (+2 applies) of corrector e_1 per step"},
            "e2e": {"value": v, "unit": "DOF*iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_apply_only(args):
    """Launches the stiffness apply of the workload's plan (all correctors as right-hand sides) --warmup + --steps
    times; used to capture the kernel under a profiler."""
    import torch
    import paper_2404_06841_gb300 as qp
    inst = instance(args.workload, args.N)
    prec_name = args.precision or ("fp64" if WORKLOADS[args.workload][1] == "fp64" else "fp32")
    prec = qp.QP_FP64 if prec_name == "fp64" else qp.QP_FP32
    plan = qp.plan_from_instance(inst, precisions=1 if prec == qp.QP_FP64 else 2)
    dt = torch.complex128 if prec == qp.QP_FP64 else torch.complex64
    h = torch.randn((inst.d, inst.D), dtype=dt, device="cuda")
    w = torch.empty_like(h)
    for _ in range(args.warmup + args.steps):
        qp.qp_apply_stiffness(plan, h, w, prec)
    torch.cuda.synchronize()
    print(json.dumps({"apply_only": args.workload, "N": inst.N, "D": inst.D, "precision": prec_name,
                      "launches": args.warmup + args.steps}))


def run_solve_only(args):
    """Launches qp_pcg_solve on the workload's corrector right-hand sides --warmup + --steps times (from U = 0);
    used to capture the solve kernels (the persistent one where it applies) under a profiler."""
    import torch
    import paper_2404_06841_gb300 as qp
    inst = instance(args.workload, args.N)
    mode = qp.QP_MODE_FP64 if (args.mode or WORKLOADS[args.workload][1]) == "fp64" else qp.QP_MODE_FP32_REFINE
    exec_mode = {"auto": qp.QP_EXEC_AUTO, "graph": qp.QP_EXEC_GRAPH, "direct": qp.QP_EXEC_DIRECT,
                 "persistent": qp.QP_EXEC_PERSISTENT}[args.exec]
    plan = qp.plan_from_instance(inst, exec_mode=exec_mode)
    F = torch.zeros((inst.d, inst.D), dtype=torch.complex128, device="cuda")
    qp.qp_corrector_rhs(plan, 0, inst.d, F)
    U = torch.zeros_like(F)
    for _ in range(args.warmup + args.steps):
        U.zero_()
        infos = qp.qp_pcg_solve(plan, F, U, tol=inst.tol, maxit=2000, mode=mode)
    torch.cuda.synchronize()
    print(json.dumps({"solve_only": args.workload, "D": inst.D, "launches": args.warmup + args.steps,
                      "iterations": [i["iterations"] for i in infos]}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg1", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default=None, choices=["fp64", "refine"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--apply-only", action="store_true",
                    help="profiling aid: build the plan and launch only the stiffness apply --steps times")
    ap.add_argument("--solve-only", action="store_true",
                    help="profiling aid: launch only qp_pcg_solve on the corrector right-hand sides --steps times")
    ap.add_argument("--N", type=int, default=None, help="modes per axis (overrides the workload's N)")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"], help="with --apply-only")
    ap.add_argument("--exec", default="auto", choices=["auto", "persistent", "graph", "direct"],
                    help="auto (default): persistent where it applies, else graph; persistent: one cooperative "
                         "launch per solve; graph: one CUDA-graph launch per solve; direct: kernel by kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if args.apply_only:
        run_apply_only(args)
        return
    if args.solve_only:
        run_solve_only(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
