#!/usr/bin/env python
"""Benchmark of the projection-method hot path on GB300: PCG DOF*iterations/s and time to the homogenized
coefficient a*, with the FP64, FP32 + FP64-refinement and batched forms and the HBM roofline of the apply.

Default workload: the large form, d = 3 lifted to n = 6, P = [[1,sqrt2,0,0,0,0],[0,0,1,sqrt3,0,0],[0,0,0,0,1,sqrt5]],
A = diag(a_i) with a_i = 4 + sum_j 0.5 cos(theta_j + phi_ij) (13 taps per component, phases seeded), 16^6 =
16,777,216 Fourier modes per field, three correctors solved by FP32 Jacobi-PCG inside FP64 iterative refinement to a
true relative residual of 1e-10, then the 3 x 3 a*. One step = corrector right-hand sides -> PCG solves -> a*
reduction -> a* on the host, with the coefficient already on the device (time-to-a*). Inputs are synthetic
(seeded); every vector of a step is larger than L2, which is also flushed before every timed step.

The line also carries: the plain FP64 solve and the Frobenius diagonal on the same workload, the 64-instance
batched workload against its instances solved one after another, the roofline of the FP32 stiffness apply as the
solve runs it and of the whole FP32 PCG iteration (per-phase CUDA-event timing of one solve), the end-to-end time
through the C ABI from host inputs, and the oracle timed on one host core and on all of them.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload cfg0..cfg4|tab2]
For N > 1 launch with torch.distributed.run; every rank solves its own replica (independent units, no
collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import os

# The CPU baseline runs the oracle in one process per core; pin numpy's helper libraries to one thread per
# process so that the reported core counts are what it used.
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
METRIC = "PCG DOF*iter/s and time-to-a* at 1e-10 (FP64 vs FP32+refine vs batched), % HBM roofline"


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
    # cfg4: the FP32 (h, Q h) batch apply of the refinement solve (k_apply_star, geometry compiled in), captured at
    # N = 14 (7.53 M modes; h and w exceed L2), scaled by 16^6 / 14^6
    ("apply32", "cfg4"): int((211014912 + 153146624) * (16 ** 6 / 14 ** 6)),
    # cfg1: one solve (33 iterations, 2 correctors) in k_pcg_persistent; vectors and stored weights stay in L2
    ("k_pcg_persistent", "cfg1"): 9733376 + 243712,
    # cfg4: k_apply_plain_star (geometry compiled in) captured at N = 14 (7.53 M modes; h and w exceed L2), scaled
    # by 16^6 / 14^6
    ("k_apply_plain", "cfg4"): int((212182400 + 153766528) * (16 ** 6 / 14 ** 6)),
    # cfg2: the three fused passes of one FP32 apply (the gradient fields stay in L2 between passes)
    ("k_fft_group", "cfg2"): 16941568 + 77568 + 46253824 + 0 + 33648384 + 256,
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


# ---------------------------------------------------------------------------------------------- in-solve timing

def phase_breakdown(qp, run_once):
    """Per-phase CUDA-event timing of one solve (the library's phase timing: the host-driven form of the same
    kernels, bitwise the same iterates). Returns ({phase: (ms, launches)}, result of run_once)."""
    import torch
    run_once()                                 # warm (graph/persistent form), so that nothing is first-use below
    torch.cuda.synchronize()
    qp.qp_set_phase_timing(True)
    try:
        out = run_once()
        torch.cuda.synchronize()
        ph = qp.qp_phase_times()
    finally:
        qp.qp_set_phase_timing(False)
    return ph, out


def apply32_bytes_per_unit_iteration(units):
    """Algorithmic bytes of the FP32 (h, Q h) apply per PCG iteration of each unit: read h, write Q h (8-byte
    complex values) for its right-hand sides, over its D modes."""
    return [2 * 8 * D * nr for (D, nr) in units]


def solve_rooflines(qp, phases, units, unit_iters, es_fft=None, grid_coef=None):
    """Rooflines of the kernels as the solve runs them, from its per-phase event times.

    units: [(D, nrhs)] per solve unit; unit_iters: the inner FP32 PCG iterations each unit took part in (the
    largest over its right-hand sides). The FP32 apply moves 16 B per mode and right-hand side (taps: read h,
    write Q h; FFT backend: the three-pass schedule's bytes, es_fft gives (d, ncomp) for it); the whole FP32
    iteration is held against the 6-stream floor of 48 B per mode and right-hand side (read and write U, r, h).
    Totals are summed over the solve, so a unit counts only in the iterations it was active in."""
    pk = peaks()
    ms_apply, n_apply = phases["apply32"]
    ms_upd, _ = phases["update32"]
    ms_hup, _ = phases["hupdate32"]
    dof_its = sum(D * nr * it for (D, nr), it in zip(units, unit_iters))
    if es_fft is None:
        apply_bytes = sum(b * it for b, it in zip(apply32_bytes_per_unit_iteration(units), unit_iters))
        what = "taps stencil: read h, write Q h (8-byte complex) per mode and right-hand side"
    else:
        d, nc = es_fft
        apply_bytes = sum(fft_apply_bytes(d, nc, nr, D, 8) * it for (D, nr), it in zip(units, unit_iters))
        what = "FFT backend, three-pass schedule: (2 + 4d) x 8 B per mode and right-hand side + the samples"
    apply = None
    if ms_apply > 0 and apply_bytes > 0:
        ach = apply_bytes / (ms_apply / 1e3) / 1e9
        apply = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": round(ach / pk["hbm_gbs"], 4), "traffic": None,
                 "kernel": "FP32 stiffness apply with its (h, Q h) reduction, as the refinement solve runs it "
                           "(per-launch CUDA events on the solve stream, host-driven form)",
                 "kernel_key": "apply32", "launches": n_apply, "us_per_launch": round(ms_apply * 1e3 / max(1, n_apply), 2),
                 "bytes_per_launch": int(apply_bytes / max(1, n_apply)), "algorithmic_bytes": what,
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs" + (" (fallback)" if pk.get("_fallback") else "")}
    it_ms = ms_apply + ms_upd + ms_hup
    iteration = None
    if it_ms > 0 and dof_its > 0:
        floor = 48.0 * dof_its
        ach = floor / (it_ms / 1e3) / 1e9
        iteration = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": round(ach / pk["hbm_gbs"], 4), "floor_bytes_per_dof": 48,
                     "what": "whole FP32 PCG iteration (apply + update + h-update) against the 6-stream floor "
                             "(read and write U, r, h: 48 B per mode and right-hand side)",
                     "us_per_iteration": round(it_ms * 1e3 / max(1, n_apply), 2),
                     "us_apply": round(ms_apply * 1e3 / max(1, n_apply), 2),
                     "us_update": round(ms_upd * 1e3 / max(1, n_apply), 2),
                     "us_hupdate": round(ms_hup * 1e3 / max(1, n_apply), 2),
                     "dof_iter_per_s": dof_its / (it_ms / 1e3)}
    return apply, iteration


def phases_json(phases):
    return {k: {"ms": round(v[0], 4), "launches": int(v[1])} for k, v in phases.items() if v[1] > 0}


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
    iteration = None
    phases = None
    if mode_name == "refine":
        # the kernels as the refinement solve runs them: per-phase events of one solve (same kernels, same iterates)
        ph, res = phase_breakdown(qp, step)
        infs = res[1]
        if name == "cfg3":
            units, unit_iters, o = [], [], 0
            for i_ in insts:
                units.append((i_.D, i_.d))
                unit_iters.append(max(x["iterations"] for x in infs[o:o + i_.d]))
                o += i_.d
        else:
            units = [(inst.D, len(infs))]
            unit_iters = [max(x["iterations"] for x in infs)]
        from qp_workloads import ncomp
        es_fft = (inst.d, ncomp(c.kind, inst.d)) if pinfo["backend"] == "fft" else None
        roof, iteration = solve_rooflines(qp, ph, units, unit_iters, es_fft)
        phases = phases_json(ph)
        tot = {k: v["ms"] for k, v in phases.items()}
        phases["dominant"] = max(tot, key=tot.get) if tot else None
    if roof is None and mode_name == "fp64" and c.taps_k is not None and name != "cfg3":
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

    # ---- the half-spectrum storage (the scheme on the Nyquist-free modes, vectors of the modes with k_{n-1} >= 0)
    if not args.no_variants and name == "cfg4" and world == 1:
        variants["half_spectrum"] = half_variant(qp, inst, mode, tol, flush, stream, max(3, min(args.steps, 10)))

    # ---- the batched form: the 64 instances in one batched solve against the same instances one after another
    if not args.no_variants and name in ("cfg3", "cfg4") and world == 1:
        variants["batched"] = batched_variant(qp, flush, stream, max(3, min(args.steps, 10)))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(name, max_seconds=args.cpu_seconds)

    out = {
        "metric": METRIC,
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
        "astar_im": (None if name in ("tab2", "cfg3") else A.imag.tolist()),
        "astar_vs_oracle": astar_vs_oracle(name, A, insts if name == "cfg3" else None, inst),
        "wall_s_timed_region": wall1 - wall0,
        "roofline": roof,
        "iteration_roofline": iteration,
        "phases": phases,
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


# The oracle's sample of each workload: the workload itself, or for the large form (one oracle apply of 16^6 modes
# takes about 40 s on a host core and 4 GB) the same coefficient, P and correctors at 10^6 modes.
CPU_SAMPLE_N = {"cfg4": 10}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_sample(name, N, max_seconds):
    """One oracle process: Algorithm 2 on corrector e_1 for as many iterations as fit in about max_seconds (at
    least one); returns (DOF-iterations, seconds, iterations) of its timed part."""
    from oracle import qp_oracle as O
    return O.timed_pcg_sample(instance(name, N), max_seconds=max_seconds)


def _oracle_workers(name, N):
    """Processes for the all-core oracle run: one per host core, as many as fit in 40% of the available memory
    (the oracle holds about 60 arrays of D complex values per process)."""
    D = instance(name, N).D
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except Exception:
        pass
    per = 60 * 16 * D + (200 << 20)
    cap = host_cores() if avail is None else max(1, int(0.4 * avail // per))
    return max(1, min(host_cores(), cap, 64))


def half_variant(qp, inst, mode, tol, flush, stream, reps):
    """Time-to-a* of the same workload on a half-spectrum plan (QP_SPECTRUM_HALF: the scheme on the Nyquist-free
    modes, about half the stored modes), its DOF*iter/s over the stored modes, and its a* against the oracle's
    Nyquist-free a* (tests/golden, written by the oracle only)."""
    import torch
    plan = qp.plan_from_instance(inst, spectrum=qp.QP_SPECTRUM_HALF)
    for _ in range(2):
        A, infs = qp.qp_homogenized(plan, tol=tol, mode=mode, maxit=2000)
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        A, infs = qp.qp_homogenized(plan, tol=tol, mode=mode, maxit=2000)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    t = statistics.median(ts)
    di = sum(plan.D * (x["iterations"] + x["outer_iterations"]) for x in infs)
    out = {"what": "QP_SPECTRUM_HALF plan: Nyquist-free modes, %d stored of %d" % (plan.D, inst.D),
           "time_to_astar_ms": round(t, 4), "dof_iter_per_s_stored": di / (t / 1e3),
           "iterations": [(x["iterations"], x["outer_iterations"]) for x in infs],
           "max_rel_residual": max(x["rel_residual"] for x in infs), "astar": np.round(A.real, 14).tolist()}
    g = golden("cfg4_half") if tuple(inst.N) == tuple(W.cfg4().N) else None
    if g is not None:
        ref = np.array(g["astar_re"])
        out["astar_vs_oracle_nyquist_free"] = float(np.abs(A.real - ref).max() / np.abs(ref).max())
    qp.qp_plan_destroy(plan)
    return out


def batched_variant(qp, flush, stream, reps):
    """Time-to-a* of the 64-instance workload (FP32 + FP64 refinement to 1e-10): all 96 correctors in one batched
    solve, against the same plans solved one after another (qp_homogenized each), and the batch's largest deviation
    from the oracle's a* (tests/golden, written by the oracle only)."""
    import torch
    insts = W.cfg3()
    plans = [qp.plan_from_instance(i) for i in insts]
    batch = qp.qp_batch_create(plans)
    mode = qp.QP_MODE_FP32_REFINE

    def timed(fn):
        for _ in range(2):
            out = fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), out

    tb, (As, infs) = timed(lambda: qp.qp_batch_homogenized(batch, tol=1e-10, mode=mode, maxit=2000))
    ts_, _ = timed(lambda: [qp.qp_homogenized(p, tol=1e-10, mode=mode, maxit=2000) for p in plans])
    tb64, _ = timed(lambda: qp.qp_batch_homogenized(batch, tol=1e-10, mode=qp.QP_MODE_FP64, maxit=2000))
    unit_D = [i.D for i in insts for _ in range(i.d)]
    di = sum(D * (x["iterations"] + x["outer_iterations"]) for D, x in zip(unit_D, infs))
    out = {"workload": "64 instances (32 d=1 n=2 N=64..512, 32 d=2 n=4 N=8..24), 96 correctors, 1e-10",
           "batched_refine_ms": round(tb, 4), "one_after_another_refine_ms": round(ts_, 4),
           "batched_fp64_ms": round(tb64, 4), "batched_dof_iter_per_s": di / (tb / 1e3),
           "max_rel_residual": max(x["rel_residual"] for x in infs)}
    gold = golden("cfg3")
    if gold is not None:
        out["max_rel_astar_err_vs_oracle"] = max(
            float(np.abs(A - np.array(g["astar_re"])).max() / np.abs(np.array(g["astar_re"])).max())
            for A, g in zip(As, gold["instances"]))
    qp.qp_batch_destroy(batch)
    for p_ in plans:
        qp.qp_plan_destroy(p_)
    return out


def astar_vs_oracle(name, A, insts, inst):
    """Largest deviation of the bench's a* from the oracle's, relative to max |a*_oracle| (Re and Im): the full-size
    values in tests/golden, or the oracle run here for the small workloads."""
    try:
        if name == "cfg3":
            gold = golden("cfg3")
            if gold is None:
                return None
            ref = {g["name"]: np.array(g["astar_re"]) for g in gold["instances"]}
            return {"re": max(float(np.abs(a - ref[i_.name]).max() / np.abs(ref[i_.name]).max())
                              for a, i_ in zip(A, insts)), "source": "tests/golden (oracle)"}
        g = golden(name)
        if g is not None and inst.N == tuple(getattr(W, name)().N):
            ref_re, ref_im = np.array(g["astar_re"]), np.array(g["astar_im"])
            src = "tests/golden (oracle, tol 1e-13)"
        elif name in ("cfg0", "cfg1"):
            from oracle import qp_oracle as O
            ref_re, _, _, ac = O.homogenized(inst, tol=1e-13)
            ref_im = ac.imag
            src = "oracle run in this process (tol 1e-13)"
        else:
            return None
        sc = np.abs(ref_re).max()
        return {"re": float(np.abs(A.real - ref_re).max() / sc), "im": float(np.abs(A.imag - ref_im).max() / sc),
                "oracle_im_max": float(np.abs(ref_im).max()), "source": src}
    except Exception as e:   # a missing or unreadable golden file leaves the field empty
        return {"error": str(e)[:200]}


def golden(name):
    """The oracle's full-size a* of a workload (tests/golden/astar_full_size.json, written by the oracle only)."""
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", "astar_full_size.json"))).get(name)
    except Exception:
        return None


def cpu_baseline(name, max_seconds=12.0):
    """The FP64 oracle (numpy, one thread per process) on a bounded sample of the same workload, on one host core
    and on all of them (one process per core, each the same sample: independent units run side by side)."""
    import multiprocessing as mp
    N = CPU_SAMPLE_N.get(name)
    inst = instance(name, N)
    dof1, sec1, it1 = _oracle_sample(name, N, max_seconds)
    workers = _oracle_workers(name, N)
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.starmap(_oracle_sample, [(name, N, max_seconds)] * workers)
    all_rate = sum(d_ / s_ for d_, s_, _ in res)
    where = "%s corrector e_1%s" % (name, "" if N is None else " at %d^%d modes (D = %d)" % (N, inst.n, inst.D))
    return {"value": all_rate, "unit": "DOF*iter/s", "cores": workers, "kind": "oracle",
            "sample": "%s: per process %d oracle PCG iterations (each apply counted as one, with the initial and the "
                      "final true residual), about %.0f s, numpy FP64, one thread per process, %d processes side by "
                      "side on %d host cores" % (where, res[0][2], res[0][1], workers, host_cores()),
            "single_core": {"value": dof1 / sec1, "unit": "DOF*iter/s", "cores": 1,
                            "sample": "the same sample in one process: %d iterations, %.1f s" % (it1, sec1)}}


# ---------------------------------------------------------------------------------------------- reference arm

def _oracle_apply_step(name, N):
    """One oracle stiffness apply of corrector e_1's right-hand side (the bulk of an oracle PCG iteration);
    returns (DOF, seconds)."""
    from oracle import qp_oracle as O
    global _REF_OP
    if _REF_OP is None:
        inst = instance(name, N)
        op = O.Operator(inst)
        _REF_OP = (op, O.corrector_rhs(op.P, op.N, op.Ahat, 0), inst.D)
    op, F, D = _REF_OP
    t0 = time.perf_counter()
    op(F)
    return D, time.perf_counter() - t0


_REF_OP = None


def run_reference(args):
    """The oracle as it stands, on all host cores (one process per core): each step is one oracle stiffness apply
    (the bulk of an oracle PCG iteration) of corrector e_1's right-hand side in every process, side by side; value =
    DOF x processes / step time, in the same unit as our arm."""
    import multiprocessing as mp
    name = args.workload
    N = CPU_SAMPLE_N.get(name)
    inst = instance(name, N)
    workers = _oracle_workers(name, N)
    with mp.get_context("spawn").Pool(workers) as pool:
        for _ in range(max(args.warmup, 1)):
            pool.starmap(_oracle_apply_step, [(name, N)] * workers)
        t0 = time.perf_counter()
        dofs = 0
        for _ in range(args.steps):
            res = pool.starmap(_oracle_apply_step, [(name, N)] * workers)
            dofs += sum(r[0] for r in res)
        secs = time.perf_counter() - t0
    v = dofs / secs
    desc = WORKLOADS[name][0]
    sample = ("one oracle stiffness apply of corrector e_1%s per process and step, %d processes side by side on %d "
              "host cores (numpy FP64, one thread each)" % ("" if N is None else " at %d^%d modes (D = %d)"
                                                             % (N, inst.n, inst.D), workers, host_cores()))
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOF*iter/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name + ": " + desc, "D": instance(name).D},
            "cpu_baseline": {"value": v, "unit": "DOF*iter/s", "cores": workers, "kind": "oracle", "sample": sample},
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
    ap.add_argument("--workload", default="cfg4", choices=sorted(WORKLOADS))
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
