#!/usr/bin/env python3
"""Benchmark of the Wilson-clover SAP-FGMRES hot path on GB300.

A step is one full solve of D x = b to a true relative residual of 1e-10 on
the 64 x 32^3 workload (T x L^3): links exp(i 0.25 H) with two stout steps
(rho = 0.1), c_sw = 1.7, m0 = -0.02, Gaussian right-hand side; Schwarz
smoother with 4^4 blocks, 4 sweeps x 4 MR steps in FP32 storage; FGMRES(16)
whose Krylov basis and true-residual Dslash are double-float (FP32 pairs,
~48-bit significands) with an FP64 least-squares update and solution
(--outer-f64: IEEE FP64 for those too). `config` names what ran.
`mixed_96x48^3` adds apply_D and the Schwarz phase with FP16, BF16 and
F16N (FP16 operator tiles, spinors as 16-bit fixed point with a per-site
scale) storage on the 96 x 48^3 mixed-precision workload.

Prints one JSON line. `value` is solves/s with all inputs resident in HBM;
`e2e` is the same metric through dd_solve with host buffers (host-to-device
copy of b and device-to-host copy of x inside the timed region). `dslash`
reports apply_D's HBM throughput, `roofline` the dominant kernel against the
measured peaks. Under torchrun (N > 1) every rank solves its own replica of
the problem (the path has no exchange between GPUs), so scaling is weak.

`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "sap_fgmres_64x32^3_fp32"
METRIC = "Dslash GB/s & % HBM peak; SAP-FGMRES solves/s, p50/p99 at 1e-10 residual"
# Per-site algorithmic traffic (reals): apply_D reads in 24, links and clover
# 72, writes out 24; the links are 72 reals in FP64 and 48 (two rows of each
# SU(3) matrix, the third rebuilt) in 32- and 16-bit storage. One Schwarz sweep
# reads links 72, A 72, A_ee^-1 36 (72 per even site), b 24, x 24 and writes
# x 24.
DSLASH_REALS = 192
DSLASH_REALS_12 = 168
SAP_REALS_PER_SWEEP = 252
# Algorithmic flops per site: Wilson-clover apply 1848 (1320 hopping + 504
# clover + 24); one Schwarz sweep with n MR steps 1848 + 1500 + 1630 n.
DSLASH_FLOPS = 1848


def sap_flops_per_site(nmr):
    return 1848 + 1500 + 1630 * nmr


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], bf16=d.get("bf16_tflops"), src="measured",
                    sm_max_mhz=d.get("sm_max_mhz", 2070.0))
    return dict(hbm_gbs=6800.0, bf16=1900.0, src="fallback", sm_max_mhz=2070.0)


def fp32_alu_peak_tflops(sm_mhz, sms):
    # SMs x 128 FP32 lanes x 2 flops (FMA) per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def kernel_traffic(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, only while the
    kernel's source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    h = hashlib.sha256()
    for src in d["sources"]:
        path = os.path.join(ROOT, src)
        if not os.path.exists(path):
            return None
        h.update(open(path, "rb").read())
    return d["bytes_per_launch"] if h.hexdigest()[:16] == d.get("source_sha256_16") else None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.samples, self.proc, self.index = [], None, index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                self.samples.append(f)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = set()
        for s in self.samples:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               s[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(self.samples[0][2]) if self.samples[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def setup_problem(wl):
    dims = wl["dims"]
    U = synth.gauge(dims, wl["eps"], wl["n_stout"], wl["rho"], wl["gauge_seed"])
    b = synth.gaussian_spinor(int(np.prod(dims)), wl["rhs_seed"])
    return U, b


def oracle_operator(wl, U):
    import oracle
    t0 = time.perf_counter()
    op = oracle.Operator(wl["dims"], U, wl["c_sw"], wl["m0"])
    return op, time.perf_counter() - t0


def cpu_model():
    """Host CPU model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def oracle_iteration(wl, op, b, threads, basis=None):
    """Time the FP64 oracle's parts of one FGMRES iteration on the full lattice
    with `threads` OpenMP threads: one apply_D, one Schwarz sweep and the
    oracle's own modified Gram-Schmidt step against the average basis length
    of a cycle (restart / 2 + 1 vectors; the oracle runs it on one thread)."""
    import oracle
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    op.apply(b)
    t_apply = time.perf_counter() - t0
    t0 = time.perf_counter()
    op.sap(wl["block"], b, 1, wl["mr_steps"])
    t_sweep = time.perf_counter() - t0
    t_orth = None
    if basis is not None:
        t0 = time.perf_counter()
        oracle.gram_schmidt(basis, b)
        t_orth = time.perf_counter() - t0
    return dict(threads=used, apply_D_s=t_apply, sweep_s=t_sweep, gram_schmidt_s=t_orth)


def gram_schmidt_basis(wl, b):
    L = wl["restart"] // 2 + 1
    return np.tile(b.reshape(1, -1), (L, 1))


def solve_seconds(wl, it, iters, cycles):
    """Seconds of one oracle solve with `iters` Arnoldi steps and `cycles`
    restarts from the measured parts of one iteration."""
    t_iter = wl["sweeps"] * it["sweep_s"] + it["apply_D_s"] + it["gram_schmidt_s"]
    return iters * t_iter + (cycles + 1) * it["apply_D_s"], t_iter


SMALL_SOLVE_DIMS = (16, 8, 8, 8)


def oracle_small_solve(wl):
    """A whole oracle SAP-FGMRES solve, measured, on a 16 x 8^3 lattice with
    the workload's gauge recipe, operator and solver parameters."""
    import oracle
    oracle.set_threads(host_cores())
    U = synth.gauge(SMALL_SOLVE_DIMS, wl["eps"], wl["n_stout"], wl["rho"], wl["gauge_seed"])
    b = synth.gaussian_spinor(int(np.prod(SMALL_SOLVE_DIMS)), wl["rhs_seed"])
    op = oracle.Operator(SMALL_SOLVE_DIMS, U, wl["c_sw"], wl["m0"])
    t0 = time.perf_counter()
    x, ok, st = op.fgmres(wl["block"], b, wl["restart"], 1e-10, 2000, wl["sweeps"], wl["mr_steps"])
    t = time.perf_counter() - t0
    return {"lattice_TZYX": list(SMALL_SOLVE_DIMS), "seconds": t, "iterations": st["iterations"],
            "cycles": st["cycles"], "true_rel_residual": st["rel_residual"], "converged": bool(ok),
            "threads": host_cores()}


def oracle_baseline(wl, U, b, iters, cycles, single_thread=True):
    """The CPU baseline of the contract line: the FP64 oracle, as it stands, on
    the host cores. Measured on the full workload lattice: the parts of one
    FGMRES iteration on all cores (and apply_D and one sweep on one thread,
    whose flop rate compares with the paper's per-core figures); a solve's
    time is the measured iteration times the GPU solve's iteration count. A
    whole oracle solve is measured on a 16 x 8^3 lattice beside it."""
    op, t_setup = oracle_operator(wl, U)
    V = int(np.prod(wl["dims"]))
    cores = host_cores()
    it = oracle_iteration(wl, op, b, cores, gram_schmidt_basis(wl, b))
    t_solve, t_iter = solve_seconds(wl, it, iters, cycles)
    out = dict(value=1.0 / t_solve, unit="solves/s", cores=it["threads"], kind="oracle", cpu_model=cpu_model(),
               sample=(f"FP64 oracle on the full {'x'.join(map(str, wl['dims']))} lattice, {it['threads']} threads: "
                       f"one apply_D ({it['apply_D_s']:.2f} s), one Schwarz sweep ({it['sweep_s']:.2f} s), the "
                       f"oracle's modified Gram-Schmidt over {wl['restart'] // 2 + 1} vectors "
                       f"({it['gram_schmidt_s']:.2f} s); one iteration {t_iter:.2f} s, a solve = {iters} iterations "
                       f"+ {cycles + 1} true residuals; operator set-up {t_setup:.1f} s not counted"),
               seconds_per_solve=t_solve, all_cores=it,
               sap_gflops_all_cores=sap_flops_per_site(wl["mr_steps"]) * V / it["sweep_s"] / 1e9,
               dslash_gbs_all_cores=DSLASH_REALS * 8 * V / it["apply_D_s"] / 1e9)
    if single_thread:
        one = oracle_iteration(wl, op, b, 1)
        out["one_thread"] = one
        out["sap_gflops_one_thread"] = sap_flops_per_site(wl["mr_steps"]) * V / one["sweep_s"] / 1e9
        out["dslash_gbs_one_thread"] = DSLASH_REALS * 8 * V / one["apply_D_s"] / 1e9
    del op
    out["measured_small_solve"] = oracle_small_solve(wl)
    return out


# iteration / cycle counts of this workload's solve (FP32 smoother), used to
# scale the oracle's measured iteration to one solve in the reference arm
REF_ITERS, REF_CYCLES = 62, 4


def run_reference(args, rank):
    """The oracle as the reference arm: one step = one FGMRES iteration of the
    FP64 oracle on the full workload lattice (4 Schwarz sweeps, apply_D and
    the Gram-Schmidt step of average length, all host cores), measured;
    `value` is solves/s = 1 / (62 measured iterations + 5 true residuals),
    the iteration count of the GPU solve of this workload."""
    if rank != 0:
        return
    import oracle
    wl = synth.WORKLOADS[args.workload]
    U, b = setup_problem(wl)
    op, t_setup = oracle_operator(wl, U)
    basis = gram_schmidt_basis(wl, b)
    cores = host_cores()
    oracle.set_threads(cores)
    steps = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(wl["sweeps"]):
            op.sap(wl["block"], b, 1, wl["mr_steps"])
        t1 = time.perf_counter()
        op.apply(b)
        t2 = time.perf_counter()
        oracle.gram_schmidt(basis, b)
        t3 = time.perf_counter()
        if i >= args.warmup:
            steps.append((t3 - t0, t2 - t1, (t1 - t0) / wl["sweeps"], t3 - t2))
    t_step = float(np.mean([s_[0] for s_ in steps]))
    t_apply = float(np.mean([s_[1] for s_ in steps]))
    t_solve = REF_ITERS * t_step + (REF_CYCLES + 1) * t_apply
    v = 1.0 / t_solve
    cb = {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
          "sample": (f"each step one FGMRES iteration of the FP64 oracle on the full "
                     f"{'x'.join(map(str, wl['dims']))} lattice on {cores} threads ({wl['sweeps']} Schwarz sweeps, "
                     f"apply_D, Gram-Schmidt over {wl['restart'] // 2 + 1} vectors), measured; value = "
                     f"1 / ({REF_ITERS} steps + {REF_CYCLES + 1} true residuals)"),
          "seconds_per_solve": t_solve, "sweep_s": float(np.mean([s_[2] for s_ in steps])),
          "apply_D_s": t_apply, "gram_schmidt_s": float(np.mean([s_[3] for s_ in steps])),
          "operator_setup_s": t_setup}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_of(wl, "f32", "df"),
           "oracle_arithmetic": "IEEE FP64 throughout (the same workload and solver parameters)",
           "step": "one FGMRES iteration of the oracle (value extrapolates 62 of them to a solve)",
           "solves_per_s_extrapolated": v, "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


OUTER = {"f64": "IEEE FP64 Krylov basis, least squares and true residual",
         "df": "double-float Krylov basis and true-residual Dslash (FP32 pairs, ~48-bit significands); "
               "FP64 least squares, x and residual norms",
         "f64_outer": "IEEE FP64 Krylov basis, least squares and true residual (outer_f64)"}


def config_of(wl, smoother, outer):
    """`smoother`: the storage precision the Schwarz smoother ran in;
    `outer`: a key of OUTER (what the FGMRES orthogonalisation and true
    residual computed in)."""
    return {"workload": WORKLOAD if wl is synth.WORKLOADS.get(WORKLOAD) else "custom",
            "dims_TZYX": list(wl["dims"]), "block_TZYX": list(wl["block"]), "sweeps": wl["sweeps"],
            "mr_steps": wl["mr_steps"], "restart": wl["restart"], "tol": 1e-10, "smoother_storage": smoother,
            "outer": OUTER[outer], "c_sw": wl["c_sw"], "m0": wl["m0"], "eps": wl["eps"], "n_stout": wl["n_stout"],
            "l2": "inputs larger than L2 (operator fields 1.8 GB, each vector 0.2-0.4 GB)"}


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time
    (each rank solves its own replica; there is no exchange between GPUs)."""
    return world * units_per_rank / seconds_max


def ev_time(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def run_ours(args, rank, world):
    import torch

    import paper_1710_07041_gb300 as dd

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    wl = synth.WORKLOADS[args.workload]
    prec = dd.PREC[args.prec]
    U, b = setup_problem(wl)
    V = int(np.prod(wl["dims"]))
    lat = dd.Lattice(wl["dims"], wl["block"])
    gauge = dd.Gauge(lat, U)
    op = dd.Op(gauge, wl["c_sw"], wl["m0"], prec)
    stream = torch.cuda.current_stream()
    L = dd.lib()
    kw = dict(tol=1e-10, restart=wl["restart"], sweeps=wl["sweeps"], mr_steps=wl["mr_steps"], max_iter=2000,
              outer_f64=args.outer_f64)
    outer = "f64" if prec == dd.F64 else ("f64_outer" if args.outer_f64 else "df")
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # kernel-level timing first (fresh device state): apply_D and one
    # Schwarz phase (launch); the first calls also run the autotuner
    fin = lat.to_field(b, dd.F32)
    fout = lat.new_field(dd.F32)
    for _ in range(5):
        op.apply_D(dd.F32, fin, fout)
    dslash_ms = ev_time(lambda: op.apply_D(dd.F32, fin, fout), 50, stream)
    fbp = lat.to_field(b, prec)
    fxp = lat.new_field(prec)
    op.sap_smooth(fbp, fxp, wl["sweeps"], wl["mr_steps"])
    sap_ms = ev_time(lambda: op.sap_smooth(fbp, fxp, wl["sweeps"], wl["mr_steps"]), 5, stream)
    sap_launch_ms = sap_ms / (2 * wl["sweeps"])

    # device-resident inputs
    b_dev = torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda()
    x_dev = torch.zeros_like(b_dev)
    for _ in range(args.warmup):
        op.solve(b_dev, x_dev, **kw)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    lat_ms, infos = [], []
    l0 = L.dd_kernel_launches()
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            _, info = op.solve(b_dev, x_dev, **kw)
            s1.record(stream)
            s1.synchronize()
            lat_ms.append(s0.elapsed_time(s1))
            infos.append(info[0])
        e1.record(stream)
        e1.synchronize()
    launches = L.dd_kernel_launches() - l0
    total_ms = max_over_ranks(e0.elapsed_time(e1), dist)
    if dist:
        dist.barrier()
    value = whole_job_rate(args.steps, world, total_ms / 1e3)

    # end to end through dd_solve with pinned host buffers
    bh = torch.from_numpy(b.view(np.float64).reshape(-1).copy()).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    bh_np, xh_np = bh.numpy(), xh.numpy()
    op.solve(bh_np, xh_np, **kw)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        op.solve(bh_np, xh_np, **kw)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / max(1, args.steps // 2), dist)

    peaks = measured_peaks()
    real_b = {dd.F64: 8, dd.F32: 4, dd.F16: 2, dd.BF16: 2}
    dslash_bytes = DSLASH_REALS_12 * 4 * V
    dslash_gbs = dslash_bytes / (dslash_ms * 1e-3) / 1e9
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or peaks["sm_max_mhz"]
    alu_peak = fp32_alu_peak_tflops(peaks["sm_max_mhz"], sms)
    sap_flops_launch = sap_flops_per_site(wl["mr_steps"]) * V / 2
    sap_tflops = sap_flops_launch / (sap_launch_ms * 1e-3) / 1e12
    sap_bytes_launch = SAP_REALS_PER_SWEEP * real_b[prec] * V / 2
    mean_info = {k: float(np.mean([i[k] for i in infos])) for k in ("ms_sap", "ms_dirac", "ms_orth", "ms_total")}
    roofline_sap = {"kernel": "k_sap_phase", "bound": "alu", "achieved": sap_tflops, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": sap_tflops / alu_peak,
                    "traffic": kernel_traffic("k_sap_phase"),
                    "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz",
                    "algorithmic_bytes_per_launch": sap_bytes_launch,
                    "hbm_frac": sap_bytes_launch / (sap_launch_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                    "ms_per_launch": sap_launch_ms}
    roofline_dslash = {"kernel": "k_dirac<float>", "bound": "hbm", "achieved": dslash_gbs,
                       "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": dslash_gbs / peaks["hbm_gbs"],
                       "traffic": kernel_traffic("k_dirac<float>"), "peak_source": peaks["src"],
                       "ms_per_launch": dslash_ms}
    dominant = roofline_sap if mean_info["ms_sap"] >= mean_info["ms_dirac"] else roofline_dslash
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == dd.F32 else args.prec,
        "data": "synthetic", "config": config_of(wl, args.prec, outer),
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99))},
        "solve": {"iterations": int(infos[-1]["iterations"]), "cycles": int(infos[-1]["cycles"]),
                  "true_rel_residual": max(i["true_rel_residual"] for i in infos), **mean_info},
        "dslash": {"GB/s": dslash_gbs, "frac_hbm": dslash_gbs / peaks["hbm_gbs"], "ms": dslash_ms,
                   "bytes_per_site": DSLASH_REALS_12 * 4,
                   "hbm_peak_gbs": peaks["hbm_gbs"], "peak_source": peaks["src"]},
        "roofline": dominant,
        "roofline_other": roofline_dslash if dominant is roofline_sap else roofline_sap,
        "e2e": {"value": whole_job_rate(1, world, e2e_s), "unit": "solves/s", "h2d_bytes_per_step": V * 24 * 8,
                "d2h_bytes_per_step": V * 24 * 8},
        "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_mixed:
        out["mixed_96x48^3"] = mixed_kernels(dd, peaks, alu_peak, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_baseline(wl, U, b, int(infos[-1]["iterations"]), int(infos[-1]["cycles"]))
    if rank == 0:
        print(json.dumps(out), flush=True)
    op.close()
    gauge.close()
    lat.close()
    if dist:
        dist.destroy_process_group()


def mixed_kernels(dd, peaks, alu_peak, stream):
    """apply_D and the Schwarz phase with FP16, BF16 and F16N storage on the
    mixed-precision workload's 96 x 48^3 lattice (exp(i 0.2 H), 3 stout steps,
    c_sw 1.7, m0 0; 4^4 blocks, 4 MR steps): time, GB/s of algorithmic bytes
    (apply_D 168 reals per site with two-row links, a phase 252 reals per
    site of its colour, 2 bytes each; F16N adds its 4-byte site scales: 2 per
    site for apply_D, 3 for a phase) and the phase's flop rate. Inputs far
    exceed L2 (one field 0.5 GB)."""
    import torch
    wl = synth.WORKLOADS["sap_fgmres_96x48^3_mixed"]
    V = int(np.prod(wl["dims"]))
    U = synth.gauge(wl["dims"], wl["eps"], wl["n_stout"], wl["rho"], wl["gauge_seed"])
    lat = dd.Lattice(wl["dims"], wl["block"])
    gauge = dd.Gauge(lat, U)
    del U
    b = synth.gaussian_spinor(V, wl["rhs_seed"])
    res = {"workload": "sap_fgmres_96x48^3_mixed", "dims_TZYX": list(wl["dims"]), "block_TZYX": list(wl["block"]),
           "mr_steps": wl["mr_steps"], "m0": wl["m0"]}
    for name, prec in (("f16", dd.F16), ("bf16", dd.BF16), ("f16n", dd.F16N)):
        scales = 4 if prec == dd.F16N else 0   # bytes of one site scale
        op = dd.Op(gauge, wl["c_sw"], wl["m0"], prec)
        fin, fout = lat.to_field(b, prec), lat.new_field(prec)
        for _ in range(5):
            op.apply_D(prec, fin, fout)
        ms_d = ev_time(lambda: op.apply_D(prec, fin, fout), 30, stream)
        op.sap_smooth(fin, fout, wl["sweeps"], wl["mr_steps"])
        ms_s = ev_time(lambda: op.sap_smooth(fin, fout, wl["sweeps"], wl["mr_steps"]), 3, stream) / (2 * wl["sweeps"])
        bytes_d, bytes_s = DSLASH_REALS_12 * 2 + 2 * scales, SAP_REALS_PER_SWEEP * 2 + 3 * scales
        gbs_d = bytes_d * V / (ms_d * 1e-3) / 1e9
        gbs_s = bytes_s * (V / 2) / (ms_s * 1e-3) / 1e9
        tf_s = sap_flops_per_site(wl["mr_steps"]) * (V / 2) / (ms_s * 1e-3) / 1e12
        res[name] = {"dslash": {"ms": ms_d, "GB/s": gbs_d, "frac_hbm": gbs_d / peaks["hbm_gbs"],
                                "bytes_per_site": bytes_d},
                     "sap_phase": {"ms": ms_s, "TFLOP/s": tf_s, "frac_fp32_peak": tf_s / alu_peak, "GB/s": gbs_s,
                                   "frac_hbm": gbs_s / peaks["hbm_gbs"]}}
        del fin, fout
        op.close()
        torch.cuda.empty_cache()
    gauge.close()
    lat.close()
    return res


def run_kernels(args):
    """Kernel-level loop for profiler captures: apply_D (F32 and the smoother
    precision) and Schwarz sweeps on the workload, plus one short solve."""
    import torch

    import paper_1710_07041_gb300 as dd

    wl = synth.WORKLOADS[args.workload]
    prec = dd.PREC[args.prec]
    U, b = setup_problem(wl)
    lat = dd.Lattice(wl["dims"], wl["block"])
    gauge = dd.Gauge(lat, U)
    op = dd.Op(gauge, wl["c_sw"], wl["m0"], prec)
    stream = torch.cuda.current_stream()
    fin, fout = lat.to_field(b, dd.F32), lat.new_field(dd.F32)
    fbp, fxp = lat.to_field(b, prec), lat.new_field(prec)
    res = {}
    kernels = [("apply_D_f32", lambda: op.apply_D(dd.F32, fin, fout), 20),
               ("sap", lambda: op.sap_smooth(fbp, fxp, wl["sweeps"], wl["mr_steps"]), 3)]
    if prec != dd.F32:
        fop = lat.new_field(prec)
        kernels.append(("apply_D_" + args.prec, lambda: op.apply_D(prec, fbp, fop), 20))
    for name, fn, reps in kernels:
        for _ in range(args.warmup):
            fn()
        res[name + "_ms"] = ev_time(fn, max(1, min(reps, args.steps)), stream)
    _, info = op.solve(b, tol=1e-10, restart=wl["restart"], sweeps=wl["sweeps"], mr_steps=wl["mr_steps"],
                       max_iter=args.solve_iters, raise_on_notconv=False)
    res["solve"] = info[0]
    print(json.dumps(res), flush=True)


def _solve_rate(op, b, kw, reps=1):
    t0 = time.perf_counter()
    infos = []
    for _ in range(reps):
        _, info = op.solve(b, **kw)
        infos += info
    return (time.perf_counter() - t0) / (reps * max(1, b.shape[0] if b.ndim == 4 else 1)), infos


def run_batched(args):
    """Batched multi-RHS workload: 48^3 x 96, 12 point sources (one per spin-colour
    at the origin) + 12 complex Z2-noise sources, FP16 storage. Autotunes the
    Schwarz block over {4^4, 8x4^3} and the RHS tile over {4, 8, 12}: the tile
    by the time of one smoother application on all 24 sources, the block by
    that time per decade of residual reduction one application achieves on a
    noise source (|b - D M b| / |b|; larger blocks are slower per application
    but stronger). Then solves all 24 to 1e-10 in as many concurrent slots as
    device memory allows, and times one plain FP64 GPU SAP-FGMRES solve for
    the speedup."""
    import torch

    import paper_1710_07041_gb300 as dd

    wl = synth.WORKLOADS["batched_48^3x96_24rhs"]
    dims = wl["dims"]
    V = int(np.prod(dims))
    U = synth.gauge(dims, wl["eps"], wl["n_stout"], wl["rho"], wl["gauge_seed"])
    srcs = [synth.point_source(V, s, c) for s in range(4) for c in range(3)]
    srcs += [synth.z2_spinor(V, wl["rhs_seed"] + k) for k in range(12)]
    B = np.stack(srcs)
    stream = torch.cuda.current_stream()
    out = {"mode": "batched", "workload": "batched_48^3x96_24rhs", "nrhs": 24, "sap": {}}
    best = None
    for block in ((4, 4, 4, 4), (8, 4, 4, 4)):
        lat = dd.Lattice(dims, block)
        gauge = dd.Gauge(lat, U)
        op = dd.Op(gauge, wl["c_sw"], wl["m0"], dd.F16)
        fb = lat.to_field(B, dd.F16, scale=1.0)
        fx = lat.new_field(dd.F16, 24)
        # residual reduction of one application (FP16 fields; a norm does not depend on the layout)
        b16 = lat.to_field(B[12], dd.F16, scale=1.0)
        x16, d16 = lat.new_field(dd.F16), lat.new_field(dd.F16)
        op.sap_smooth(b16, x16, wl["sweeps"], wl["mr_steps"])
        op.apply_D(dd.F16, x16, d16)
        bv, dv = b16.view(torch.float16).float(), d16.view(torch.float16).float()
        rho = float(torch.linalg.norm(bv - dv) / torch.linalg.norm(bv))
        del b16, x16, d16, bv, dv
        bkey = "x".join(map(str, block))
        best_tile = None
        for tile in (4, 8, 12):
            op.sap_smooth(fb, fx, wl["sweeps"], wl["mr_steps"], nrhs=24, rhs_tile=tile)
            ms = ev_time(lambda: op.sap_smooth(fb, fx, wl["sweeps"], wl["mr_steps"], nrhs=24, rhs_tile=tile), 3,
                         stream)
            out["sap"][f"block {bkey} tile {tile}"] = {"ms_per_application_24rhs": ms, "ms_per_rhs": ms / 24}
            if best_tile is None or ms < best_tile[0]:
                best_tile = (ms, tile)
        decades = max(1e-3, -math.log10(max(rho, 1e-12)))
        cost = best_tile[0] / decades
        out["sap"][f"block {bkey}"] = {"residual_reduction_per_application": rho,
                                        "ms_per_decade_24rhs": cost}
        if best is None or cost < best[0]:
            best = (cost, block, best_tile[1])
        del fb, fx
        op.close(); gauge.close(); lat.close()
        torch.cuda.empty_cache()
    out["chosen"] = {"block": list(best[1]), "rhs_tile": best[2]}
    lat = dd.Lattice(dims, best[1])
    gauge = dd.Gauge(lat, U)
    op = dd.Op(gauge, wl["c_sw"], wl["m0"], dd.F16)
    kw = dict(tol=1e-10, restart=wl["restart"], sweeps=wl["sweeps"], mr_steps=wl["mr_steps"], max_iter=3000)
    t0 = time.perf_counter()
    x, infos = op.solve(B, **kw)
    t = time.perf_counter() - t0
    out["solve_all_24"] = {"seconds": t, "rhs_per_s": 24 / t,
                           "max_true_rel_residual": max(i["true_rel_residual"] for i in infos),
                           "iterations": [int(i["iterations"]) for i in infos]}
    op.close()
    op64 = dd.Op(gauge, wl["c_sw"], wl["m0"], dd.F64)
    t64, info64 = _solve_rate(op64, B[12], dict(kw, inner_reduction=0.0))
    out["plain_fp64_one_rhs"] = {"seconds": t64, "iterations": int(info64[0]["iterations"]),
                                 "true_rel_residual": info64[0]["true_rel_residual"]}
    out["speedup_vs_plain_fp64"] = (24 / t) / (1 / t64)
    op64.close(); gauge.close(); lat.close()
    print(json.dumps(out), flush=True)


# two-level configuration (DD-alpha-AMG style, Sec. 1): test vectors, their
# smoothing iterations, coarse GMRES steps and tolerance, Schwarz post-smoother
MG = {"n_vectors": 16, "setup_iters": 6, "coarse_max_iter": 24, "coarse_tol": 0.05, "sweeps": 3, "mr_steps": 4,
      "tv_seed": 7000}


def run_oracle(args):
    """The FP64 oracle's apply_D and one Schwarz sweep on the full 64 x 32^3
    and 96 x 48^3 lattices of the benchmark and mixed-precision workloads, on
    one host thread and on all host cores (OpenMP), with the host CPU named:
    time, GB/s of algorithmic bytes (192 reals of 8 bytes per site for
    apply_D) and GFlop/s of the sweep (9868 flops per site at 4 MR steps).
    Needs about 80 GB of host memory for the 96 x 48^3 site matrices."""
    import oracle
    out = {"mode": "oracle", "cpu_model": cpu_model(), "cores": host_cores()}
    for name in ("sap_fgmres_64x32^3_fp32", "sap_fgmres_96x48^3_mixed"):
        wl = synth.WORKLOADS[name]
        V = int(np.prod(wl["dims"]))
        U, b = setup_problem(wl)
        op, t_setup = oracle_operator(wl, U)
        del U
        res = {"dims_TZYX": list(wl["dims"]), "operator_setup_s": t_setup}
        for threads in (host_cores(), 1):
            it = oracle_iteration(wl, op, b, threads)
            res[f"threads_{it['threads']}"] = {
                "apply_D_s": it["apply_D_s"], "sweep_s": it["sweep_s"],
                "dslash_GB/s": DSLASH_REALS * 8 * V / it["apply_D_s"] / 1e9,
                "sweep_GFlop/s": sap_flops_per_site(wl["mr_steps"]) * V / it["sweep_s"] / 1e9}
        out[name] = res
        del op
    oracle.set_threads(host_cores())
    print(json.dumps(out), flush=True)


def run_mma(args):
    """The tensor-core question for the 12-source link product: time the
    FP32 CUDA-core form, the warp-MMA form (FP16 operands, two
    site-directions block-diagonal per m16n8k16 tile) and the FP16-operand
    CUDA-core form on the same products (dd_bench_link_product), in useful
    flops (1728 per site-direction: a 6x6 real matrix times 24 columns)."""
    import paper_1710_07041_gb300 as dd
    ctas, reps = 152 * 8, 200
    out = {"mode": "mma", "sites_x_directions": ctas * 64, "reps": reps, "rhs_tile": 12}
    for method, name in ((0, "fp32_cuda_cores"), (1, "fp16_mma_sync"), (2, "fp16_operands_cuda_cores")):
        ms, n, diff = dd.bench_link_product(method, ctas, reps)
        out[name] = {"ms": ms, "useful_TFLOP/s": 1728.0 * n * reps / (ms * 1e-3) / 1e12,
                     "rel_diff_vs_fp32": diff}
    print(json.dumps(out), flush=True)


def run_mg(args):
    """Two-level preconditioner on the benchmark workload: SAP-FGMRES against
    FGMRES preconditioned by the aggregation coarse-grid correction plus
    Schwarz post-smoothing, both to 1e-10 (FP64 true residual). Reports the
    setup time, solve times and iterations, and after how many solves the
    setup has paid for itself."""
    import torch

    import paper_1710_07041_gb300 as dd

    wl = synth.WORKLOADS[args.workload]
    prec = {"f32": dd.F32, "f16": dd.F16, "bf16": dd.BF16, "f64": dd.F64}[args.prec]
    U, b = setup_problem(wl)
    lat = dd.Lattice(wl["dims"], wl["block"])
    gauge = dd.Gauge(lat, U)
    op = dd.Op(gauge, wl["c_sw"], wl["m0"], prec)
    V = lat.V
    bd = torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda()
    xd = torch.zeros_like(bd)
    kw = dict(tol=1e-10, restart=wl["restart"], sweeps=wl["sweeps"], mr_steps=wl["mr_steps"], max_iter=3000)
    reps = max(1, args.steps)

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            info = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps, info

    t_sap, (_, info_sap) = timed(lambda: op.solve(bd, xd, **kw))
    tv = np.stack([synth.gaussian_spinor(V, MG["tv_seed"] + k) for k in range(MG["n_vectors"])])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mg = dd.Multigrid(op, tv, setup_iters=MG["setup_iters"], coarse_max_iter=MG["coarse_max_iter"],
                      coarse_tol=MG["coarse_tol"], sweeps=MG["sweeps"], mr_steps=MG["mr_steps"])
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    t_mg, (_, info_mg) = timed(lambda: op.solve(bd, xd, mg=mg, **kw))
    mg.close()
    op.close()
    gauge.close()
    lat.close()
    i0, i1 = info_sap[0], info_mg[0]
    out = {"mode": "mg", "workload": args.workload, "smoother_dtype": args.prec, "tol": 1e-10, "mg": MG,
           "sap_fgmres": {"ms_per_solve": t_sap * 1e3, "solves_per_s": 1 / t_sap, "iterations": int(i0["iterations"]),
                          "true_rel_residual": i0["true_rel_residual"]},
           "two_level": {"ms_per_solve": t_mg * 1e3, "solves_per_s": 1 / t_mg, "iterations": int(i1["iterations"]),
                         "true_rel_residual": i1["true_rel_residual"], "setup_s": t_setup,
                         "ms_preconditioner": i1["ms_sap"], "ms_orth": i1["ms_orth"], "ms_dirac": i1["ms_dirac"]},
           "speedup_per_solve": t_sap / t_mg,
           "break_even_solves": (t_setup / (t_sap - t_mg)) if t_sap > t_mg else None}
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Served stream: Poisson arrivals at 200 req/s over lattices 16^3x32,
    24^3x48 and 32^3x64 (equal mix), 1-12 right-hand sides each, on 8 resident
    gauge fields (3 + 3 + 2; exp(i 0.25 H) + 2 stout, seeds 500..507), m0 drawn
    from {-0.03, -0.0033, 0.0233, 0.05} (uniform grid over [-0.03, 0.05]),
    mixed-precision (FP16) solves to 1e-10 through the continuous-batching
    server. Reports p50/p99 latency and solves/s next to the plain FP64 GPU
    solve of the same request mix (estimated from one timed FP64 solve per
    lattice size). --rate sets the offered request rate: 200/s overloads the
    GPU ~100x (latency is then queueing); a rate below capacity measures the
    service latency of requests that find the server idle or lightly loaded."""
    import torch

    import paper_1710_07041_gb300 as dd

    sizes = [(32, 16, 16, 16), (48, 24, 24, 24), (64, 32, 32, 32)]
    fields = [(sizes[0], 500), (sizes[0], 501), (sizes[0], 502), (sizes[1], 503), (sizes[1], 504), (sizes[1], 505),
              (sizes[2], 506), (sizes[2], 507)]
    m0s = [-0.03, -0.0033, 0.0233, 0.05]
    lats = {d: dd.Lattice(d, (4, 4, 4, 4)) for d in sizes}
    gauges = [dd.Gauge(lats[d], synth.gauge(d, 0.25, 2, 0.1, seed)) for d, seed in fields]
    ops = {}

    def op_for(fi, mi, prec=dd.F16):
        k = (fi, mi, prec)
        if k not in ops:
            ops[k] = dd.Op(gauges[fi], 1.7, m0s[mi], prec)
        return ops[k]

    nreq = args.requests
    rate = float(args.rate)
    u = synth.uniform(4 * nreq, 51)
    arrivals = np.cumsum(-np.log(u[:nreq]) / rate)
    reqs = []
    for k in range(nreq):
        size = int(u[nreq + k] * 3) % 3
        fi = [i for i, (d, _) in enumerate(fields) if d == sizes[size]][int(u[2 * nreq + k] * 8) % (3 if size < 2 else 2)]
        nrhs = 1 + int(u[3 * nreq + k] * 12) % 12
        mi = k % len(m0s)
        reqs.append((arrivals[k], fi, mi, nrhs, 1000 + k))
    for _, fi, mi, _, _ in reqs:   # resident operators before the stream starts
        op_for(fi, mi)
    srv = dd.Server(max_slots=8, max_batch_rhs=12)
    # warm-up: one small request per lattice size (autotuning, graphs)
    for d in sizes:
        fi = [i for i, (dd_, _) in enumerate(fields) if dd_ == d][0]
        t = srv.submit(op_for(fi, 0), synth.gaussian_spinor(int(np.prod(d)), 7))
        srv.wait(t)
    srv.close()
    srv = dd.Server(max_slots=8, max_batch_rhs=12)
    tickets = []
    t0 = time.perf_counter()
    for at, fi, mi, nrhs, seed in reqs:
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        # the right-hand sides are drawn at submission (the server copies them)
        V = int(np.prod(fields[fi][0]))
        b = synth.gaussian(12 * V * nrhs, seed).reshape(nrhs, V, 4, 3)
        tickets.append((srv.submit(op_for(fi, mi), b if nrhs > 1 else b[0]), nrhs))
        del b
    worst, nrhs_done = 0.0, 0
    for t, nrhs in tickets:
        st, x, info = srv.wait(t, timeout=3600)
        if st != dd.DONE:
            raise RuntimeError(f"request {t} ended in state {st}")
        del x
        worst = max(worst, max(i["true_rel_residual"] for i in info))
        nrhs_done += nrhs
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    # plain FP64 GPU solves: one per lattice size, scaled to the mix
    kw = dict(tol=1e-10, restart=16, sweeps=4, mr_steps=4, max_iter=3000, inner_reduction=0.0)
    t64 = {}
    for si, d in enumerate(sizes):
        fi = [i for i, (dd_, _) in enumerate(fields) if dd_ == d][0]
        op64 = op_for(fi, 1, dd.F64)
        t64[si], _ = _solve_rate(op64, synth.gaussian_spinor(int(np.prod(d)), 9), kw)
    fp64_seconds = sum(t64[[s for s, dd_ in enumerate(sizes) if dd_ == fields[fi][0]][0]] * nrhs
                       for _, fi, _, nrhs, _ in reqs)
    out = {"mode": "serve", "requests": nreq, "offered_req_per_s": rate, "rhs": nrhs_done,
           "wall_s": wall, "achieved_req_per_s": nreq / wall, "rhs_per_s": nrhs_done / wall,
           "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "max_true_rel_residual": worst,
           "plain_fp64_seconds_per_rhs": {f"{'x'.join(map(str, d))}": t64[i] for i, d in enumerate(sizes)},
           "plain_fp64_rhs_per_s_same_mix": nrhs_done / fp64_seconds,
           "speedup_vs_plain_fp64": (nrhs_done / wall) / (nrhs_done / fp64_seconds)}
    print(json.dumps(out), flush=True)
    for o in ops.values():
        o.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--prec", default="f32", choices=["f64", "f32", "f16", "bf16", "f16n"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 96x48^3 FP16/BF16 kernel measurements")
    ap.add_argument("--outer-f64", action="store_true",
                    help="IEEE FP64 Krylov basis and true residual with a mixed-precision smoother")
    ap.add_argument("--mode", default="bench",
                    choices=["bench", "kernels", "batched", "serve", "mg", "mma", "oracle"],
                    help="kernels: short kernel loop for profiler captures; batched: the 24-source "
                         "48^3x96 workload; serve: the Poisson request stream; mg: two-level "
                         "preconditioner against SAP alone; mma: tensor-core link-product "
                         "measurement; oracle: the FP64 oracle's apply_D and sweep at 64x32^3 and "
                         "96x48^3 on 1 thread and all cores (no contract line)")
    ap.add_argument("--requests", type=int, default=40, help="requests in --mode serve")
    ap.add_argument("--rate", type=float, default=200.0, help="offered requests/s in --mode serve")
    ap.add_argument("--solve-iters", type=int, default=20, help="iteration cap of the solve in --mode kernels")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.mode == "kernels":
        run_kernels(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "mg":
        run_mg(args)
    elif args.mode == "mma":
        run_mma(args)
    elif args.mode == "oracle":
        run_oracle(args)
    elif args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
