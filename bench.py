#!/usr/bin/env python
"""Benchmark: time to solve the 32^4 Wilson-clover quark equation D phi = eta
to |eta - D phi| / |eta| <= 1e-10 on one GB300.

Workload (the paper's lattice size, Sec. 5, with synthetic seeded inputs in
place of the authors' configuration): 32^4 sites, antiperiodic time, random
SU(3) links U = exp(i 0.3 H) (gauge seed 1), kappa = 0.125, c_sw = 1, complex
Gaussian source (seed 2).  One step = one whole pass of the hot path: gauge
import and clover build, then the mixed-precision nested solve (FP64 defect
correction around the FP16-storage / FP32-arithmetic inner BiCGStab, right-
preconditioned by RAS).  The plain FP64 BiCGStab on the same GPU is timed
beside it (the comparison the metric names), and the CPU oracle on a bounded
sample of the same workload.

Prints one JSON line on stdout (rank 0).  Usage:
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own replica of the workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "32^4 solve time to 1e-10 FP64 residual (RAS FP16/32 vs plain FP64); dslash GB/s/HBM"
DIMS = (32, 32, 32, 32)
BC = (1, 1, 1, -1)
EPS, KAPPA, CSW, GSEED, SSEED, TOL = 0.3, 0.125, 1.0, 1, 2, 1e-10
WORKLOAD = "32^4 lattice, eps=0.3 links (seed 1), kappa=0.125, c_sw=1.0, Gaussian source (seed 2), tol 1e-10"
BYTES_PER_SITE = {"f64": 1536, "f32": 672, "f16": 348}   # compulsory D traffic: spinor in/out, links, clover
SPINOR_BYTES = {"f64": 192, "f32": 96, "f16": 52}
# The paper's own 32^4 measurement (Table 1), on other hardware and to another
# tolerance: context only, not a target.
PAPER_TABLE1 = {"hardware": "8x GeForce GTX 285 in 4 PCs, 4x GigE (Open-MX, OpenMPI)", "tolerance": 1e-14,
                "solve_s_ras_d0": 27.977, "solve_s_no_preconditioner": 53.305,
                "dv_total_s_no_preconditioner": 48.243, "note": "whole quark solve, dominated by GigE communication"}
FLOPS_PER_SITE_D = 1872                                    # spin-projected hop 1320 + clover 504 + combine 48
NOMINAL = {"hbm_gbs": 7900.0, "sms": 152, "fp32_lanes": 128, "sm_max_mhz": 2070.0, "fp64_tflops": 1.25}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ helpers
# the files that define device code: a change to any of them invalidates the
# committed ncu traffic figures
KERNEL_SOURCES = ("device.cuh", "pair.cuh", "df64.cuh", "tma.cuh", "tmem.cuh", "qdd_internal.h", "lib.h", "dslash.cu",
                  "ras.cu", "blas.cu", "lattice.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1011_3318_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class):
    """DRAM bytes per launch of a kernel class (with the RAS block shape of
    the solve it was captured in, e.g. "ras 4x4x4x2") from the committed ncu
    summary profiles/traffic.md, if it was taken on the current kernel
    sources (its 'sources hash' line matches), else None."""
    p = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m = re.search(r"sources hash: `([0-9a-f]+)`", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    for line in text.splitlines():
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] == kernel_class:
            try:
                return int(cells[2])
            except ValueError:
                return None
    return None


def ras_sweep_flops(blk, ov, n_dominv):
    """Algorithmic flops of one RAS sweep over the 32^4 lattice: per domain
    and MR iteration, the clover term and combine on every site of the
    extended domain, only the hops that stay inside it (the Dirichlet
    operator drops the others), and the two dot products and two axpys."""
    ext = [b if b == L else b + 2 * ov for b, L in zip(blk, DIMS)]
    nloc = 1
    for e in ext:
        nloc *= e
    ndom = 1
    for b, L in zip(blk, DIMS):
        ndom *= L // b
    kept_hops = sum(2 * nloc * ((e - 1) / e if b < L else 1.0) for e, b, L in zip(ext, blk, DIMS))
    hop = (FLOPS_PER_SITE_D - 504 - 48) / 8
    per_iter = nloc * (504 + 48 + 96 + 48) + kept_hops * hop
    return ndom * n_dominv * per_iter


def oracle_solve(op, eta):
    """One whole plain FP64 BiCGStab solve of the oracle to the benchmark's
    tolerance (continued from the true residual), timed; the true residual of
    its answer is computed afterwards, outside the timing."""
    t0 = time.perf_counter()
    phi, info = op.solve(eta, TOL)
    t = time.perf_counter() - t0
    return t, info, op.true_residual(eta, phi)


def cpu_baseline(U, eta):
    """The oracle (plain FP64 C, OpenMP on all host cores) on the same
    workload: its clover build and one whole measured plain-BiCGStab solve to
    1e-10 at 32^4 (about 30 s on 16 host cores), nothing extrapolated."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    op = oracle.Op(DIMS, BC, U, KAPPA, CSW)
    t_clover = time.perf_counter() - t0
    t_solve, info, res = oracle_solve(op, eta)
    value = t_clover + t_solve
    sample = (f"measured full solve: the oracle's clover build ({t_clover:.2f} s) and one whole plain FP64 "
              f"BiCGStab solve of the 32^4 workload to 1e-10 ({t_solve:.2f} s, {info['inner_iters']} iterations, "
              f"true residual {res:.2e})")
    return {"value": round(value, 3), "unit": "s", "cores": oracle.get_threads(), "kind": "oracle",
            "sample": sample, "converged": bool(info["status"] == 0 and res <= TOL)}


def host_cpu():
    """CPU model and core count of this host."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                if key == "model name":
                    break
    except OSError:
        pass
    import platform
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
                 "0xd49": "Arm Neoverse N2"}
    if model in arm_parts:
        model = f"{arm_parts[model]} (CPU part {model})"
    return {"model": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "nproc": os.cpu_count()}


def oracle_timing(U32=None, eta32=None):
    """The oracle's D at 8^4, 16^4 and 32^4 on one thread and on all host
    threads, and its plain FP64 BiCGStab solves at 8^4 (config kappa 0.12)
    and 16^4 on all threads: context for the CPU baseline (a few seconds)."""
    import oracle
    import synth
    oracle.build()
    n_all = oracle.get_threads()
    out = {"cpu": host_cpu(), "threads_all": n_all, "d_apply_s": {}, "plain_solve": {}}
    for dims, kappa in (((8, 8, 8, 8), 0.12), ((16, 16, 16, 16), 0.12), (DIMS, KAPPA)):
        if dims == DIMS and U32 is not None:
            U, eta = U32, eta32
        else:
            U = synth.gauge_field(dims, EPS, GSEED)
            eta = synth.gaussian_source(dims, SSEED)
        op = oracle.Op(dims, BC, U, kappa, CSW)
        name = "x".join(map(str, dims))
        row = {}
        for nthr in (1, n_all):
            oracle.set_threads(nthr)
            op.dslash(eta)
            t0 = time.perf_counter()
            op.dslash(eta)
            row[f"{nthr}_threads"] = round(time.perf_counter() - t0, 4)
        oracle.set_threads(n_all)
        out["d_apply_s"][name] = row
        if dims != DIMS:
            t0 = time.perf_counter()
            _, info = op.solve(eta, TOL)
            out["plain_solve"][name] = {"s": round(time.perf_counter() - t0, 3), "threads": n_all,
                                        "inner_iters": info.get("inner_iters")}
    return out


# ------------------------------------------------------------------ replicas
def reduce_max(value: float, dist=None, device: str = "cpu") -> float:
    """Largest value over all ranks (the slowest replica sets the job time);
    the value itself when not distributed."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_seconds_per_solve(ms_max: float, world: int) -> float:
    """Replicas only: every rank solves its own copy of the workload, so the
    job solves `world` systems in the slowest rank's time."""
    return ms_max / 1e3 / world


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, budget_s=240.0):
    """The reference arm: the FP64 CPU oracle on this machine's host cores, on the
    benchmark's workload and metric.  Warm-up steps are oracle D applications
    (a CPU needs no repeated solve to warm up); each timed step is one whole
    measured plain-BiCGStab solve to 1e-10 at 32^4.  Steps stop once the timed
    solves have taken budget_s, so that the run ends within a few minutes:
    "steps" is the number of solves actually timed (at least one)."""
    if rank != 0:
        return 0
    import synth
    log("reference arm: the FP64 CPU oracle on this box's host cores")
    U = synth.gauge_field(DIMS, EPS, GSEED)
    eta = synth.gaussian_source(DIMS, SSEED)
    import oracle
    oracle.build()
    op = oracle.Op(DIMS, BC, U, KAPPA, CSW)
    for _ in range(args.warmup):
        op.dslash(eta)
    times, infos, res = [], [], []
    for _ in range(max(1, args.steps)):
        t, info, r = oracle_solve(op, eta)
        times.append(t)
        infos.append(info)
        res.append(r)
        log(f"oracle solve {len(times)}: {t:.2f} s, {info['inner_iters']} iterations, true residual {r:.2e}")
        if sum(times) >= budget_s:
            break
    value = statistics.mean(times)
    sample = (f"{len(times)} whole plain FP64 BiCGStab solves of the 32^4 workload to 1e-10, each measured "
              f"({infos[-1]['inner_iters']} iterations, true residual {max(res):.2e}); warm-up: "
              f"{args.warmup} oracle D applications")
    cb = {"value": round(value, 3), "unit": "s", "cores": oracle.get_threads(), "kind": "oracle", "sample": sample}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "s",
                      "n_gpus": args.gpus, "steps": len(times), "steps_requested": args.steps,
                      "warmup": args.warmup, "ms_per_step": round(value * 1e3, 1), "higher_is_better": False,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": WORKLOAD, "method": "plain FP64 BiCGStab (oracle)"},
                      "all_timed_solves_converged": all(i["status"] == 0 for i in infos) and max(res) <= TOL,
                      "cpu_baseline": cb, "e2e": {"value": round(value, 3), "unit": "s", "h2d_bytes_per_step": 0,
                                                  "d2h_bytes_per_step": 0}}), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def time_steps(torch, stream, fn, steps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    infos = [fn() for _ in range(steps)]
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps, infos


def dslash_roofline(torch, qdd, lat, stream, deta, prec, pk, reps=50):
    a = qdd.field_create(lat, prec)
    b = qdd.field_create(lat, prec)
    qdd.field_import(a, deta)
    for _ in range(3):
        qdd.dslash_field(lat, b, a, KAPPA, CSW)
    ms, _ = time_steps(torch, stream, lambda: qdd.dslash_field(lat, b, a, KAPPA, CSW), reps)
    V = lat.V
    gbs = BYTES_PER_SITE[prec] * V / (ms * 1e-3) / 1e9
    qdd.field_destroy(a)
    qdd.field_destroy(b)
    return {"us_per_launch": round(ms * 1e3, 1), "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / pk, 3),
            "D_per_s": round(1e3 / ms, 1), "bytes_per_site": BYTES_PER_SITE[prec]}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import synth
    from paper_1011_3318_gb300 import qdd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pk, pk_kind = peaks()
    hbm = float(pk["hbm_gbs"])

    log(f"rank {rank}: generating the 32^4 workload")
    U = synth.gauge_field(DIMS, EPS, GSEED)
    eta = synth.gaussian_source(DIMS, SSEED)
    V = int(np.prod(DIMS))
    stream = torch.cuda.Stream()
    lat = qdd.create_lattice(DIMS, BC, stream=stream)
    dU = torch.from_numpy(U).cuda()
    deta = torch.from_numpy(eta).cuda()
    dphi = torch.empty_like(deta)
    params = qdd.default_params(inner_prec=args.prec, use_ras=1, block=args.block, overlap=args.overlap,
                                n_dominv=args.n_dominv, n_ras=args.n_ras, inner_tol=args.inner_tol)
    plain = qdd.default_params(inner_prec="f64", use_ras=0)
    tune = None
    if not args.no_autotune:
        qdd.load_gauge(lat, dU)
        t0 = time.perf_counter()
        params, best_ms = qdd.autotune(lat, deta, KAPPA, CSW, TOL, params, max_trials=args.tune_trials)
        tune = {"seconds": round(time.perf_counter() - t0, 2), "best_solve_ms": round(best_ms, 2),
                "block": list(params.block), "overlap": params.overlap, "n_dominv": params.n_dominv,
                "n_ras": params.n_ras, "ras_kernel": params.ras_kernel,
                "inner_prec": {0: "f64", 1: "f32", 2: "f16"}[params.inner_prec], "inner_tol": params.inner_tol}
        log(f"autotune: {tune}")
    blk, ov, nd, nr = list(params.block), params.overlap, params.n_dominv, params.n_ras
    args.prec = {1: "f32", 2: "f16"}.get(params.inner_prec, args.prec)
    args.inner_tol = params.inner_tol

    def step():
        qdd.load_gauge(lat, dU)           # gauge import + invalidates the clover: rebuilt inside the solve
        return qdd.solve(lat, dphi, deta, KAPPA, CSW, TOL, params)

    for _ in range(args.warmup):
        step()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    n0 = qdd.kernel_launches()
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the timed steps: the production path (solves run as CUDA graphs)
    torch.cuda.nvtx.range_push("timed")   # profilers select the timed steps with this range
    ms, infos = time_steps(torch, stream, step, args.steps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        ms = reduce_max(ms, dist, "cuda")
        dist.barrier()
    launches = qdd.kernel_launches() - n0
    # the same steps again with per-kernel CUDA events on the lattice stream
    # (event-record nodes inside the graphs), for the per-class times and the
    # rooflines; the events cost about 2% of a step, so this pass is not the value
    qdd.set_profiling(lat, True)
    qdd.profile_read(lat, reset=True)
    torch.cuda.nvtx.range_push("profiled")
    ms_prof, pinfos_ = time_steps(torch, stream, step, args.steps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    prof = qdd.profile_read(lat, reset=True)
    qdd.set_profiling(lat, False)
    ok = all(i["status"] == 0 and i["true_rel_residual"] <= TOL for i in infos + pinfos_)
    info = infos[-1]

    # plain FP64 BiCGStab on the same GPU (the comparison of the metric)
    qdd.solve(lat, dphi, deta, KAPPA, CSW, TOL, plain)
    ms_plain, pinfos = time_steps(torch, stream, lambda: qdd.solve(lat, dphi, deta, KAPPA, CSW, TOL, plain),
                                  max(1, min(3, args.steps)))
    # mixed precision without RAS (context)
    nor = qdd.default_params(inner_prec=args.prec, use_ras=0, inner_tol=args.inner_tol)
    qdd.solve(lat, dphi, deta, KAPPA, CSW, TOL, nor)
    ms_nor, ninfos = time_steps(torch, stream, lambda: qdd.solve(lat, dphi, deta, KAPPA, CSW, TOL, nor),
                                max(1, min(3, args.steps)))

    # the dslash kernel alone, same launch configuration as inside the solve
    dsl = {p: dslash_roofline(torch, qdd, lat, stream, deta, p, hbm) for p in ("f16", "f32", "f64")}

    # roofline of the dominant kernel class inside the timed solves
    total = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    sm_mhz = clocks.get("sm_mhz") or NOMINAL["sm_max_mhz"]
    fp32_alu_peak = NOMINAL["sms"] * NOMINAL["fp32_lanes"] * 2 * NOMINAL["sm_max_mhz"] * 1e6 / 1e12
    if dom == "ras":
        ms_l = prof["ras"][0] / max(1, prof["ras"][1])
        flops = ras_sweep_flops(blk, ov, nd)
        ach = flops / (ms_l * 1e-3) / 1e12
        tma = (params.ras_kernel == 0 and ov == 0 and blk[0] * blk[1] * blk[2] * blk[3] in (128, 256)
               and blk[0] % 4 == 0 and DIMS[0] % 4 == 0)
        name = "ras_tma_kernel (RAS sweep, TMA staging)" if tma else "ras_smem_kernel (RAS sweep)"
        roof = {"kernel": name, "bound": "alu", "achieved": round(ach, 2),
                "peak": round(fp32_alu_peak, 1), "unit": "TFLOP/s", "frac": round(ach / fp32_alu_peak, 3),
                "traffic": ncu_traffic("ras " + "x".join(map(str, blk))),
                "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "us_per_launch": round(ms_l * 1e3, 1), "share": round(prof["ras"][0] / total, 3)}
    else:
        cls = dom if dom in ("dslash", "dslash_f64") else "dslash"
        ms_l = prof[cls][0] / max(1, prof[cls][1])
        prec = "f64" if cls == "dslash_f64" else args.prec
        ach = BYTES_PER_SITE[prec] * V / (ms_l * 1e-3) / 1e9
        roof = {"kernel": f"dslash_kernel ({prec})", "bound": "hbm", "achieved": round(ach, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(ach / hbm, 3), "traffic": ncu_traffic(cls),
                "peak_kind": f"{pk_kind} (MEASURED_PEAKS.json hbm_gbs)", "us_per_launch": round(ms_l * 1e3, 1),
                "share": round(prof[cls][0] / total, 3)}
    # the inner-precision dslash inside the solves (fused epilogues included)
    # (each launch also reads its epilogue vector: one more spinor per site)
    ms_d = prof["dslash"][0] / max(1, prof["dslash"][1])
    bps_d = BYTES_PER_SITE[args.prec] + SPINOR_BYTES[args.prec]
    ach_d = bps_d * V / (ms_d * 1e-3) / 1e9
    roof_dslash = {"kernel": f"dslash kernel ({args.prec}, D with fused dot-product epilogue, in the solve)",
                   "bound": "hbm", "achieved": round(ach_d, 1), "peak": hbm, "unit": "GB/s",
                   "frac": round(ach_d / hbm, 3), "traffic": ncu_traffic("dslash " + "x".join(map(str, blk))),
                   "bytes_per_site": bps_d,
                   "us_per_launch": round(ms_d * 1e3, 1)}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hU = torch.from_numpy(U).pin_memory()
    heta = torch.from_numpy(eta).pin_memory()
    hphi = torch.empty_like(heta).pin_memory()

    def e2e_step():
        qdd.load_gauge(lat, hU)
        return qdd.solve(lat, hphi, heta, KAPPA, CSW, TOL, params)

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_infos = [e2e_step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e_ok = all(i["status"] == 0 for i in e_infos)
    # one more step, its two calls timed apart (host clock, each call returns synchronised)
    t0 = time.perf_counter()
    qdd.load_gauge(lat, hU)
    t1 = time.perf_counter()
    e_last = qdd.solve(lat, hphi, heta, KAPPA, CSW, TOL, params)
    t2 = time.perf_counter()
    e2e_split = {"load_gauge_ms": round((t1 - t0) * 1e3, 2), "solve_ms": round((t2 - t1) * 1e3, 2),
                 "solve_t_total_ms": round(e_last["t_total_ms"], 2)}

    # the box's pinned-copy bandwidth, which sets the end-to-end overhead
    # (it has varied between boxes of this pool): one copy of the links each way
    dev = torch.empty(hU.shape, dtype=hU.dtype, device="cuda")
    xfer = {}
    for name, dst, src in (("h2d_GBps", dev, hU), ("d2h_GBps", hU, dev)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        dst.copy_(src, non_blocking=True)
        ev1.record()
        torch.cuda.synchronize()
        xfer[name] = round(hU.numel() * hU.element_size() / (ev0.elapsed_time(ev1) * 1e-3) / 1e9, 1)
    del dev

    # the oracle's check of the last answer (FP64 true residual with the oracle's D)
    oracle_res = None
    cb = None
    ot = None
    if rank == 0:
        import oracle
        oracle.build()
        op = oracle.Op(DIMS, BC, U, KAPPA, CSW, store_clover=False)
        oracle_res = op.true_residual(eta, hphi.numpy())
        if world == 1 and not args.no_cpu_baseline:
            cb = cpu_baseline(U, eta)
            ot = oracle_timing(U, eta)

    if rank == 0:
        value = whole_job_seconds_per_solve(ms, world)
        rec = {
            "metric": METRIC, "value": round(value, 5), "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16-storage/f32-arith + f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS),
                       "method": f"FP64 defect correction + {args.prec}-storage/FP32 inner BiCGStab, RAS "
                                 f"block {'x'.join(map(str, blk))} s={ov} "
                                 f"N_dominv={nd} NRAS={nr}, inner tol {args.inner_tol}",
                       "autotune": tune,
                       "l2": "inputs larger than L2 (links 604 MB, source 201 MB FP64 per replica)",
                       "parallelism": f"{world} independent replica(s)"},
            "solve": {k: info[k] for k in ("outer_iters", "inner_iters", "dv_count", "ras_sweeps",
                                            "true_rel_residual")},
            "all_timed_solves_converged": ok,
            "oracle_true_rel_residual": oracle_res,
            "paper_context": PAPER_TABLE1,
            "oracle_timing": ot,
            "plain_fp64": {"s": round(ms_plain / 1e3, 4), "inner_iters": pinfos[-1]["inner_iters"],
                           "true_rel_residual": pinfos[-1]["true_rel_residual"],
                           "speedup_of_value": round(ms_plain / ms, 2)},
            "mixed_no_ras": {"s": round(ms_nor / 1e3, 4), "inner_iters": ninfos[-1]["inner_iters"],
                             "outer_iters": ninfos[-1]["outer_iters"]},
            "profiled_ms_per_step": round(ms_prof, 3),
            "kernel_time_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in prof.items()},
            "kernel_launches_per_step": {k: v[1] / args.steps for k, v in prof.items()},
            "roofline": roof, "roofline_dslash": roof_dslash, "dslash_alone": dsl,
            "e2e": {"value": round(e2e_s, 5), "unit": "s",
                    "h2d_bytes_per_step": int(U.nbytes + eta.nbytes), "d2h_bytes_per_step": int(eta.nbytes),
                    "converged": e_ok, "pinned_copy": xfer, "one_step_split": e2e_split},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "cpu_baseline": cb,
            "kernel_source_hash": kernel_source_hash(),
        }
        print(json.dumps(rec), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_workload(args):
    """Batched workloads (one JSON line each; the default run is the 32^4 solve):
      mrhs  -- 24^3 x 48, eps 0.25 (seed 1), kappa 0.124, c_sw 1, 12 unit point
               sources at the origin (one per spin-colour) in one 12-RHS lattice,
               FP16 inner / FP64 outer, RAS parameters autotuned;
      batch -- 16 independent systems drawn by synth.uneven_batch(16, 1) from
               8^4, 12^4, 16^4, 8^3 x 24, 24^4, each on its own stream, solved in
               lockstep with one CUDA graph;
      table1 -- the paper's experiment (Table 1) emulated: 8 x-slab domains of
               4 x 32^3, d = 0, 2, 4, NRAS 3, N_dominv 5, FP32 inner, kappa
               0.126, tolerance 1e-14, and no preconditioner; Dv counts and
               times beside the paper's (context only);
      schwarz -- the 32^4 workload solved with each member of the Schwarz
               family as K (RAS, red/black SAP, plain AS; Sec. 1, Sec. 2), 4^4
               blocks, N_dominv 4, FP16 inner, 1..3 cycles, d in {0, 2} (AS:
               one cycle, d in {2, 4}, as AS with d = 0 is RAS), each solve
               timed once after an untimed one;
      small -- the 8^4 plain FP64 configuration and the 16^4 FP32-inner
               configuration without and with RAS (4^4, N_dominv 4, NRAS 3):
               time, iterations, global D count and sweeps, 3 timed solves;
      blocks -- the 32^4 workload over the RAS block shapes 8^4, 4^4, 8x4^3,
               overlap s = 0, 1, 2 (d = 0, 2, 4) and FP32 / FP16 inner solves,
               NRAS 1, N_dominv 4, each solve timed once after an untimed one;
      outer -- the 32^4 workload solved with FP64 defect correction and with
               the paper's FP64 outer BiCGStab (Sec. 3) around the same inner
               solve (4^4 blocks, NRAS 1, N_dominv 4), inner tolerance 1e-1,
               1e-2, 1e-3, FP16 and FP32 inner;
      survey -- the paper's parameter survey (Sec. 5) on the 32^4 workload:
               NRAS 1..10 x N_dominv 1..20 x d = 2s in {0, 2, 4}, 4^4 blocks,
               FP16 inner, each solve timed once after one untimed solve of the
               same parameters; reports the grid and the best point against the
               paper's choice (NRAS 3, N_dominv 5, d 0).
    Every answer is checked with the oracle's FP64 D (the survey checks the
    residual the library recomputes in FP64)."""
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_1011_3318_gb300 import qdd
    oracle.build()
    torch.cuda.set_device(0)
    t_all = time.perf_counter()
    n0 = qdd.kernel_launches()
    if args.workload == "table1":
        # the paper's own experiment (Table 1) emulated on one GPU: 8 x-slab
        # domains of 4 x 32^3 (one per GPU there, one CTA here), overlap d = 2s
        # in {0, 2, 4}, NRAS 3, N_dominv 5, FP32 inner, kappa 0.126, c_sw 1,
        # stopping at 1e-14; synthetic field and source as in the headline
        kappa, tol = 0.126, 1e-14
        U = synth.gauge_field(DIMS, EPS, GSEED)
        eta = synth.gaussian_source(DIMS, SSEED)
        st = torch.cuda.Stream()
        lat = qdd.create_lattice(DIMS, BC, stream=st)
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        d_eta = torch.from_numpy(eta).cuda()
        d_phi = torch.empty_like(d_eta)
        op = oracle.Op(DIMS, BC, U, kappa, CSW, store_clover=False)
        paper = {"none": {"dv_count": 1328, "total_s": 53.305}, "d0": {"dv_count": 484, "total_s": 27.977},
                 "d2": {"dv_count": 496, "total_s": 35.234}, "d4": {"dv_count": 416, "total_s": 37.195}}
        runs = {}
        for name, use_ras, s_ in (("none", 0, 0), ("d0", 1, 0), ("d2", 1, 1), ("d4", 1, 2)):
            p = qdd.default_params(inner_prec="f32", use_ras=use_ras, block=(4, 32, 32, 32), overlap=s_, n_ras=3,
                                   n_dominv=5)
            t0 = time.perf_counter()
            info = qdd.solve(lat, d_phi, d_eta, kappa, CSW, tol, p, raise_on_failure=False)
            torch.cuda.synchronize()
            runs[name] = {"s": round(time.perf_counter() - t0, 3), "dv_count": info["dv_count"],
                          "inner_iters": info["inner_iters"], "outer_iters": info["outer_iters"],
                          "ras_sweeps": info["ras_sweeps"], "status": info["status"],
                          "true_rel_residual": info["true_rel_residual"],
                          "oracle_true_rel_residual": op.true_residual(eta, d_phi.cpu().numpy())}
        rec = {"workload": "table1", "metric": "Table 1 emulated: 32^4, 8 x-slab domains, solve to 1e-14",
               "kappa": kappa, "tol": tol, "ras": {"block": [4, 32, 32, 32], "n_ras": 3, "n_dominv": 5,
                                                  "inner_prec": "f32"},
               "runs": runs, "paper_context": paper,
               "dv_ratio_none_over_d0": round(runs["none"]["dv_count"] / max(1, runs["d0"]["dv_count"]), 2),
               "paper_dv_ratio_none_over_d0": round(1328 / 484, 2),
               "note": "each slab domain is spread over many CTAs (the phased sweep, one launch per MR step, "
                       "as the paper's one domain per GPU); with 8 domains the sweep's launches and per-domain "
                       "reductions cost more than the tuned 4^4 blocks (4096 CTAs, one launch per sweep)"}
    elif args.workload == "survey":
        U = synth.gauge_field(DIMS, EPS, GSEED)
        eta = synth.gaussian_source(DIMS, SSEED)
        st = torch.cuda.Stream()
        lat = qdd.create_lattice(DIMS, BC, stream=st)
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        d_eta = torch.from_numpy(eta).cuda()
        d_phi = torch.empty_like(d_eta)
        grid = []
        budget_s, t_start, skipped = 300.0, time.perf_counter(), 0
        for s_ in (0, 1, 2):
            for nr in range(1, 11):
                for nd in range(1, 21):
                    if time.perf_counter() - t_start > budget_s:
                        skipped += 1
                        continue
                    p = qdd.default_params(inner_prec="f16", block=(4, 4, 4, 4), overlap=s_, n_ras=nr, n_dominv=nd,
                                           max_inner=400, max_outer=12)
                    t0 = time.perf_counter()
                    i = qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p, raise_on_failure=False)
                    torch.cuda.synchronize()
                    ms = (time.perf_counter() - t0) * 1e3
                    if ms < 500:  # a second, event-timed solve when the first was quick
                        ms, infos = time_steps(torch, st, lambda: qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p,
                                                                            raise_on_failure=False), 1)
                        i = infos[0]
                    ok = i["status"] == 0 and i["true_rel_residual"] <= TOL
                    grid.append([nr, nd, 2 * s_, round(ms, 2) if ok else None, i["inner_iters"], i["dv_count"]])
        done = [g for g in grid if g[3] is not None]
        best = min(done, key=lambda g: g[3])
        paper = next((g for g in grid if g[0] == 3 and g[1] == 5 and g[2] == 0), None)
        rec = {"workload": "survey", "metric": "32^4 solve time to 1e-10 over NRAS x N_dominv x d (Sec. 5 survey)",
               "unit": "ms", "grid_columns": ["n_ras", "n_dominv", "d", "ms", "inner_iters", "dv_count"],
               "best": dict(zip(["n_ras", "n_dominv", "d", "ms", "inner_iters", "dv_count"], best)),
               "paper_choice": dict(zip(["n_ras", "n_dominv", "d", "ms", "inner_iters", "dv_count"], paper))
               if paper else None,
               "converged": len(done), "points": len(grid), "skipped_over_budget": skipped,
               "budget_s": budget_s, "grid": grid}
    elif args.workload == "schwarz":
        U = synth.gauge_field(DIMS, EPS, GSEED)
        eta = synth.gaussian_source(DIMS, SSEED)
        st = torch.cuda.Stream()
        lat = qdd.create_lattice(DIMS, BC, stream=st)
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        d_eta = torch.from_numpy(eta).cuda()
        d_phi = torch.empty_like(d_eta)
        op = oracle.Op(DIMS, BC, U, KAPPA, CSW, store_clover=False)
        grid = []
        for sch, ds in (("ras", (0, 2)), ("sap", (0, 2)), ("as", (2, 4))):
            for d in ds:
                # AS: one cycle only; with overlap its Richardson iteration
                # amplifies the residual, so further cycles only hurt
                for cyc in ((1,) if sch == "as" else (1, 2, 3)):
                    p = qdd.default_params(inner_prec="f16", block=(4, 4, 4, 4), overlap=d // 2, n_ras=cyc,
                                           n_dominv=4, schwarz=sch, max_inner=400, max_outer=12)
                    qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p, raise_on_failure=False)  # untimed
                    ms, infos = time_steps(torch, st, lambda: qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p,
                                                                        raise_on_failure=False), 1)
                    i = infos[0]
                    res = op.true_residual(eta, d_phi.cpu().numpy())
                    ok = i["status"] == 0 and res <= TOL
                    grid.append({"schwarz": sch, "d": d, "cycles": cyc, "ms": round(ms, 2) if ok else None,
                                 "inner_iters": i["inner_iters"], "outer_iters": i["outer_iters"],
                                 "dv_count": i["dv_count"], "domain_solves_per_site": i["ras_sweeps"]
                                 // (2 if sch == "sap" else 1), "oracle_true_rel_residual": res})
        done = [g for g in grid if g["ms"] is not None]
        best = {sch: min((g for g in done if g["schwarz"] == sch), key=lambda g: g["ms"], default=None)
                for sch in ("ras", "sap", "as")}
        rec = {"workload": "schwarz",
               "metric": "32^4 solve time to 1e-10 with RAS, SAP (red/black multiplicative) or AS as K",
               "unit": "ms", "ras": {"block": [4, 4, 4, 4], "n_dominv": 4, "inner_prec": "f16"},
               "equal_cost": "a cycle solves every domain once in each variant (SAP: red then black); "
                             "domain_solves_per_site counts them over the whole solve",
               "best": best, "grid": grid}
    elif args.workload == "small":
        # the two small configurations: 8^4 plain FP64 BiCGStab (kappa 0.12),
        # and 16^4 FP32 inner + FP64 defect correction without and with RAS
        # (4^4, s = 0, N_dominv 4, NRAS 3, inner tol 1e-3), kappa 0.12
        runs = {}
        for name, dims, kw in (("8^4 plain FP64", (8, 8, 8, 8), dict(inner_prec="f64")),
                               ("16^4 FP32 inner, no RAS", (16, 16, 16, 16), dict(inner_prec="f32", use_ras=0)),
                               ("16^4 FP32 inner, RAS 4^4", (16, 16, 16, 16),
                                dict(inner_prec="f32", block=(4, 4, 4, 4), n_ras=3, n_dominv=4))):
            U = synth.gauge_field(dims, EPS, GSEED)
            eta = synth.gaussian_source(dims, SSEED)
            st = torch.cuda.Stream()
            lat = qdd.create_lattice(dims, BC, stream=st)
            qdd.load_gauge(lat, torch.from_numpy(U).cuda())
            d_eta = torch.from_numpy(eta).cuda()
            d_phi = torch.empty_like(d_eta)
            p = qdd.default_params(inner_tol=1e-3, **kw)
            qdd.solve(lat, d_phi, d_eta, 0.12, CSW, TOL, p)  # untimed
            ms, infos = time_steps(torch, st, lambda: qdd.solve(lat, d_phi, d_eta, 0.12, CSW, TOL, p), 3)
            i = infos[-1]
            op = oracle.Op(dims, BC, U, 0.12, CSW, store_clover=False)
            runs[name] = {"ms": round(ms, 3), "outer_iters": i["outer_iters"], "inner_iters": i["inner_iters"],
                          "dv_count": i["dv_count"], "ras_sweeps": i["ras_sweeps"],
                          "oracle_true_rel_residual": op.true_residual(eta, d_phi.cpu().numpy())}
            qdd.destroy_lattice(lat)
        rec = {"workload": "small", "metric": "time to 1e-10 on the 8^4 and 16^4 configurations",
               "unit": "ms", "runs": runs}
    elif args.workload == "blocks":
        U = synth.gauge_field(DIMS, EPS, GSEED)
        eta = synth.gaussian_source(DIMS, SSEED)
        st = torch.cuda.Stream()
        lat = qdd.create_lattice(DIMS, BC, stream=st)
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        d_eta = torch.from_numpy(eta).cuda()
        d_phi = torch.empty_like(d_eta)
        op = oracle.Op(DIMS, BC, U, KAPPA, CSW, store_clover=False)
        grid = []
        for blk in ((8, 8, 8, 8), (4, 4, 4, 4), (8, 4, 4, 4)):
            for ov in (0, 1, 2):
                for prec in ("f32", "f16"):
                    p = qdd.default_params(inner_prec=prec, block=blk, overlap=ov, n_ras=1, n_dominv=4,
                                           max_inner=400, max_outer=12)
                    qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p, raise_on_failure=False)  # untimed
                    ms, infos = time_steps(torch, st, lambda: qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p,
                                                                        raise_on_failure=False), 1)
                    i = infos[0]
                    res = op.true_residual(eta, d_phi.cpu().numpy())
                    ok = i["status"] == 0 and res <= TOL
                    grid.append({"block": list(blk), "d": 2 * ov, "inner_prec": prec, "ms": round(ms, 2) if ok else None,
                                 "inner_iters": i["inner_iters"], "dv_count": i["dv_count"],
                                 "oracle_true_rel_residual": res})
        done = [g for g in grid if g["ms"] is not None]
        rec = {"workload": "blocks",
               "metric": "32^4 solve time to 1e-10 over RAS block shapes 8^4, 4^4, 8x4^3, d = 0, 2, 4, FP32 and FP16 inner",
               "unit": "ms", "ras": {"n_ras": 1, "n_dominv": 4}, "best": min(done, key=lambda g: g["ms"]),
               "converged": len(done), "points": len(grid), "grid": grid}
    elif args.workload == "outer":
        U = synth.gauge_field(DIMS, EPS, GSEED)
        eta = synth.gaussian_source(DIMS, SSEED)
        st = torch.cuda.Stream()
        lat = qdd.create_lattice(DIMS, BC, stream=st)
        qdd.load_gauge(lat, torch.from_numpy(U).cuda())
        d_eta = torch.from_numpy(eta).cuda()
        d_phi = torch.empty_like(d_eta)
        op = oracle.Op(DIMS, BC, U, KAPPA, CSW, store_clover=False)
        grid = []
        for prec in ("f16", "f32"):
            for itol in (1e-1, 1e-2, 1e-3):
                for mode in (0, 1):
                    p = qdd.default_params(inner_prec=prec, block=(4, 4, 4, 4), n_ras=1, n_dominv=4,
                                           inner_tol=itol, outer_mode=mode)
                    qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p, raise_on_failure=False)  # untimed
                    ms, infos = time_steps(torch, st, lambda: qdd.solve(lat, d_phi, d_eta, KAPPA, CSW, TOL, p,
                                                                        raise_on_failure=False), 1)
                    i = infos[0]
                    res = op.true_residual(eta, d_phi.cpu().numpy())
                    ok = i["status"] == 0 and res <= TOL
                    grid.append({"outer": "defect correction" if mode == 0 else "BiCGStab", "inner_prec": prec,
                                 "inner_tol": itol, "ms": round(ms, 2) if ok else None,
                                 "outer_iters": i["outer_iters"], "inner_iters": i["inner_iters"],
                                 "oracle_true_rel_residual": res})
        done = [g for g in grid if g["ms"] is not None]
        rec = {"workload": "outer",
               "metric": "32^4 solve time to 1e-10: FP64 defect correction vs the paper's FP64 outer BiCGStab",
               "unit": "ms", "ras": {"block": [4, 4, 4, 4], "n_ras": 1, "n_dominv": 4},
               "best": {o: min((g for g in done if g["outer"] == o), key=lambda g: g["ms"], default=None)
                        for o in ("defect correction", "BiCGStab")},
               "grid": grid}
    elif args.workload == "mrhs":
        dims, kappa, eps = (24, 24, 24, 48), 0.124, 0.25
        U = synth.gauge_field(dims, eps, 1)
        src = np.stack([synth.point_source(dims, s_, c_) for s_ in range(4) for c_ in range(3)])
        st = torch.cuda.Stream()
        lat = qdd.create_lattice(dims, BC, n_rhs=12, stream=st)
        dU = torch.from_numpy(U).cuda()
        qdd.load_gauge(lat, dU)
        d_src = torch.from_numpy(src).cuda()
        d_phi = torch.empty_like(d_src)
        # tune on a one-RHS lattice of the same field (the parameters do not depend on the RHS count)
        lat1 = qdd.create_lattice(dims, BC, stream=st)
        qdd.load_gauge(lat1, dU)
        p, best_ms = qdd.autotune(lat1, d_src[0].contiguous(), kappa, CSW, TOL, qdd.default_params(inner_prec="f16"),
                                  max_trials=args.tune_trials)
        # the single-right-hand-side FP16 D on the same lattice, for the per-RHS ratio
        a1, b1 = qdd.field_create(lat1, "f16"), qdd.field_create(lat1, "f16")
        qdd.field_import(a1, d_src[0].contiguous())
        for _ in range(3):
            qdd.dslash_field(lat1, b1, a1, kappa, CSW)
        ms_d1, _ = time_steps(torch, st, lambda: qdd.dslash_field(lat1, b1, a1, kappa, CSW), 20)
        qdd.field_destroy(a1)
        qdd.field_destroy(b1)
        qdd.destroy_lattice(lat1)

        def step():
            qdd.load_gauge(lat, dU)
            return qdd.solve(lat, d_phi, d_src, kappa, CSW, TOL, p)
        for _ in range(args.warmup):
            step()
        n0 = qdd.kernel_launches()
        ms, infos = time_steps(torch, st, step, args.steps)
        launches = (qdd.kernel_launches() - n0) // args.steps
        # the multi-RHS dslash against one RHS at a time (FP16, internal fields)
        a = qdd.field_create(lat, "f16")
        b = qdd.field_create(lat, "f16")
        qdd.field_import(a, d_phi)
        ms_d, _ = time_steps(torch, st, lambda: qdd.dslash_field(lat, b, a, kappa, CSW), 20)
        phi = d_phi.cpu().numpy()
        op = oracle.Op(dims, BC, U, kappa, CSW, store_clover=False)
        res = [op.true_residual(src[r], phi[r]) for r in range(12)]
        V = int(np.prod(dims))
        bytes_12 = 12 * (52 + 52) * V + (96 + 148) * V
        rec = {"workload": "mrhs", "metric": "time to solve 12 point sources to 1e-10 on 24^3x48",
               "value": round(ms / 1e3, 4), "unit": "s", "per_rhs_s": round(ms / 1e3 / 12, 5),
               "steps": args.steps, "warmup": args.warmup,
               "ras": {"block": list(p.block), "overlap": p.overlap, "n_dominv": p.n_dominv, "n_ras": p.n_ras,
                       "tuned_best_ms_one_rhs": round(best_ms, 2)},
               "inner_iters": [i["inner_iters"] for i in infos[-1]],
               "outer_iters": [i["outer_iters"] for i in infos[-1]],
               "oracle_true_rel_residual_max": max(res),
               "dslash_12rhs_f16": {"us_per_launch": round(ms_d * 1e3, 1),
                                     "us_per_rhs": round(ms_d * 1e3 / 12, 1),
                                     "us_one_rhs_lattice": round(ms_d1 * 1e3, 1),
                                     "per_rhs_over_one_rhs": round(ms_d / 12 / ms_d1, 3),
                                     "algorithmic_GB/s": round(bytes_12 / (ms_d * 1e-3) / 1e9, 1),
                                     "note": "links and clover counted once for the 12 right-hand sides"},
               "gpu_launches_per_step": int(launches)}
    else:
        draws = synth.uneven_batch(16, 1)
        lats, etas, phis, checks = [], [], [], []
        streams = [torch.cuda.Stream() for _ in draws]
        dUs = []
        for d, st in zip(draws, streams):
            U = synth.gauge_field(d["dims"], d["eps"], d["gauge_seed"])
            eta = synth.gaussian_source(d["dims"], d["source_seed"])
            lat = qdd.create_lattice(d["dims"], BC, stream=st)
            dUs.append(torch.from_numpy(U).cuda())
            qdd.load_gauge(lat, dUs[-1])
            lats.append(lat)
            etas.append(torch.from_numpy(eta).cuda())
            phis.append(torch.empty_like(etas[-1]))
            checks.append((U, eta))
        kap = [d["kappa"] for d in draws]
        # the parameter survey once per lattice shape (on the first system of
        # that shape); the tuning cache then feeds every system of the shape
        tuned = {}
        for i, d in enumerate(draws):
            key = tuple(d["dims"])
            if key in tuned:
                continue
            tp, tms = qdd.autotune(lats[i], etas[i], kap[i], CSW, TOL, qdd.default_params(inner_prec="f16"),
                                   max_trials=min(args.tune_trials, 24))
            tuned[key] = {"block": list(tp.block), "overlap": tp.overlap, "n_dominv": tp.n_dominv, "n_ras": tp.n_ras,
                          "inner_prec": {1: "f32", 2: "f16"}[tp.inner_prec], "inner_tol": tp.inner_tol,
                          "tuned_solve_ms": round(tms, 2)}
        shared = qdd.default_params(inner_prec="f16", block=(4, 4, 4, 4), n_dominv=3, n_ras=2)

        def run_batch(params):
            for lat, dU in zip(lats, dUs):
                qdd.load_gauge(lat, dU)
            return qdd.solve_batch(lats, phis, etas, kap, [CSW] * len(lats), TOL, params)

        def timed(params, lists=True):
            prev = qdd.set_batch_lists(lists)
            try:
                for _ in range(args.warmup):
                    run_batch(params)
                torch.cuda.synchronize()
                n0 = qdd.kernel_launches()
                t0 = time.perf_counter()
                for _ in range(args.steps):
                    infos = run_batch(params)
                torch.cuda.synchronize()
            finally:
                qdd.set_batch_lists(prev)
            return (time.perf_counter() - t0) / args.steps * 1e3, (qdd.kernel_launches() - n0) // args.steps, infos

        # with the work lists (compatible lattices share each launch of an
        # iteration) and without (every lattice launches its own kernels)
        ms_shared, launches_shared, _ = timed(shared)
        ms_shared_own, launches_shared_own, _ = timed(shared, lists=False)
        ms, launches, infos = timed([None] * len(lats))   # per-size tuned parameters from the cache
        ms_own, launches_own, _ = timed([None] * len(lats), lists=False)
        res = []
        for d, (U, eta), phi in zip(draws, checks, phis):
            op = oracle.Op(d["dims"], BC, U, d["kappa"], CSW, store_clover=False)
            res.append(op.true_residual(eta, phi.cpu().numpy()))
        # the same systems solved one at a time with their tuned parameters
        ms_single = 0.0
        for i in range(len(lats)):
            qdd.solve(lats[i], phis[i], etas[i], kap[i], CSW, TOL, qdd.tuned_params(lats[i]))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            qdd.load_gauge(lats[i], dUs[i])
            qdd.solve(lats[i], phis[i], etas[i], kap[i], CSW, TOL, qdd.tuned_params(lats[i]))
            torch.cuda.synchronize()
            ms_single += (time.perf_counter() - t0) * 1e3
        rec = {"workload": "batch", "metric": "time to solve 16 uneven systems to 1e-10 in one graph",
               "value": round(ms / 1e3, 4), "unit": "s", "steps": args.steps, "warmup": args.warmup,
               "systems": [{"dims": d["dims"], "kappa": round(d["kappa"], 4), "eps": round(d["eps"], 3)} for d in draws],
               "inner_iters": [i[0]["inner_iters"] for i in infos],
               "oracle_true_rel_residual_max": max(res),
               "tuned_per_shape": {"x".join(map(str, k)): v for k, v in tuned.items()},
               "one_shared_setting_s": round(ms_shared / 1e3, 4),
               "shared_setting": {"block": list(shared.block), "n_dominv": shared.n_dominv, "n_ras": shared.n_ras},
               "work_lists": {"tuned_s": round(ms / 1e3, 4), "tuned_own_launches_s": round(ms_own / 1e3, 4),
                              "shared_s": round(ms_shared / 1e3, 4),
                              "shared_own_launches_s": round(ms_shared_own / 1e3, 4),
                              "launches_per_step": {"tuned": int(launches), "tuned_own": int(launches_own),
                                                    "shared": int(launches_shared),
                                                    "shared_own": int(launches_shared_own)},
                              "note": "own launches: every lattice launches its own kernels (forked in the graph)"},
               "sum_of_single_tuned_solves_s": round(ms_single / 1e3, 4),
               "gpu_launches_per_step": int(launches), "note": "graph replays count the launches they contain"}
    rec["total_wall_s"] = round(time.perf_counter() - t_all, 1)
    print(json.dumps(rec), flush=True)
    return 0


def run_kernels(spec, dims=None):
    """Kernel microbenchmark for profilers: builds the 32^4 workload (or the
    lattice `dims`, with the same generators) and runs
    one kernel a few times -- dslash:<prec>,
    ras:<prec>[:<s>[:<bx>x<by>x<bz>x<bt>[:<n_dominv>]]] (one RAS sweep,
    extension s, default 0, blocks default 4^4, N_dominv default 4: s = 1, 2
    run the thread-block-cluster sweep, 4x32x32x32 slabs the phased sweep),
    mrhs:<n> (the FP16 D on n right-hand sides) or clover (the clover build)."""
    import torch

    import synth
    from paper_1011_3318_gb300 import qdd
    kind, _, prec = spec.partition(":")
    prec, _, ext = prec.partition(":")
    ext, _, blk = ext.partition(":")
    blk, _, ndv = blk.partition(":")
    block = tuple(int(b) for b in blk.split("x")) if blk else (4, 4, 4, 4)
    n_dominv = int(ndv) if ndv else 4
    dims = tuple(dims or DIMS)
    U = synth.gauge_field(dims, EPS, GSEED)
    eta = synth.gaussian_source(dims, SSEED)
    lat = qdd.create_lattice(dims, BC)
    qdd.load_gauge(lat, torch.from_numpy(U).cuda())
    deta = torch.from_numpy(eta).cuda()
    out = torch.empty_like(deta)
    if kind == "dslash":
        a = qdd.field_create(lat, prec)
        b = qdd.field_create(lat, prec)
        qdd.field_import(a, deta)
        for _ in range(3):
            qdd.dslash_field(lat, b, a, KAPPA, CSW)
    elif kind == "ras":
        p = qdd.default_params(inner_prec=prec, n_ras=1, n_dominv=n_dominv, overlap=int(ext or 0), block=block)
        for _ in range(3):
            qdd.ras_apply(lat, out, deta, KAPPA, CSW, p)
        # then the sweep alone, timed by the library's per-class CUDA events
        qdd.set_profiling(lat, True)
        qdd.profile_read(lat, True)
        for _ in range(5):
            qdd.ras_apply(lat, out, deta, KAPPA, CSW, p)
        ms, n = qdd.profile_read(lat, True)["ras"]
        qdd.set_profiling(lat, False)
        log(f"RAS sweep {spec}: {1e3 * ms / max(n, 1):.1f} us per sweep (CUDA events, {n} sweeps)")
    elif kind == "clover":
        for k in range(3):
            qdd.dslash(lat, out, deta, KAPPA + 0.001 * k, CSW, "f32")
    elif kind == "mrhs":
        # the FP16 D on a lattice with n right-hand sides (two per thread)
        n = int(prec or 12)
        latm = qdd.create_lattice(dims, BC, n_rhs=n)
        qdd.load_gauge(latm, torch.from_numpy(U).cuda())
        src = torch.stack([torch.from_numpy(synth.gaussian_source(dims, SSEED + r)) for r in range(n)]).cuda()
        a = qdd.field_create(latm, "f16")
        b = qdd.field_create(latm, "f16")
        qdd.field_import(a, src)
        for _ in range(3):
            qdd.dslash_field(latm, b, a, KAPPA, CSW)
    else:
        raise SystemExit(f"unknown kernel {spec}")
    torch.cuda.synchronize()
    log(f"ran {spec}")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--prec", choices=("f16", "f32"), default="f16")
    ap.add_argument("--block", type=lambda s: tuple(int(x) for x in s.split(",")), default=(4, 4, 4, 4))
    ap.add_argument("--overlap", type=int, default=0)
    ap.add_argument("--n-dominv", dest="n_dominv", type=int, default=4)
    ap.add_argument("--n-ras", dest="n_ras", type=int, default=3)
    ap.add_argument("--inner-tol", dest="inner_tol", type=float, default=1e-3)
    ap.add_argument("--no-cpu-baseline", dest="no_cpu_baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="no_autotune", action="store_true",
                    help="use --block/--overlap/--n-dominv/--n-ras as given instead of tuning them")
    ap.add_argument("--tune-trials", dest="tune_trials", type=int, default=56)
    ap.add_argument("--workload", choices=("solve", "mrhs", "batch", "survey", "table1", "schwarz", "outer",
                                           "blocks", "small"),
                    default="solve",
                    help="solve: the 32^4 headline; mrhs / batch: the batched workloads; survey: the Sec. 5 "
                         "parameter survey; table1: the paper's slab-domain experiment emulated; schwarz: RAS, "
                         "SAP and AS compared as the preconditioner; outer: defect correction vs outer BiCGStab; "
                         "blocks: block shapes x overlaps x inner precisions; small: the 8^4 and 16^4 configurations")
    ap.add_argument("--kernels", default=None,
                    help="profiler workload: dslash:f16|f32|f64, ras:f16|f32[:s[:bxxbyxbzxbt[:n_dominv]]], "
                         "mrhs:<n right-hand sides> (FP16) or clover, three launches at 32^4")
    ap.add_argument("--kernel-dims", dest="kernel_dims", type=lambda s: tuple(int(x) for x in s.split(",")),
                    default=None, help="lattice of the --kernels workload (default 32,32,32,32)")
    args = ap.parse_args()
    if args.kernels:
        return run_kernels(args.kernels, args.kernel_dims)
    if args.workload != "solve":
        return run_workload(args)
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
