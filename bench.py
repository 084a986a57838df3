#!/usr/bin/env python3
"""Benchmark of randomized QRCP (Alg. 2) on GB300.

Default workload: plain FP64 full RQRCP (k = n) of an 8192 x 8192 matrix with i.i.d.
N(0,1) entries, b = 64, p = 8.  A step is one whole factorization (sketch, every pivot
search, swap, panel, compact-WY update and Eq. (4) sketch update) of a fresh copy of the
input; the 512 MB input is larger than L2 and is rewritten before every step.

metric value = counted flops / time, counted flops F = 2 l m n + 4 m n k - 2 (m+n) k^2 + 4 k^3/3
(sketch + Householder QR to rank k).  One JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded sample of
the same workload on the host cores.  With torchrun (N > 1) every rank factors its own
matrix (independent replicas: the single-matrix path has no data-parallel split), value
is the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RQRCP ms & GFLOP/s, mixed vs plain FP64 at rel. residual ≤1e-6; % roofline"

WORKLOADS = {
    "fp64_8192_iid": dict(m=8192, n=8192, k=8192, b=64, p=8, kind="iid", prec="fp64",
                          desc="plain FP64 full RQRCP 8192x8192, i.i.d. N(0,1), b=64, p=8"),
    "fp64_8192_rank500": dict(m=8192, n=8192, k=8192, b=64, p=8, kind="rank500", prec="fp64",
                              desc="plain FP64 full RQRCP 8192x8192, exactly rank 500 (G1 G2), b=64, p=8"),
    "fp64_4096_iid": dict(m=4096, n=4096, k=4096, b=64, p=8, kind="iid", prec="fp64",
                          desc="plain FP64 full RQRCP 4096x4096, i.i.d. N(0,1), b=64, p=8 (profiling size)"),
    "fp64_1000_k64": dict(m=1000, n=1000, k=64, b=32, p=8, kind="logspec", prec="fp64",
                          desc="plain FP64 partial RQRCP k=64 on 1000x1000 U diag(10^(-6i/1000)) V^T, b=32, p=8"),
    "diff_4096_k256": dict(m=4096, n=4096, k=256, b=64, p=8, kind="invsq", prec="diff",
                           desc="differentiable truncated RQRCP: FP32 forward + backward of "
                                "||A - Q1 [R11 R12] Pi^T||_F^2 + random upstream on (Q1, R), 4096x4096, "
                                "sigma_i = 1/(1+i)^2, k=256, b=64, p=8"),
    "batched_512": dict(m=4096, n=2048, k=256, b=64, p=8, kind="batch", prec="batched",
                        desc="batched RQRCP: 512 FP32 matrices, m~U[256,4096], n~U[128,min(m,2048)], "
                             "k~U[16,256], sigma_i = exp(-i/(0.1 n)), p=8, b per shape from the autotuner, "
                             "one persistent launch replayed from a CUDA graph"),
    "mixed_16384x8192_k128": dict(m=16384, n=8192, k=128, b=64, p=16, kind="expspec200", prec="mixed",
                                  desc="mixed partial RQRCP k=128 on 16384x8192 FP32 U diag(exp(-i/200)) V^T, "
                                       "b=64, p=16 (profiling size)"),
    "mixed_32768x16384_k512": dict(m=32768, n=16384, k=512, b=64, p=16, kind="expspec200", prec="mixed",
                                   desc="mixed partial RQRCP k=512 on 32768x16384 FP32 U diag(exp(-i/200)) V^T, "
                                        "b=64, p=16"),
}

# FP64 peak of a GB300 from the recipe's nominal table (DFMA pipe; no measured FP64 entry
# exists in MEASURED_PEAKS.json).
FP64_NOMINAL_TFLOPS = 1.25

# DRAM bytes per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) divided
# by the launch's algorithmic bytes, on the 4096^2 FP64 capture summarised in
# profiles/gemm_fp64_4096_wy_kernels.md; scaled to a full launch by the algorithmic bytes.
MEASURED_TRAFFIC_RATIO = {"fp64": {"wy_gemm_tn": 1.011, "wy_update": 0.609}}


# Roofline of each kernel class.  FP64 form: the SIMT contractions run on the DFMA pipe; the
# tensor-core contractions of the FP32 form stream A once per launch and are bound by HBM; the
# remaining kernels (pivot search, panel QR, small reductions, swaps) are latency-bound chains of
# grid-wide steps, reported against HBM for their algorithmic bytes.
ALU_CLASSES = {"fp64": {"sketch_gemm", "wy_gemm_tn", "wy_update"}, "mixed": set()}


LATENCY_CLASSES = {"pivot", "panel"}  # one grid-wide step per pivot / per panel column


def kernel_rooflines(prof, prec, hbm_peak_gbs, steps_per_launch=None):
    """Per kernel class: time, share, launches and the roofline fraction against its bound;
    the latency-bound classes report microseconds per grid-wide step (steps_per_launch = the
    mean block width bb) next to their HBM fraction."""
    total = sum(v["ms"] for v in prof.values()) or 1e-9
    table = {}
    for name, v in prof.items():
        if not v["launches"] or v["ms"] <= 0:
            continue
        row = {"launches": v["launches"], "ms": round(v["ms"], 4), "share": round(v["ms"] / total, 4)}
        if name in LATENCY_CLASSES and steps_per_launch:
            row["us_per_step"] = round(1e3 * v["ms"] / (v["launches"] * steps_per_launch), 3)
        if name in ALU_CLASSES.get(prec, set()):
            ach = v["flops"] / (v["ms"] * 1e-3) / 1e12
            row.update(bound="alu", achieved=round(ach, 4), peak=FP64_NOMINAL_TFLOPS, unit="TFLOP/s",
                       frac=round(ach / FP64_NOMINAL_TFLOPS, 4))
        else:
            ach = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            row.update(bound="hbm", achieved=round(ach, 2), peak=hbm_peak_gbs, unit="GB/s",
                       frac=round(ach / hbm_peak_gbs, 4))
        table[name] = row
    return table


def counted_flops(m, n, k, l):
    return 2.0 * l * m * n + 4.0 * m * n * k - 2.0 * (m + n) * k * k + 4.0 * k ** 3 / 3.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------------------ inputs
def make_input_torch(w, device, seed=1):
    import torch
    from paper_1804_05138_gb300 import inputs
    m, n = w["m"], w["n"]
    dt = torch.float64 if w["prec"] == "fp64" else torch.float32
    if w["kind"] == "invsq":
        return inputs.spectrum_matrix_torch(m, n, inputs.sigma_inverse_square(min(m, n)), device=device, dtype=dt)
    if w["kind"] == "iid":
        return inputs.gaussian_torch(m, n, seed, device=device, dtype=dt)
    if w["kind"] == "rank500":
        return inputs.rank_r_product_torch(m, n, 500, device=device, dtype=dt)
    if w["kind"] == "logspec":
        return inputs.spectrum_matrix_torch(m, n, inputs.sigma_log_decay(min(m, n)), device=device, dtype=dt)
    if w["kind"] == "expspec200":
        # sigma_i = exp(-i/200): beyond i = 4096 every sigma_i is below 1e-8 sigma_1, under one FP32
        # rounding of the stored entries, so the draw keeps the leading 4096 triplets.
        return inputs.spectrum_matrix_torch(m, n, inputs.sigma_exp_decay(min(m, n), 200.0), device=device,
                                            dtype=dt, rank_cap=4096)
    raise ValueError(w["kind"])


def make_input_numpy(w, m, n):
    from paper_1804_05138_gb300 import inputs
    if w["kind"] == "iid":
        return inputs.gaussian(m, n, seed=1)
    if w["kind"] == "rank500":
        return inputs.rank_r_product(m, n, 500)
    if w["kind"] == "logspec":
        return inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    if w["kind"] == "invsq":
        return inputs.spectrum_matrix(m, n, inputs.sigma_inverse_square(min(m, n)))
    return inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(min(m, n), 200.0))


# ------------------------------------------------------------------------------ CPU oracle leg
def oracle_sample(w, target_s=15.0):
    """Time the FP64 oracle on a bounded sample of workload w: the same m x n matrix but
    only the first blocks (k_sample columns).  Returns (GFLOP/s, cores, description)."""
    import numpy as np
    from oracle import oracle
    oracle.build()
    m, n, b, p = w["m"], w["n"], w["b"], w["p"]
    # keep the sample's memory modest on the host: cap rows/cols at 8192
    ms, ns = min(m, 8192), min(n, 8192)
    A = make_input_numpy(w, ms, ns)
    Om = oracle.omega(b + p, ms, seed=0)
    k_s = min(w["k"], b)
    t0 = time.perf_counter()
    oracle.rqrcp(A, k_s, b, p, Om)
    dt = time.perf_counter() - t0
    # grow the sample to roughly target_s of CPU work
    blocks = max(1, min(int(target_s / max(dt, 1e-3)), max(1, min(w["k"], min(ms, ns)) // b)))
    k_s = min(w["k"], blocks * b, min(ms, ns))
    t0 = time.perf_counter()
    oracle.rqrcp(A, k_s, b, p, Om)
    dt = time.perf_counter() - t0
    gf = counted_flops(ms, ns, k_s, b + p) / dt / 1e9
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    omp = os.environ.get("OMP_NUM_THREADS")
    cores = int(omp) if omp else cores
    desc = f"first {k_s} of {w['k']} pivots ({k_s // b} blocks) on a {ms}x{ns} matrix of the same recipe, {dt:.1f} s"
    return gf, cores, desc, dt


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def gpu_smi_id(dev_index):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev_index] if vis else dev_index


# ------------------------------------------------------------------------------ our arm
# ---- N GPUs: replicas (one process per GPU, each factoring its own matrix; no collective on the
# data path).  The job's time is its slowest rank's; its throughput counts the work of all ranks.
def replica_seed(base, rank):
    """Input seed of a rank's matrix: every replica draws its own matrix of the same recipe."""
    return base + 4096 * rank


def max_over_ranks(x, world, device):
    """max of x over the ranks (x itself when world == 1); device: where the collective runs."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput per second: the units all ranks processed over the job's time (ms)."""
    return world * units_per_rank / (ms * 1e-3)


def gpu_local_cpus(dev):
    """CPUs local to the GPU (the sysfs local_cpulist of its PCI function, within this process's
    affinity), or None when that is not available."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (pr.pci_domain_id, pr.pci_bus_id,
                                                                         pr.pci_device_id)
        with open(path) as f:
            txt = f.read().strip()
        cpus = set()
        for part in txt.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


class NearGpu:
    """Context in which the process runs on the GPU's local CPUs, so that pinned host buffers
    allocated in it land on the GPU's NUMA node; the previous affinity comes back on exit.
    `placement` says what happened ("gpu-local" or "default")."""

    def __init__(self, dev):
        self.dev = dev
        self.old = None
        self.placement = "default"

    def __enter__(self):
        cpus = gpu_local_cpus(self.dev)
        self.old = os.sched_getaffinity(0)
        if cpus:
            try:
                os.sched_setaffinity(0, cpus)
                self.placement = "gpu-local"
            except OSError:
                pass
        return self

    def __exit__(self, *exc):
        try:
            os.sched_setaffinity(0, self.old)
        except OSError:
            pass
        return False


def run_ours(args, w, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1804_05138_gb300 import binding, build as libbuild

    libbuild.build()
    binding.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    m, n, k, b, p = w["m"], w["n"], w["k"], w["b"], w["p"]
    l = b + p
    mixed = w["prec"] in ("mixed", "diff")
    diff = w["prec"] == "diff"
    F = counted_flops(m, n, k, l)
    if diff:  # forward (factor + Q1) and backward (thin-QR adjoint with the wide block)
        F += 4.0 * m * k * k + 4.0 * m * (n - k) * k + 5.0 * m * k * k
    A0 = binding.colmajor(make_input_torch(w, dev, seed=replica_seed(1, rank)))
    A = torch.empty_like(A0.t()).t()
    jpvt = torch.empty(n, dtype=torch.int32, device=dev)
    tau = torch.empty(k, dtype=torch.float64, device=dev)
    need = binding.rqrcp_workspace_size(m, n, k, b, p, binding.RQRCP_PREC_MIXED if mixed else binding.RQRCP_PREC_FP64)
    work = binding.workspace(need, dev)
    stream = torch.cuda.current_stream(dev)
    call = binding.rqrcp_factor_mixed if mixed else binding.rqrcp_factor
    if args.formula == 5:
        if mixed:
            raise SystemExit("--formula 5 applies to the plain FP64 workloads")

        def call(A, k, b, p, seed, jpvt, tau, work):
            return binding.rqrcp_factor_ex(A, k, b, p, seed, None, binding.RQRCP_UPDATE_EQ5, jpvt, tau, work)

    if diff:
        from paper_1804_05138_gb300 import autograd as rq_autograd
        gq = torch.randn((m, k), device=dev, generator=torch.Generator(device=dev).manual_seed(5)) * 1e-3
        gr = torch.randn((k, n), device=dev, generator=torch.Generator(device=dev).manual_seed(6)) * 1e-3

    def one_step(timed_events=None):
        A.copy_(A0)
        if timed_events is not None:
            timed_events[0].record(stream)
        if diff:
            Ag = A.detach().requires_grad_(True)
            Q1, R, jp = rq_autograd.rqrcp_truncated(Ag, k, b, p, 0)
            E = Ag[:, jp.long()] - Q1 @ R
            loss = (E * E).sum() + (gq * Q1).sum() + (gr * R).sum()
            loss.backward()
            code = 0
        else:
            code = call(A, k, b, p, 0, jpvt, tau, work)
        if timed_events is not None:
            timed_events[1].record(stream)
        if code != 0:
            raise binding.RQRCPError(code, "factor")

    for _ in range(args.warmup):
        one_step()
    rank_out = k
    if not diff:  # the differentiable step checks the status of its own workspaces
        code, rank_out = binding.rqrcp_read_status(work)
        if code != 0:
            raise binding.RQRCPError(code, "device status (warm-up)")

    sampler = ClockSampler(gpu_smi_id(local_rank))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    binding.rqrcp_profile_begin()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        one_step(evs[i])
    torch.cuda.synchronize()
    prof = binding.rqrcp_profile_end()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(bv) for a, bv in evs]
    if not diff:
        code, rank_out = binding.rqrcp_read_status(work)
        if code != 0:
            raise binding.RQRCPError(code, "device status (timed)")
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(F, world, ms_per_step) / 1e9

    # dominant kernel and its roofline (alu: FP64 DFMA pipe; mixed: FP32 SIMT)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    launches_total = sum(v["launches"] for v in prof.values())
    kernels_per_launch_class = {"swap": 2, "bupdate": 2}
    if mixed:  # tensor-core contractions: an operand-splitting kernel, then the contraction
        kernels_per_launch_class.update({"sketch_gemm": 2, "wy_gemm_tn": 2, "wy_update": 2})
    gpu_launches = sum(v["launches"] * kernels_per_launch_class.get(kname, 1) for kname, v in prof.items())
    gpu_launches += args.steps  # status/jpvt init kernel, one per factorization
    achieved_tflops = d["flops"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
    peaks = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (copy, measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    kernels = kernel_rooflines(prof, "mixed" if mixed else "fp64", hbm_peak, steps_per_launch=k / ((k + b - 1) // b))
    if mixed:
        # every kernel of the FP32 form is bound by memory traffic or by latency: HBM roofline
        kr = kernels.get(dname, {})
        roof = {"bound": "hbm", "achieved": kr.get("achieved"), "peak": hbm_peak, "unit": "GB/s",
                "frac": kr.get("frac"), "traffic": None, "kernel": dname, "peak_source": hbm_src + ", of measured",
                "algorithmic_bytes_per_launch": round(d["bytes"] / max(1, d["launches"]))}
    else:
        ratio = MEASURED_TRAFFIC_RATIO["fp64"].get(dname)
        traffic = None
        if ratio is not None and d["launches"]:
            traffic = round(ratio * d["bytes"] / d["launches"])
        roof = {"bound": "alu", "achieved": round(achieved_tflops, 4), "peak": FP64_NOMINAL_TFLOPS,
                "unit": "TFLOP/s", "frac": round(achieved_tflops / FP64_NOMINAL_TFLOPS, 4), "traffic": traffic,
                "kernel": dname, "peak_source": "FP64 nominal 1.25 TFLOP/s (recipe table; DFMA pipe)",
                "algorithmic_bytes_per_launch": round(d["bytes"] / max(1, d["launches"])),
                "traffic_source": "ncu 4096^2 capture scaled by algorithmic bytes (profiles/gemm_fp64_4096_wy_kernels.md)"}
    kernel_share = {kname: round(v["ms"] / max(1e-9, sum(x["ms"] for x in prof.values())), 4)
                    for kname, v in prof.items() if v["launches"]}

    # end to end through the public API with host buffers
    # host buffers hold the column-major matrix as a contiguous (n, m) row-major array
    with NearGpu(dev) as near:
        host_A = A0.t().contiguous().cpu().pin_memory()
        host_out = torch.empty_like(host_A).pin_memory()
        host_jpvt = torch.empty(n, dtype=torch.int32).pin_memory()
        host_tau = torch.empty(k, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_e2e = []
    for _ in range(e2e_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        A.t().copy_(host_A, non_blocking=True)
        if diff:
            Ag = A.detach().requires_grad_(True)
            Q1, R, jp = rq_autograd.rqrcp_truncated(Ag, k, b, p, 0)
            E = Ag[:, jp.long()] - Q1 @ R
            ((E * E).sum() + (gq * Q1).sum() + (gr * R).sum()).backward()
            host_out.copy_(Ag.grad.t(), non_blocking=True)
            host_jpvt.copy_(jp, non_blocking=True)
        else:
            code = call(A, k, b, p, 0, jpvt, tau, work)
            if code != 0:
                raise binding.RQRCPError(code, "factor (e2e)")
            host_out.copy_(A.t(), non_blocking=True)
            host_jpvt.copy_(jpvt, non_blocking=True)
            host_tau.copy_(tau, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(sum(t_e2e) / len(t_e2e), world, dev)
    esz = A.element_size()
    e2e = {"value": round(job_rate(F, world, e2e_ms) / 1e9, 3), "unit": "GFLOP/s",
           "h2d_bytes_per_step": m * n * esz, "d2h_bytes_per_step": m * n * esz + n * 4 + k * 8,
           "ms_per_step": round(e2e_ms, 3), "host_buffers": "pinned, " + near.placement}

    extra = {}
    if not diff and not args.no_other_form:
        # the other form on the same matrix: plain FP64 for the mixed workload, mixed for FP64
        other = "fp64" if mixed else "mixed"
        Ao = binding.colmajor(A0.double() if other == "fp64" else A0.float())
        Aw = torch.empty_like(Ao.t()).t()
        jo = torch.empty(n, dtype=torch.int32, device=dev)
        to = torch.empty(k, dtype=torch.float64, device=dev)
        wo = binding.workspace(binding.rqrcp_workspace_size(
            m, n, k, b, p, binding.RQRCP_PREC_FP64 if other == "fp64" else binding.RQRCP_PREC_MIXED), dev)
        co = binding.rqrcp_factor if other == "fp64" else binding.rqrcp_factor_mixed
        times = []
        for it in range(3):
            Aw.copy_(Ao)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            code = co(Aw, k, b, p, 0, jo, to, wo)
            e1.record(stream)
            if code != 0:
                raise binding.RQRCPError(code, "factor (other form)")
            torch.cuda.synchronize()
            if it > 0:
                times.append(e0.elapsed_time(e1))
        code, _ = binding.rqrcp_read_status(wo)
        if code != 0:
            raise binding.RQRCPError(code, "device status (other form)")
        oms = sum(times) / len(times)
        fp64_ms, mixed_ms = (oms, ms_per_step) if other == "fp64" else (ms_per_step, oms)
        extra["same_problem"] = {"form": other, "ms_per_step": round(oms, 3),
                                 "plain_fp64_ms": round(fp64_ms, 3), "mixed_ms": round(mixed_ms, 3),
                                 "mixed_speedup": round(fp64_ms / mixed_ms, 3),
                                 "sketch": "bf16"}
        del Ao, Aw, wo
    if mixed and not diff:
        # FP64 Q1 / R of the factorization just timed, with the CholQR pass forced (tol = 0)
        Q1 = torch.empty((k, m), dtype=torch.float64, device=dev).t()
        R64 = torch.empty((n, k), dtype=torch.float64, device=dev).t()
        orth = torch.zeros(1, dtype=torch.float64, device=dev)
        rw = binding.workspace(binding.rqrcp_reorth_workspace_size(m, n, k), dev)
        t_re = []
        for it in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            code = binding.rqrcp_lowrank_reorth(A, k, tau, Q1, R64, 0.0, orth, rw)
            e1.record(stream)
            if code != 0:
                raise binding.RQRCPError(code, "lowrank_reorth")
            torch.cuda.synchronize()
            t_re.append(e0.elapsed_time(e1))
        code, _ = binding.rqrcp_read_status(rw)
        if code != 0:
            raise binding.RQRCPError(code, "device status (reorth)")
        G = Q1.t() @ Q1
        extra["lowrank_reorth"] = {"ms": round(min(t_re), 3), "orth_before": float(orth.item()),
                                   "orth_after": float(torch.linalg.norm(G - torch.eye(k, dtype=G.dtype, device=dev)))}

    if args.srqr and not mixed and not diff:
        # Alg. 3 (SRQR) on the same matrix: RQRCP to rank L, the extra pivot, the g2 estimate and
        # any swaps; beside it the RQRCP stage alone to k = L
        L = args.srqr
        Aw = torch.empty_like(A0.t()).t()
        ws = binding.workspace(binding.load().rqrcp_srqr_workspace_size(m, n, L, b, p, 8), dev)
        t_sr, t_rq = [], []
        for it in range(3):
            for which in ("srqr", "rqrcp"):
                Aw.copy_(A0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if which == "srqr":
                    f = binding.srqr(Aw, L, b, p, seed=0, g=5.0, d=8, max_swaps=50, work=ws, stream=stream,
                                     overwrite=True)
                else:
                    code = binding.rqrcp_factor(Aw, L, b, p, 0, jpvt, tau, work, stream)
                    if code != 0:
                        raise binding.RQRCPError(code, "factor (rank l)")
                e1.record(stream)
                torch.cuda.synchronize()
                (t_sr if which == "srqr" else t_rq).append(e0.elapsed_time(e1))
        extra["srqr"] = {"l": L, "g": 5.0, "d": 8, "max_swaps": 50, "ms": round(min(t_sr[1:]), 3),
                         "rqrcp_to_l_ms": round(min(t_rq[1:]), 3), "swaps": f.swaps, "g2": f.g2}
        del Aw, ws

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "m": m, "n": n, "k": k, "b": b, "p": p,
                   "sketch_update": "Eq. (5)" if args.formula == 5 else "Eq. (4)",
                   "counted_gflop_per_step": round(F / 1e9, 3),
                   "l2": "inputs larger than L2: the 512 MB+ input is rewritten from a pristine copy before every step",
                   "parallelism": "replicas" if world > 1 else "single", "rank_out": rank_out},
        "roofline": roof,
        "kernel_time_share": kernel_share,
        "kernels": kernels,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if extra:
        out["extra"] = extra
    return out


def run_batched(args, w, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1804_05138_gb300 import autotune, binding, build as libbuild, inputs

    libbuild.build()
    binding.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    p = w["p"]
    shapes = inputs.batched_shapes(args.count, seed=0)
    table = autotune.load_or_tune(shapes, p=p)
    bs = [autotune.choose(table, m, n, k) for (m, n, k) in shapes]
    # the matrices are column-major views (ld = m) into one device pool, so the end-to-end run
    # moves the batch with one copy each way and the restore between steps is one copy
    pool = torch.empty(sum(m * n for m, n, _ in shapes), dtype=torch.float32, device=dev)
    mats = []
    off = 0
    for i, (m, n, _) in enumerate(shapes):
        sig = inputs.sigma_exp_decay(min(m, n), 0.1 * n)
        view = pool[off:off + m * n].view(n, m).t()
        view.copy_(inputs.spectrum_matrix_torch(m, n, sig, seed_u=replica_seed(1000 + 2 * i, rank),
                                                seed_v=replica_seed(1001 + 2 * i, rank), device=dev,
                                                dtype=torch.float32))
        mats.append(view)
        off += m * n
    pristine_pool = pool.clone()
    batch = binding.Batch(mats, [k for _, _, k in shapes], bs, p=p, seed=0)
    F = batch.flops
    stream = torch.cuda.Stream(device=dev)

    def restore():
        pool.copy_(pristine_pool)

    # capture the batched call in a CUDA graph
    restore()
    code = batch.run()
    if code != 0:
        raise binding.RQRCPError(code, "rqrcp_factor_batched")
    graph = torch.cuda.CUDAGraph()
    stream.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            code = batch.run(stream=stream)
    torch.cuda.current_stream(dev).wait_stream(stream)
    if code != 0:
        raise binding.RQRCPError(code, "rqrcp_factor_batched (capture)")
    for _ in range(args.warmup):
        restore()
        graph.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_smi_id(local_rank))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    step_ms = []
    cur = torch.cuda.current_stream(dev)
    for _ in range(args.steps):
        restore()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        graph.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ranks = batch.ranks.cpu().numpy()
    bad = int(np.sum(ranks != np.array([k for _, _, k in shapes])))
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(F, world, ms_per_step) / 1e9
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = F / (ms_per_step * 1e-3) / 1e12
    # end to end: H2D of every matrix from pinned host memory, the batched call, D2H of every result
    with NearGpu(dev) as near:
        host_in = pristine_pool.cpu().pin_memory()  # the batch as stored on the device, one buffer
        host_out = torch.empty_like(host_in).pin_memory()
        host_jall = torch.empty(sum(j.numel() for j in batch.jpvts), dtype=torch.int32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(cur)
    pool.copy_(host_in, non_blocking=True)
    code = batch.run(stream=cur)
    host_out.copy_(pool, non_blocking=True)
    host_jall.copy_(torch.cat(batch.jpvts), non_blocking=True)  # every pivot vector, one copy
    e1.record(cur)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    nbytes = sum(A.numel() * 4 for A in batch.mats)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"] if args.count == 512 else
                   w["desc"].replace("512 FP32 matrices", f"the first {args.count} of the 512 FP32 matrices"),
                   "count": len(shapes), "p": p, "b_histogram":
                   {str(b): int(c) for b, c in zip(*np.unique(bs, return_counts=True))},
                   "counted_gflop_per_step": round(F / 1e9, 3), "bytes_per_step": nbytes,
                   "l2": "inputs larger than L2: 2.6 GB of matrices restored before every step",
                   "parallelism": "replicas" if world > 1 else "single", "ranks_not_k": bad},
        "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / fp32_peak, 4), "traffic": None, "kernel": "batched_kernel",
                     "peak_source": "FP32 SIMT nominal: 152 SMs x 128 lanes x 2 x 2070 MHz"},
        "e2e": {"value": round(job_rate(F, world, e2e_ms) / 1e9, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + host_jall.numel() * 4,
                "ms_per_step": round(e2e_ms, 3), "host_buffers": "pinned, " + near.placement},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="fp64_8192_iid", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count", type=int, default=512,
                    help="batched workload only: factor the first COUNT matrices of the 512-matrix draw "
                         "(a smaller case for profiling; the workload is 512)")
    ap.add_argument("--formula", type=int, default=4, choices=[4, 5],
                    help="plain FP64 workloads: update the sketch between blocks with Eq. (4) (default) "
                         "or Eq. (5)")
    ap.add_argument("--srqr", type=int, default=0, metavar="L",
                    help="plain FP64 workloads: also time SRQR (Alg. 3) to rank L on the same matrix")
    ap.add_argument("--no-other-form", action="store_true",
                    help="skip timing the other form (mixed / plain FP64) on the same matrix")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        per_step = []
        desc = cores = None
        gf_last = None
        for _ in range(args.warmup):
            oracle_sample(w, target_s=2.0)
        for _ in range(args.steps):
            gf, cores, desc, dt = oracle_sample(w, target_s=8.0)
            per_step.append(dt)
            gf_last = gf
        line = {"impl": "reference", "metric": METRIC, "value": round(gf_last, 4), "unit": "GFLOP/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * sum(per_step) / len(per_step), 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": w["desc"], "m": w["m"], "n": w["n"], "k": w["k"], "b": w["b"], "p": w["p"]},
                "cpu_baseline": {"value": round(gf_last, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": round(gf_last, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_batched(args, w, rank, world, local_rank) if w["prec"] == "batched" else \
        run_ours(args, w, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gf, cores, desc, dt = oracle_sample(w, target_s=15.0)
        out["cpu_baseline"] = {"value": round(gf, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                               "sample": desc}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
