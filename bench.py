#!/usr/bin/env python3
"""Benchmark of randomized QRCP (Alg. 2) on GB300.

Default workload: the mixed-vs-plain comparison on a 32768 x 16384 matrix U diag(exp(-i/200)) V^T
stored in FP32, target rank k = 512, b = 64, p = 16.  A step is one whole factorization (sketch,
every pivot search, swap, panel, compact-WY update and Eq. (4) sketch update) of a fresh copy of
the input by the plain FP64 form (the line's `value`); the mixed form (BF16 sketch, 3xTF32 WY
updates, FP64 reflectors) factors the same matrix in `extra.same_problem`.  Both forms report the
backward error ||A Pi - Q R||_F / ||A||_F (estimated from sampled columns in FP64) and
||R22||_2 / sigma_{k+1} (power iteration on the device).  Inputs are larger than L2 and are
rewritten from a pristine device copy before every step.

metric value = counted flops / time, counted flops F = 2 l m n + 4 m n k - 2 (m+n) k^2 + 4 k^3/3
(sketch + Householder QR to rank k).  One JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
  python bench.py --peaks      # the compute-throughput probes only (DFMA, FFMA, tcgen05 TF32/BF16)

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded sample of the same
workload on the host cores.  With torchrun (N > 1) every rank factors its own matrix (independent
replicas: a single matrix has no exchange-free split); the batched workload gives each rank its
LPT-balanced share of the one batch.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RQRCP ms & GFLOP/s, mixed vs plain FP64 at rel. residual ≤1e-6; % roofline"

WORKLOADS = {
    "c3_mixed_vs_fp64": dict(m=32768, n=16384, k=512, b=64, p=16, kind="expspec200", prec="fp64", gen="f32",
                             other="mixed",
                             desc="mixed vs plain FP64 partial RQRCP, k=512, on 32768x16384 U diag(exp(-i/200)) V^T "
                                  "stored in FP32 (the plain form factors its exact FP64 copy), b=64, p=16; value: "
                                  "plain FP64, extra.same_problem: mixed (BF16 sketch, 3xTF32 WY updates, FP64 "
                                  "reflectors)"),
    "fp64_8192_iid": dict(m=8192, n=8192, k=8192, b=64, p=8, kind="iid", prec="fp64", other="mixed",
                          desc="plain FP64 full RQRCP 8192x8192, i.i.d. N(0,1), b=64, p=8"),
    "fp64_8192_rank500": dict(m=8192, n=8192, k=8192, b=64, p=8, kind="rank500", prec="fp64", other=None,
                              desc="plain FP64 full RQRCP 8192x8192, exactly rank 500 (G1 G2), b=64, p=8"),
    "fp64_4096_iid": dict(m=4096, n=4096, k=4096, b=64, p=8, kind="iid", prec="fp64", other="mixed",
                          desc="plain FP64 full RQRCP 4096x4096, i.i.d. N(0,1), b=64, p=8 (profiling size)"),
    "fp64_1000_k64": dict(m=1000, n=1000, k=64, b=32, p=8, kind="logspec", prec="fp64", other="mixed",
                          desc="plain FP64 partial RQRCP k=64 on 1000x1000 U diag(10^(-6i/1000)) V^T, b=32, p=8"),
    "diff_4096_k256": dict(m=4096, n=4096, k=256, b=64, p=8, kind="invsq", prec="diff", other=None,
                           desc="differentiable truncated RQRCP: FP32 forward + backward of "
                                "||A - Q1 [R11 R12] Pi^T||_F^2 + random upstream on (Q1, R), 4096x4096, "
                                "sigma_i = 1/(1+i)^2, k=256, b=64, p=8"),
    "batched_512": dict(m=4096, n=2048, k=256, b=64, p=8, kind="batch", prec="batched", other=None,
                        desc="batched RQRCP: 512 FP32 matrices, m~U[256,4096], n~U[128,min(m,2048)], "
                             "k~U[16,256], sigma_i = exp(-i/(0.1 n)), p=8, b per shape from the autotuner, "
                             "one persistent launch replayed from a CUDA graph"),
    "mixed_16384x8192_k128": dict(m=16384, n=8192, k=128, b=64, p=16, kind="expspec200", prec="mixed", other=None,
                                  desc="mixed partial RQRCP k=128 on 16384x8192 FP32 U diag(exp(-i/200)) V^T, "
                                       "b=64, p=16 (profiling size)"),
    "mixed_32768x16384_k512": dict(m=32768, n=16384, k=512, b=64, p=16, kind="expspec200", prec="mixed",
                                   other="fp64",
                                   desc="mixed partial RQRCP k=512 on 32768x16384 FP32 U diag(exp(-i/200)) V^T, "
                                        "b=64, p=16"),
}
DEFAULT_WORKLOAD = "c3_mixed_vs_fp64"

# FP64 peak of a GB300 from the recipe's nominal table (DFMA pipe), kept beside the measured one.
FP64_NOMINAL_TFLOPS = 1.25

# DRAM bytes per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) divided by the
# launch's algorithmic bytes, on a 4096^2 FP64 capture; scaled to a full launch by its algorithmic bytes.
MEASURED_TRAFFIC_RATIO = {"fp64": {"wy_gemm_tn": 1.011, "wy_update": 0.609}}
TRAFFIC_SOURCE = "ncu capture of the 4096^2 FP64 factorization, scaled by algorithmic bytes"

# Roofline of each kernel class.  FP64 form: the SIMT contractions run on the DFMA pipe; the
# tensor-core contractions of the FP32 form stream A once per launch and are bound by HBM; the
# remaining kernels (pivot search, panel QR, small reductions, swaps) are latency-bound chains of
# grid-wide steps, reported against HBM for their algorithmic bytes.
ALU_CLASSES = {"fp64": {"sketch_gemm", "wy_gemm_tn", "wy_update"}, "mixed": set()}


LATENCY_CLASSES = {"pivot", "panel"}  # one grid-wide step per pivot / per panel column


def kernel_rooflines(prof, prec, hbm_peak_gbs, fp64_peak, steps_per_launch=None):
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
            row.update(bound="alu", achieved=round(ach, 4), peak=round(fp64_peak, 4), unit="TFLOP/s",
                       frac=round(ach / fp64_peak, 4), frac_of_nominal=round(ach / FP64_NOMINAL_TFLOPS, 4))
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
def make_input_torch(w, device, seed=1, dtype=None):
    """The workload's matrix on the device, column-major, in `dtype` (default: the value form's)."""
    import torch
    from paper_1804_05138_gb300 import inputs
    m, n = w["m"], w["n"]
    if dtype is None:
        dtype = torch.float64 if w["prec"] == "fp64" else torch.float32
    if w["kind"] == "invsq":
        return inputs.spectrum_matrix_torch(m, n, inputs.sigma_inverse_square(min(m, n)), device=device, dtype=dtype)
    if w["kind"] == "iid":
        return inputs.gaussian_torch(m, n, seed, device=device, dtype=dtype)
    if w["kind"] == "rank500":
        return inputs.rank_r_product_torch(m, n, 500, device=device, dtype=dtype)
    if w["kind"] == "logspec":
        return inputs.spectrum_matrix_torch(m, n, inputs.sigma_log_decay(min(m, n)), device=device, dtype=dtype)
    if w["kind"] == "expspec200":
        # sigma_i = exp(-i/200): beyond i = 4096 every sigma_i is below 1e-8 sigma_1, under one FP32
        # rounding of the stored entries, so the draw keeps the leading 4096 triplets.
        return inputs.spectrum_matrix_torch(m, n, inputs.sigma_exp_decay(min(m, n), 200.0), device=device,
                                            dtype=dtype, rank_cap=4096)
    raise ValueError(w["kind"])


def sigma_of(w):
    """The workload's prescribed singular values (sigma_1 first), or None where it has none."""
    from paper_1804_05138_gb300 import inputs
    n = min(w["m"], w["n"])
    if w["kind"] == "expspec200":
        return inputs.sigma_exp_decay(n, 200.0)
    if w["kind"] == "logspec":
        return inputs.sigma_log_decay(n)
    if w["kind"] == "invsq":
        return inputs.sigma_inverse_square(n)
    return None


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
    A = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(min(m, n), 200.0), rank_cap=4096)
    return A.astype(np.float32).astype(np.float64) if w.get("gen") == "f32" else A


# ------------------------------------------------------------------------------ CPU oracle leg
def oracle_sample(w, target_s=15.0, A=None):
    """Time the FP64 oracle on a bounded sample of workload w: the workload's m x n matrix (A, when
    given: the very matrix the GPU factored) but only its first blocks.  Returns (GFLOP/s, cores,
    description, seconds)."""
    from oracle import oracle
    oracle.build()
    m, n, b, p = w["m"], w["n"], w["b"], w["p"]
    if A is None:
        A = make_input_numpy(w, m, n)
    Om = oracle.omega(b + p, m, seed=0)
    k_s = min(w["k"], b)
    t0 = time.perf_counter()
    oracle.rqrcp(A, k_s, b, p, Om)
    dt = time.perf_counter() - t0
    # grow the sample to roughly target_s of CPU work
    blocks = max(1, min(int(target_s / max(dt, 1e-3)), max(1, min(w["k"], min(m, n)) // b)))
    if blocks > 1:
        k_s = min(w["k"], blocks * b, min(m, n))
        t0 = time.perf_counter()
        oracle.rqrcp(A, k_s, b, p, Om)
        dt = time.perf_counter() - t0
    gf = counted_flops(m, n, k_s, b + p) / dt / 1e9
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    omp = os.environ.get("OMP_NUM_THREADS")
    cores = int(omp) if omp else cores
    desc = (f"the sketch and the first {k_s} of {w['k']} pivots ({k_s // b} blocks) of the same "
            f"{m}x{n} matrix, {dt:.1f} s")
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


def sum_over_ranks(x, world, device):
    """sum of x over the ranks (x itself when world == 1)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
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


def measured_peaks(stream):
    """DFMA / FFMA / tcgen05 TF32 / tcgen05 BF16 probes of the library (rqrcp_peak_probe)."""
    from paper_1804_05138_gb300 import binding
    out = {}
    for name, kind in (("fp64_dfma", binding.RQRCP_PROBE_DFMA), ("fp32_ffma", binding.RQRCP_PROBE_FFMA),
                       ("tf32_tcgen05", binding.RQRCP_PROBE_TC_TF32), ("bf16_tcgen05", binding.RQRCP_PROBE_TC_BF16)):
        best = 0.0
        for _ in range(3):
            tf, _ms = binding.rqrcp_peak_probe(kind, stream)
            best = max(best, tf)
        out[name] = round(best, 4)
    return out


def apply_q_cols(V, tau, k, Y):
    """Y <- H_0 ... H_{k-1} Y in FP64 on the device (V: the factored array, reflectors below the
    diagonal; Y: m x s).  Measurement only: checks the factorization's output."""
    import torch
    V = V.double()
    for h in range(k - 1, -1, -1):
        v = V[h:, h].clone()
        v[0] = 1.0
        w = float(tau[h]) * (v @ Y[h:])
        Y[h:] -= torch.outer(v, w)
    return Y


def sampled_backward_error(A0, Af, tau, jpvt, k, nsample=64, seed=7):
    """||A Pi - Q R||_F / ||A||_F estimated from `nsample` uniformly drawn columns (plus the block
    boundaries 0, k-1, k, n-1), in FP64 on the device: column j of A Pi - Q R is
    a(:, jpvt[j]) - Q r_j with r_j the j-th column of R (R22 included).  Returns (estimate, max
    relative column error)."""
    import torch
    m, n = A0.shape
    rng = np.random.default_rng(seed)
    cols = np.unique(np.concatenate([rng.integers(0, n, nsample), [0, k - 1, min(k, n - 1), n - 1]]))
    ci = torch.from_numpy(cols).long().to(A0.device)
    R = Af[:, ci].double().clone()
    for t, j in enumerate(cols):
        if j < k:
            R[j + 1:, t] = 0.0
    QR = apply_q_cols(Af, tau.cpu().numpy(), k, R)
    Ac = A0[:, jpvt.long()[ci]].double()
    E = Ac - QR
    col_rel = (torch.linalg.norm(E, dim=0) / torch.linalg.norm(Ac, dim=0).clamp_min(1e-300)).max().item()
    est = (torch.linalg.norm(E).item() * (n / len(cols)) ** 0.5) / torch.linalg.norm(A0.double()).item()
    return est, col_rel


def r22_over_sigma(Af, k, sigma, iters=60):
    """||R22||_2 / sigma_{k+1} by power iteration on R22 = A(k:m, k:n) on the device."""
    import torch
    if sigma is None or k >= min(Af.shape):
        return None
    R22 = Af[k:, k:]
    g = torch.Generator(device=Af.device)
    g.manual_seed(0)
    x = torch.randn(R22.shape[1], device=Af.device, generator=g, dtype=R22.dtype)
    for _ in range(iters):
        x = R22.t() @ (R22 @ x)
        x = x / torch.linalg.norm(x)
    return torch.linalg.norm(R22 @ x).item() / float(sigma[k])


def gpu_launch_count(prof, mixed):
    """Kernels the library launched in the profiled region: classes x kernels per launch of each."""
    per = {"swap": 2, "bupdate": 2, "omega": 0}
    if mixed:  # tensor-core contractions: an operand-splitting kernel, then the contraction; the
        # CholeskyQR2 panel: two Gram, reduce and Cholesky passes, the row solve between them, the
        # rebuild, the row solve below it and the (normally idle) Householder fallback
        per.update({"sketch_gemm": 2, "wy_gemm_tn": 2, "wy_update": 2, "panel": 9})
    return sum(v["launches"] * per.get(kname, 1) for kname, v in prof.items())


class Form:
    """One form of the factorization (plain FP64 or mixed) on one matrix, with its device
    buffers and the sketching matrix Omega on the device (the seeded draw, made once)."""

    def __init__(self, prec, A0, w, dev, pivot="greedy"):
        import torch
        from paper_1804_05138_gb300 import binding
        self.prec, self.w, self.dev, self.pivot = prec, w, dev, pivot
        m, n, k, b, p = w["m"], w["n"], w["k"], w["b"], w["p"]
        self.mixed = prec == "mixed"
        self.A0 = A0
        self.A = torch.empty_like(A0.t()).t()
        self.jpvt = torch.empty(n, dtype=torch.int32, device=dev)
        self.tau = torch.empty(k, dtype=torch.float64, device=dev)
        self.rank = torch.zeros(1, dtype=torch.int64, device=dev)
        self.work = binding.workspace(binding.rqrcp_workspace_size(
            m, n, k, b, p, binding.RQRCP_PREC_MIXED if self.mixed else binding.RQRCP_PREC_FP64), dev)
        self.omega = torch.empty((b + p, m), dtype=A0.dtype, device=dev)
        binding._check(binding.rqrcp_generate_omega(b + p, m, 0, self.omega), "rqrcp_generate_omega")

    def call(self, stream, formula=4, seeded=False):
        """One factorization of self.A in place (seeded: the public seeded entry point, which copies
        the host draw of Omega; else Omega already on the device)."""
        from paper_1804_05138_gb300 import binding
        k, b, p = self.w["k"], self.w["b"], self.w["p"]
        if self.pivot == "tournament":  # QR with tournament pivoting on B, automatic leaf groups
            om = None if seeded else self.omega
            if self.mixed:
                return binding.rqrcp_factor_mixed_tournament(self.A, k, b, p, 0, binding.RQRCP_SKETCH_BF16, 0,
                                                             self.jpvt, self.tau, self.work, stream, Omega=om,
                                                             rank_out=self.rank)
            return binding.rqrcp_factor_tournament(self.A, k, b, p, 0, om, 0, self.jpvt, self.tau, self.work, stream,
                                                   rank_out=self.rank)
        if self.mixed:
            om = None if seeded else self.omega
            return binding.rqrcp_factor_mixed_ex(self.A, k, b, p, 0, binding.RQRCP_SKETCH_BF16, self.jpvt, self.tau,
                                                 self.work, stream, Omega=om, rank_out=self.rank)
        if formula == 5:
            return binding.rqrcp_factor_ex(self.A, k, b, p, 0, None if seeded else self.omega,
                                           binding.RQRCP_UPDATE_EQ5, self.jpvt, self.tau, self.work, stream,
                                           rank_out=self.rank)
        if seeded:
            return binding.rqrcp_factor(self.A, k, b, p, 0, self.jpvt, self.tau, self.work, stream,
                                        rank_out=self.rank)
        return binding.rqrcp_factor_with_omega(self.A, k, b, p, self.omega, self.jpvt, self.tau, self.work, stream,
                                               rank_out=self.rank)

    def timed(self, stream, steps, warmup, formula=4, profile=True):
        """Warm-up, then `steps` factorizations of a fresh copy of A0, each bracketed by CUDA
        events on `stream`; returns (ms per step list, per-class profile or None)."""
        import torch
        from paper_1804_05138_gb300 import binding
        for _ in range(warmup):
            self.A.copy_(self.A0)
            binding._check(self.call(stream, formula), "factor (warm-up)")
        code, _ = binding.rqrcp_read_status(self.work, stream)
        binding._check(code, "device status (warm-up)")
        torch.cuda.synchronize()
        if profile:
            binding.rqrcp_profile_begin()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            self.A.copy_(self.A0)
            evs[i][0].record(stream)
            binding._check(self.call(stream, formula), "factor")
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        prof = binding.rqrcp_profile_end() if profile else None
        code, _ = binding.rqrcp_read_status(self.work, stream)
        binding._check(code, "device status")
        return [a.elapsed_time(bv) for a, bv in evs], prof

    def accuracy(self, A_ref):
        """Backward error (sampled, FP64) and ||R22||_2 / sigma_{k+1} of the factorization in self.A."""
        k = self.w["k"]
        est, col = sampled_backward_error(A_ref, self.A, self.tau, self.jpvt, k)
        ratio = r22_over_sigma(self.A, k, sigma_of(self.w))
        out = {"rel_residual_sampled": float("%.4g" % est), "max_column_rel_residual": float("%.4g" % col),
               "rank": int(self.rank.item())}
        if ratio is not None:
            out["r22_over_sigma_k1"] = round(ratio, 4)
        return out


def roofline_of(prof, kernels, prec, hbm_peak, hbm_src, fp64_peak, fp64_src):
    """The line's roofline object for the dominant kernel class of one form's profile."""
    dname, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    kr = kernels.get(dname, {})
    per_launch = round(d["bytes"] / max(1, d["launches"]))
    if kr.get("bound") == "alu":
        ratio = MEASURED_TRAFFIC_RATIO.get(prec, {}).get(dname)
        traffic = round(ratio * d["bytes"] / d["launches"]) if ratio is not None and d["launches"] else None
        return {"bound": "alu", "achieved": kr["achieved"], "peak": kr["peak"], "unit": "TFLOP/s",
                "frac": kr["frac"], "traffic": traffic, "kernel": dname, "peak_source": fp64_src,
                "peak_nominal": FP64_NOMINAL_TFLOPS, "frac_of_nominal": kr.get("frac_of_nominal"),
                "algorithmic_bytes_per_launch": per_launch, "algorithmic_flops_per_launch":
                round(d["flops"] / max(1, d["launches"])), "traffic_source": TRAFFIC_SOURCE}
    return {"bound": "hbm", "achieved": kr.get("achieved"), "peak": hbm_peak, "unit": "GB/s", "frac": kr.get("frac"),
            "traffic": None, "kernel": dname, "peak_source": hbm_src + ", of measured",
            "algorithmic_bytes_per_launch": per_launch}


def run_ours(args, w, rank, world, local_rank):
    import torch
    from paper_1804_05138_gb300 import binding, build as libbuild

    libbuild.build()
    binding.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    m, n, k, b, p = w["m"], w["n"], w["k"], w["b"], w["p"]
    l = b + p
    diff = w["prec"] == "diff"
    mixed = w["prec"] in ("mixed", "diff")
    F = counted_flops(m, n, k, l)
    if diff:  # forward (factor + Q1) and backward (thin-QR adjoint with the wide block)
        F += 4.0 * m * k * k + 4.0 * m * (n - k) * k + 5.0 * m * k * k
    peaks = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (copy, measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    probes = measured_peaks(stream)
    fp64_peak = probes["fp64_dfma"]
    fp64_src = ("measured: rqrcp_peak_probe DFMA register chains (bench.py --peaks), %.3f TFLOP/s; nominal %.2f"
                % (fp64_peak, FP64_NOMINAL_TFLOPS))
    gen_dtype = torch.float32 if (mixed or w.get("gen") == "f32") else torch.float64
    Agen = binding.colmajor(make_input_torch(w, dev, seed=replica_seed(1, rank), dtype=gen_dtype))
    value_dtype = torch.float32 if mixed else torch.float64
    A0 = Agen if Agen.dtype == value_dtype else binding.colmajor(Agen.to(value_dtype))

    extra = {}
    if diff:
        value_ms, prof, acc = run_diff_steps(args, w, A0, stream)
        rank_out = k
    else:
        form = Form("mixed" if mixed else "fp64", A0, w, dev)
        clocks_sampler = ClockSampler(gpu_smi_id(local_rank))
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        clocks_sampler.start()
        value_ms, prof = form.timed(stream, args.steps, args.warmup, formula=args.formula)
        clocks = clocks_sampler.stop()
        rank_out = int(form.rank.item())
        acc = form.accuracy(A0)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if diff:
        clocks = acc.pop("clocks")
    total_ms = max_over_ranks(sum(value_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(F, world, ms_per_step) / 1e9
    prec_key = "mixed" if mixed else "fp64"
    kernels = kernel_rooflines(prof, prec_key, hbm_peak, fp64_peak, steps_per_launch=k / ((k + b - 1) // b))
    roof = roofline_of(prof, kernels, prec_key, hbm_peak, hbm_src, fp64_peak, fp64_src)
    kernel_share = {kname: v["share"] for kname, v in kernels.items()}
    gpu_launches = gpu_launch_count(prof, mixed) + args.steps  # + the status/jpvt init kernel per call

    # end to end through the public seeded entry point with host buffers: H2D of A, the factorization
    # (its host draw of Omega and that copy included), D2H of the factored A, jpvt and tau
    e2e = run_e2e(args, w, A0, dev, stream, world, F, diff, form if not diff else None)

    other = w.get("other")
    if other and not diff and not args.no_other_form:
        extra["same_problem"] = run_other_form(args, w, Agen, other, dev, stream, ms_per_step, acc, hbm_peak,
                                               hbm_src, fp64_peak, fp64_src)
    if not diff:
        extra["accuracy"] = acc
    if mixed and not diff and not args.no_tournament:
        extra["tournament"] = run_tournament_extra(args, w, A0, dev, stream, ms_per_step, acc, hbm_peak, fp64_peak)
    if args.srqr and not mixed and not diff:
        extra["srqr"] = run_srqr_extra(args, w, A0, dev, stream)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "m": m, "n": n, "k": k, "b": b, "p": p,
                   "sketch_update": "Eq. (5)" if args.formula == 5 else "Eq. (4)",
                   "counted_gflop_per_step": round(F / 1e9, 3),
                   "l2": "inputs larger than L2: the input is rewritten from a pristine device copy before every step",
                   "omega": "seeded draw (host Philox4x64-10 + Box-Muller) copied to the device once, outside the "
                            "timed region; e2e times the seeded entry point with its copy",
                   "parallelism": "replicas" if world > 1 else "single", "rank_out": rank_out},
        "roofline": roof,
        "kernel_time_share": kernel_share,
        "kernels": kernels,
        "peaks_measured": probes,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if extra:
        out["extra"] = extra
    if not diff and not args.no_cpu_baseline and world == 1 and rank == 0:
        out["_A_host"] = A0.double().cpu().numpy()  # the matrix the GPU factored, for the oracle's sample
    return out


def run_diff_steps(args, w, A0, stream):
    """Forward + backward of the differentiable workload, timed per step; the library's profile."""
    import torch
    from paper_1804_05138_gb300 import autograd as rq_autograd, binding
    m, n, k, b, p = w["m"], w["n"], w["k"], w["b"], w["p"]
    dev = A0.device
    gq = torch.randn((m, k), device=dev, generator=torch.Generator(device=dev).manual_seed(5)) * 1e-3
    gr = torch.randn((k, n), device=dev, generator=torch.Generator(device=dev).manual_seed(6)) * 1e-3
    A = torch.empty_like(A0.t()).t()

    def step():
        A.copy_(A0)
        Ag = A.detach().requires_grad_(True)
        Q1, R, jp = rq_autograd.rqrcp_truncated(Ag, k, b, p, 0)
        # A Pi as index_select: its backward is one index_add (each gradient column receives one
        # column), where advanced indexing's backward sorts all m n indices (3-4 ms here)
        E = Ag.index_select(1, jp.long()) - Q1 @ R
        ((E * E).sum() + (gq * Q1).sum() + (gr * R).sum()).backward()

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(gpu_smi_id(dev.index))
    torch.cuda.synchronize()
    sampler.start()
    binding.rqrcp_profile_begin()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = binding.rqrcp_profile_end()
    return ms, prof, {"clocks": sampler.stop()}


def run_e2e(args, w, A0, dev, stream, world, F, diff, form):
    """The metric end to end through the public API at this rank: every step copies the input from
    pinned host memory, factors it and copies the result back; the copies' own rates are reported."""
    import torch
    m, n, k, b, p = w["m"], w["n"], w["k"], w["b"], w["p"]
    with NearGpu(dev) as near:
        host_A = torch.empty((n, m), dtype=A0.dtype, pin_memory=True)
        host_A.copy_(A0.t())
        host_out = torch.empty((n, m), dtype=A0.dtype, pin_memory=True)
        host_jpvt = torch.empty(n, dtype=torch.int32, pin_memory=True)
        host_tau = torch.empty(k, dtype=torch.float64, pin_memory=True)
    if diff:
        from paper_1804_05138_gb300 import autograd as rq_autograd
        gq = torch.randn((m, k), device=dev, generator=torch.Generator(device=dev).manual_seed(5)) * 1e-3
        gr = torch.randn((k, n), device=dev, generator=torch.Generator(device=dev).manual_seed(6)) * 1e-3
        A = torch.empty_like(A0.t()).t()
    else:
        A = form.A
    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t_all, t_h2d, t_d2h = [], [], []
    for _ in range(steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        A.t().copy_(host_A, non_blocking=True)
        ev[1].record(stream)
        if diff:
            Ag = A.detach().requires_grad_(True)
            Q1, R, jp = rq_autograd.rqrcp_truncated(Ag, k, b, p, 0)
            E = Ag.index_select(1, jp.long()) - Q1 @ R
            ((E * E).sum() + (gq * Q1).sum() + (gr * R).sum()).backward()
            ev[2].record(stream)
            host_out.copy_(Ag.grad.t(), non_blocking=True)
            host_jpvt.copy_(jp, non_blocking=True)
        else:
            from paper_1804_05138_gb300 import binding
            binding._check(form.call(stream, args.formula, seeded=True), "factor (e2e)")
            ev[2].record(stream)
            host_out.copy_(A.t(), non_blocking=True)
            host_jpvt.copy_(form.jpvt, non_blocking=True)
            host_tau.copy_(form.tau, non_blocking=True)
        ev[3].record(stream)
        torch.cuda.synchronize()
        t_all.append(ev[0].elapsed_time(ev[3]))
        t_h2d.append(ev[0].elapsed_time(ev[1]))
        t_d2h.append(ev[2].elapsed_time(ev[3]))
    e2e_ms = max_over_ranks(sum(t_all) / len(t_all), world, dev)
    esz = A0.element_size()
    h2d = m * n * esz
    d2h = m * n * esz + n * 4 + (0 if diff else k * 8)
    return {"value": round(job_rate(F, world, e2e_ms) / 1e9, 3), "unit": "GFLOP/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
            "h2d_gbs": round(h2d / (min(t_h2d) * 1e-3) / 1e9, 1), "d2h_gbs": round(d2h / (min(t_d2h) * 1e-3) / 1e9, 1),
            "host_buffers": "pinned, " + near.placement}


def run_other_form(args, w, Agen, other, dev, stream, value_ms, value_acc, hbm_peak, hbm_src, fp64_peak, fp64_src):
    """The other form (mixed for the FP64 value, FP64 for the mixed value) on the same matrix: its
    time, kernels and roofline, accuracy, and the mixed-over-plain speed-up."""
    import torch
    from paper_1804_05138_gb300 import binding
    k, b = w["k"], w["b"]
    dt = torch.float64 if other == "fp64" else torch.float32
    A0 = Agen if Agen.dtype == dt else binding.colmajor(Agen.to(dt))
    form = Form(other, A0, w, dev)
    steps = 3 if other == "fp64" else max(3, args.steps)
    ms, prof = form.timed(stream, steps, 2)
    oms = sum(ms) / len(ms)
    kernels = kernel_rooflines(prof, other, hbm_peak, fp64_peak, steps_per_launch=k / ((k + b - 1) // b))
    acc = form.accuracy(A0)
    fp64_ms, mixed_ms = (oms, value_ms) if other == "fp64" else (value_ms, oms)
    fp64_acc, mixed_acc = (acc, value_acc) if other == "fp64" else (value_acc, acc)
    out = {"form": other, "ms_per_step": round(oms, 3), "steps": steps,
           "value": round(counted_flops(w["m"], w["n"], k, b + w["p"]) / (oms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
           "plain_fp64_ms": round(fp64_ms, 3), "mixed_ms": round(mixed_ms, 3),
           "mixed_speedup": round(fp64_ms / mixed_ms, 3), "sketch": "bf16",
           "accuracy": acc,
           "mixed_meets_target": bool(mixed_acc["rel_residual_sampled"] <= 1e-6),
           "mixed_r22_ratio_vs_plain": (round(mixed_acc["r22_over_sigma_k1"] / fp64_acc["r22_over_sigma_k1"], 4)
                                        if "r22_over_sigma_k1" in mixed_acc and "r22_over_sigma_k1" in fp64_acc
                                        else None),
           "roofline": roofline_of(prof, kernels, other, hbm_peak, hbm_src, fp64_peak, fp64_src),
           "kernels": kernels, "gpu_launches": gpu_launch_count(prof, other == "mixed") + steps}
    if other == "mixed":
        out["lowrank_reorth"] = reorth_extra(form, w, dev, stream)
    del form
    if other == "mixed" and not args.no_tournament:
        out["tournament"] = run_tournament_extra(args, w, A0, dev, stream, oms, acc, hbm_peak, fp64_peak)
    return out


def run_tournament_extra(args, w, A0, dev, stream, greedy_ms, greedy_acc, hbm_peak, fp64_peak):
    """The same form with QR with tournament pivoting on B in place of Alg. 2's partial QRCP:
    time, the pivot search's time per pivot against the greedy search's, accuracy."""
    k, b = w["k"], w["b"]
    mixed = A0.element_size() == 4
    form = Form("mixed" if mixed else "fp64", A0, w, dev, pivot="tournament")
    steps = max(3, args.steps) if mixed else 3
    ms, prof = form.timed(stream, steps, 2)
    tms = sum(ms) / len(ms)
    kernels = kernel_rooflines(prof, "mixed" if mixed else "fp64", hbm_peak, fp64_peak,
                               steps_per_launch=k / ((k + b - 1) // b))
    acc = form.accuracy(A0)
    out = {"pivot": "tournament (leaf groups max(2b, (n-i)/SMs), fan-in 4)", "ms_per_step": round(tms, 3),
           "steps": steps, "value": round(counted_flops(w["m"], w["n"], k, b + w["p"]) / (tms * 1e-3) / 1e9, 3),
           "unit": "GFLOP/s", "greedy_ms": round(greedy_ms, 3), "speedup_over_greedy": round(greedy_ms / tms, 4),
           "pivot_us_per_step": kernels.get("pivot", {}).get("us_per_step"), "accuracy": acc,
           "r22_ratio_vs_greedy": (round(acc["r22_over_sigma_k1"] / greedy_acc["r22_over_sigma_k1"], 4)
                                   if "r22_over_sigma_k1" in acc and "r22_over_sigma_k1" in greedy_acc else None),
           "kernel_time_share": {kname: v["share"] for kname, v in kernels.items()}}
    del form
    return out


def reorth_extra(form, w, dev, stream):
    """FP64 Q1 / R of the mixed factorization just timed, with the CholQR pass forced (tol = 0)."""
    import torch
    from paper_1804_05138_gb300 import binding
    m, n, k = w["m"], w["n"], w["k"]
    Q1 = torch.empty((k, m), dtype=torch.float64, device=dev).t()
    R64 = torch.empty((n, k), dtype=torch.float64, device=dev).t()
    orth = torch.zeros(1, dtype=torch.float64, device=dev)
    rw = binding.workspace(binding.rqrcp_reorth_workspace_size(m, n, k), dev)
    t_re = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        binding._check(binding.rqrcp_lowrank_reorth(form.A, k, form.tau, Q1, R64, 0.0, orth, rw, stream),
                       "lowrank_reorth")
        e1.record(stream)
        torch.cuda.synchronize()
        t_re.append(e0.elapsed_time(e1))
    code, _ = binding.rqrcp_read_status(rw, stream)
    binding._check(code, "device status (reorth)")
    G = Q1.t() @ Q1
    return {"ms": round(min(t_re), 3), "orth_before": float(orth.item()),
            "orth_after": float(torch.linalg.norm(G - torch.eye(k, dtype=G.dtype, device=dev)))}


def run_srqr_extra(args, w, A0, dev, stream):
    """Alg. 3 (SRQR) on the same matrix: RQRCP to rank L, the extra pivot, the g2 estimate and any
    swaps; beside it the RQRCP stage alone to k = L."""
    import torch
    from paper_1804_05138_gb300 import binding
    m, n, b, p = w["m"], w["n"], w["b"], w["p"]
    L = args.srqr
    Aw = torch.empty_like(A0.t()).t()
    ws = binding.workspace(binding.load().rqrcp_srqr_workspace_size(m, n, L, b, p, 8), dev)
    wf = binding.workspace(binding.rqrcp_workspace_size(m, n, L, b, p), dev)
    jpvt = torch.empty(n, dtype=torch.int32, device=dev)
    tau = torch.empty(L, dtype=torch.float64, device=dev)
    t_sr, t_rq = [], []
    f = None
    for _ in range(3):
        for which in ("srqr", "rqrcp"):
            Aw.copy_(A0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if which == "srqr":
                f = binding.srqr(Aw, L, b, p, seed=0, g=5.0, d=8, max_swaps=50, work=ws, stream=stream,
                                 overwrite=True)
            else:
                binding._check(binding.rqrcp_factor(Aw, L, b, p, 0, jpvt, tau, wf, stream), "factor (rank l)")
            e1.record(stream)
            torch.cuda.synchronize()
            (t_sr if which == "srqr" else t_rq).append(e0.elapsed_time(e1))
    return {"l": L, "g": 5.0, "d": 8, "max_swaps": 50, "ms": round(min(t_sr[1:]), 3),
            "rqrcp_to_l_ms": round(min(t_rq[1:]), 3), "swaps": f.swaps, "g2": f.g2}


def run_batched(args, w, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1804_05138_gb300 import autotune, binding, build as libbuild, inputs

    libbuild.build()
    binding.load()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    from paper_1804_05138_gb300 import partition
    p = w["p"]
    all_shapes = inputs.batched_shapes(args.count, seed=0)
    table = autotune.load_or_tune(all_shapes, p=p)
    all_bs = [autotune.choose(table, m, n, k) for (m, n, k) in all_shapes]
    all_tiles = [autotune.choose_tiles(table, m, n, k) for (m, n, k) in all_shapes]
    # N ranks: each factors its LPT share of the one batch (independent matrices, no exchange)
    costs = [binding.batch_cost(m, n, k, b, p) for (m, n, k), b in zip(all_shapes, all_bs)]
    mine = sorted(partition.lpt_partition(costs, world)[rank]) if world > 1 else list(range(len(all_shapes)))
    shapes = [all_shapes[i] for i in mine]
    bs = [all_bs[i] for i in mine]
    tiles = [all_tiles[i] for i in mine]
    # the matrices are column-major views (ld = m) into one device pool, so the end-to-end run
    # moves the batch with one copy each way and the restore between steps is one copy
    pool = torch.empty(sum(m * n for m, n, _ in shapes), dtype=torch.float32, device=dev)
    mats = []
    off = 0
    for i, (m, n, _) in zip(mine, shapes):
        sig = inputs.sigma_exp_decay(min(m, n), 0.1 * n)
        view = pool[off:off + m * n].view(n, m).t()
        view.copy_(inputs.spectrum_matrix_torch(m, n, sig, seed_u=1000 + 2 * i, seed_v=1001 + 2 * i, device=dev,
                                                dtype=torch.float32))
        mats.append(view)
        off += m * n
    pristine_pool = pool.clone()
    batch = binding.Batch(mats, [k for _, _, k in shapes], bs, p=p, seed=0, tiles=tiles)
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
    F_job = sum_over_ranks(F, world, dev)  # the whole batch's counted flops
    value = F_job / (ms_per_step * 1e-3) / 1e9
    fp32_peak = round(measured_peaks(cur)["fp32_ffma"], 3)
    achieved = F / (ms_per_step * 1e-3) / 1e12
    # end to end: H2D of every matrix from pinned host memory, the batched call, D2H of every result
    with NearGpu(dev) as near:
        host_in = torch.empty(pristine_pool.shape, dtype=torch.float32, pin_memory=True)
        host_in.copy_(pristine_pool)  # the batch as stored on the device, one buffer
        host_out = torch.empty_like(host_in, pin_memory=True)
        host_jall = torch.empty(sum(j.numel() for j in batch.jpvts), dtype=torch.int32, pin_memory=True)
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
                   "count": len(all_shapes), "p": p, "b_histogram":
                   {str(b): int(c) for b, c in zip(*np.unique(bs, return_counts=True))},
                   "tiles_histogram": {str(t): int(c) for t, c in zip(*np.unique(tiles, return_counts=True))},
                   "autotune_table": {key: {"b": v["b"], "tiles": v["tiles"]} if isinstance(v, dict) else v
                                      for key, v in sorted(table.items())},
                   "counted_gflop_per_step": round(F / 1e9, 3), "bytes_per_step": nbytes,
                   "l2": "inputs larger than L2: 2.6 GB of matrices restored before every step",
                   "parallelism": f"batch partitioned over {world} ranks (LPT on counted flops)" if world > 1
                   else "single", "matrices_this_rank": len(shapes), "ranks_not_k": bad},
        "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": round(achieved / fp32_peak, 4), "traffic": None, "kernel": "batched_kernel",
                     "peak_source": "measured: rqrcp_peak_probe FFMA register chains (bench.py --peaks)"},
        "e2e": {"value": round(F_job / (e2e_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + host_jall.numel() * 4,
                "ms_per_step": round(e2e_ms, 3), "host_buffers": "pinned, " + near.placement},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    return out


def run_reference(args, w):
    """The oracle (test infrastructure, as it stands) on the host cores: each step a bounded sample
    of the workload (its sketch and first pivot blocks on the same-recipe matrix)."""
    per_step = []
    desc = cores = None
    gf_last = None
    A = make_input_numpy(w, w["m"], w["n"])
    target = 4.0 if w["m"] * w["n"] > 1e8 else 2.0
    for _ in range(args.warmup):
        oracle_sample(w, target_s=1.0, A=A)
    for _ in range(args.steps):
        gf, cores, desc, dt = oracle_sample(w, target_s=target, A=A)
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


def run_peaks():
    import torch
    from paper_1804_05138_gb300 import binding, build as libbuild
    libbuild.build()
    binding.load()
    torch.cuda.set_device(0)
    sampler = ClockSampler(gpu_smi_id(0))
    sampler.start()
    probes = measured_peaks(torch.cuda.current_stream())
    clocks = sampler.stop()
    print(json.dumps({"peaks": probes, "unit": "TFLOP/s", "clocks": clocks,
                      "how": "rqrcp_peak_probe: best of 3 timed launches per probe, CUDA events"}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--peaks", action="store_true", help="run the compute-throughput probes only")
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
    ap.add_argument("--no-tournament", action="store_true",
                    help="skip the mixed form with QR with tournament pivoting on the sketch (extra.tournament)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.formula == 5 and w["prec"] != "fp64":
        raise SystemExit("--formula 5 applies to the plain FP64 workloads")

    if args.peaks:
        return run_peaks() if rank == 0 else 0
    if args.impl == "reference":
        return run_reference(args, w) if rank == 0 else 0

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_batched(args, w, rank, world, local_rank) if w["prec"] == "batched" else \
        run_ours(args, w, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        A_host = None
        if w["prec"] != "batched" and w["m"] * w["n"] > 1 << 26:
            # the very matrix the GPU factored (FP64), for the oracle's sample
            A_host = out.pop("_A_host", None)
        gf, cores, desc, dt = oracle_sample(w, target_s=15.0, A=A_host)
        out["cpu_baseline"] = {"value": round(gf, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                               "sample": desc}
    out.pop("_A_host", None)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
