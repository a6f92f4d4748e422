"""Benchmark: fp64 Jacobi-PCG time to a 1e-8 relative residual on one GB300.

Default workload: 3-D 7-point Poisson on a 256^3 grid (n = 16,777,216,
nnz = 117,047,296), FP64 CSR with int32 indices, x* uniform[-1, 1) from seed 0,
b = A x*, x0 = 0, Jacobi-PCG to ||b - A x|| / ||b|| <= 1e-8.  One step = one
whole solve (every phase of the hot path: SpMV + p.q, x/r update + r.z/r.r,
p update, device-side convergence test, final fp64 true residual) through
the C ABI.  The matrix (1.4 GB) and vectors exceed the 129 MB L2, so no
explicit flush is needed between steps.

Printed JSON line (rank 0):
  value / ms_per_step  solves per second over all ranks and the time to tolerance
                       (inputs resident in HBM, CUDA events on the current stream);
  e2e                  the same through the host-buffer entry point (H2D of b and
                       x0, D2H of x inside the timed region);
  roofline             the dominant kernel of the loop (the SpMV fused with p.q)
                       launched alone on its loop grid, its own bytes per launch
                       over its event-timed launch duration, against the measured
                       HBM copy bandwidth; "fp64_pipe" gives the same kernel's
                       fp64 FMA rate against the pipe's peak (it co-limits);
  loop                 the whole CG loop's own bytes per iteration over its time,
                       and the caller-CSR byte model (column indices, row pointers and
                       the diagonal streamed too) as a separate figure;
  config.setup_ms      cg_create + cg_prepare (validation, loop matrix, vectors);
  cpu_baseline         the CPU oracle on all host cores (OpenMP row-split build)
                       and on one core, each on a bounded sample of iterations
                       scaled to the oracle's own count, with a whole-solve check
                       of that scaling on a smaller system;
  extra                (default workload, one rank) the other configurations
                       timed in the same run: 64x64 Poisson, the 27-point
                       diffusion in fp32 with fp64 reliable updates against
                       plain fp64, the 512-system batch against solving the
                       systems one by one, learned FSAI on the 1024^2 Q1 matrix
                       against plain fp64 Jacobi-PCG, and a general sparse
                       (non-stencil) matrix.

--impl reference times the CPU oracle (the reference arm: the paper ships no code)
on a bounded sample of the same workload.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

Q1_1024 = {"s": 1024, "sigma_a": 1.5, "theta": 0.7, "eps": 0.01, "seed": 3}
FSAI_WEIGHTS = os.path.join(ROOT, "paper_2608_09647_gb300", "fsai_q1aniso_bf16.npy")
DEFAULT = "poisson3d_256"

WORKLOADS = {
    # name: (builder, kwargs, precond, precision, tol, maxit, description)
    "poisson3d_256": ("lap3d7", {"N": 256}, "jacobi", "fp64", 1e-8, 10000,
                      "3-D 7-point Poisson 256^3, FP64 Jacobi-PCG to 1e-8"),
    "poisson2d_64": ("lap2d", {"N": 64}, "none", "fp64", 1e-8, 1000,
                     "2-D 5-point Poisson 64x64, FP64 CG to 1e-8"),
    "poisson2d_96": ("lap2d", {"N": 96}, "none", "fp64", 1e-8, 5000,
                     "2-D 5-point Poisson 96x96 (9216 rows), FP64 CG to 1e-8"),
    "poisson2d_128": ("lap2d", {"N": 128}, "none", "fp64", 1e-8, 5000,
                      "2-D 5-point Poisson 128x128 (16384 rows), FP64 CG to 1e-8"),
    "poisson3d_32": ("lap3d7", {"N": 32}, "jacobi", "fp64", 1e-8, 5000,
                     "3-D 7-point Poisson 32^3 (32768 rows), FP64 Jacobi-PCG to 1e-8"),
    "poisson3d_128": ("lap3d7", {"N": 128}, "jacobi", "fp64", 1e-8, 10000,
                      "3-D 7-point Poisson 128^3, FP64 Jacobi-PCG to 1e-8"),
    "poisson3d_192": ("lap3d7", {"N": 192}, "jacobi", "fp64", 1e-8, 10000,
                      "3-D 7-point Poisson 192^3, FP64 Jacobi-PCG to 1e-8 (profiling size: "
                      "larger than L2, a few GB on the device)"),
    "diffusion27_160": ("diff3d27", {"N": 160, "sigma": 1.0, "seed": 0}, "jacobi", "fp32_ir",
                        1e-10, 100000,
                        "3-D 27-point lognormal diffusion 160^3, FP32 inner / FP64 refinement to 1e-10"),
    "diffusion27_160_ru": ("diff3d27", {"N": 160, "sigma": 1.0, "seed": 0}, "jacobi", "fp32_ru", 1e-10, 100000,
                           "3-D 27-point lognormal diffusion 160^3, FP32 Jacobi-PCG with FP64 reliable "
                           "updates to 1e-10"),
    "diffusion27_160_fp64": ("diff3d27", {"N": 160, "sigma": 1.0, "seed": 0}, "jacobi", "fp64",
                             1e-10, 100000,
                             "3-D 27-point lognormal diffusion 160^3, FP64 Jacobi-PCG to 1e-10"),
    "q1aniso_1024_learned": ("q1aniso", Q1_1024, "fsai_learned", "fp32_ir", 1e-8, 200000,
                             "2-D rotated-anisotropy Q1 diffusion 1024^2 (a_c lognormal sigma 1.5, theta 0.7, "
                             "eps 0.01), learned FSAI, FP32 inner / FP64 refinement to 1e-8"),
    "q1aniso_1024_learned_ru": ("q1aniso", Q1_1024, "fsai_learned", "fp32_ru", 1e-8, 200000,
                                "the same matrix, learned FSAI, FP32 PCG with FP64 reliable updates to 1e-8"),
    "q1aniso_1024_classic": ("q1aniso", Q1_1024, "fsai_classic", "fp32_ir", 1e-8, 200000,
                             "the same matrix, classic FSAI, FP32 inner / FP64 refinement to 1e-8"),
    "q1aniso_1024_jacobi_fp64": ("q1aniso", Q1_1024, "jacobi", "fp64", 1e-8, 200000,
                                 "the same matrix, plain FP64 Jacobi-PCG to 1e-8"),
    "q1aniso_1024_learned_fp64": ("q1aniso", Q1_1024, "fsai_learned", "fp64", 1e-8, 200000,
                                  "the same matrix, learned FSAI, FP64 PCG to 1e-8"),
    "graph_spd_12m": ("graph_spd", {"n": 12_000_000, "dmax": 600, "seed": 0}, "jacobi", "fp64", 1e-8, 20000,
                      "general sparse SPD (graph Laplacian, power-law degrees 1-223 nonzeros per row, "
                      "70 % local / 30 % random couplings), n = 12M, nnz = 71M; FP64 Jacobi-PCG to 1e-8 "
                      "(the row-block CSR loop layout)"),
    "graph_spd_2m": ("graph_spd", {"n": 2_000_000, "dmax": 600, "seed": 0}, "jacobi", "fp64", 1e-8, 20000,
                     "the same family at n = 2M (profiling size)"),
    "batch16": ("batch", {"count": 16, "seed": 0}, "jacobi", "fp64", 1e-8, 20000,
                "the first 16 systems of the 512-system batch (small profiling case)"),
    "batch64": ("batch", {"count": 64, "seed": 0}, "jacobi", "fp64", 1e-8, 20000,
                "the first 64 systems of the 512-system batch (profiling size)"),
    "batch512": ("batch", {"count": 512, "seed": 0}, "jacobi", "fp64", 1e-8, 20000,
                 "512 systems in one launch: 2-D 5-/9-point anisotropic Laplacians, side uniform "
                 "in [32, 512], eps log-uniform in [1e-3, 1]; FP64 Jacobi-PCG to 1e-8 each"),
    "batch512_fp32": ("batch", {"count": 512, "seed": 0}, "jacobi", "fp32_ru", 1e-8, 20000,
                      "the same 512 systems in one launch, FP32 Jacobi-PCG with FP64 reliable "
                      "updates to 1e-8 each"),
}
BATCH_GOLDEN = os.path.join(ROOT, "tests", "golden", "batch512_oracle.json")

# Configurations timed beside the default workload (one rank): (label, workload,
# steps) and the pairs compared on the same GPU (faster form, plain fp64 form).
EXTRAS = ("poisson2d_64", "diffusion27_160_ru", "diffusion27_160_fp64", "q1aniso_1024_learned_ru",
          "q1aniso_1024_jacobi_fp64", "batch512", "batch512_fp32", "graph_spd_12m")
EXTRA_PAIRS = (("diffusion27_160_ru", "diffusion27_160_fp64"),
               ("q1aniso_1024_learned_ru", "q1aniso_1024_jacobi_fp64"),
               ("batch512_fp32", "batch512"))


def bytes_per_iter(n, nnz, precond, precision):
    """Modelled (algorithmic) HBM bytes of one CG iteration on the caller's CSR: the
    CSR stream plus the vector streams of the three phases (SpMV + p.q, x/r update,
    p update)."""
    if precision == "fp64":
        return 12 * nnz + 4 * (n + 1) + (104 if precond == "jacobi" else 88) * n
    return 8 * nnz + 4 * (n + 1) + (52 if precond == "jacobi" else 44) * n


def load_peaks():
    """(HBM GB/s, how it was obtained, fp64 FMA per second of the pipe at max clock)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mhz = 2070.0
    if os.path.exists(p):
        d = json.load(open(p))
        mhz = float(d.get("sm_max_mhz", mhz))
        return float(d["hbm_gbs"]), "measured", fp64_fma_peak(mhz)
    return 6800.0, "fallback", fp64_fma_peak(mhz)


def fp64_fma_peak(sm_mhz, sms=152, dfma_per_clk_per_sm=2):
    """fp64 FMAs per second: GB300 issues 2 fp64 FMAs per clock per SM (ncu's
    sm__sass_thread_inst_executed_op_dfma_pred_on.avg.peak_sustained), 152 SMs."""
    return sms * dfma_per_clk_per_sm * sm_mhz * 1e6


# Sources that define each workload's timed kernels: a committed traffic figure
# counts only while these files are unchanged.
KERNEL_SOURCES = {
    "single": ("cg_exact.cuh", "cg_device.cuh", "cg_csr.cuh", "cg_kernels.cuh", "cg_graph.cuh"),
    "batch": ("cg_exact.cuh", "cg_device.cuh", "cg_csr.cuh", "cg_kernels.cuh", "cg_batch.cu"),
    "fsai": ("cg_exact.cuh", "cg_device.cuh", "cg_csr.cuh", "cg_kernels.cuh", "cg_graph.cuh", "cg_fsai.cu",
             "cg_fsai.cuh"),
}


def _code_only(text):
    """Source text without its comments and blank lines: editing a comment does not
    change the kernels a traffic figure was measured on."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_sha(kind="single"):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2608_09647_gb300", "csrc")
    for f in KERNEL_SOURCES[kind]:
        h.update(_code_only(open(os.path.join(csrc, f)).read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kind="single", loop_form=None):
    """DRAM bytes of the timed kernels from the committed ncu summary, if it was taken
    from the current kernel sources and, where it names one, in the loop form that
    ran (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(workload)
    if not d or d.get("kernel_sha") != kernel_source_sha(kind):
        return None
    if loop_form is not None and d.get("loop_form", loop_form) != loop_form:
        return None
    return d


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def build_matrix(workload):
    import cgproblems as gen
    builder, kw, *_ = WORKLOADS[workload]
    return getattr(gen, builder)(**kw)


def golden_iters(workload):
    p = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if workload in d:
            return int(d[workload]["iters"])
    return None


def time_oracle_sample(A, b, precond, precision, budget_s, lib=None):
    """Time the oracle on a bounded sample of the workload: PCG iterations on the full
    matrix, as many as fit the budget.  lib: the all-core (OpenMP) build for fp64 PCG.
    Returns (seconds per iteration, iterations run)."""
    import oracle
    pc = 1 if precond == "jacobi" else 0
    g = None
    if precond.startswith("fsai"):  # the oracle's own factor (setup not timed)
        from oracle import fsai
        import numpy as np
        if precond == "fsai_classic":
            g = fsai.classic(A)
        else:
            bits = np.load(FSAI_WEIGHTS)
            g = fsai.learned(A, (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64))
    m = 2
    while True:
        t0 = time.perf_counter()
        if g is not None and precision == "fp64":
            fsai.pcg(A, g, b, tol=0.0, maxit=m, max_restarts=0)
        elif g is not None:
            fsai.pcg_ir(A, g, b, tol=0.0, tol_in=1e-30, maxit=m, max_outer=1)
        elif precision == "fp64":
            oracle.pcg(A, b, tol=0.0, maxit=m, precond=pc, max_restarts=0, lib=lib)
        else:
            oracle.pcg_ir(A, b, tol=0.0, tol_in=1e-30, maxit=m, max_outer=1, precond=pc)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 3 or m >= 4096:
            return dt / m, m
        m = max(m * 2, int(m * (budget_s / 3) / max(dt, 1e-3)))


def oracle_scaling_check(lib=None, N=64):
    """A whole oracle solve of a smaller system of the default family (3-D 7-point
    Poisson N^3, Jacobi-PCG to 1e-8) against the estimate the sampling method makes
    for it (seconds per iteration from a short sample x the solve's iterations)."""
    import oracle
    import cgproblems as gen
    A = gen.lap3d7(N)
    b = oracle.spmv(A, gen.xstar(A.n, 0))
    s_iter, m = time_oracle_sample(A, b, "jacobi", "fp64", 1.5, lib)
    t0 = time.perf_counter()
    r = oracle.pcg(A, b, tol=1e-8, maxit=10000, precond=1, lib=lib)
    whole = time.perf_counter() - t0
    return {"system": f"3-D 7-point Poisson {N}^3, Jacobi-PCG to 1e-8", "iters": r.iters,
            "whole_solve_s": whole, "sampled_estimate_s": s_iter * r.iters,
            "estimate_over_measured": s_iter * r.iters / whole}


def cpu_baseline_single(A, b, workload, precond_s, precision_s, budget_s, iters_fallback):
    """The oracle on the host cores: all cores (OpenMP build, fp64 PCG) and one core,
    each a bounded sample of iterations on the full matrix scaled to the oracle's own
    iteration count."""
    import oracle
    it_ref = golden_iters(workload) or iters_fallback
    s1, m1 = time_oracle_sample(A, b, precond_s, precision_s, budget_s)
    one = {"value": 1.0 / (s1 * it_ref), "unit": "solves/s", "cores": 1,
           "sample": (f"{m1} oracle iterations of the same system on 1 host core "
                      f"({s1 * 1e3:.1f} ms/iter), scaled to {it_ref} iterations"),
           "ms_per_solve": s1 * it_ref * 1e3, "check": oracle_scaling_check()}
    lib, threads = oracle.openmp()
    out = dict(one)
    out["kind"] = "oracle"
    out["one_core"] = one
    out["all_cores"] = None
    if lib is not None and precision_s == "fp64" and not precond_s.startswith("fsai"):
        sa, ma = time_oracle_sample(A, b, precond_s, precision_s, budget_s / 2, lib)
        allc = {"value": 1.0 / (sa * it_ref), "unit": "solves/s", "cores": threads,
                "sample": (f"{ma} iterations of the OpenMP row-split build on {threads} host "
                           f"threads ({sa * 1e3:.1f} ms/iter), scaled to {it_ref} iterations"),
                "ms_per_solve": sa * it_ref * 1e3, "check": oracle_scaling_check(lib, 128)}
        out.update({k: allc[k] for k in ("value", "cores", "sample", "ms_per_solve", "check")})
        out["all_cores"] = allc
    elif lib is None:
        out["all_cores_unavailable"] = "no OpenMP build of the oracle on this host"
    else:
        out["all_cores_unavailable"] = "the OpenMP build covers the fp64 (Jacobi-)PCG loops only"
    return out


def max_over_ranks(x, world, device=None):
    """x from every rank reduced to its maximum (the job's time is its slowest
    rank's); x itself with one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, t_max_s):
    """Whole-job units per second: every rank processes `steps` units in the
    slowest rank's time."""
    return world * steps / t_max_s


def run_reference(args):
    """The oracle as the reference arm: rank 0 times bounded samples on the host cores
    (all of them through the OpenMP build where it covers the workload)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import cgproblems as gen
    builder, _, precond, precision, tol, maxit, desc = WORKLOADS[args.workload]
    per_step_budget = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    if builder == "batch":
        _, systems = batch_systems(args.workload)
        gold = batch_golden_iters(len(systems))
        if gold is None:
            print(json.dumps({"impl": "reference", "unavailable":
                              "no golden oracle iteration counts for the batch (tests/golden)"}))
            return
        for _ in range(args.warmup):
            time_oracle_batch_sample(systems, gold, per_step_budget)
        times = []
        for _ in range(args.steps):
            t, sample = time_oracle_batch_sample(systems, gold, per_step_budget)
            times.append(t)
        solve_s = statistics.median(times)
        value = 1.0 / solve_s
        line = {"impl": "reference",
                "metric": "batched PCG time to 1e-8 rel. residual, all systems (batches/s)",
                "value": value, "unit": "batches/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": solve_s * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "description": desc, "systems": len(systems),
                           "rows": int(sum(A.n for A in systems))},
                "cpu_baseline": {"value": value, "unit": "batches/s", "cores": 1, "kind": "oracle",
                                 "sample": sample, "extrapolated": True},
                "e2e": {"value": value, "unit": "batches/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    A = build_matrix(args.workload)
    b = oracle.spmv(A, gen.xstar(A.n, 0))
    iters = golden_iters(args.workload)
    lib, threads = oracle.openmp()
    if lib is None or precision != "fp64" or precond.startswith("fsai"):
        lib, threads = None, 1
    for _ in range(args.warmup):
        time_oracle_sample(A, b, precond, precision, per_step_budget, lib)
    samples = []
    for _ in range(args.steps):
        s, m = time_oracle_sample(A, b, precond, precision, per_step_budget, lib)
        samples.append((s, m))
    s_iter = statistics.median(s for s, _ in samples)
    solve_s = s_iter * iters if iters else None
    value = 1.0 / solve_s if solve_s else None
    sample = (f"{samples[0][1]} oracle {precision} {'Jacobi-' if precond == 'jacobi' else ''}PCG "
              f"iterations on the full matrix per step ({'OpenMP build, ' if lib else ''}{threads} "
              f"host threads), scaled to {iters if iters else '?'} iterations (the oracle's own count "
              f"to tol): an extrapolation, not a whole solve")
    line = {"impl": "reference", "metric": "PCG time to 1e-8 rel. residual (solves/s)",
            "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": solve_s * 1e3 if solve_s else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": A.n, "nnz": A.nnz},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "s_per_iter": s_iter, "extrapolated": True},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_systems(workload):
    import cgproblems as gen
    kw = WORKLOADS[workload][1]
    params = gen.batch_members(512, kw["seed"])[:kw["count"]]
    return params, [gen.lap2d(side, pts, eps) for side, pts, eps in params]


def batch_golden_iters(count):
    """The oracle's own iteration count of every batch member (committed golden file)."""
    if not os.path.exists(BATCH_GOLDEN):
        return None
    d = json.load(open(BATCH_GOLDEN))
    if d.get("count") != count:
        return None
    return [m["iters"] for m in d["members"]]


def time_oracle_batch_sample(systems, iters, budget_s):
    """Time the oracle on a bounded sample of a batch: fixed Jacobi-PCG iterations on a few
    members spread over the size range; seconds per (row x iteration) from the sample,
    scaled to sum_i n_i k_i.  Returns (seconds per batch solve, sample description)."""
    import oracle
    import cgproblems as gen
    order = sorted(range(len(systems)), key=lambda i: systems[i].n)
    picks = [order[int(q * (len(order) - 1))] for q in (0.0, 0.25, 0.5, 0.75, 1.0)]
    rows_iters, secs, m = 0, 0.0, 4
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < budget_s / 2:
        for i in picks:
            A = systems[i]
            b = oracle.spmv(A, gen.xstar(A.n, i))
            t0 = time.perf_counter()
            oracle.pcg(A, b, tol=0.0, maxit=m, precond=1, max_restarts=0)
            secs += time.perf_counter() - t0
            rows_iters += A.n * m
        m *= 2
    per = secs / rows_iters
    total = sum(A.n * k for A, k in zip(systems, iters))
    desc = (f"oracle Jacobi-PCG iterations on members {picks} (n = "
            f"{[systems[i].n for i in picks]}), {rows_iters} row-iterations in {secs:.1f} s on 1 core, "
            f"scaled to sum_i n_i k_i = {total}")
    return per * total, desc


def _barrier(world, torch):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def _uuid(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


def bench_batch(args, workload, steps, warmup, world, rank, dev, torch, cg, full=True):
    """The batched workload: every system of the batch in one cg_solve_batch per step."""
    _, kw, precond_s, precision_s, tol, maxit, desc = WORKLOADS[workload]
    precond = cg.CG_PRECOND_JACOBI if precond_s == "jacobi" else cg.CG_PRECOND_NONE
    precision = {"fp64": cg.CG_PREC_FP64, "fp32_ir": cg.CG_PREC_FP32_IR, "fp32_ru": cg.CG_PREC_FP32_RU}[precision_s]
    params, systems = batch_systems(workload)
    import numpy as np
    import cgproblems as gen
    ns = [A.n for A in systems]
    off = np.concatenate([[0], np.cumsum(ns)])
    ntot = int(off[-1])
    # one flat buffer per vector kind; member i is a view (x is reset by one fill per step)
    b_flat = torch.empty(ntot, dtype=torch.float64, device=dev)
    x_flat = torch.zeros(ntot, dtype=torch.float64, device=dev)
    for i, A in enumerate(systems):
        bi = A.to_scipy() @ gen.xstar(A.n, i)  # b = A x* (scipy, input preparation)
        b_flat[off[i]:off[i + 1]].copy_(torch.from_numpy(bi))
    bs = [b_flat[off[i]:off[i + 1]] for i in range(len(systems))]
    xs = [x_flat[off[i]:off[i + 1]] for i in range(len(systems))]
    dev_csr = [tuple(torch.from_numpy(a).to(dev) for a in (A.rowptr, A.colind, A.vals)) for A in systems]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = cg.cg_batch_create([c[0] for c in dev_csr], [c[1] for c in dev_csr], [c[2] for c in dev_csr])
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    if args.loop_mode in ("persistent", "graph"):
        assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, 1 if args.loop_mode == "persistent" else 2) == cg.CG_OK
    if args.grid:
        assert cg.cg_set_option(h, cg.CG_OPT_GRID_CTAS, args.grid) == cg.CG_OK

    def step():
        x_flat.zero_()
        st, its, rels = cg.cg_solve_batch(h, bs, xs, tol, maxit, precond, precision)
        if st != cg.CG_OK:
            raise RuntimeError(f"batch solve failed: {cg.status_string(st)} {cg.cg_last_error(h)}")
        return its, rels, cg.cg_get_solve_info(h)

    t0 = time.perf_counter()
    step()                                       # the first solve runs the autotuner
    first_ms = (time.perf_counter() - t0) * 1e3
    for _ in range(max(0, warmup - 1)):
        step()
    tuning = cg.cg_batch_get_tuning(h, precond, precision)

    infos = []
    _barrier(world, torch)
    with ClockSampler(_uuid(torch, dev)) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            infos.append(step())
        ev1.record()
        _barrier(world, torch)
    t_max = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ms_per_step = t_max / steps
    value = job_throughput(world, steps, t_max / 1e3)
    its = infos[0][0]
    relres = max(max(r) for _, r, _ in infos)
    kern_ms = sum(inf["kernel_ms"] for _, _, inf in infos)
    kern_bytes = sum(inf["bytes_moved"] for _, _, inf in infos)
    peak, peak_kind, _ = load_peaks()
    achieved = kern_bytes / (kern_ms / 1e3) / 1e9
    launches = sum(inf["kernel_launches"] for _, _, inf in infos)
    form = {1: "persistent", 2: "graph"}.get(infos[0][2]["loop_form"], "?")
    # DRAM bytes of one launch from the committed ncu capture (a smaller batch, scaled by
    # the row-iterations processed), while the kernel sources are unchanged
    row_iters = int(sum(n_i * k_i for n_i, k_i in zip(ns, its)))
    tr = ncu_traffic(workload, "batch") if precision_s == "fp64" else None
    traffic = int(tr["dram_bytes_per_row_iter"] * row_iters) if tr else None
    # the fp64 kernel's algorithmic bytes: a member whose off-diagonal entries lie on
    # d <= 8 offsets is stored by diagonal, and one of its row-iterations streams the d
    # slot values (8 B each) plus p, q (phase A), q, r read and r written (B), and
    # x, p, r read and x, p written (C): 8 d + 80 bytes
    own_bytes = None
    if precision_s == "fp64":
        own_bytes = 0
        for A, k_i in zip(systems, its):
            rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
            offs = np.unique(A.colind.astype(np.int64) - rows)
            d = int(np.count_nonzero(offs))
            w = d if d <= 8 else int(np.max(np.diff(A.rowptr)))
            own_bytes += ((8 if d <= 8 else 12) * w + 80) * A.n * int(k_i)
    own_achieved = own_bytes / (kern_ms / steps / 1e3) / 1e9 if own_bytes else None

    e2e = None
    if full and not args.no_e2e:
        bh = b_flat.cpu().pin_memory()
        x0h = torch.zeros(ntot, dtype=torch.float64).pin_memory()
        xh = torch.empty(ntot, dtype=torch.float64).pin_memory()
        _barrier(world, torch)
        t0 = time.perf_counter()
        for _ in range(steps):
            b_flat.copy_(bh, non_blocking=True)
            x_flat.copy_(x0h, non_blocking=True)
            st, _, _ = cg.cg_solve_batch(h, bs, xs, tol, maxit, precond, precision)
            if st != cg.CG_OK:
                raise RuntimeError(f"batch solve failed: {cg.status_string(st)}")
            xh.copy_(x_flat, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        _barrier(world, torch)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_throughput(world, steps, e2e_s), "unit": "batches/s",
               "h2d_bytes_per_step": 16 * ntot, "d2h_bytes_per_step": 8 * ntot}

    # the same systems solved one after another by cg_solve (plain FP64 Jacobi-PCG,
    # one launch per system), for comparison on the same GPU
    seq = None
    if not args.no_sequential and precision_s == "fp64":
        handles = [cg.cg_create(A.n, *c) for A, c in zip(systems, dev_csr)]
        bsq = [b.clone() for b in bs]  # own (16-byte aligned) vectors per system
        xsq = [torch.zeros_like(b) for b in bsq]
        for hs, bi, xi in zip(handles, bsq, xsq):  # warm: build each handle's loop matrix
            cg.cg_solve(hs, bi, xi, tol, maxit, precond)
        for xi in xsq:
            xi.zero_()
        _barrier(world, torch)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for hs, bi, xi in zip(handles, bsq, xsq):
            st, _, _ = cg.cg_solve(hs, bi, xi, tol, maxit, precond)
            if st != cg.CG_OK:
                raise RuntimeError(f"sequential solve failed: {cg.status_string(st)}")
        e1.record()
        _barrier(world, torch)
        seq_ms = e0.elapsed_time(e1)
        for hs in handles:
            cg.cg_destroy(hs)
        seq = {"ms": seq_ms, "what": "cg_solve on each system in turn (FP64 Jacobi-PCG, auto loop form)",
               "batched_speedup": seq_ms / ms_per_step}

    cpu = None
    if full and rank == 0 and world == 1 and not args.no_cpu_baseline:
        gold = batch_golden_iters(len(systems))
        k_used = gold if gold else its
        solve_s, sample = time_oracle_batch_sample(systems, k_used, args.cpu_budget)
        sample += " (oracle's own counts)" if gold else " (this run's counts: no golden file)"
        cpu = {"value": 1.0 / solve_s, "unit": "batches/s", "cores": 1, "kind": "oracle",
               "sample": sample, "ms_per_batch": solve_s * 1e3, "extrapolated": True}
    cg.cg_destroy(h)
    return {
        "metric": "batched PCG time to 1e-8 rel. residual, all systems (batches/s)",
        "value": value, "unit": "batches/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision_s == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": workload, "description": desc, "systems": len(systems),
                   "precision": precision_s,
                   "rows": ntot, "nnz": int(sum(A.nnz for A in systems)), "tol": tol,
                   "iters_max": max(its), "iters_sum": int(sum(its)), "row_iterations": row_iters,
                   "relres_true_max": relres, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (no flush)",
                   "setup_ms": setup_ms, "first_solve_ms": first_ms,
                   "grid_ctas": infos[0][2]["grid_ctas"], "autotuner": tuning,
                   "loop_mode": args.loop_mode},
        "roofline": {"bound": "hbm", "achieved": own_achieved, "peak": peak, "unit": "GB/s",
                     "frac": own_achieved / peak if own_achieved else None, "traffic": traffic,
                     "peak_kind": peak_kind,
                     "achieved_is": "the fp64 kernel's algorithmic bytes (8 d + 80 per row-iteration "
                                    "of a member stored by its d diagonals) / the launch's device "
                                    "time; traffic = ncu DRAM bytes per row-iteration x the "
                                    "row-iterations (null without a current ncu figure)",
                     "timed_unit": "one batched solve: the persistent batch kernel (whole launch)",
                     "loop_form": form,
                     "achieved_survey_model": achieved, "frac_survey_model": achieved / peak,
                     "bytes_model": ("sum over systems of iters x (12 nnz + 4 (n+1) + 104 n)"
                                     if precision_s == "fp64" else
                                     "sum over systems of inner iters x (8 nnz + 4 (n+1) + 52 n)")},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
        "sequential_fp64": seq,
    }


def dominant_kernel(h, A, precond, precision, torch, cg, dev, peak, fma_peak, reps=50):
    """The loop's SpMV fused with p.q (the graph form's per-iteration SpMV kernel) launched
    alone on its loop grid, `reps` times between CUDA events on the current stream."""
    fp64 = precision == cg.CG_PREC_FP64
    dt = torch.float64 if fp64 else torch.float32
    p = torch.rand(A.n, dtype=dt, device=dev) - 0.5
    q = torch.empty_like(p)
    st, nbytes = cg.cg_loop_spmv(h, p, q, precond, precision, reps=3)   # warm
    if st != cg.CG_OK:
        return None
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    cg.cg_loop_spmv(h, p, q, precond, precision, reps=reps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    mi = cg.cg_get_matrix_info(h)
    # fp64 FMAs of one launch: each stored off-diagonal slot and the p.q term per row
    # (the diagonal starts the chain; without Jacobi it is one more multiply)
    ent = nbytes  # placeholder for clarity below
    fmas = None
    if fp64:
        od = (nbytes - (16 if precond == cg.CG_PRECOND_JACOBI else 24) * A.n) / 8  # diagonal layout
        fmas = od + A.n * (1 if precond == cg.CG_PRECOND_JACOBI else 2)
    del ent
    out = {"kernel": "g_spmv (loop SpMV fused with p.q, graph-form kernel, launched alone)",
           "ms_per_launch": ms, "bytes_per_launch": nbytes, "achieved_gbs": nbytes / ms / 1e6,
           "frac": nbytes / ms / 1e6 / peak, "launches_timed": reps, "n": mi["n"]}
    if fmas is not None:
        out["fp64_fma_per_launch"] = int(fmas)
        out["fp64_pipe"] = {"achieved_gfma_s": fmas / ms / 1e6, "peak_gfma_s": fma_peak / 1e9,
                            "frac": fmas / ms / 1e6 / (fma_peak / 1e9)}
    return out


def bench_single(args, workload, steps, warmup, world, rank, dev, torch, cg, full=True):
    """One single-system workload: setup, warm-up, `steps` timed solves, and (full) the
    end-to-end, dominant-kernel, SpMV-comparison and CPU-baseline legs."""
    import numpy as np
    import cgproblems as gen
    builder, kw, precond_s, precision_s, tol, maxit, desc = WORKLOADS[workload]
    precond = {"jacobi": cg.CG_PRECOND_JACOBI, "none": cg.CG_PRECOND_NONE}.get(precond_s, cg.CG_PRECOND_FSAI)
    precision = {"fp64": cg.CG_PREC_FP64, "fp32_ir": cg.CG_PREC_FP32_IR, "fp32_ru": cg.CG_PREC_FP32_RU}[precision_s]

    # every rank solves its own copy of the system (replicas: weak scaling)
    A = build_matrix(workload)
    rp, ci, va = (torch.from_numpy(a).to(dev) for a in (A.rowptr, A.colind, A.vals))
    xs = torch.from_numpy(gen.xstar(A.n, 0)).to(dev)
    torch.cuda.synchronize()
    # setup: validation, row blocks, diagonal (cg_create), loop matrix and vectors (cg_prepare)
    t0 = time.perf_counter()
    h = cg.cg_create(A.n, rp, ci, va)
    st = cg.cg_prepare(h, cg.CG_PRECOND_JACOBI if precond_s.startswith("fsai") else precond, precision)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    if st != cg.CG_OK:
        raise RuntimeError(f"cg_prepare failed: {cg.cg_last_error(h)}")
    mode = {"auto": 0, "persistent": 1, "graph": 2, "unrolled": 3, "cluster": 4}[args.loop_mode]
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
    b = torch.empty_like(xs)
    assert cg.cg_spmv(h, xs, b) == cg.CG_OK        # b = A x* on the device
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    precond_setup_ms = None
    if precond_s.startswith("fsai"):  # the factor, once per matrix (timed on its own)
        def setup(hh):
            if precond_s == "fsai_classic":
                r = cg.cg_fsai_classic(hh)
            else:
                bits = np.load(FSAI_WEIGHTS)
                r = cg.cg_fsai_load(hh, (bits.astype(np.uint32) << 16).view(np.float32))
            if r != cg.CG_OK:
                raise RuntimeError(f"FSAI setup failed: {cg.cg_last_error(hh)}")
        # once on a scratch handle first: the first use of the setup kernels
        # (module loading) is not part of a factor's cost
        hw = cg.cg_create(A.n, rp, ci, va)
        setup(hw)
        cg.cg_destroy(hw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        setup(h)  # the whole setup on a fresh handle: pattern, factor, loop layouts
        precond_setup_ms = (time.perf_counter() - t0) * 1e3

    def step():
        x.zero_()
        r, it, rel = cg.cg_solve(h, b, x, tol, maxit, precond, precision)
        if r != cg.CG_OK:
            raise RuntimeError(f"solve failed: {cg.status_string(r)} {cg.cg_last_error(h)}")
        return it, rel, cg.cg_get_solve_info(h)

    t0 = time.perf_counter()
    step()                                         # first solve: also builds the loop graph
    first_ms = (time.perf_counter() - t0) * 1e3
    for _ in range(max(0, warmup - 1)):
        step()

    infos = []
    _barrier(world, torch)
    with ClockSampler(_uuid(torch, dev)) as clocks:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            infos.append(step())
        ev1.record()
        _barrier(world, torch)
    elapsed_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(elapsed_ms, world, dev)
    ms_per_step = t_max / steps
    value = job_throughput(world, steps, t_max / 1e3)

    iters = [i for i, _, _ in infos]
    relres = max(r for _, r, _ in infos)
    kern_ms = sum(inf["kernel_ms"] for _, _, inf in infos)
    kern_bytes = sum(inf["bytes_moved"] for _, _, inf in infos)
    own_bytes = sum(inf["kernel_bytes_per_iter"] * inf["iters"] for _, _, inf in infos)
    peak, peak_kind, fma_peak = load_peaks()
    achieved_model = kern_bytes / (kern_ms / 1e3) / 1e9
    achieved_own = own_bytes / (kern_ms / 1e3) / 1e9
    form = {1: "persistent", 2: "graph", 3: "unrolled", 4: "cluster"}.get(infos[0][2]["loop_form"], "?")
    launches = sum(inf["kernel_launches"] for _, _, inf in infos)
    tr = ncu_traffic(workload, "fsai" if precond_s.startswith("fsai") else "single", form)
    loop_traffic = int(tr["dram_bytes_per_iter"] * statistics.mean(iters)) if tr else None
    loop = {"achieved_gbs": achieved_own, "frac": achieved_own / peak,
            "bytes_per_iter": infos[0][2]["kernel_bytes_per_iter"],
            "iter_us": 1e3 * kern_ms / sum(iters), "loop_form": form,
            "timed_unit": {"persistent": "the CG loop of one solve: the persistent kernel",
                           "cluster": "the CG loop of one solve: one thread-block cluster kernel"}.get(
                               form, "the CG loop of one solve: SpMV, r-update and x/p-update kernels"),
            "traffic_per_solve": loop_traffic,
            "achieved_gbs_survey_model": achieved_model, "frac_survey_model": achieved_model / peak,
            "bytes_per_iter_survey_model": kern_bytes / max(1, sum(iters)),
            "survey_model": "12 nnz + 4 (n+1) + 104 n (Jacobi) / 88 n bytes per iteration on the "
                            "caller's CSR, fp64; this design moves neither the column indices, rowptr "
                            "nor the diagonal in the loop"}

    dom = None
    if not args.no_dominant and not precond_s.startswith("fsai") and form != "cluster":
        # (the cluster form runs no separate SpMV kernel: its loop is one kernel)
        dom = dominant_kernel(h, A, precond, precision, torch, cg, dev, peak, fma_peak)
    if dom is not None:
        trd = ncu_traffic(workload + ":g_spmv", "single")
        roofline = {"bound": "hbm", "achieved": dom["achieved_gbs"], "peak": peak, "unit": "GB/s",
                    "frac": dom["frac"],
                    "traffic": int(trd["dram_bytes_per_launch"]) if trd else None,
                    "peak_kind": peak_kind, "kernel": dom["kernel"],
                    "bytes_per_launch": dom["bytes_per_launch"], "ms_per_launch": dom["ms_per_launch"],
                    "fp64_pipe": dom.get("fp64_pipe"),
                    "bytes_are": "the loop matrix slots (8 B each in the diagonal layout, +4 B column "
                                 "otherwise), p read once and q written: this kernel's algorithmic bytes"}
    elif form == "cluster" and loop["bytes_per_iter"] == 0:
        # vectors and CSR in the cluster's shared memory: nothing moves from outside the
        # SMs, and the iteration's time is a latency chain (row products, two exchanges
        # of partial sums across the cluster, two fp64 divisions), not a throughput
        roofline = {"bound": "latency", "achieved": loop["iter_us"], "peak": None, "unit": "us/iteration",
                    "frac": None, "traffic": None, "peak_kind": None,
                    "kernel": "the whole CG loop (" + loop["timed_unit"] + ")",
                    "note": "no bytes from outside the SMs per iteration: vectors and CSR held in the "
                            "cluster's shared memory"}
        loop["frac"] = None
    else:
        roofline = {"bound": "hbm", "achieved": achieved_own, "peak": peak, "unit": "GB/s",
                    "frac": achieved_own / peak, "traffic": loop_traffic, "peak_kind": peak_kind,
                    "kernel": "the whole CG loop (" + loop["timed_unit"] + ")"}
    # a loop whose working set fits the 129 MB L2 (an FSAI loop near 10^6 rows) can
    # move its own bytes faster than HBM: its fraction is not an HBM roofline
    ws = loop["bytes_per_iter"]
    loop["l2_resident"] = bool(ws and ws < 129e6)
    if dom is None and roofline["bound"] != "latency":
        if loop["l2_resident"]:
            roofline["bound"] = "l2"
        if roofline["frac"] is not None and roofline["frac"] > 1.0:
            roofline["note"] = (f"above 1: the loop's own bytes ({ws / 1e6:.0f} MB an iteration) are partly "
                                "served by the 129 MB L2")
    elif roofline["frac"] is not None and roofline["frac"] > 1.1:
        # above the measured copy bandwidth by more than a copy kernel's own spread:
        # the byte count does not describe what the kernel moves
        raise RuntimeError(f"roofline fraction {roofline['frac']:.2f} exceeds the measured peak")

    e2e = None
    if full and not args.no_e2e:
        bh = torch.from_numpy(b.cpu().numpy()).pin_memory()
        xh = torch.zeros(A.n, dtype=torch.float64).pin_memory()
        cg.cg_solve_host(h, bh, xh, tol, maxit, precond, precision)   # warm the staging buffers
        _barrier(world, torch)
        t0 = time.perf_counter()
        for _ in range(steps):
            xh.zero_()
            r, it, rel = cg.cg_solve_host(h, bh, xh, tol, maxit, precond, precision)
            if r != cg.CG_OK:
                raise RuntimeError(f"host solve failed: {cg.status_string(r)}")
        _barrier(world, torch)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_throughput(world, steps, e2e_s), "unit": "solves/s",
               "h2d_bytes_per_step": 16 * A.n, "d2h_bytes_per_step": 8 * A.n}

    # the caller-CSR SpMV (cg_spmv) against cuSPARSE through torch's CSR tensor, the
    # comparison the paper makes for its own kernel (Sec. 4.1)
    spmv = None
    if full and not args.no_spmv_compare:
        spmv = spmv_compare(h, A, rp, ci, va, xs, torch, cg, peak)

    cpu = None
    if full and rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        bo = oracle.spmv(A, gen.xstar(A.n, 0))
        cpu = cpu_baseline_single(A, bo, workload, precond_s, precision_s, args.cpu_budget,
                                  int(statistics.median(iters)))

    cg.cg_destroy(h)
    return {
        "metric": "PCG time to 1e-8 rel. residual (solves/s)",
        "value": value, "unit": "solves/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision_s == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": workload, "description": desc, "n": A.n, "nnz": A.nnz,
                   "tol": tol, "iters": iters[0], "relres_true_max": relres, "precond": precond_s,
                   "precision": precision_s, "setup_ms": setup_ms, "precond_setup_ms": precond_setup_ms,
                   "first_solve_ms": first_ms,
                   "setup_plus_solve_ms": setup_ms + (precond_setup_ms or 0.0) + ms_per_step,
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (no flush)",
                   "grid_ctas": infos[0][2]["grid_ctas"], "loop_mode": args.loop_mode},
        "iter_us": loop["iter_us"],
        "roofline": roofline,
        "loop": loop,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
        "spmv": spmv,
    }


def spmv_compare(h, A, rp, ci, va, xs, torch, cg, peak):
    """cg_spmv against cuSPARSE's CSR SpMV (through torch's sparse CSR tensor), both
    timed into preallocated outputs, on the same byte model."""
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        At = torch.sparse_csr_tensor(rp, ci, va, size=(A.n, A.n))
    y1 = torch.empty_like(xs)
    y2 = torch.empty_like(xs)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_lib = timed(lambda: cg.cg_spmv(h, xs, y1))
    how = "torch.mv(csr, x, out=y)"
    try:
        torch.mv(At, xs, out=y2)
        t_cus = timed(lambda: torch.mv(At, xs, out=y2))
    except (RuntimeError, TypeError, NotImplementedError):
        how = "At @ x (output from torch's caching allocator, no copy)"
        t_cus = timed(lambda: At @ xs)
        y2 = At @ xs
    torch.cuda.synchronize()
    agree = bool(torch.allclose(y1, y2, rtol=1e-12, atol=1e-12))
    sb = 12 * A.nnz + 4 * (A.n + 1) + 16 * A.n
    return {"libcg_ms": t_lib, "cusparse_ms": t_cus, "libcg_gbs": sb / t_lib / 1e6,
            "cusparse_gbs": sb / t_cus / 1e6, "libcg_frac": sb / t_lib / 1e6 / peak,
            "libcg_vs_cusparse": t_cus / t_lib, "bytes_model": sb, "results_agree": agree,
            "cusparse_call": how}


def run_extras(args, dev, torch, cg):
    """The other configurations of the build, each timed over a few solves in this run,
    and the speed of each faster form against plain fp64 Jacobi-PCG on the same GPU."""
    out = {}
    for w in EXTRAS:
        try:
            if WORKLOADS[w][0] == "batch":
                r = bench_batch(args, w, args.extra_steps, 3, 1, 0, dev, torch, cg, full=False)
            else:
                r = bench_single(args, w, args.extra_steps, 3, 1, 0, dev, torch, cg, full=False)
        except Exception as e:  # report and go on: the default line must still print
            out[w] = {"error": f"{type(e).__name__}: {e}"}
            continue
        c = r["config"]
        e = {"description": c["description"], "ms_per_step": r["ms_per_step"], "steps": r["steps"],
             "iters": c.get("iters", c.get("iters_max")), "relres_true_max": c["relres_true_max"],
             "tol": c["tol"], "dtype": r["dtype"], "setup_ms": c.get("setup_ms"),
             "precond_setup_ms": c.get("precond_setup_ms"), "gpu_launches": r["gpu_launches"],
             "clocks": r["clocks"]}
        if "loop" in r:
            e["loop"] = {k: r["loop"][k] for k in ("achieved_gbs", "frac", "iter_us", "loop_form",
                                                    "frac_survey_model")}
            if "ms_per_launch" in r["roofline"]:
                e["dominant_kernel"] = {k: r["roofline"].get(k) for k in ("kernel", "achieved", "frac",
                                                                          "ms_per_launch", "fp64_pipe")}
        else:
            e["roofline"] = {k: r["roofline"][k] for k in ("achieved", "frac", "frac_survey_model",
                                                            "traffic")}
            e["sequential_fp64"] = r.get("sequential_fp64")
            e["systems"] = c["systems"]
        out[w] = e
        torch.cuda.empty_cache()
    cmp = {}
    for fast, base in EXTRA_PAIRS:
        if "ms_per_step" in out.get(fast, {}) and "ms_per_step" in out.get(base, {}):
            f = out[fast]
            cmp[f"{fast}_vs_{base}"] = {
                "time_ratio": f["ms_per_step"] / out[base]["ms_per_step"],
                "time_ratio_with_setup": (f["ms_per_step"] + (f["precond_setup_ms"] or 0.0))
                / out[base]["ms_per_step"]}
    if "batch512" in out and out["batch512"].get("sequential_fp64"):
        cmp["batch512_vs_sequential_fp64"] = {
            "time_ratio": out["batch512"]["ms_per_step"] / out["batch512"]["sequential_fp64"]["ms"]}
    out["compare"] = cmp
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libcg", choices=["libcg", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle CPU time for the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-spmv-compare", action="store_true",
                    help="skip the cg_spmv vs cuSPARSE comparison")
    ap.add_argument("--no-dominant", action="store_true",
                    help="skip the stand-alone timing of the loop's SpMV kernel")
    ap.add_argument("--no-sequential", action="store_true",
                    help="batch workloads: skip the one-system-at-a-time comparison")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other configurations timed beside the default workload")
    ap.add_argument("--extra-steps", type=int, default=3)
    ap.add_argument("--loop-mode", default="auto", choices=["auto", "persistent", "graph", "unrolled", "cluster"])
    ap.add_argument("--grid", type=int, default=0, help="force the persistent grid (CTAs; 0 = automatic)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import paper_2608_09647_gb300 as cg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    if WORKLOADS[args.workload][0] == "batch":
        line = bench_batch(args, args.workload, args.steps, args.warmup, world, rank, dev, torch, cg)
    else:
        line = bench_single(args, args.workload, args.steps, args.warmup, world, rank, dev, torch, cg)
    # the other configurations: one rank, default workload only (the multi-GPU scaling
    # runs time the default workload alone)
    if world == 1 and args.workload == DEFAULT and not args.no_extra:
        line["extra"] = run_extras(args, dev, torch, cg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
