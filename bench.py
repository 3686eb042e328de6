#!/usr/bin/env python
"""Benchmark of the GB300 Top-K sparse eigensolver.

Workload (default): symmetric R-MAT graph, n = 2^24, edge factor 8 (about
268M stored non-zeros after symmetrisation), (a, b, c, d) = (0.57, 0.19, 0.19,
0.05), no self-loops, normalised adjacency D^-1/2 A D^-1/2, seed 1; top K = 24
eigenpairs with 2K = 48 Lanczos steps.  Synthetic stand-in for the paper's
SuiteSparse / GAP graphs.

One step = one complete Top-K solve (Lanczos with full reorthogonalisation,
Jacobi on T, Ritz vectors) in the chosen mixed precision FDF (binary32
values and basis, double-float arithmetic) with the delayed form of the
reorthogonalisation (two passes over the basis per step), launched as one
CUDA graph with the matrix already resident in HBM.  The plain FP64 path (DDD) and the K = 8,
m = 16 solves are timed alongside and reported as extra keys.

--impl reference times the CPU oracle (plain FP64 C) on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "top-K solve ms, SpMV GB/s vs FP64 plain at fixed error; solves/s, p99 ms"


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--scale", type=int, default=24)
    p.add_argument("--edge-factor", type=int, default=8)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--K", type=int, default=24)
    p.add_argument("--m", type=int, default=48)
    p.add_argument("--order", choices=["keep", "degree"], default="degree",
                   help="degree: the plans relabel the rows by length (longest first) so that "
                        "the SpMV's reads of the most connected columns share cache lines")
    p.add_argument("--reorth", choices=["full", "delayed"], default="delayed",
                   help="full: classical Gram-Schmidt twice per step (three passes); delayed: "
                        "the second sweep folded into the next step (two passes)")
    p.add_argument("--e2e-steps", type=int, default=3, help="0 skips the end-to-end leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the DDD and K=8 timings")
    p.add_argument("--oracle-steps", type=int, default=2,
                   help="Lanczos steps of the oracle timed with all host cores and with one")
    p.add_argument("--no-small", action="store_true",
                   help="skip the latency leg (uniform n = 10^4, K = 8, m = 16, FP64)")
    p.add_argument("--no-fixed-error", action="store_true",
                   help="skip the fixed-error leg (planted communities, n = 2^24, K = 24, m = 48)")
    p.add_argument("--no-serving", action="store_true",
                   help="skip the serving leg (Poisson arrivals of small solves)")
    p.add_argument("--serving-requests", type=int, default=10000,
                   help="requests per arrival rate >= 1000/s (1000 at the lower rates)")
    p.add_argument("--no-ooc", action="store_true",
                   help="skip the host-streamed solve (R-MAT 2^25, edge factor 16, 4 GB budget)")
    p.add_argument("--no-sweep", action="store_true",
                   help="skip the precision sweep (R-MAT 2^22, edge factor 16, K=16, m=32)")
    p.add_argument("--spmv-order-probe", default=None,
                   choices=["degree", "keep", "rcm", "hubs32k_rcm", "hubs256k_rcm",
                            "degbucket_rcm"],
                   help="only time one FDF SpMV under this row order on the --scale / "
                        "--edge-factor / --seed R-MAT graph and exit (for the order study)")
    p.add_argument("--no-banded", action="store_true",
                   help="skip the SpMV on a banded matrix of the same size (cache-friendly gathers)")
    p.add_argument("--serving-only", default=None, metavar="RATES",
                   help="only run the serving leg at these comma-separated arrival rates "
                        "(--serving-requests requests each) and print its JSON (for profiling "
                        "the engine)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup(args):
    """Rank, world size and local rank from the launcher's environment; for
    N > 1 one process group over NCCL (one GPU per rank), or over gloo on a
    host without a GPU (the CPU reference arm, the plumbing's tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def make_inputs(args):
    import synth
    t0 = time.perf_counter()
    A = synth.rmat_sym(args.scale, args.edge_factor, args.seed)
    gen_s = time.perf_counter() - t0
    v1 = synth.start_vector(A.n, args.seed)
    return A, v1, gen_s


# DRAM bytes per SpMV step (slice kernel + cut-row finaliser) measured by ncu
# on the small case of the same kernels and layout (R-MAT scale 22, edge
# factor 8, rows by degree: 557.4 MB against 605.8 MB of algorithmic bytes,
# 0.920x; profiles/spmv_dram_fdf_rmat22_ef8.md) and scaled to this workload
# by its algorithmic bytes per step (2,442,972,024: x 4.03); valid for the
# kernel and layout sources whose SHA-256 is recorded with it
SPMV_TRAFFIC = {
    "workload": "rmat24_ef8_normadj_seed1",
    "order": "degree",
    "bytes_per_step": 2.248e9,
    "measured_on": "rmat22_ef8_normadj_seed1 (557.4 MB per step), scaled by algorithmic bytes",
    "sources": {
        "paper_2201_07498_gb300/csrc/te_spmv.cu":
            "0ddeb9b3a8d19cd98cc189d7eb2a82f624f922edd1a0ad9b13b9a3ea11ef81ea",
        "paper_2201_07498_gb300/csrc/te_common.cuh":
            "4a92b110c7810ee9286055e9629f3bb8af147b489cdb6326cff63482fe82bba1",
        "paper_2201_07498_gb300/csrc/te_layout.cu":
            "2e04e36f6ff8dddb6c1ec280a506a01b4a00e23d1e40214dc16daa4f7279106c",
        "paper_2201_07498_gb300/csrc/te_layout_dev.cu":
            "b9794931a840a978b7559adc0fdccd1090315f9189c296e3e5a4ca4dde7a83e2",
        "paper_2201_07498_gb300/csrc/te_internal.h":
            "ee27e2ed3bc30a8907acafd806e9458318e59c3f91e7fbdc16be11a9f6e74a8c",
    },
}


def spmv_traffic(workload, order):
    """The measured traffic when the SpMV sources are unchanged since the
    capture and the workload and row order match, else None."""
    import hashlib
    if not workload.startswith(SPMV_TRAFFIC["workload"]) or order != SPMV_TRAFFIC["order"]:
        return None
    for path, digest in SPMV_TRAFFIC["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return SPMV_TRAFFIC["bytes_per_step"]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle, timed on the host cores
# ---------------------------------------------------------------------------
def oracle_solve_timed(A, v1, K, m, seed, vectors=True):
    """One complete oracle solve (m Lanczos steps with MGS, Jacobi, selection
    and, with `vectors`, the K Ritz vectors), timed once: (ms, result)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.topk_eigs(A, K, m, v1, seed=seed, want_vectors=vectors)
    return (time.perf_counter() - t0) * 1e3, r


def oracle_thread_scaling(A, v1, steps, seed):
    """The oracle's first `steps` Lanczos steps on the full matrix, timed with
    every host core and with one thread (the same sample both times)."""
    import oracle
    full = oracle.num_threads()
    out = {"sample": f"the oracle's first {steps} Lanczos steps (SpMV + MGS) on the full matrix",
           "threads": full}
    try:
        for th, key in ((full, "ms_all_threads"), (1, "ms_1_thread")):
            oracle.set_num_threads(th)
            t0 = time.perf_counter()
            oracle.lanczos(A, v1, steps, seed=seed)
            out[key] = (time.perf_counter() - t0) * 1e3
    finally:
        oracle.set_num_threads(full)
    out["speedup"] = out["ms_1_thread"] / out["ms_all_threads"]
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_config(args, A):
    c = workload_config(args, A)
    c["precision"] = "FP64 oracle: binary64 values, vectors and arithmetic"
    c["reorthogonalisation"] = "modified Gram-Schmidt, one pass per step (Algorithm 1)"
    c["row_order"] = "the generator's order"
    return c


def run_reference(args, world, rank):
    """The oracle, as it stands, on the benchmark's workload: every timed step
    is one complete solve (no sampling or extrapolation); each warm-up step is
    one oracle SpMV over the whole matrix (it pages the matrix in)."""
    if rank != 0:
        return
    import oracle
    A, v1, _ = make_inputs(args)
    for _ in range(args.warmup):
        oracle.spmv(A, v1)
    times = []
    for _ in range(args.steps):
        ms, _ = oracle_solve_timed(A, v1, args.K, args.m, args.seed)
        times.append(ms)
    ms = sum(times) / len(times)
    cores = oracle.num_threads()
    sample = (f"{args.steps} complete oracle solves ({args.m} Lanczos steps with MGS, Jacobi, "
              f"{args.K} Ritz vectors) on the full matrix, each timed; median "
              f"{statistics.median(times):.0f} ms")
    out = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": oracle_config(args, A),
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def workload_config(args, A):
    return {
        "workload": f"rmat{args.scale}_ef{args.edge_factor}_normadj_seed{args.seed}"
                    f"_K{args.K}_m{args.m}",
        "n": int(A.n), "nnz": int(A.nnz), "K": args.K, "krylov_steps": args.m,
        "rmat": [0.57, 0.19, 0.19, 0.05],
        "precision": "FDF: f32 values + f32 Lanczos basis, double-float arithmetic, "
                     "f64 cross-block sums and Jacobi",
        "reorthogonalisation": ("classical Gram-Schmidt twice per step" if args.reorth == "full"
                                else "classical Gram-Schmidt twice, second sweep delayed "
                                     "into the next step"),
        "row_order": ("rows relabelled by length, longest first (the caller sees its own "
                      "order)" if args.order == "degree" else "the generator's order"),
        "l2": "no flush: inputs larger than L2 (CSR and basis are several GB each)",
        "parallelism": "replicas",
    }


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def converged_match_err(ev_test, ev_ref, res_ref, tol=1e-9):
    """Largest relative distance from each converged reference Ritz value
    (residual <= tol |theta|) to the nearest value of the tested form, and how
    many reference pairs were converged."""
    import numpy as np
    errs = []
    for th, r in zip(ev_ref, res_ref):
        if r <= tol * abs(th):
            errs.append(float(np.min(np.abs(ev_test - th)) / abs(th)))
    return (max(errs) if errs else None), len(errs)


def nearest_rel_err(ev_test, ev_ref):
    """Largest relative distance from a tested value to the nearest reference value."""
    import numpy as np
    return float(max(np.min(np.abs(ev_ref - t)) / abs(t) for t in ev_test))


def small_latency(te, world, solves=200, warmup=20, oracle_runs=20):
    """The small FP64 case: uniform-random symmetric n = 10^4 (10 draws per
    row, values uniform(0,1), A + A^T), seed 0, K = 8, m = 16, plain FP64
    (DDD), one CUDA graph per solve with the matrix resident.  Latency-bound:
    reports microseconds and kernels per solve, with the oracle timed beside
    it (median of `oracle_runs` complete solves on the host cores)."""
    import numpy as np
    import oracle
    import synth
    A = synth.uniform_sym(10_000, 10, 0)
    K, m, seed = 8, 16, 0
    plan = te.Plan(te.CSR.from_host(A, "ddd"), K, m, "ddd", seed=seed)
    ms, ev, _ = time_plan(plan, solves, warmup, world, want_vectors=True)
    ev_g, _, _ = plan.solve(vectors=False)
    kernels = plan.kernel_count + 1
    del plan
    v1 = synth.start_vector(A.n, seed)
    t_o = []
    for _ in range(oracle_runs):
        t, r = oracle_solve_timed(A, v1, K, m, seed)
        t_o.append(t)
    rel = float(np.max(np.abs(np.sort(ev_g.numpy()) - np.sort(r.eigvals))
                       / np.abs(np.sort(r.eigvals))))
    return {"workload": "uniform_n10000_10perrow_seed0_K8_m16_ddd", "n": int(A.n),
            "nnz": int(A.nnz), "us_per_solve": ms * 1e3, "solves_per_s": 1e3 / ms,
            "kernels_per_solve": kernels, "graph": True,
            "oracle_ms_median": statistics.median(t_o), "oracle_runs": oracle_runs,
            "oracle_cores": oracle.num_threads(),
            "max_rel_err_vs_oracle": rel}


def fixed_error_planted(te, world, steps, warmup):
    """Solve time at a fixed error.  Workload: the uniform background of the
    small case at n = 2^24 (8 draws per row, values uniform(0,1), A + A^T) plus
    24 planted unit cliques of sizes round(16 * 1.25^k), seed 6: 24 eigenvalues
    (about 15 to 2,700) stand out of the background's spectrum, so an m = 48
    Lanczos run converges all K = 24 of them (the community structure that
    spectral clustering, Section I, looks for).  The oracle solves it once on
    the host (binary64 values); each GPU form is timed as one CUDA graph per
    solve, and its K values are compared with the oracle's, sorted."""
    import numpy as np
    import synth
    t0 = time.perf_counter()
    A = synth.planted_sym(1 << 24, 8, 24, 16, 1.25, 6)
    gen_s = time.perf_counter() - t0
    K, m, seed = 24, 48, 6
    v1 = synth.start_vector(A.n, seed)
    ms_o, r_o = oracle_solve_timed(A, v1, K, m, seed, vectors=False)
    ev_o = np.sort(r_o.eigvals)
    conv = int(np.sum(r_o.residuals <= 1e-9 * np.abs(r_o.eigvals)))
    out = {"workload": "planted24_n16777216_8perrow_smin16_ratio1.25_seed6_K24_m48",
           "n": int(A.n), "nnz": int(A.nnz), "generate_s": gen_s, "oracle_ms": ms_o,
           "oracle_converged_pairs": conv,
           "oracle_max_rel_residual": float(np.max(r_o.residuals / np.abs(r_o.eigvals))),
           "forms": {}}
    csr64 = te.CSR.from_host(A, "ddd")
    for name, prec, refine in (("ddd", "ddd", False), ("fdf", "fdf", False),
                               ("fdf_refined", "fdf", True), ("bdf", "bdf", False)):
        plan = te.Plan(csr64, K, m, prec, seed=seed, refine=refine, reorth="delayed",
                       order="degree")
        ms, _, _ = time_plan(plan, max(3, steps // 2), warmup, world)
        ev, _, res = plan.solve(vectors=False, residuals=True)
        del plan
        ev = np.sort(ev.numpy())
        out["forms"][name] = {
            "solve_ms": ms,
            "max_rel_err_vs_oracle": float(np.max(np.abs(ev - ev_o) / np.abs(ev_o)))}
    d = out["forms"]["ddd"]["solve_ms"]
    for name, row in out["forms"].items():
        row["speedup_vs_ddd"] = d / row["solve_ms"]
    return out


def precision_sweep(te, world, steps=5, warmup=3):
    """Every supported form on R-MAT scale 22, edge factor 16, seed 2
    (normalised adjacency), K = 16, m = 32: solve time, and the error of the
    Ritz values against the plain FP64 path, without and with the binary64
    Rayleigh-quotient refinement."""
    import numpy as np
    import synth
    A = synth.rmat_sym(22, 16, 2)
    K, m, seed = 16, 32, 2
    csr = te.CSR.from_host(A, "ddd")  # binary64 values serve every form
    opts = {"reorth": "delayed", "order": "degree"}  # the benchmark's plan options
    out = {"workload": "rmat22_ef16_normadj_seed2_K16_m32", "n": int(A.n), "nnz": int(A.nnz),
           "plan_options": opts, "forms": {}}
    plan = te.Plan(csr, K, m, "ddd", seed=seed, **opts)
    ms_d, _, _ = time_plan(plan, steps, warmup, world)
    ev_d, _, res_d = plan.solve(vectors=False, residuals=True)
    ev_d, res_d = ev_d.numpy(), res_d.numpy()
    out["forms"]["ddd"] = {"solve_ms": ms_d, "spmv_value_bytes": 8,
                           "fp64_converged_pairs": int(np.sum(res_d <= 1e-9 * np.abs(ev_d)))}
    del plan
    for prec, vb in (("fdf", 4), ("bdf", 2), ("8df", 1)):
        row = {"spmv_value_bytes": vb}
        plan = te.Plan(csr, K, m, prec, seed=seed, **opts)
        row["solve_ms"], ev, _ = time_plan(plan, steps, warmup, world)
        sp = plan.profile()["spmv"]
        row["spmv_ms"] = sp[0]
        row["spmv_gbs"] = sp[2] / (sp[0] * 1e-3) / 1e9
        del plan
        row["max_rel_err_vs_fp64_converged"] = converged_match_err(ev, ev_d, res_d)[0]
        row["max_rel_err_vs_fp64_nearest"] = nearest_rel_err(ev, ev_d)
        plan = te.Plan(csr, K, m, prec, seed=seed, refine=True, **opts)
        ms_r, _, _ = time_plan(plan, steps, warmup, world)
        ev_r, _, res_r = plan.solve(vectors=False, residuals=True)
        ev_r, res_r = ev_r.numpy(), res_r.numpy()
        del plan
        row["refined"] = {
            "solve_ms": ms_r,
            "max_rel_err_vs_fp64_converged": converged_match_err(ev_r, ev_d, res_d)[0],
            "max_rel_err_vs_fp64_nearest": nearest_rel_err(ev_r, ev_d),
            "max_rel_residual": float(np.max(res_r / np.abs(ev_r))),
        }
        out["forms"][prec] = row
    return out


def spmv_banded(te, peak, peak_kind):
    """The SpMV kernel of each mixed form (binary32, bfloat16 and FP8 E4M3
    values) on a banded matrix of the benchmark's size (n = 2^24; each row
    draws 8 columns among the 1024 right of the diagonal, then A + A^T: about
    16 non-zeros per row), rows in their own order.  Its x reads stay within
    a few KB of the slice's rows and hit cache, so this measures how close
    the kernel streams to the HBM peak when random gathers do not bound it.
    Algorithmic bytes and time per SpMV from the plan's per-kernel CUDA
    events (best of three un-graphed solves)."""
    import synth
    A = synth.banded_sym(1 << 24, 8, 1024, 5)
    csr = te.CSR.from_host(A, "ddd")  # binary64 values: each plan rounds them
    out = {"workload": "banded_n16777216_8perrow_hw1024_seed5_K8_m16", "n": int(A.n),
           "nnz": int(A.nnz), "peak": peak, "peak_kind": peak_kind, "forms": {}}
    for prec, vb in (("fdf", 4), ("bdf", 2), ("8df", 1)):
        plan = te.Plan(csr, 8, 16, prec, seed=5)
        plan.solve(vectors=False)
        ms, launches, by = min(plan.profile()["spmv"] for _ in range(3))
        del plan
        gbs = by / (ms * 1e-3) / 1e9
        out["forms"][prec] = {"value_bytes": vb, "spmv_ms_per_launch": ms / launches,
                              "algorithmic_bytes_per_launch": by / launches, "gbs": gbs,
                              "frac": gbs / peak}
    return out


def h2d_probe(nbytes=1 << 30, reps=5):
    """Pinned host -> device copy bandwidth (GB/s, best of reps, CUDA events)."""
    import torch
    src = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    best = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del src, dst
    return best


def out_of_core(te, world, steps=2, warmup=1):
    """Host-streamed solve: R-MAT scale 25, edge factor 16, seed 3 (normalised
    adjacency), int32 columns + binary32 values in pinned host memory, device
    matrix budget 4 GB, binary64 vectors and arithmetic (FDD), K = 8, m = 16."""
    import synth
    t0 = time.perf_counter()
    A = synth.rmat_sym(25, 16, 3)
    gen_s = time.perf_counter() - t0
    n, nnz = int(A.n), int(A.nnz)
    # a caller whose values are binary32 already (half the pinned host memory
    # of binary64 values)
    host = te.CSR.from_host(A.with_f32_values(), "fdd", device="cpu", pin=True)
    del A
    t0 = time.perf_counter()
    plan = te.Plan(host, 8, 16, "fdd", seed=3, matrix_budget=4 << 30)
    build_s = time.perf_counter() - t0
    ms, _, _ = time_plan(plan, steps, warmup, world)
    prof = plan.profile()
    sp_ms, sp_n, sp_bytes = prof["spmv"]
    blocks = plan.stream_blocks
    del plan, host
    link = h2d_probe()
    spmv_gbs = sp_bytes / (sp_ms * 1e-3) / 1e9
    return {"workload": "rmat25_ef16_normadj_seed3_K8_m16_fdd_budget4GB", "n": n, "nnz": nnz,
            "solve_ms": ms, "stream_blocks": blocks, "spmv_ms_per_step": sp_ms / max(sp_n, 1),
            "spmv_gbs": spmv_gbs, "h2d_probe_gbs": link,
            "roofline": {"bound": "host link", "achieved": spmv_gbs, "peak": link,
                         "frac": spmv_gbs / link, "unit": "GB/s"},
            "generate_s": gen_s, "plan_build_s": build_s}


def serving(te, nreq_high, nreq_low=1000, npool=256, rates=(100, 300, 1000, 3000, 5000),
            seed=4, max_slots=64):
    """Continuous-batching serving: Poisson arrivals of solve requests drawn
    from synth's serving mix (n log-uniform in [2^10, 2^18], degree 4-64,
    uniform or R-MAT, K in {4, 8, 16}, m = 2K, binary32 or bfloat16 values;
    binary32 requests carry binary32 values, bfloat16 ones binary64 values).
    `npool` distinct matrices are generated and request i solves matrix
    i mod npool (with its own K, m, form) from its own start vector (seed i);
    `nreq_high` requests arrive at rates >= 1000/s and `nreq_low` at lower
    rates (so that a rate's arrivals span at most about ten seconds).  A client
    loop submits each request on arrival, runs engine steps and collects the
    finished requests from the completion queue (eigenvalues, and Ritz
    vectors into a pinned host buffer the client reuses).  Latency =
    completion minus scheduled arrival.  One
    server runs every rate, with the per-class layout autotuner on; a warm-up
    pass over the pool (untimed) tunes its classes first."""
    import numpy as np
    import synth
    t0 = time.perf_counter()
    # the binary32-storage requests arrive with binary32 values, the bfloat16
    # ones with binary64 values (the library rounds them)
    pool = [(A.with_f32_values() if prec == "fdf" else A, K, m, prec)
            for A, K, m, prec in synth.serving_requests(npool, seed)]
    gen_s = time.perf_counter() - t0
    nnz = [int(A.nnz) for A, _, _, _ in pool]
    out = {"workload": f"serving_mix_seed{seed}", "distinct_matrices": npool,
           "requests_per_rate": {str(r): (nreq_high if r >= 1000 else nreq_low) for r in rates},
           "mean_nnz": float(np.mean(nnz)), "generate_s": gen_s, "rates": {}}
    rng = np.random.default_rng(seed + 1)
    # one long-running server with the per-class layout autotuner; a warm-up
    # pass over the pool lets it tune every request class first
    srv = te.Server(max_slots=max_slots, max_krylov_steps=32, budget=24 << 30, autotune=True)
    # the client collects each request's Ritz vectors into one pinned buffer
    import torch
    ubuf = torch.empty(max(A.n * K for A, K, _, _ in pool), dtype=torch.float64).pin_memory()
    t0 = time.perf_counter()
    pend = set(srv.submit(A, K, m, prec, seed=i) for i, (A, K, m, prec) in enumerate(pool))
    while pend:
        srv.step()
        for t in srv.completed():
            srv.poll(t, vectors=False)
            pend.discard(t)
    out["warmup_s"] = time.perf_counter() - t0
    out["tuned_classes"] = {str(k): list(v) for k, v in srv.classes().items()}
    for rate in rates:
        nreq = nreq_high if rate >= 1000 else nreq_low
        arrive = np.cumsum(rng.exponential(1.0 / rate, nreq))
        lat, tickets, max_live, steps = [], {}, 0, 0
        host0, an0 = srv.timing(), srv.analysis()
        client = {"submit_s": 0.0, "step_s": 0.0, "collect_s": 0.0}  # the client loop's wall time
        i = 0
        start = time.perf_counter()
        while len(lat) < nreq:
            c0 = time.perf_counter()
            now = c0 - start
            while i < nreq and arrive[i] <= now:
                A, K, m, prec = pool[i % npool]
                tickets[srv.submit(A, K, m, prec, seed=i)] = arrive[i]
                i += 1
            c1 = time.perf_counter()
            client["submit_s"] += c1 - c0
            if not tickets:
                time.sleep(max(0.0, min(arrive[i] - now, 0.01)))
                continue
            live, _ = srv.step()
            c2 = time.perf_counter()
            client["step_s"] += c2 - c1
            steps += 1
            max_live = max(max_live, live)
            for t in srv.completed():
                if srv.poll(t, out=ubuf) is not None:
                    lat.append(time.perf_counter() - start - tickets.pop(t))
            client["collect_s"] += time.perf_counter() - c2
        wall = time.perf_counter() - start
        lat_ms = np.array(lat) * 1e3
        host1, an1 = srv.timing(), srv.analysis()
        an = {k: an1[k] - an0[k] for k in an1}
        out["rates"][str(rate)] = {
            "requests": nreq, "solves_per_s": nreq / (wall - arrive[0]),
            "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "engine_steps": steps,
            "max_resident": max_live, "wall_s": wall,
            "host_s": {k: host1[k] - host0[k] for k in host1},
            "mean_batch": an["resident_steps"] / max(an["engine_steps"], 1),
            "client_s": client,
            "analysis_threads_s": {k: an[k] for k in ("layout_s", "gather_s", "copy_s",
                                                      "stage_wait_s")}}
    srv.close()
    return out


def spmv_order_probe(args):
    """One FDF SpMV per launch (best of three un-graphed solves, K = 8,
    m = 16) under a row order: the plans' degree order, the generator's, or a
    locality order computed on the host (reverse Cuthill-McKee of the
    symmetric pattern, alone, after the 32 K / 256 K most connected rows, or
    inside log2-degree buckets) with the matrix relabelled before the plan
    is made."""
    import numpy as np
    import synth
    import paper_2201_07498_gb300 as te
    te.load_library(build_if_missing=True)
    A = synth.rmat_sym(args.scale, args.edge_factor, args.seed)
    n, deg, order = A.n, np.diff(A.row_ptr), args.spmv_order_probe
    if order in ("degree", "keep"):
        M, plan_order = A, order
    else:
        import scipy.sparse as sp
        from scipy.sparse.csgraph import reverse_cuthill_mckee
        G = sp.csr_matrix((np.ones(A.nnz, dtype=np.float32), A.col, A.row_ptr), shape=(n, n))
        rcm = reverse_cuthill_mckee(G, symmetric_mode=True)
        del G
        if order == "rcm":
            perm = rcm
        elif order.startswith("hubs"):
            H = 32768 if order == "hubs32k_rcm" else 262144
            hubs = np.argsort(-deg, kind="stable")[:H]
            is_hub = np.zeros(n, bool)
            is_hub[hubs] = True
            perm = np.concatenate([hubs, rcm[~is_hub[rcm]]])
        else:
            b = np.floor(np.log2(np.maximum(deg, 1))).astype(int)
            pos = np.empty(n, dtype=np.int64)
            pos[rcm] = np.arange(n)
            perm = np.lexsort((pos, -b))
        iperm = np.empty(n, dtype=np.int64)
        iperm[perm] = np.arange(n)
        rows = np.repeat(np.arange(n), deg)
        M = synth.from_triplets(n, iperm[rows].astype(np.int32), iperm[A.col].astype(np.int32),
                                A.val)
        plan_order = "keep"
    plan = te.Plan(te.CSR.from_host(M, "fdf"), 8, 16, "fdf", seed=1, order=plan_order)
    ms, launches, _ = min(plan.profile()["spmv"] for _ in range(3))
    print(json.dumps({"order": order, "scale": args.scale, "edge_factor": args.edge_factor,
                      "nnz": int(A.nnz), "spmv_ms_per_launch": ms / launches}), flush=True)


def time_plan(plan, steps, warmup, world, want_vectors=True):
    import torch
    ev = torch.empty(plan.K, dtype=torch.float64, device="cuda")
    U = torch.empty((plan.K, plan.n), dtype=torch.float64, device="cuda") if want_vectors else None
    for _ in range(warmup):
        plan.launch(ev, U)
    torch.cuda.synchronize()
    plan.status()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(steps):
        plan.launch(ev, U)
    e1.record(s)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / steps
    plan.status()
    return ms, ev.cpu().numpy(), U


def main():
    args = parse()
    if args.spmv_order_probe:
        spmv_order_probe(args)
        return
    if args.serving_only:
        import paper_2201_07498_gb300 as te
        te.load_library(build_if_missing=True)
        rates = tuple(int(r) for r in args.serving_only.split(","))
        print(json.dumps(serving(te, args.serving_requests, min(1000, args.serving_requests),
                                 rates=rates)), flush=True)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    import paper_2201_07498_gb300 as te
    torch.cuda.set_device(local)
    te.load_library(build_if_missing=True)
    A, v1, gen_s = make_inputs(args)
    K, m = args.K, args.m

    csr_f = te.CSR.from_host(A, "fdf")
    plan_f = te.Plan(csr_f, K, m, "fdf", seed=args.seed, reorth=args.reorth, order=args.order)
    kernels_per_solve = plan_f.kernel_count + 1  # + the per-solve set-up kernel

    peak, peak_kind = measured_peaks()
    clocks = ClockSampler(local)
    clocks.start()
    ms_f, ev_f, _ = time_plan(plan_f, args.steps, args.warmup, world)
    clk = clocks.stop()
    ms_f_max = max_over_ranks(ms_f, world)

    # per-kernel durations (CUDA events on the launch stream, one un-graphed solve)
    prof = plan_f.profile()
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    d_ms, d_n, d_bytes = kinds[dom]
    achieved = d_bytes / (d_ms * 1e-3) / 1e9
    sp_ms, sp_n, sp_bytes = prof["spmv"]
    spmv_gbs = sp_bytes / (sp_ms * 1e-3) / 1e9
    # the gather ceiling: random reads of a table the size of x (binary32)
    gather_rate = te.probe_gather(int(A.n))
    spmv_gather_rate = A.nnz * sp_n / (sp_ms * 1e-3)

    extras = {}
    if not args.no_extras:
        # the plain FP64 path (DDD) on the same workload
        csr_d = te.CSR.from_host(A, "ddd")
        plan_d = te.Plan(csr_d, K, m, "ddd", seed=args.seed, reorth=args.reorth,
                         order=args.order)
        ms_d, _, _ = time_plan(plan_d, max(2, args.steps // 2), args.warmup, world)
        ev_d, _, res_d = plan_d.solve(vectors=False, residuals=True)
        ev_d, res_d = ev_d.numpy(), res_d.numpy()
        prof_d = plan_d.profile()
        spd_ms, _, spd_bytes = prof_d["spmv"]
        del plan_d
        # the chosen form with the binary64 Rayleigh-quotient refinement
        csr_r = te.CSR.from_host(A, "fdf")
        plan_r = te.Plan(csr_r, K, m, "fdf", seed=args.seed, refine=True, reorth=args.reorth,
                         order=args.order)
        ms_r, _, _ = time_plan(plan_r, max(2, args.steps // 2), args.warmup, world)
        ev_r, _, res_r = plan_r.solve(vectors=False, residuals=True)
        ev_r, res_r = ev_r.numpy(), res_r.numpy()
        del plan_r, csr_r
        err_f, n_conv = converged_match_err(ev_f, ev_d, res_d)
        err_r, _ = converged_match_err(ev_r, ev_d, res_d)
        extras.update({
            "fp64_plain_solve_ms": ms_d,
            "speedup_vs_fp64_plain": ms_d / ms_f,
            "spmv_gbs": spmv_gbs,
            "spmv_gbs_fp64_plain": spd_bytes / (spd_ms * 1e-3) / 1e9,
            "fixed_error": {
                "fp64_converged_pairs": n_conv,
                "max_rel_err_fdf_vs_fp64_converged": err_f,
                "max_rel_err_fdf_refined_vs_fp64_converged": err_r,
                "fdf_refined_solve_ms": ms_r,
                "fdf_refined_speedup_vs_fp64_plain": ms_d / ms_r,
                "fdf_refined_max_rel_residual": float(np.max(res_r / np.abs(ev_r))),
                "note": "eigenvalues +-1 have huge multiplicity here; a converged FP64 pair "
                        "(residual <= 1e-9 |theta|) must appear in the mixed form's list; "
                        "the refined residual bounds each value's distance to an eigenvalue",
            },
        })
        # the layout autotuner on this matrix
        t0 = time.perf_counter()
        plan_t = te.Plan(csr_f, K, m, "fdf", seed=args.seed, autotune=True, reorth=args.reorth,
                         order=args.order)
        tune_s = time.perf_counter() - t0
        ms_t, _, _ = time_plan(plan_t, max(2, args.steps // 2), args.warmup, world)
        extras["autotune"] = {"layout_window_vmax": list(plan_t.layout), "solve_ms": ms_t,
                              "spmv_ms": plan_t.profile()["spmv"][0], "plan_create_s": tune_s,
                              "default_layout_spmv_ms": sp_ms}
        del plan_t
        Ks, ms_ = max(1, K // 3), max(2, m // 3)
        plan_fs = te.Plan(csr_f, Ks, ms_, "fdf", seed=args.seed, reorth=args.reorth,
                          order=args.order)
        ms_fs, ev_fs, _ = time_plan(plan_fs, args.steps, args.warmup, world)
        plan_ds = te.Plan(csr_d, Ks, ms_, "ddd", seed=args.seed, reorth=args.reorth,
                          order=args.order)
        ms_ds, ev_ds, _ = time_plan(plan_ds, max(2, args.steps // 2), args.warmup, world)
        extras[f"solve_ms_K{Ks}_m{ms_}"] = {
            "fdf": ms_fs, "ddd": ms_ds,
            "max_rel_err_fdf_vs_fp64": float(np.max(
                [np.min(np.abs(ev_fs - t)) / abs(t) for t in ev_ds]))}
        del plan_fs, plan_ds, csr_d
    else:
        extras["spmv_gbs"] = spmv_gbs

    # end to end through the public API: host (pinned) CSR in, host results out
    # the caller's binary64 CSR in pinned host memory: the library copies it
    # and rounds the values to binary32 inside the timed call
    host = te.CSR.from_host(A, "fdf", device="cpu", pin=True)
    h2d = sum(t.numel() * t.element_size() for t in (host.row_ptr, host.col, host.val))
    d2h = K * 8 + A.n * K * 8
    e2e_ms = []
    ev_out = torch.empty(K, dtype=torch.float64).pin_memory()
    U_out = torch.empty((K, A.n), dtype=torch.float64).pin_memory()
    for it in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s)
        te.topk_eigs(host, K, m, "fdf", seed=args.seed, reorth=args.reorth, order=args.order,
                     out=(ev_out, U_out))
        a1.record(s)
        torch.cuda.synchronize()
        if it > 0:
            e2e_ms.append(a0.elapsed_time(a1))
    e2e = max_over_ranks(statistics.median(e2e_ms), world) if e2e_ms else None

    if not args.no_small and world == 1:
        extras["small_latency"] = small_latency(te, world)
    if not args.no_fixed_error and world == 1:
        extras["fixed_error_planted"] = fixed_error_planted(te, world, args.steps, args.warmup)
    if not args.no_sweep and world == 1:
        extras["precision_sweep"] = precision_sweep(te, world)
    if not args.no_banded and world == 1:
        extras["spmv_banded"] = spmv_banded(te, peak, peak_kind)
    if not args.no_serving and world == 1:
        extras["serving"] = serving(te, args.serving_requests,
                                    min(1000, args.serving_requests))
    if not args.no_ooc and world == 1:
        extras["out_of_core"] = out_of_core(te, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ms_o, _ = oracle_solve_timed(A, v1, K, m, args.seed)
        cpu = {"value": ms_o, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"one complete oracle solve on the full workload ({m} Lanczos steps "
                         f"with MGS, Jacobi, {K} Ritz vectors), timed once, not extrapolated",
               "thread_scaling": oracle_thread_scaling(A, v1, args.oracle_steps, args.seed)}

    if rank == 0:
        out = {
            "metric": METRIC, "value": ms_f_max, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_f_max,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/df64", "data": "synthetic",
            "config": workload_config(args, A),
            "solves_per_s": 1e3 * world / ms_f_max,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (spmv_traffic(workload_config(args, A)["workload"], args.order)
                                     if dom == "spmv" else None),
                         "traffic_unit": "bytes per SpMV step (ncu, DRAM read + write)",
                         "traffic_source": SPMV_TRAFFIC["measured_on"],
                         "algorithmic_bytes_per_step": d_bytes / max(d_n, 1),
                         "gather_ceiling": {
                             "note": "the SpMV reads one scattered 4-byte x value per "
                                     "non-zero; te_probe_gather measures the GPU's rate of "
                                     "uniformly random reads from a table the size of x. "
                                     "With rows relabelled by degree the reads of the most "
                                     "connected columns share cache lines, so the SpMV can "
                                     "exceed that rate (frac > 1)",
                             "probe_gathers_per_s": gather_rate,
                             "spmv_gathers_per_s": spmv_gather_rate,
                             "frac": spmv_gather_rate / gather_rate},
                         "peak_kind": peak_kind,
                         "launches_per_solve": d_n, "ms_per_solve": d_ms,
                         "algorithmic_bytes_per_solve": d_bytes},
            "kernels": {k: {"ms": v[0], "launches": v[1], "gbs": (v[2] / (v[0] * 1e-3) / 1e9
                                                                  if v[0] > 0 and v[2] > 0
                                                                  else None)}
                        for k, v in kinds.items()},
            "e2e": ({"value": e2e, "unit": "ms", "h2d_bytes_per_step": int(h2d),
                     "d2h_bytes_per_step": int(d2h)} if e2e is not None else None),
            "gpu_launches": int(kernels_per_solve * args.steps),
            "clocks": clk,
            "cpu_baseline": cpu,
            "generate_s": gen_s,
        }
        out.update(extras)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
