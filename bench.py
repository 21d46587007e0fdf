#!/usr/bin/env python
"""Throughput benchmark of the Strang-preconditioned BVM/GMRES solver on GB300.

Metric: space-time FDE solves/s at rel.err 1e-8.  One step = one complete solve
of the space-time system of a problem whose inputs (u0, f, d+, d-) are already
resident in HBM: bvm_assemble (Grunwald weights, symbols, right-hand side) +
strang_precond_factor (129 complex 2047 x 2047 block LUs) + pgmres_solve
(flexible GMRES(--restart, default 30) to a true FP64 relative residual of --tol).

Default workload: m=2047 interior points, s=256 time steps, alpha=1.8,
d+(x)=1+x, d-(x)=2-x, 5-step GBDF, manufactured source (exact solution
exp(-t) x^2 (1-x)^2); 524,032 unknowns.  Synthetic, seeded-free (deterministic).

The default run also reports, as extra keys of its JSON line: the plain FP64 PGMRES
on the same workload (one warm-up, --fp64-steps timed), the same solve end to end
through the C ABI from pinned host buffers (e2e), the 64-instance batched workload
(batch64) and the m=4095 precision study (precision_m4095), the stage split of an
untimed profiled pass, and cuBLAS-measured TF32 / FP32 / FP64 peaks.  The headline
runs the product path (iteration CUDA graphs); the block solves are timed by event
pairs recorded inside those graphs.  --impl reference times complete solves of the
CPU oracle.

Other configurations (--config): batch (64 uneven instances in one call), rhs (many
right-hand sides of one operator), precision (m=4095, s=128 factor precisions),
learned (warm start), bccb (S^(2) and its modified form), example41 (Tables 1-2),
timevar (the default shape with d+-(x, t) varying in time).

Multi-GPU: one process per GPU (torchrun), each solving its own instance; the
instances are independent, so there is no data-path collective (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "space-time FDE solves/s at rel.err 1e-8: mixed+batched vs plain FP64 PGMRES"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def rank_max_ms(total_ms: float, dist, device) -> float:
    """The timed region of the slowest replica: the maximum of total_ms over the ranks
    (one process per GPU, each solving its own instance; no data-path collective)."""
    if dist is None:
        return total_ms
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="tf32", choices=["fp64", "fp32", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--storage", default="bf16", choices=["fp32", "bf16"],
                    help="storage of the factor copy the block solves stream (fde_factor_storage)")
    ap.add_argument("--matvec", default="fp64", choices=["fp64", "fp32"],
                    help="precision of the Toeplitz apply in the Arnoldi products (the restart residual is FP64)")
    ap.add_argument("--relax", type=float, default=0.0,
                    help="--matvec fp32: FP32 products while the residual estimate is above this (0: always)")
    ap.add_argument("--tune", default="",
                    help="force launch shapes instead of autotuning, e.g. 'trsv=1,matvec=2,lu=1' (fde_tune_set)")
    ap.add_argument("--batch-precision", default="tf32", choices=["fp32", "tf32", "bf16", "tf32x3"],
                    help="factor precision of the batched workload")
    ap.add_argument("--m", type=int, default=2047)
    ap.add_argument("--s", type=int, default=256)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--restart", type=int, default=30,
                    help="GMRES restart length of the benchmark legs (the paper's Tables 1-2 use 20; the example41 "
                         "and bccb configurations keep 20)")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="plain FP64 solves timed for comparison, after one FP64 warm-up solve (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="untimed solves with the full stage profiler after the timed region (stage split)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (64 instances) and precision (m=4095) legs of the default run")
    ap.add_argument("--reference-budget", type=float, default=150.0,
                    help="--impl reference: seconds of complete oracle solves (at least one solve)")
    ap.add_argument("--oracle-single-thread", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--single-its", type=int, default=20, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--config", choices=["scale", "batch", "learned", "precision", "bccb", "example41", "rhs", "timevar"],
                    default="scale",
                    help="scale: one m=2047/s=256 instance per step; batch: 64 uneven instances per step; "
                         "learned: train the warm-start operator on m=1023/s=256 solves, then compare guesses; "
                         "precision: m=4095/s=128, alpha=1.9, every preconditioner precision; "
                         "bccb: the scale workload with the Strang-type BCCB preconditioners; "
                         "example41: every row of Tables 1-2 with the columns I, S, S^(2), S~^(2); "
                         "rhs: --rhs right-hand sides of the scale operator sharing one factorisation")
    ap.add_argument("--rhs", type=int, default=16, help="rhs: number of right-hand sides")
    ap.add_argument("--block-solver", default="auto", choices=["auto", "cuda_cores", "tensor_cores"],
                    help="rhs: block solves of the shared operator")
    ap.add_argument("--train", type=int, default=4096, help="learned: method-generated training solves")
    ap.add_argument("--epochs", type=int, default=40, help="learned: passes over the training set")
    ap.add_argument("--eval", type=int, default=32, help="learned: held-out instances")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), \
            "measured"
    except OSError:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def lu_update_flops(mp: int, nblk: int, nb: int = 32) -> float:
    """Algorithmic FP flops of the trailing complex updates: sum_p 8 NB rem_p^2 per block."""
    tot = 0.0
    p = 0
    while (p + 1) * nb < mp:
        rem = mp - (p + 1) * nb
        tot += 8.0 * nb * rem * rem
        p += 1
    return tot * nblk


def tc_update_flops(mp: int, nblk: int, tb: int = 128) -> float:
    """Algorithmic flops of the rank-128 tensor-core updates: sum_o 8 TB R_o^2 per block, R_o = mp - o - TB."""
    tot = 0.0
    o = 0
    while o + tb < mp:
        r = mp - o - tb
        tot += 8.0 * tb * r * r
        o += tb
    return tot * nblk


def tc_update_bytes(mp: int, nblk: int, tb: int = 128) -> float:
    """Algorithmic HBM bytes of the same updates: each trailing C entry (Re, Im FP32) read and written once."""
    tot = 0.0
    o = 0
    while o + tb < mp:
        r = mp - o - tb
        tot += 16.0 * r * r
        o += tb
    return tot * nblk


def matvec_flops(m: int, s: int, L: int, mu: int) -> float:
    """Algorithmic FP64 flops of one space-time matvec launch (s time rows).  Per row:
    the real-input forward FFT as a length-L/2 complex FFT (radix-4 passes of L/8
    butterflies at 34 flops, one radix-2 pass of L/4 at 4 flops when log2(L/2) is
    odd), the split and symbol product (30 flops per output), the length-L inverse
    radix-4 FFT, the (mu+1)-tap band (4 flops per tap and point) and the output
    combination (8 flops per point)."""
    import math
    n = L // 2
    ln = int(math.log2(n))
    fwd = (ln // 2) * (n // 4) * 34 + (ln % 2) * (n // 2) * 4
    lL = int(math.log2(L))
    inv = (lL // 2) * (L // 4) * 34 + (lL % 2) * (L // 2) * 4
    return float(s) * (fwd + 30 * n + inv + 4 * (mu + 1) * m + 8 * m)


FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64 (no measured FP64 figure in MEASURED_PEAKS.json)
# DRAM bytes / algorithmic bytes of block_trsv_kernel<float> (ncu, m=1023, s=256), by the
# element size of the factor copy it streams (4: FP32, 2: bfloat16)
TRSV_TRAFFIC_RATIO = {4: 1.034, 2: 1.098}


def trsv_bytes(mp: int, nblk: int, esz: int, fac_esz: int | None = None) -> float:
    """Algorithmic bytes of one block-substitution launch: every factor entry once
    (L below, U on/above the diagonal; Re and Im planes; fac_esz bytes each, the
    stored copy's element) + the RHS in and out (esz per real part)."""
    return nblk * (2.0 * mp * mp * (fac_esz or esz) + 4.0 * mp * esz)


def path_roofline(m: int, s: int, mp: int, esz: int, its: int, precision: str, bf16_peak: float,
                  hbm_peak: float, ms_measured: float, restart: int = 20, tf32_peak: float | None = None,
                  fp64_peak: float | None = None, fac_esz: int | None = None) -> dict:
    """Whole-path roofline of one solve: the time it would take at the roofs over the
    measured time.  The block LUs' (s/2+1)(8/3)m^3 real flops at the factor
    precision's peak, plus, per iteration at Arnoldi step j, the factor stream
    (trsv_bytes) and (4 + 4(j+1)) n FP64 vector reads and writes at the HBM peak."""
    nblk = s // 2 + 1
    n = m * s
    setup_flops = nblk * (8.0 / 3.0) * float(m) ** 3
    tf32 = tf32_peak if tf32_peak else bf16_peak * 1.1 / 2.25
    setup_peak = {"tf32": tf32, "tf32x3": tf32, "bf16": bf16_peak,
                  "fp32": FP32_ALU_PEAK_TFLOPS, "fp64": fp64_peak if fp64_peak else FP64_PEAK_TFLOPS}[precision]
    iter_bytes = sum(trsv_bytes(mp, nblk, esz, fac_esz) + (4 + 4 * (i % restart + 1)) * 8.0 * n for i in range(its))
    roof_ms = setup_flops / (setup_peak * 1e12) * 1e3 + iter_bytes / (hbm_peak * 1e9) * 1e3
    return {"setup_flops": setup_flops, "setup_peak_tflops": setup_peak, "iteration_bytes": iter_bytes,
            "iterations": its, "ms_at_roofs": roof_ms, "ms_measured": ms_measured, "frac": roof_ms / ms_measured}


# ---------------------------------------------------------------------------
# the CPU oracle: bounded sample (cpu_baseline) and complete solves (--impl reference)
# ---------------------------------------------------------------------------

def oracle_cores() -> int:
    """Threads the oracle's BLAS/LAPACK use (threadpoolctl where installed, else the
    environment's OpenBLAS/OMP setting, else the host's core count)."""
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
            if os.environ.get(k, "").isdigit():
                return int(os.environ[k])
        return os.cpu_count() or 1


def oracle_sample(prob, iterations: int, its_source: str) -> dict:
    """Time the FP64 oracle on a bounded sample of one solve and compose the time of
    a full solve from it (a complete oracle solve of the benchmark workload takes
    about a minute of host time; the reference arm times complete solves).

    Sample, on the full workload: the right-hand side, the dense LUs of all s/2+1
    Strang blocks, and the work of one FGMRES iteration (one preconditioner apply,
    one matvec, classical Gram-Schmidt with re-orthogonalisation against the mean
    basis size of GMRES(20), 10 vectors).  Composition:
    t = t_rhs + t_factor + its * t_iteration, its = `iterations` (`its_source` says
    where that count comes from)."""
    import numpy as np

    import oracle as O

    s, m = prob.s, prob.m
    t0 = time.perf_counter()
    J = O.j_of(prob)
    O.reduced_rhs(prob, J=J)
    t_rhs = time.perf_counter() - t0
    AB = O.bvm_matrices(prob.family, prob.mu, s)
    t0 = time.perf_counter()
    P = O.StrangPreconditioner(prob, J=J)
    t_fac = time.perf_counter() - t0
    nblk = len(P.lu)
    V = np.random.default_rng(2).standard_normal((11, prob.n))
    t0 = time.perf_counter()
    z = P.apply(V[0])
    w = O.matvec(prob, z, J=J, AB=AB)
    for _ in range(2):  # CGS2: two passes of dots and updates against 10 vectors
        h = V[:10] @ w
        w = w - V[:10].T @ h
    float(np.linalg.norm(w))
    t_it = time.perf_counter() - t0
    del P
    t_solve = t_rhs + t_fac + iterations * t_it
    sampled = t_rhs + t_fac + t_it
    return {
        "value": 1.0 / t_solve, "unit": "solves/s", "cores": oracle_cores(), "kind": "oracle", "composed": True,
        "sample": (f"m={m}, s={s}: right-hand side ({t_rhs:.2f} s), dense LUs of all {nblk} Strang blocks "
                   f"({t_fac:.1f} s) and one FGMRES iteration ({t_it:.2f} s: preconditioner apply, matvec, CGS2 "
                   f"against 10 vectors), composed to {iterations} iterations ({its_source}); {sampled:.1f} s of "
                   f"CPU work"),
        "seconds_per_solve": t_solve,
    }


def oracle_complete_solve(prob, tol: float, restart: int) -> dict:
    """One complete solve by the oracle as it stands: right-hand side, the Strang
    preconditioner (dense DFT along time, one LAPACK LU per frequency block), and its
    right-preconditioned FGMRES(restart) to a true relative residual of tol (the steps
    of oracle.solve_strang_gmres, timed one by one)."""
    import oracle as O

    t0 = time.perf_counter()
    J = O.j_of(prob)
    AB = O.bvm_matrices(prob.family, prob.mu, prob.s)
    b = O.reduced_rhs(prob, J=J)
    t1 = time.perf_counter()
    P = O.StrangPreconditioner(prob, J=J)
    t2 = time.perf_counter()
    _, its, ok, _ = O.gmres(lambda z: O.matvec(prob, z, J=J, AB=AB), b, precond=P.apply, side="right",
                            restart=restart, tol=tol, maxit=400, reference="b")
    t3 = time.perf_counter()
    return {"seconds": t3 - t0, "rhs_s": t1 - t0, "factor_s": t2 - t1, "fgmres_s": t3 - t2, "iterations": its,
            "converged": bool(ok), "blocks": len(P.lu)}


def oracle_single_thread_sample(prob, iterations: int) -> dict:
    """Single-thread oracle (run in a child process with one BLAS thread): the right-
    hand side and one matvec, DFT pair and Gram-Schmidt at full size, ONE dense block
    LU and ONE block solve, composed to a full solve: t_rhs + nblk t_lu +
    its (s t_blocksolve + t_rest)."""
    import numpy as np
    import scipy.linalg as sla

    import oracle as O

    s, m = prob.s, prob.m
    t0 = time.perf_counter()
    J = O.j_of(prob)
    O.reduced_rhs(prob, J=J)
    t_rhs = time.perf_counter() - t0
    AB = O.bvm_matrices(prob.family, prob.mu, s)
    phi, psi = O.strang_symbols(prob.family, prob.mu, s)
    k = s // 4
    Bk = phi[k] * np.eye(m) - prob.h * psi[k] * J
    t0 = time.perf_counter()
    lu = sla.lu_factor(Bk, check_finite=False)
    t_lu = time.perf_counter() - t0
    r = np.random.default_rng(3).standard_normal(m) + 0j
    t0 = time.perf_counter()
    sla.lu_solve(lu, r, check_finite=False)
    t_bs = time.perf_counter() - t0
    V = np.random.default_rng(2).standard_normal((11, prob.n))
    n_ = np.arange(s)
    F = np.exp(-2j * np.pi * np.outer(n_, n_) / s)
    t0 = time.perf_counter()
    R = F @ V[0].reshape(s, m)
    z = (np.conj(F) @ R).real.reshape(-1) / s
    w = O.matvec(prob, z, J=J, AB=AB)
    for _ in range(2):
        h = V[:10] @ w
        w = w - V[:10].T @ h
    t_rest = time.perf_counter() - t0
    nblk = s // 2 + 1
    t_solve = t_rhs + nblk * t_lu + iterations * (s * t_bs + t_rest)
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "composed": True,
            "sample": (f"one thread: right-hand side {t_rhs:.2f} s, one {m}x{m} complex block LU {t_lu:.2f} s "
                       f"(x {nblk}), one block solve {t_bs * 1e3:.1f} ms (x {s} per iteration), DFT pair + matvec "
                       f"+ CGS2 {t_rest:.2f} s per iteration; composed to {iterations} iterations")}


def bench_reference(args, rank, prob, workload):
    """--impl reference: the CPU oracle (no GPU) timed on COMPLETE solves of the
    workload, as many as fit in --reference-budget seconds (at least one, at most
    --steps); `steps` is the number of complete solves timed.  A complete solve takes
    about a minute, so --warmup is not run (the oracle has no warm-up effects beyond
    the first numpy import, done before the clock starts)."""
    if rank != 0:
        return
    import numpy  # noqa: F401  (import cost outside the timed solves)
    solves = []
    t_start = time.perf_counter()
    while True:
        r = oracle_complete_solve(prob, args.tol, args.restart)
        solves.append(r)
        elapsed = time.perf_counter() - t_start
        if len(solves) >= max(1, args.steps) or elapsed + r["seconds"] > args.reference_budget:
            break
    total = sum(r["seconds"] for r in solves)
    t = total / len(solves)
    v = 1.0 / t
    cores = oracle_cores()
    single = None
    try:  # the single-thread leg, in a child process with one BLAS thread
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-single-thread",
                              "--m", str(args.m), "--s", str(args.s), "--single-its", str(solves[-1]["iterations"])],
                             env=env, capture_output=True, text=True, timeout=600)
        single = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, never fatal
        single = {"unavailable": f"{type(e).__name__}: {e}"}
    stage = {k: round(sum(r[k] for r in solves) / len(solves), 3) for k in ("rhs_s", "factor_s", "fgmres_s")}
    sample = (f"{len(solves)} complete oracle solve(s) of the workload (m={prob.m}, s={prob.s}): right-hand side, "
              f"dense LAPACK LUs of all {solves[-1]['blocks']} Strang blocks, FGMRES({args.restart}) to a true residual of "
              f"{args.tol:g} ({solves[-1]['iterations']} iterations); mean wall per stage {stage}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": len(solves), "warmup": 0, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload,
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "composed": False},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_iterations": [r["iterations"] for r in solves],
            "oracle_converged": all(r["converged"] for r in solves),
            "oracle_stage_seconds": stage, "single_thread": single,
            "note": (f"--steps {args.steps} / --warmup {args.warmup} requested; a complete oracle solve takes "
                     f"{t:.0f} s, so the arm times complete solves for at most {args.reference_budget:.0f} s "
                     f"(steps = solves timed) and runs no warm-up")}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# batched workload: 64 independent instances per step
# ---------------------------------------------------------------------------

def measure_batch(args, steps: int, warmup: int, sequential: bool = True, sample_clocks: bool = False,
                  local_rank: int = 0) -> dict:
    """The 64-instance batched workload (fde_inputs.config_batch): one step = assemble +
    factor + solve of all instances in one fde_batch_* call sequence, inputs resident in
    HBM.  Optionally the same instances one at a time through the single-problem API."""
    import numpy as np
    import torch

    import fde_inputs
    import paper_1305_6653_gb300 as fde

    probs = fde_inputs.config_batch()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    outs = [torch.empty(p.n, dtype=torch.float64, device="cuda") for p in probs]
    b = fde.FDEBatch(probs, device_inputs=True)

    def step():
        b.assemble().factor(args.batch_precision, storage=args.storage)
        _, st = b.solve(tol=args.tol, restart=args.restart, maxit=400, outs=outs)
        return st

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    if sample_clocks:
        sampler.start()
    l0 = fde.fde_launch_count()
    times, stats = [], None
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        stats = step()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = fde.fde_launch_count() - l0
    clocks = sampler.stop() if sample_clocks else None
    b.close()
    ms = sum(times) / len(times)
    out = {"value": len(probs) / (ms / 1e3), "unit": "solves/s", "instances": len(probs), "steps": steps,
           "warmup": warmup, "ms_per_step": ms, "per_step_ms": times, "precision": args.batch_precision,
           "factor_storage": args.storage,
           "tol_true_residual": args.tol, "gpu_launches": launches, "clocks": clocks,
           "iterations": [s_["iterations"] for s_ in stats],
           "unknowns_total": int(sum(p.n for p in probs))}
    if sequential:  # the same 64 instances one at a time through the single-problem API
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for pr, o in zip(probs, outs):
            with fde.FDEProblem.from_inputs(pr, device_inputs=True) as p:
                p.assemble().factor(args.batch_precision, storage=args.storage)
                p.solve(tol=args.tol, restart=args.restart, maxit=400, out=o)
        e1.record()
        e1.synchronize()
        seq_s = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0)
        out["sequential_single_api"] = {"value": len(probs) / seq_s, "unit": "solves/s", "seconds": seq_s}
    import oracle as O
    worst = 0.0
    for pr, o in zip(probs, outs):
        xs = o.cpu().numpy()
        bb = O.reduced_rhs(pr)
        worst = max(worst, float(np.linalg.norm(bb - O.matvec(pr, xs)) / np.linalg.norm(bb)))
    out["worst_rel_residual_oracle_matvec"] = worst
    return out


def bench_batch(args, world, rank, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    r = measure_batch(args, args.steps, args.warmup, sequential=True, sample_clocks=not args.no_clocks,
                      local_rank=local_rank)
    if rank == 0:
        line = {"metric": METRIC, "value": world * r["value"], "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": "batch64_m255-2047_s64-256_etr3_gbdf3_gam4", "instances": r["instances"],
                           "unknowns_total": r["unknowns_total"], "precision": args.batch_precision,
                           "factor_storage": args.storage,
                           "tol_true_residual": args.tol, "restart": args.restart,
                           "l2": "flushed (512 MiB write) before every timed step"},
                "roofline": None, "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
                "iterations": r["iterations"], "sequential_single_api": r["sequential_single_api"],
                "worst_rel_residual_oracle_matvec": r["worst_rel_residual_oracle_matvec"],
                "per_step_ms": r["per_step_ms"]}
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# many right-hand sides of the benchmark operator: one factorisation, shared block solves
# ---------------------------------------------------------------------------

def bench_many_rhs(args, world, rank, local_rank):
    import numpy as np
    import torch

    import fde_inputs
    import paper_1305_6653_gb300 as fde

    torch.cuda.set_device(local_rank)
    count = args.rhs
    probs = fde_inputs.config_many_rhs(count=count, m=args.m, s=args.s)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    outs = [torch.empty(p.n, dtype=torch.float64, device="cuda") for p in probs]

    def timed(solver, steps, warmup, sample_clocks):
        b = fde.FDEBatch(probs, device_inputs=True).share_operator().block_solver(solver)

        def step():
            b.assemble().factor(args.precision)
            _, st = b.solve(tol=args.tol, restart=args.restart, maxit=400, outs=outs)
            return st

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        sampler = ClockSampler(local_rank)
        if sample_clocks:
            sampler.start()
        l0 = fde.fde_launch_count()
        times, stats = [], None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            stats = step()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        launches = fde.fde_launch_count() - l0
        clocks = sampler.stop() if sample_clocks else None
        b.close()
        return sum(times) / len(times), stats, launches, clocks

    ms, stats, launches, clocks = timed(args.block_solver, args.steps, args.warmup, not args.no_clocks)
    value = world * count / (ms / 1e3)
    other = {}
    for solver in ("cuda_cores", "tensor_cores"):  # the block solvers side by side (a short run each)
        if solver == args.block_solver:
            continue
        try:
            oms, ost, _, _ = timed(solver, min(args.steps, 2), 1, False)
            other[solver] = {"value": world * count / (oms / 1e3), "unit": "solves/s", "ms_per_step": oms,
                             "iterations": [st["iterations"] for st in ost]}
        except fde.FdeError as e:
            other[solver] = {"unavailable": str(e)}
    # the same right-hand sides one at a time through the single-problem API (own factors each)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for pr, out in zip(probs, outs):
        with fde.FDEProblem.from_inputs(pr, device_inputs=True) as p:
            p.assemble().factor(args.precision)
            p.solve(tol=args.tol, restart=args.restart, maxit=400, out=out)
    e1.record()
    e1.synchronize()
    seq_s = e0.elapsed_time(e1) / 1e3
    import oracle as O
    J = O.j_of(probs[0])
    AB = O.bvm_matrices(probs[0].family, probs[0].mu, probs[0].s)
    worst = 0.0
    for pr, out in zip(probs[:4], outs[:4]):  # bounded host check
        xs = out.cpu().numpy()
        bb = O.reduced_rhs(pr, J=J)
        worst = max(worst, float(np.linalg.norm(bb - O.matvec(pr, xs, J=J, AB=AB)) / np.linalg.norm(bb)))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": f"many_rhs{count}_m{args.m}_s{args.s}_gbdf5_alpha1.8_variable_d",
                           "right_hand_sides": count, "m": args.m, "s": args.s, "precision": args.precision,
                           "block_solver": args.block_solver,
                           "tol_true_residual": args.tol, "restart": args.restart,
                           "l2": "flushed (512 MiB write) before every timed step; factors (4.3 GB) exceed L2"},
                "roofline": None, "gpu_launches": launches, "clocks": clocks,
                "iterations": [st["iterations"] for st in stats],
                "sequential_single_api": {"value": count / seq_s, "unit": "solves/s", "seconds": seq_s},
                "other_block_solvers": other,
                "worst_rel_residual_oracle_matvec_first4": worst}
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# precision study: one m=4095/s=128 instance, every preconditioner precision
# ---------------------------------------------------------------------------

def measure_precision(args, steps: int, warmup: int, precisions=("fp64", "fp32", "tf32", "tf32x3", "bf16"),
                      sample_clocks: bool = False, local_rank: int = 0) -> dict:
    """The precision study: one m=4095, s=128, alpha=1.9, GBDF3 instance, solved to a true
    residual of 1e-8 (the tolerance it is specified at) with each factor precision; one
    step = assemble + factor + solve.  TF32 and BF16 factors do not precondition it
    (kappa(B_k) u >> 1): they are run to maxit = 100 and reported as not converged."""
    import numpy as np
    import torch

    import fde_inputs
    import paper_1305_6653_gb300 as fde

    prob = fde_inputs.config_precision()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    xbuf = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    p = fde.FDEProblem.from_inputs(prob, device_inputs=True)
    tol = 1e-8

    def step(precision):
        p.assemble().factor(precision)
        _, st = p.solve(tol=tol, restart=args.restart, maxit=100, out=xbuf, raise_on_error=False)
        return st

    variants, sols = {}, {}
    l0 = fde.fde_launch_count()
    sampler = ClockSampler(local_rank)
    if sample_clocks:
        sampler.start()
    for prec in precisions:
        for _ in range(warmup):
            step(prec)
        times, st = [], None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            st = step(prec)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = sum(times) / len(times)
        sols[prec] = xbuf.cpu().numpy()
        variants[prec] = {"solves_per_s": 1e3 / ms, "ms_per_step": ms, "steps": steps, "warmup": warmup,
                          "iterations": st["iterations"], "rel_residual": st["rel_residual"],
                          "converged": st["status"] == 0}
    clocks = sampler.stop() if sample_clocks else None
    launches = fde.fde_launch_count() - l0
    p.close()
    if "fp64" in sols:
        ref = sols["fp64"]
        for prec, v in variants.items():
            v["rel_diff_vs_gpu_fp64"] = float(np.linalg.norm(sols[prec] - ref) / np.linalg.norm(ref))
    conv = [k for k, v in variants.items() if v["converged"]]
    best = max(conv, key=lambda k: variants[k]["solves_per_s"]) if conv else None
    return {"workload": f"precision_m{prob.m}_s{prob.s}_gbdf3_alpha1.9", "m": prob.m, "s": prob.s,
            "unknowns": prob.n, "tol_true_residual": tol, "variants": variants, "fastest_converged": best,
            "gpu_launches": launches, "clocks": clocks,
            "note": "rel_diff_vs_gpu_fp64 compares with the FP64 GPU solve of the same run; the error of every "
                    "variant against the CPU oracle is checked by tests/test_gpu_precision.py"}


def bench_precision(args, world, rank, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    r = measure_precision(args, args.steps, args.warmup, sample_clocks=not args.no_clocks, local_rank=local_rank)
    best = r["fastest_converged"] or "fp64"
    head = r["variants"][best]
    if rank == 0:
        line = {"metric": METRIC, "value": world * head["solves_per_s"], "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": r["workload"], "m": r["m"], "s": r["s"], "unknowns": r["unknowns"],
                           "precision": best, "tol_true_residual": r["tol_true_residual"], "restart": args.restart,
                           "l2": "flushed (512 MiB write) before every timed step"},
                "roofline": None, "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
                "variants": r["variants"], "note": r["note"]}
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# Strang-type BCCB preconditioners S^(2) / S~^(2) on the benchmark workload
# ---------------------------------------------------------------------------

def bench_timevar(args, world, rank, local_rank):
    """Time-dependent coefficients d+-(x, t) (eq. (1.1) allows them): the default
    workload's shape (m=2047, s=256, alpha=1.8, 5-step GBDF) with
    d+(x,t) = (1+x)(1 + sin(pi t)/2), d-(x,t) = (2-x)(1 + t/2).  The matvec applies
    J(t_n) on every time level; the block-circulant preconditioner uses the
    time-averaged J.  The oracle's time-level matvec checks the last solution."""
    import numpy as np
    import torch

    import fde_inputs
    import oracle as O
    import paper_1305_6653_gb300 as fde

    torch.cuda.set_device(local_rank)
    prob = fde_inputs.manufactured_time_varying(args.m, args.s, 1.8, "GBDF5", name=f"timevar_m{args.m}_s{args.s}")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    xbuf = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    p = fde.FDEProblem.from_inputs(prob, device_inputs=True)

    def step():
        p.assemble().factor(args.precision)
        _, st = p.solve(tol=args.tol, restart=args.restart, maxit=400, out=xbuf)
        return st

    for _ in range(args.warmup):
        step()
    l0 = fde.fde_launch_count()
    sampler = ClockSampler(local_rank)
    if not args.no_clocks:
        sampler.start()
    p.profile(True)
    times, stats = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        stats.append(step())
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    prof = p.profile_read()
    p.profile(False)
    clocks = sampler.stop() if not args.no_clocks else None
    launches = fde.fde_launch_count() - l0
    p.close()
    ms = rank_max_ms(sum(times), None, "cuda") / args.steps
    mp = (prob.m + 63) // 64 * 64
    nblk = prob.s // 2 + 1
    esz = 8 if args.precision == "fp64" else 4
    roof = None
    if prof.get("trsv", (0, 0))[1] > 0:
        tms, tn = prof["trsv"]
        per_launch = trsv_bytes(mp, nblk, esz)
        ach = per_launch / (tms / tn / 1e3) / 1e9
        hbm_peak, _, _, peak_kind = peaks()
        roof = {"kernel": "block_trsv_kernel", "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": TRSV_TRAFFIC_RATIO[4] * per_launch if esz == 4 else None,
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": per_launch,
                "traffic_source": "ncu capture at m=1023, s=256 scaled by the factor bytes" if esz == 4 else None}
    xs = xbuf.cpu().numpy()
    bor = O.reduced_rhs(prob)
    res_oracle = float(np.linalg.norm(bor - O.matvec(prob, xs)) / np.linalg.norm(bor))
    if rank == 0:
        line = {"metric": METRIC, "value": world * 1e3 / ms, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if args.precision != "fp64" else "f64", "data": "synthetic",
                "config": {"workload": f"timevar_m{prob.m}_s{prob.s}_gbdf5_alpha1.8_d_of_x_t", "m": prob.m,
                           "s": prob.s, "unknowns": prob.n, "scheme": "GBDF5", "alpha": 1.8,
                           "d": "d+=(1+x)(1+sin(pi t)/2), d-=(2-x)(1+t/2)", "precision": args.precision,
                           "tol_true_residual": args.tol, "restart": args.restart,
                           "l2": "flushed (512 MiB write) before every timed step; factors exceed L2"},
                "roofline": roof, "gpu_launches": launches, "clocks": clocks,
                "iterations": [s["iterations"] for s in stats], "rel_residual": stats[-1]["rel_residual"],
                "rel_residual_oracle_matvec": res_oracle,
                "stage_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items()},
                "stage_launches_per_step": {k: v[1] // args.steps for k, v in prof.items()}}
        print(json.dumps(line))


def bench_bccb(args, world, rank, local_rank):
    import numpy as np
    import torch

    import fde_inputs
    import paper_1305_6653_gb300 as fde

    torch.cuda.set_device(local_rank)
    prob = fde_inputs.config_scale(args.m, args.s)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    xbuf = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    p = fde.FDEProblem.from_inputs(prob, device_inputs=True)
    bprec = "fp32" if args.precision in ("fp32", "tf32", "bf16", "tf32x3") else "fp64"

    def step(modified):
        p.assemble().bccb(modified=modified, precision=bprec)
        _, st = p.solve(tol=args.tol, restart=20, maxit=20000, out=xbuf, raise_on_error=False)
        return st

    variants = {}
    l0 = fde.fde_launch_count()
    sampler = ClockSampler(local_rank)
    if not args.no_clocks:
        sampler.start()
    mv_ms, mv_launches = 0.0, 0
    for name, modified in (("S2", False), ("S2_modified", True)):
        for _ in range(args.warmup):
            step(modified)
        times, st = [], None
        p.profile(True)
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            st = step(modified)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        prof = p.profile_read()
        p.profile(False)
        ms = sum(times) / len(times)
        stages = {k: v[0] / args.steps for k, v in prof.items() if v[1]}
        variants[name] = {"solves_per_s": 1e3 / ms, "ms_per_step": ms, "iterations": st["iterations"],
                          "rel_residual": st["rel_residual"], "converged": st["status"] == 0,
                          "stage_ms_per_step": stages}
        if name == "S2":
            mv_ms, mv_launches = prof["matvec"]
    clocks = sampler.stop() if not args.no_clocks else None
    launches = fde.fde_launch_count() - l0
    p.close()
    conv = [k for k, v in variants.items() if v["converged"]]
    best = max(conv, key=lambda k: variants[k]["solves_per_s"]) if conv else "S2"
    head = variants[best]
    flops = matvec_flops(prob.m, prob.s, 1 << (2 * prob.m - 1).bit_length(), prob.mu)
    per_launch_s = mv_ms / max(mv_launches, 1) / 1e3
    achieved = flops / per_launch_s / 1e12 if per_launch_s > 0 else None
    roof = {"kernel": "st_matvec_kernel", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
            "peak_kind": "nominal FP64 (152 SMs x 2 FP64 FMA per clock x 2.07 GHz)",
            "algorithmic_flops_per_launch": flops}
    if rank == 0:
        line = {"metric": METRIC, "value": world * head["solves_per_s"], "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if bprec == "fp64" else "f32+f64", "data": "synthetic",
                "config": {"workload": f"bccb_scale_m{prob.m}_s{prob.s}_gbdf5_alpha1.8_variable_d", "m": prob.m,
                           "s": prob.s, "unknowns": prob.n, "preconditioner": best, "apply_precision": bprec,
                           "tol_true_residual": args.tol, "restart": 20,
                           "l2": "flushed (512 MiB write) before every timed step"},
                "roofline": roof, "gpu_launches": launches, "clocks": clocks, "variants": variants}
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# Example 4.1 (Sec. 4, Tables 1-2): every row with the columns I, S, S^(2), S~^(2)
# ---------------------------------------------------------------------------

def bench_example41(args, world, rank, local_rank):
    import os

    import torch

    import fde_inputs
    import paper_1305_6653_gb300 as fde

    torch.cuda.set_device(local_rank)
    golden = {}
    for fn, cols in (("paper_tables_its.txt", ("I", "S")), ("paper_tables_bccb_its.txt", ("S2", "S2_modified"))):
        for line in open(os.path.join(ROOT, "tests", "golden", fn)):
            if line.strip() and not line.startswith("#"):
                a, n, s_, c1, c2 = line.split()
                golden.setdefault((float(a), int(n), int(s_)), {}).update({cols[0]: int(c1), cols[1]: int(c2)})
    setups = {"I": lambda p: p.no_precond(), "S": lambda p: p.factor("fp64"), "S2": lambda p: p.bccb(),
              "S2_modified": lambda p: p.bccb(modified=True)}
    rows, total_ms, nsolves = [], 0.0, 0
    l0 = fde.fde_launch_count()
    sampler = ClockSampler(local_rank)
    if not args.no_clocks:
        sampler.start()
    for (alpha, n, s_), paper in sorted(golden.items()):
        prob = fde_inputs.example_4_1(alpha, n, s_)
        xbuf = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        row = {"alpha": alpha, "n": n, "s": s_}
        with fde.FDEProblem.from_inputs(prob, device_inputs=True) as p:
            for name, setup in setups.items():
                def step():
                    setup(p.assemble())
                    return p.solve(tol=1e-8, restart=20, maxit=5000, out=xbuf, raise_on_error=False)[1]
                for _ in range(args.warmup):
                    step()
                times, st = [], None
                for _ in range(args.steps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    st = step()
                    e1.record()
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = sum(times) / len(times)
                total_ms += ms
                nsolves += 1
                row[name] = {"its": st["iterations"], "paper_its": paper[name], "ms": ms,
                             "converged": st["status"] == 0}
        rows.append(row)
    clocks = sampler.stop() if not args.no_clocks else None
    launches = fde.fde_launch_count() - l0
    if rank == 0:
        line = {"metric": METRIC, "value": world * nsolves * 1e3 / total_ms, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / nsolves,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "example_4_1_tables_1_2", "rows": len(rows),
                           "preconditioners": list(setups), "tol": 1e-8, "restart": 20,
                           "stopping": "true residual relative to ||b|| (x0 = 0, so ||r0|| = ||b||); the paper's "
                                       "counts use the left-preconditioned residual",
                           "l2": "inputs of a few MB; every solve re-assembles and re-sets up its preconditioner"},
                "roofline": None, "gpu_launches": launches, "clocks": clocks, "rows": rows}
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# learned warm start: train on method-generated solves, compare initial guesses
# ---------------------------------------------------------------------------

def bench_learned(args, world, rank, local_rank):
    import numpy as np
    import torch

    import fde_inputs
    import paper_1305_6653_gb300 as fde

    torch.cuda.set_device(local_rank)
    m, s, modes = 1023, 256, 16
    net = fde.FDENop(m, s, modes=modes, width=64, layers=6, ksize=5, seed=1305)
    X = torch.empty((args.train, net.cin * modes), dtype=torch.float32, device="cuda")
    Y = torch.empty((args.train, s * modes), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    its_train = []
    for c0 in range(0, args.train, 64):
        chunk = [fde_inputs.config_learned_family(seed=i, m=m, s=s) for i in range(c0, min(c0 + 64, args.train))]
        with fde.FDEBatch(chunk, device_inputs=True) as b:
            b.assemble().factor(args.precision)
            xs, st = b.solve(tol=args.tol)
            its_train += [x_["iterations"] for x_ in st]
            for i, x in enumerate(xs):
                net.features(b.problem(i), X[c0 + i])
                net.coefficients(x, Y[c0 + i])
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    B = 32
    steps = args.epochs * (args.train // B)
    t0 = time.perf_counter()
    loss = None
    for step in range(steps):
        i0 = (step * B) % (args.train - B + 1)
        lr = 2e-3 if step < 0.6 * steps else (6e-4 if step < 0.85 * steps else 2e-4)
        loss, _ = net.loss_grad(X[i0:i0 + B].reshape(-1), Y[i0:i0 + B].reshape(-1), B)
        net.adam_step(lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = {"zero": {"its": [], "ms": []}, "learned": {"its": [], "ms": [], "rejected": 0}}
    x0 = torch.empty(s * m, dtype=torch.float64, device="cuda")
    for k in range(args.eval):
        prob = fde_inputs.config_learned_family(seed=10**6 + k, m=m, s=s)
        with fde.FDEProblem.from_inputs(prob, device_inputs=True) as p:
            for mode in ("zero", "learned"):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                p.assemble().factor(args.precision)
                if mode == "learned":
                    net.warm_start(p.h, x0)
                    _, st = p.solve(tol=args.tol, x0=x0)
                    res[mode]["rejected"] += st["x0_rejected"]
                else:
                    _, st = p.solve(tol=args.tol)
                e1.record()
                e1.synchronize()
                res[mode]["its"].append(st["iterations"])
                res[mode]["ms"].append(e0.elapsed_time(e1))
    out = {}
    for mode in ("zero", "learned"):
        ms = float(np.mean(res[mode]["ms"]))
        out[mode] = {"solves_per_s": 1e3 / ms, "mean_iterations": float(np.mean(res[mode]["its"])),
                     "iterations": res[mode]["its"], "ms_per_solve": ms}
    out["learned"]["x0_rejected"] = res["learned"]["rejected"]
    if rank == 0:
        line = {"metric": METRIC, "value": out["learned"]["solves_per_s"], "unit": "solves/s", "n_gpus": world,
                "steps": args.eval, "warmup": 0, "ms_per_step": out["learned"]["ms_per_solve"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64+f16",
                "data": "synthetic",
                "config": {"workload": "learned_family_m1023_s256_gbdf3", "train_solves": args.train,
                           "epochs": args.epochs, "batch": B,
                           "network": "6 conv1d layers along 16 sine modes, width 64, kernel 5",
                           "precision": args.precision, "tol_true_residual": args.tol},
                "training": {"data_gen_s": t_gen, "train_s": t_train, "final_loss": loss, "steps": steps,
                             "mean_train_iterations": float(np.mean(its_train))},
                "zero_x0": out["zero"], "learned_x0": out["learned"]}
        print(json.dumps(line))


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def measure_peaks() -> dict:
    """Microbenchmarks of the peaks that MEASURED_PEAKS.json lacks, on this GPU: TF32
    tensor-core GEMM (float32 matmul with TF32 allowed), FP32 CUDA-core GEMM (TF32
    off) and FP64 GEMM, 8192^3 / 8192^3 / 4096^3, best of several CUDA-event timings
    (2 N^3 flops).  cuBLAS through torch: a measurement of the hardware, not a part of
    the solver."""
    import torch

    def best(n, dtype, reps, tf32):
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            a = torch.randn(n, n, device="cuda", dtype=dtype)
            b = torch.randn(n, n, device="cuda", dtype=dtype)
            c = a @ b
            torch.cuda.synchronize()
            t = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                t.append(e0.elapsed_time(e1))
            del a, b, c
            return 2.0 * n ** 3 / (min(t) / 1e3) / 1e12
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old

    def copy_gbs(reps=5):
        # device-to-device copy of 2 GiB (read + write bytes), best of several timings: this box's
        # HBM rate, to set the block solves' roofline fraction beside the pool-wide measurement
        n = 1 << 29
        a = torch.ones(n, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        b.copy_(a)
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            b.copy_(a)
            e1.record()
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        del a, b
        return 2.0 * n * 4 / (min(t) / 1e3) / 1e9

    return {"tf32_tflops": best(8192, torch.float32, 8, True), "fp32_tflops": best(8192, torch.float32, 3, False),
            "fp64_tflops": best(4096, torch.float64, 3, False), "hbm_copy_gbs": copy_gbs(),
            "how": "torch.matmul (cuBLAS) best of 3-8 CUDA-event timings: float32 8192^3 with TF32 on / off, "
                   "float64 4096^3 (2 N^3 flops); hbm_copy_gbs: a 2 GiB device-to-device copy, read + write "
                   "bytes, best of 5"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    import fde_inputs

    if args.oracle_single_thread:  # child process of the reference arm (one BLAS thread)
        print(json.dumps(oracle_single_thread_sample(fde_inputs.config_scale(args.m, args.s), args.single_its)))
        return
    if args.config == "batch" and args.impl == "ours":
        return bench_batch(args, world, rank, local_rank)
    if args.config == "learned" and args.impl == "ours":
        return bench_learned(args, world, rank, local_rank)
    if args.config == "rhs" and args.impl == "ours":
        return bench_many_rhs(args, world, rank, local_rank)
    if args.config == "example41" and args.impl == "ours":
        return bench_example41(args, world, rank, local_rank)
    if args.config == "bccb" and args.impl == "ours":
        return bench_bccb(args, world, rank, local_rank)
    if args.config == "precision" and args.impl == "ours":
        return bench_precision(args, world, rank, local_rank)
    if args.config == "timevar" and args.impl == "ours":
        return bench_timevar(args, world, rank, local_rank)
    prob = fde_inputs.config_scale(args.m, args.s)
    workload = {"workload": f"scale_m{args.m}_s{args.s}_gbdf5_alpha1.8_variable_d", "m": args.m, "s": args.s,
                "unknowns": args.m * args.s, "scheme": "GBDF5", "alpha": 1.8, "d": "d+=1+x, d-=2-x",
                "tol_true_residual": args.tol, "restart": args.restart, "precision": args.precision,
                "arnoldi_matvec": args.matvec if args.matvec == "fp64" else f"fp32 (relax {args.relax:g})",
                "factor_storage": args.storage,
                "l2": "flushed (512 MiB write) before every timed step; factors (4.3 GB fp32; the bfloat16 copy the "
                      "block solves read, 2.2 GB) exceed L2"}

    if args.impl == "reference":
        return bench_reference(args, rank, prob, workload)

    import numpy as np
    import torch

    import paper_1305_6653_gb300 as fde

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the solver has no CPU path)")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for item in filter(None, args.tune.split(",")):
        name, v = item.split("=")
        fde.fde_tune_set({"matvec": 0, "trsv": 1, "lu": 2}[name.strip()], int(v))
    hbm_peak, bf16_peak, _, peak_kind = peaks()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    xbuf = torch.empty(prob.n, dtype=torch.float64, device="cuda")

    p = fde.FDEProblem.from_inputs(prob, device_inputs=True)

    def step(precision, matvec=None):
        p.assemble()
        p.factor(precision, storage=args.storage)
        mv = args.matvec if matvec is None else matvec
        _, st = p.solve(tol=args.tol, restart=args.restart, maxit=400, out=xbuf, matvec=mv, relax=args.relax)
        return st

    # the block-solve timer is selected before the warm-up, so that the iteration graphs
    # the warm-up captures already carry its event-record nodes
    p.profile_select(["trsv"])
    for _ in range(args.warmup):
        step(args.precision)
    barrier()

    # ---- timed region: the product path (iteration graphs replayed), with CUDA-event
    # pairs around the block solves only, recorded inside those graphs
    sampler = ClockSampler(local_rank)
    if not args.no_clocks:
        sampler.start()
    p.profile_select(["trsv"])  # same selection (graphs kept): clears the warm-up's records
    launches0 = fde.fde_launch_count()
    per_step = []
    stats = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        stats.append(step(args.precision))
        e1.record()
        e1.synchronize()
        per_step.append(e0.elapsed_time(e1))
    barrier()
    launches = fde.fde_launch_count() - launches0
    timed_prof = p.profile_read()
    p.profile_select([])
    clocks = sampler.stop() if not args.no_clocks else None

    total_ms = rank_max_ms(sum(per_step), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = world * args.steps / (total_ms / 1e3)

    # ---- untimed profiled pass: every stage with its own event pair (direct launches)
    prof = {}
    if args.profile_steps > 0:
        p.profile(True)
        for _ in range(args.profile_steps):
            flush.zero_()
            step(args.precision)
        torch.cuda.synchronize()
        prof = p.profile_read()
        p.profile(False)

    measured = measure_peaks() if rank == 0 else None
    tf32_peak = measured["tf32_tflops"] if measured else bf16_peak * 1.1 / 2.25
    fp64_peak = measured["fp64_tflops"] if measured else FP64_PEAK_TFLOPS

    # roofline of the dominant kernel, the block solves: algorithmic bytes per launch over
    # their mean CUDA-event duration in the timed region
    mp = (prob.m + 63) // 64 * 64
    nblk = prob.s // 2 + 1
    esz = 8 if args.precision == "fp64" else 4
    # the block solves stream the bfloat16 copy of the factors where the tensor-core LU wrote one
    fac_esz = 2 if (args.storage == "bf16" and args.precision in ("tf32", "bf16", "tf32x3") and mp % 128 == 0) \
        else esz
    dom_ms, dom_n = timed_prof["trsv"]
    per_launch = trsv_bytes(mp, nblk, esz, fac_esz)
    ach = per_launch / (dom_ms / dom_n / 1e3) / 1e9
    # DRAM traffic of one launch: ncu's dram__bytes_read.sum + dram__bytes_write.sum on the
    # m=1023, s=256 case was TRSV_TRAFFIC_RATIO[element bytes] x its algorithmic bytes; the
    # bytes grow with the factor planes, so a launch here moves the same multiple
    ratio = TRSV_TRAFFIC_RATIO.get(fac_esz) if esz == 4 else None
    traffic = ratio * per_launch if ratio else None
    roof = {"kernel": "block_trsv_kernel", "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
            "frac": ach / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": per_launch, "launches_timed": dom_n,
            "frac_of_this_gpu_copy": ach / measured["hbm_copy_gbs"] if measured else None,
            "timing": "CUDA events recorded inside the replayed iteration graphs, over the timed region",
            "traffic_source": "ncu capture at m=1023, s=256 scaled by the factor bytes" if traffic else None}
    # the tensor-core update beside it (profiled pass)
    tc_line = None
    if prof.get("lu_tc", (0, 0))[0] > 0:
        tms, tn = prof["lu_tc"]
        nps = args.profile_steps
        tfl = tc_update_flops(mp, nblk) * nps * (3 if args.precision == "tf32x3" else 1)
        tpeak = tf32_peak if args.precision in ("tf32", "tf32x3") else bf16_peak
        tbytes = tc_update_bytes(mp, nblk) * nps
        tc_line = {"kernel": "lu_update_tc2_kernel, lu_update_tc2p_kernel (cross tiles) + lu_update_tc2s_kernel "
                             "(interior, consecutive steps merged)",
                   "launches_per_step": tn // nps,
                   "timing": "profiled pass; CUDA events on both LU streams (the interior updates overlap the "
                             "panel chain)",
                   "ms_per_step": tms / nps, "tflops": tfl / (tms / 1e3) / 1e12,
                   "tensor_peak": tpeak, "tensor_peak_kind": "measured (cuBLAS TF32 GEMM, this run)" if measured
                   and args.precision in ("tf32", "tf32x3") else "measured bf16",
                   "c_tile_gbs": tbytes / (tms / 1e3) / 1e9, "hbm_peak": hbm_peak}
    matvec_line = None
    nps_ = max(args.profile_steps, 1)
    if prof.get("matvec", (0, 0))[1] > 0:
        mms, mn = prof["matvec"]
        L = 1
        while L < 2 * prob.m:
            L *= 2
        mfl = matvec_flops(prob.m, prob.s, L, prob.mu) * mn
        matvec_line = {"kernel": "st_matvec_kernel", "ms_per_launch": mms / mn, "launches_per_step": mn // nps_,
                       "tflops": mfl / (mms / 1e3) / 1e12, "timing": "profiled pass"}
        if args.matvec == "fp64":  # every launch is the FP64 product: bound by the FP64 rate
            matvec_line.update({"bound": "fp64 alu", "fp64_peak": fp64_peak,
                                "frac": mfl / (mms / 1e3) / 1e12 / fp64_peak})
        else:
            matvec_line["note"] = ("mixed: FP32 Arnoldi products and FP64 restart residuals; no single-precision "
                                   "roofline")
    path_roof = path_roofline(prob.m, prob.s, mp, esz, stats[-1]["iterations"], args.precision, bf16_peak,
                              hbm_peak, ms_per_step, restart=args.restart, tf32_peak=tf32_peak, fp64_peak=fp64_peak,
                              fac_esz=fac_esz)
    nps = max(args.profile_steps, 1)
    stage_ms = {k: round(v[0] / nps, 4) for k, v in prof.items()}
    stage_n = {k: v[1] // nps for k, v in prof.items()}

    # accuracy of the last solution: true residual with the oracle's independent matvec
    import oracle as O
    xs = xbuf.cpu().numpy()
    J = O.j_of(prob)
    bor = O.reduced_rhs(prob, J=J)
    res_oracle = float(np.linalg.norm(bor - O.matvec(prob, xs, J=J)) / np.linalg.norm(bor))

    # plain FP64 PGMRES on the same workload (the comparison the metric names): one
    # FP64 warm-up solve (allocates the 8.7 GB of FP64 factors), then timed solves
    plain = None
    if args.fp64_steps > 0:
        step("fp64", "fp64")
        tms, st64 = [], None
        for _ in range(args.fp64_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            st64 = step("fp64", "fp64")
            e1.record()
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        tms_sorted = sorted(tms)
        plain = {"value": 1e3 / (sum(tms) / len(tms)), "unit": "solves/s", "ms_per_step": sum(tms) / len(tms),
                 "ms_median": tms_sorted[len(tms) // 2], "per_step_ms": tms, "steps": len(tms), "warmup": 1,
                 "iterations": st64["iterations"], "rel_residual": st64["rel_residual"],
                 "speedup_of_mixed": (sum(tms) / len(tms)) / ms_per_step}
    p.close()

    # end-to-end through the C ABI from pinned host buffers: create copies the inputs in,
    # pgmres_solve copies the solution out (host x_out), destroy
    e2e = None
    if args.e2e_steps > 0:
        host = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k))).pin_memory()
                for k in ("dplus", "dminus", "u0", "f")}
        xh = torch.empty(prob.n, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * 8 for t in host.values())
        d2h = prob.n * 8

        def e2e_step():
            q = fde.FDEProblem(m=prob.m, s=prob.s, alpha=prob.alpha, xL=prob.xL, xR=prob.xR, t0=prob.t0, T=prob.T,
                               dplus=host["dplus"].numpy(), dminus=host["dminus"].numpy(), u0=host["u0"].numpy(),
                               f=host["f"].numpy(), family=prob.family, mu=prob.mu, device_inputs=False)
            q.assemble().factor(args.precision, storage=args.storage)
            q.solve(tol=args.tol, restart=args.restart, maxit=400, out=xh, matvec=args.matvec,
                    relax=args.relax)  # returns after the copy to xh
            q.close()

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.e2e_steps):
            e2e_step()
        e1.record()
        e1.synchronize()
        wall = time.perf_counter() - t0
        ev = e0.elapsed_time(e1) / 1e3
        e2e = {"value": world * args.e2e_steps / max(ev, wall), "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "path": "fde_problem_create (host desc) -> bvm_assemble -> strang_precond_factor -> pgmres_solve "
                       "(host x_out) -> fde_problem_destroy"}

    # the batched and precision legs (the metric's "mixed+batched"), driver-visible
    batch = precision = None
    if not args.no_extras and world == 1:
        batch = measure_batch(args, steps=3, warmup=1, sequential=False)
        precision = measure_precision(args, steps=1, warmup=1,
                                      precisions=("tf32x3", "fp32", "tf32", "bf16", "fp64"))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        its = plain["iterations"] if plain else 20
        cpu = oracle_sample(prob, iterations=its,
                            its_source="the plain FP64 solve's iteration count in this run" if plain
                            else "assumed")
        cpu.pop("seconds_per_solve", None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if args.precision != "fp64" else "f64", "data": "synthetic",
            "config": workload, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "iterations": [s["iterations"] for s in stats],
            "matvecs_fp32": [s["matvecs_fp32"] for s in stats],
            "rel_residual": stats[-1]["rel_residual"], "rel_residual_oracle_matvec": res_oracle,
            "plain_fp64": plain, "batch64": batch, "precision_m4095": precision,
            "tensor_core_update": tc_line, "matvec": matvec_line, "path_roofline": path_roof,
            "peaks_measured": measured,
            "launch_shapes": {"matvec": fde.fde_tune_query(0, mp, prob.s, "fp64"),
                              "trsv": fde.fde_tune_query(1, mp, nblk, {8: "fp64", 4: "fp32", 2: "bf16"}[fac_esz])},
            "stage_ms_per_step": stage_ms, "stage_launches_per_step": stage_n,
            "stage_split_source": f"untimed profiled pass of {args.profile_steps} solves after the timed region "
                                  "(every stage with its own event pair, direct launches)",
            "per_step_ms": per_step,
            # setup-excluded rate: the GMRES phase alone (pgmres_solve's device time)
            "gmres_phase": {"ms_per_solve": sum(s["ms_solve"] for s in stats) / len(stats),
                            "iterations_per_s": sum(s["iterations"] for s in stats) /
                            (sum(s["ms_solve"] for s in stats) / 1e3)},
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
