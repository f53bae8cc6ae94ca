"""Benchmark: block-CG RHS*iterations/s on the 128^3 7-point Laplacian (FP64).

Workload (the configuration the headline metric is quoted on): 3D 7-point
Laplacian on a 128^3 grid (n = 2,097,152), matrix-free stencil, FP64,
s = 8 right-hand sides drawn N(0,1) (seed 0), block CG with residual-block
QR stabilisation in every iteration (eta = inf, Alg. "bcgaro" scheduled as
Alg. "2R-CG").  One step = one BCG iteration: SpMM with the fused alpha Gram,
s x s solve, fused X/R update with the Gram of R-tilde, the normaliser
(CholeskyQR2: two row passes with their Grams and two s x s factors; the
Householder TSQR for blocks it declines), s x s step, direction update.

  value      RHS*iterations/s = s * K / (device time of K steady-state iterations);
             the K iterations are timed as the difference of two solves with
             maxit = W + K and maxit = W (setup cancels), each bracketed by
             CUDA events on the library's stream;
  e2e        the same metric through the C ABI with HOST buffers (B and X0 copied
             in, X copied out inside the call), host wall clock around the call;
  roofline   the dominant single-kernel phase, timed live with CUDA events (profiled
             solve), against the measured HBM bandwidth or the FP64 FMA rate of this
             GPU, whichever it comes closer to (the FP64 ridge point is ~0.19
             flop/byte; the operator and update passes sit near it at s = 8);
  iteration  the whole iteration's algorithmic FP64 flops and HBM bytes per second;
  cpu_baseline  the FP64 oracle (numpy/scipy) on the host cores, a bounded
             number of iterations of the same workload;
  sweep      s in {1, 4, 8, 16, 32}, stencil and CSR: RHS*iter/s, the FP64 and HBM
             fractions of the iteration, the FP32 fused operator + Gram against HBM;
  scalar_cg  time to 1e-8 of block CG against s independent scalar CG solves (one
             after another, and side by side in the subalgebra with p = 1);
  ir         FP32 + FP64 refinement against FP64 BCG, time to 1e-10 at 192^3.

--impl reference times the oracle alone as the reference arm: W warm-up and
exactly K timed BCG iterations of the same workload on the host cores (the K
timed as the difference of a (W + K)- and a W-iteration oracle solve).

Every n x s block is 134 MB > 129 MB L2, so no L2 flush is needed between
timed iterations ("inputs larger than L2").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "block-CG RHS*iter/s (128^3 Laplacian, FP64, QR-stabilised BCG)"
UNIT = "RHS*iter/s"
# FP64 FMA peak of a GB300: 152 SMs x 2.07 GHz x 2 DFMA/clk/SM x 2 flops = 1.259 TFLOP/s
# (the part's nominal 1.25 TFLOP/s FP64 rate at its maximum SM clock)
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12

# DRAM bytes (read + write) per launch of a kernel phase, from one ncu capture of the current
# kernel on the same workload (the level-0 TSQR leaf factor at 128^3, s = 8: 134.349 MB read +
# 79.423 MB written; the FP64 update with the Gram of R-tilde: 536.946 MB read + 226.509 MB
# written); keyed by (phase, grid, s, operator).
NCU_TRAFFIC = {("tsqr_leaf_factor", 128, 8, "stencil"): 134.349056e6 + 79.423488e6,
               ("update_rho", 128, 8, "stencil"): 536.935936e6 + 225.641472e6}


def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0   # fallback copy bandwidth of a GB300


HBM_PEAK_GBS = _hbm_peak()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default 300 for the native arm, 20 for the reference arm)")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--s", type=int, default=8)
    p.add_argument("--grid", type=int, default=128)
    p.add_argument("--op", default="stencil", choices=["stencil", "csr"])
    p.add_argument("--no-extra", action="store_true",
                   help="skip the rest of the metric (the s sweep, block vs scalar CG, and the FP32+IR vs FP64 "
                        "time to 1e-10)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--probe", choices=["bcg_fp64", "bcg_fp32_ir"],
                   help="run one short solve (a target for ncu) on --workload/--grid/--s and exit")
    p.add_argument("--phases", action="store_true",
                   help="per-phase device time of FP32+IR and FP64 BCG iterations on --workload")
    p.add_argument("--micro", action="store_true",
                   help="stand-alone FP32 operator product and block inner product timings")
    p.add_argument("--micro-case", default=None,
                   help="with --micro: one case only, as workload:s (e.g. laplace3d:8)")
    p.add_argument("--workload", default=None, help="workload of --probe / --phases")
    p.add_argument("--maxit", type=int, default=3)
    p.add_argument("--eta", type=float, default=math.inf,
                   help="re-orthonormalisation parameter of --probe / --phases (inf: every iteration)")
    p.add_argument("--jacobi", action="store_true", help="point-Jacobi preconditioner in --probe / --phases")
    p.add_argument("--subalgebra", action="store_true",
                   help="block-parallel subalgebra S_BP^p: cost per iteration and time to 1e-8 over p")
    p.add_argument("--tt", action="store_true",
                   help="time-to-tolerance of every workload's solver (median of 5 after 1 warm-up)")
    p.add_argument("--precond", action="store_true",
                   help="point-Jacobi preconditioned BCG against M = I on the variable-coefficient "
                        "workloads: time and iterations to tolerance, cost per iteration, and the "
                        "fused M^-1 + Gram pass against its roofline")
    p.add_argument("--one-reduction", action="store_true",
                   help="BCG with one reduction per iteration (Alg. 1R-CG) against the default "
                        "two-reduction schedule: time per iteration and to tolerance")
    p.add_argument("--ir", action="store_true",
                   help="time-to-1e-10 of FP32+IR vs plain FP64 BCG on the 192^3 log-normal diffusion "
                        "workload (s = 16) instead of the default line")
    a = p.parse_args()
    if a.steps is None:
        a.steps = 20 if a.impl == "reference" else 300
    return a


def run_ir(args):
    """FP32 inner BCG (to 1e-5) + FP64 refinement vs plain FP64 BCG, both to 1e-10; then the
    same pair with point Jacobi, the refinement's inner solve with the adaptive criterion
    (eta = 1: a QR only when kappa_D(alpha) > 1 / sqrt(eps_fp32)) and FP64 with eta = 1e4."""
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    build()
    grid = args.grid if args.grid != 128 else 192
    prob = W.problem("vardiff3d", s=16, grid=grid, with_csr=False)
    h = Handle(0)
    op = operator_from_problem(h, prob, "stencil")
    M = h.op_jacobi(op)
    Bd = torch.from_numpy(prob.B).cuda()
    nb = torch.linalg.vector_norm(Bd, dim=0)
    out = {}
    runs = [("fp32_ir", "fp32_ir", math.inf, None), ("fp64", "fp64", math.inf, None),
            ("fp32_ir_jacobi_eta1", "fp32_ir", 1.0, M), ("fp64_jacobi_eta1e4", "fp64", 1e4, M)]
    for name, prec, eta, pre in runs:
        X = torch.zeros_like(Bd)
        t0 = time.perf_counter()
        X, info = h.solve("bcg", op, Bd, X, tol=1e-10, maxit=20000, eta=eta, prec=prec, record=False,
                          precond=pre)
        wall = time.perf_counter() - t0
        R = h.residual(op, Bd, X)
        rel = float((torch.linalg.vector_norm(R, dim=0) / nb).max())
        out[name] = {"device_s": info.elapsed_ms / 1000.0, "wall_s": wall, "iters": info.iters,
                     "outer": info.outer, "reorths": info.reorths, "converged": info.converged,
                     "true_relres_max": rel, "eta": eta, "jacobi": pre is not None}
    line = {"metric": "time to max-column relative residual 1e-10 (192^3 log-normal diffusion, s=16)",
            "value": out["fp32_ir"]["device_s"], "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "dtype": "f32 inner + f64 refinement", "data": "synthetic",
            "config": {"workload": f"vardiff3d {grid}^3 var7 stencil, s=16, eta=inf"},
            "fp64_reference": out["fp64"], "fp32_ir": out["fp32_ir"],
            "speedup_vs_fp64": out["fp64"]["device_s"] / out["fp32_ir"]["device_s"],
            "jacobi": {"fp32_ir_eta1": out["fp32_ir_jacobi_eta1"], "fp64_eta1e4": out["fp64_jacobi_eta1e4"],
                       "speedup_vs_fp64": out["fp64_jacobi_eta1e4"]["device_s"]
                       / out["fp32_ir_jacobi_eta1"]["device_s"]}}
    print(json.dumps(line))
    M.close()
    h.close()


def dist_init(args):
    if args.gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist.get_rank(), dist.get_world_size(), dist


def aggregate(ms: float, units_per_rank: float, dist=None):
    """Whole-job throughput of independent replicas: every rank's units over the slowest rank's time.

    Returns (max_ms, value) with value = world * units_per_rank / (max_ms / 1000).  The only
    cross-rank operation of the bench is this max (a host-side gloo all-reduce of one float).
    """
    world = 1
    if dist is not None:
        import torch
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        world = dist.get_world_size()
    return ms, world * units_per_rank / (ms / 1000.0)


def spmm_alpha_ms(h, op, B, prec, iters=6):
    """Device time per launch of the fused SpMM + alpha Gram kernel in a profiled solve."""
    import math as _m
    h.profile_reset()
    h.solve("bcg", op, B, tol=0.0, maxit=iters, eta=_m.inf, prec=prec, ir_max_outer=1, profile=True,
            record=False)
    for nm, ms, nl in h.profile():
        if nm == "spmm_alpha" and nl:
            return ms / nl
    return float("nan")


def iteration_flops(n, s, cholqr=True):
    """Algorithmic FP64 flops of one BCG iteration (stencil, eta = inf); FMA = 2 flops.

    SpMM 7-point 14ns; the Grams alpha and rho (upper triangles) 2 n s(s+1);
    the block updates X += P lx, R -= Q lam, P = R + P beta: 6ns^2; the
    normaliser: CholeskyQR2's two triangular products Y <- Y U^-1, 2 n s(s+1), and the
    Gram of the first, n s(s+1) (its first Gram is rho's; the second pass's Gram is I
    by construction and not formed), or the Householder factor 2ns^2 and
    Q [sigma~; 0] 2ns^2.  The s x s work, the WY factors and the TSQR tree are
    O(n s^2 / tile) and not counted.
    """
    norm = 3 * n * s * (s + 1) if cholqr else 4 * n * s * s
    return 14 * n * s + 2 * n * s * (s + 1) + 6 * n * s * s + norm


def iteration_bytes(n, s, cholqr=True, elem=8):
    """Algorithmic HBM bytes of one BCG iteration (stencil, eta = inf): the SpMM reads P
    and writes Q, the update reads P, Q, X, R and writes X, R, the normaliser reads and
    writes the block (CholeskyQR2's first pass; the TSQR's factor and apply: twice), and
    the P update reads R, P and writes P (and R-bar with CholeskyQR2)."""
    return elem * n * s * ((2 + 6 + 2 + 4) if cholqr else (2 + 6 + 4 + 3))


PHASE_FLOPS = {
    # algorithmic flops per iteration of each kernel phase, as functions of (n, s)
    "spmm_alpha": lambda n, s: 14 * n * s + n * s * (s + 1),
    "update_rho": lambda n, s: 4 * n * s * s + n * s * (s + 1),
    # Householder QR of the tiles (2 n s^2) and the strict upper triangle of
    # V^T V that defines their compact WY factors (n s (s - 1))
    "tsqr_leaf_factor": lambda n, s: 2 * n * s * s + n * s * (s - 1),
    "tsqr_leaf_apply": lambda n, s: 2 * n * s * s + n * s * (s + 1),
    # P = R-bar + P beta with R-bar = Y1 U2^-1 formed on the way (CholeskyQR2 iterations)
    "p_update": lambda n, s: 2 * n * s * s + n * s * (s + 1),
}
PHASE_BYTES = {
    # algorithmic bytes per iteration (FP64): blocks read + written
    "spmm_alpha": lambda n, s: 2 * 8 * n * s,
    "update_rho": lambda n, s: 6 * 8 * n * s,
    "tsqr_leaf_factor": lambda n, s: 2 * 8 * n * s,
    "tsqr_leaf_apply": lambda n, s: 2 * 8 * n * s,
    "p_update": lambda n, s: 4 * 8 * n * s,
}
# The CholeskyQR2 phase per iteration (M = I): one row pass (read + write of the block,
# the triangular product and the Gram, 2 n s(s+1) flops) and two one-CTA s x s kernels;
# the second triangular product runs inside p_update.
PHASE_ITER_FLOPS = {"cholqr": lambda n, s: 2 * n * s * (s + 1)}
PHASE_ITER_BYTES = {"cholqr": lambda n, s: 2 * 8 * n * s}


class Clocks:
    """nvidia-smi sampling (every 100 ms) while the GPU work of the run executes: the timed
    region first, then the sweep and refinement parts of the line.  Samples with the GPU
    more than half busy count as under load; the median SM clock is taken over those."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, dev=0):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        if not self.p or not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons, total = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                clk, mx_, util = float(f[1]), float(f[2]), float(f[9])
            except ValueError:
                continue
            total += 1
            mx = mx_
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
            if util > 50:
                sm.append(clk)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": total, "samples_under_load": len(sm),
                "covers": "timed region, then the sweep, scalar CG and refinement runs"}


def cpu_baseline(prob, s, iters=3):
    """The FP64 oracle on the host cores: `iters` BCG-ARO iterations of the same workload."""
    import oracle
    t0 = time.perf_counter()
    oracle.bcg(prob.A, prob.B, tol=0.0, maxit=iters, eta=math.inf)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return {"value": s * iters / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{iters} BCG iterations (setup included) of the full {prob.A.n}-row, s={s} "
                      f"workload, CSR operator, numpy/scipy FP64 ({cores} host cores visible; "
                      f"BLAS calls threaded, sparse product single-threaded)",
            "seconds": dt}


def run_reference(args):
    """The oracle as the reference arm: W untimed warm-up iterations, then exactly K timed ones.

    One step is one BCG-ARO iteration of the same workload.  The oracle runs a whole solve per
    call, so the K steady-state iterations are timed as the difference of two runs from the same
    start, one of W + K iterations and one of W (the setup, R0 and its QR, cancels)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workloads as W
    prob = W.problem("laplace3d", s=args.s, grid=args.grid)
    K, Wm = max(1, args.steps), max(0, args.warmup)

    def solve_time(iters):
        t0 = time.perf_counter()
        oracle.bcg(prob.A, prob.B, tol=0.0, maxit=iters, eta=math.inf)
        return time.perf_counter() - t0

    dt = solve_time(Wm + K) - solve_time(Wm)
    value = args.s * K / dt
    cores = len(os.sched_getaffinity(0))
    cpu = {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{K} BCG iterations after {Wm} warm-up iterations of the full {prob.A.n}-row, "
                     f"s={args.s} workload, CSR operator, numpy/scipy FP64 ({cores} host cores visible; "
                     f"BLAS calls threaded, sparse product single-threaded), timed as the difference "
                     f"of a {Wm + K}-iteration and a {Wm}-iteration solve"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": K, "warmup": Wm,
            "ms_per_step": 1000.0 * dt / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"laplace3d {args.grid}^3 s={args.s} BCG eta=inf (oracle, CSR)"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def time_iters(h, op, Bd, s, W, K, torch):
    """Device ms of K steady-state iterations: solve(W+K) - solve(W), best of 2."""
    best = math.inf
    for _ in range(2):
        X1 = torch.zeros_like(Bd)
        _, i1 = h.solve("bcg", op, Bd, X1, tol=0.0, maxit=W + K, eta=math.inf, sync_every=W + K,
                        record=False)
        X0 = torch.zeros_like(Bd)
        _, i0 = h.solve("bcg", op, Bd, X0, tol=0.0, maxit=W, eta=math.inf, sync_every=max(W, 1),
                        record=False)
        assert i1.iters == W + K and i0.iters == W
        best = min(best, i1.elapsed_ms - i0.elapsed_ms)
    return best


def _diag_setup(args, workload, s_default):
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    build()
    s = args.s if args.s != 8 or workload == "laplace3d" else s_default
    prob = W.problem(workload, s=s, grid=args.grid, with_csr=(args.op == "csr"))
    h = Handle(0)
    op = operator_from_problem(h, prob, args.op)
    return h, op, prob, torch.from_numpy(prob.B).cuda(), torch


def run_probe(args):
    """One short solve, e.g. as the target of an ncu capture."""
    wl = args.workload or ("laplace3d" if args.probe == "bcg_fp64" else "vardiff3d")
    h, op, prob, B, torch = _diag_setup(args, wl, 16)
    prec = "fp64" if args.probe == "bcg_fp64" else "fp32_ir"
    M = h.op_jacobi(op) if args.jacobi else None
    X, info = h.solve("bcg", op, B, tol=0.0, maxit=args.maxit, eta=args.eta, prec=prec, ir_max_outer=1,
                      record=False, precond=M)
    torch.cuda.synchronize()
    print(json.dumps({"probe": args.probe, "workload": wl, "n": prob.B.shape[0], "s": prob.B.shape[1],
                      "iters": info.iters}))


def run_phases(args):
    """Per-phase device time per launch of FP32+IR (inner) and FP64 BCG iterations."""
    wl = args.workload or "vardiff3d"
    h, op, prob, B, torch = _diag_setup(args, wl, 16)
    out = {"workload": wl, "n": prob.B.shape[0], "s": prob.B.shape[1], "iterations": args.maxit,
           "eta": args.eta, "jacobi": args.jacobi}
    M = h.op_jacobi(op) if args.jacobi else None
    for prec in ("fp32_ir", "fp64"):
        for _ in range(2):   # the second run is reported
            h.profile_reset()
            X, info = h.solve("bcg", op, B, tol=0.0, maxit=args.maxit, eta=args.eta, prec=prec,
                              ir_max_outer=1, profile=True, record=False, precond=M)
        out[prec] = {nm: {"ms_per_launch": ms / nl, "launches": nl} for nm, ms, nl in h.profile() if nl}
    print(json.dumps(out))


def run_micro(args):
    """Stand-alone FP32 kernels against HBM: the operator product alone and with its fused
    Gram (alpha = P^T A P), block inner products of one and two blocks, and a copy.  Every
    repetition is timed on its own with CUDA events after an L2 flush (a 512 MB write)."""
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    build()
    h = Handle(0)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timeit(fn, reps=20):
        for _ in range(3):
            fn()
        tot = 0.0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            # two 512 MB writes: the L2 flush, and ~80 us more device work so that the host
            # has enqueued fn's kernels before e0 is reached (no host time in the window)
            flush.zero_()
            flush.zero_()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    out = {"hbm_peak_gbs": HBM_PEAK_GBS, "l2": "flushed before every timed launch"}
    cases = [("laplace3d", 8, 128), ("laplace3d", 16, 128), ("laplace3d", 32, 128), ("vardiff3d", 8, 192),
             ("vardiff3d", 16, 192)]
    if args.micro_case:
        kind, s = args.micro_case.split(":")
        cases = [c for c in cases if c[0] == kind and c[1] == int(s)]
        if not cases:
            raise SystemExit(f"no micro case {args.micro_case!r}")
    for kind, s, grid in cases:
        prob = W.problem(kind, s=s, grid=grid if args.grid == 128 else args.grid, with_csr=False)
        op = operator_from_problem(h, prob, "stencil")
        n = prob.B.shape[0]
        P = torch.randn(n, s, device="cuda", dtype=torch.float32)
        Q = torch.empty_like(P)
        G = torch.empty(s, s, device="cuda", dtype=torch.float64)
        by = 4 * n * s
        coef = 4 * n if kind == "vardiff3d" else 0     # one coefficient k per cell (algorithmic)
        r = {"spmm": timeit(lambda: h.spmm(op, P, Q)),
             "spmm_gram": timeit(lambda: h.spmm_gram(op, P, Q, G=G)),
             "bdot_two_blocks": timeit(lambda: h.bdot(P, Q, G=G)),
             "bdot_one_block": timeit(lambda: h.bdot(P, P, sym=True, G=G)),
             "copy": timeit(lambda: Q.copy_(P))}
        gbs = {"spmm": 2 * by + coef, "spmm_gram": 2 * by + coef, "bdot_two_blocks": 2 * by,
               "bdot_one_block": by, "copy": 2 * by}
        out[f"{kind}{grid}_s{s}"] = {k: {"ms": v, "gbs": gbs[k] / (v / 1000.0) / 1e9,
                                        "hbm_frac": gbs[k] / (v / 1000.0) / 1e9 / HBM_PEAK_GBS}
                                    for k, v in r.items()}
        op.close()
        del P, Q
        torch.cuda.empty_cache()
    print(json.dumps(out))


def run_tt(args):
    """Time to tolerance of the solve call for each workload (device time, CUDA events around
    the whole solve inside the library; median of 5 runs after 1 warm-up, of 3 for the
    refinement case)."""
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    build()
    h = Handle(0)
    cases = [
        ("poisson2d 64^2 5-point CSR, s=4, BCG eta=inf, 1e-8", "poisson2d", "csr", "bcg",
         dict(tol=1e-8, eta=math.inf)),
        ("laplace3d 128^3 stencil, s=8, BCG eta=inf, 1e-8", "laplace3d", "stencil", "bcg",
         dict(tol=1e-8, eta=math.inf)),
        ("laplace3d 128^3 stencil, s=8, BCG eta=1e4 (adaptive), 1e-8", "laplace3d", "stencil", "bcg",
         dict(tol=1e-8, eta=1e4)),
        ("convdiff3d 96^3 upwind stencil, s=8, BBiCGStab eta=100, 1e-8", "convdiff3d", "stencil",
         "bbicgstab", dict(tol=1e-8, eta=100.0)),
        ("convdiff3d 96^3 upwind stencil, s=8, BGMRes(30) CGS2 + TSQR, 1e-8", "convdiff3d", "stencil",
         "bgmres", dict(tol=1e-8, restart=30, ortho="cgs2")),
        ("convdiff3d 96^3 upwind stencil, s=8, BGMRes(30) localized Arnoldi, 1e-8", "convdiff3d", "stencil",
         "bgmres", dict(tol=1e-8, restart=30, ortho="localized")),
        ("convdiff3d 96^3 upwind stencil, s=8, BGMRes(30) block MGS, 1e-8", "convdiff3d", "stencil",
         "bgmres", dict(tol=1e-8, restart=30, ortho="mgs")),
        ("vardiff3d 192^3 var7 stencil, s=16, FP32 BCG + FP64 refinement, 1e-10", "vardiff3d", "stencil",
         "bcg", dict(tol=1e-10, eta=math.inf, prec="fp32_ir")),
        ("vardiff3d 192^3 var7 stencil, s=16, FP32 BCG (Jacobi, eta=1) + FP64 refinement, 1e-10", "vardiff3d",
         "stencil", "bcg", dict(tol=1e-10, eta=1.0, prec="fp32_ir", jacobi=True)),
        ("edge2d 512^2 per-edge stencil, s=32, BCG eta=1e4, 1e-8", "edge2d", "stencil", "bcg",
         dict(tol=1e-8, eta=1e4)),
    ]
    out = []
    for label, wl, use, method, kw in cases:
        prob = W.problem(wl, with_csr=(use == "csr"))
        op = operator_from_problem(h, prob, use)
        B = torch.from_numpy(prob.B).cuda()
        kw = dict(kw)
        M = h.op_jacobi(op) if kw.pop("jacobi", False) else None
        times, info = [], None
        nrep = 4 if kw.get("prec") == "fp32_ir" else 6     # the refinement case runs ~15 s
        for rep in range(nrep):
            X, info = h.solve(method, op, B, maxit=20000, record=False, precond=M, **kw)
            if rep:
                times.append(info.elapsed_ms)
        times.sort()
        out.append({"case": label, "median_ms": times[len(times) // 2], "min_ms": times[0],
                     "iters": info.iters, "converged": info.converged, "relres_max": info.relres_max,
                     "n": prob.B.shape[0], "s": prob.B.shape[1]})
        if M is not None:
            M.close()
        op.close()
        del B
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "time to tolerance (solve call, device time)", "unit": "ms",
                      "results": out}))


def run_subalgebra(args):
    """S_BP^p on the 128^3 Laplacian (stencil, FP64, eta = inf): device time per iteration
    (20 iterations after 3) and time / iterations to a max-column relative residual of 1e-8,
    for s in {16, 32} and p from s (the block case S_B) down to 1 (S_P)."""
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    build()
    h = Handle(0)
    out = []
    for s in (16, 32):
        prob = W.problem("laplace3d", s=s, grid=args.grid, with_csr=False)
        op = operator_from_problem(h, prob, "stencil")
        B = torch.from_numpy(prob.B).cuda()
        for p in [q for q in (32, 16, 8, 4, 2, 1) if q <= s]:
            h.solve("bcg", op, B, tol=0.0, maxit=3, eta=math.inf, record=False, p=p)
            _, i20 = h.solve("bcg", op, B, tol=0.0, maxit=23, eta=math.inf, record=False, p=p)
            _, i3 = h.solve("bcg", op, B, tol=0.0, maxit=3, eta=math.inf, record=False, p=p)
            ms_it = (i20.elapsed_ms - i3.elapsed_ms) / 20
            _, it = h.solve("bcg", op, B, tol=1e-8, maxit=5000, eta=math.inf, record=False, p=p)
            out.append({"s": s, "p": p, "ms_per_iter": ms_it, "rhs_iter_per_s": s / (ms_it / 1000.0),
                        "iters_to_1e-8": it.iters, "time_to_1e-8_ms": it.elapsed_ms,
                        "converged": it.converged})
        op.close()
        del B
    print(json.dumps({"workload": f"laplace3d {args.grid}^3 stencil, FP64, eta=inf", "results": out}))


def run_precond(args):
    """Point Jacobi (M = diag(A)) against M = I for BCG on the variable-coefficient
    workloads.  Per case and M: device time and iterations to tolerance (two runs after a
    short warm-up, the smaller time kept), device time per iteration (23 minus 3
    iterations, over 20), and for Jacobi the profiled per-launch time of the fused pass
    Z = M^-1 R-bar, rho = R-bar^T Z with its algorithmic bytes n (2s + 1) w and flops
    n (s + s (s + 1))."""
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    build()
    h = Handle(0)
    cases = [
        ("vardiff3d 192^3 var7 stencil, s=16, FP32 BCG + FP64 refinement, 1e-10", "vardiff3d", None, 16,
         dict(tol=1e-10, eta=math.inf, prec="fp32_ir")),
        ("vardiff3d 128^3 var7 stencil, s=8, FP64 BCG eta=1e4, 1e-8", "vardiff3d", 128, 8,
         dict(tol=1e-8, eta=1e4)),
        ("edge2d 512^2 per-edge stencil, s=32, FP64 BCG eta=1e4, 1e-8", "edge2d", None, 32,
         dict(tol=1e-8, eta=1e4)),
    ]
    out = []
    for label, wl, grid, s, kw in cases:
        prob = W.problem(wl, s=s, grid=grid, with_csr=False)
        op = operator_from_problem(h, prob, "stencil")
        Mj = h.op_jacobi(op)
        B = torch.from_numpy(prob.B).cuda()
        n = prob.B.shape[0]
        w = 4 if kw.get("prec") == "fp32_ir" else 8
        row = {"case": label, "n": n, "s": s}
        for name, M in (("identity", None), ("jacobi", Mj)):
            h.solve("bcg", op, B, maxit=3, record=False, precond=M, **kw)
            times = []
            for _ in range(2):
                _, info = h.solve("bcg", op, B, maxit=20000, record=False, precond=M, **kw)
                times.append(info.elapsed_ms)
            pk = dict(kw, prec="fp64" if w == 8 else "fp32_ir", tol=0.0)
            if w == 4:
                pk["ir_max_outer"] = 1
            _, i23 = h.solve("bcg", op, B, maxit=23, record=False, precond=M, **pk)
            _, i3 = h.solve("bcg", op, B, maxit=3, record=False, precond=M, **pk)
            r = {"time_ms": min(times), "iters": info.iters, "converged": info.converged,
                 "relres_max": info.relres_max, "outer": info.outer,
                 "ms_per_iter": (i23.elapsed_ms - i3.elapsed_ms) / 20}
            if M is not None:
                h.profile_reset()
                h.solve("bcg", op, B, maxit=20, record=False, precond=M, profile=True, **pk)
                prof = {p[0]: (p[1], p[2]) for p in h.profile()}
                ms, nl = prof["precond_rho"]
                per = ms / max(nl, 1)
                nbytes = n * (2 * s + 1) * w
                flops = n * (s + s * (s + 1))
                r["precond_pass"] = {"ms_per_launch": per, "launches": nl,
                                     "gbs": nbytes / (per / 1e3) / 1e9,
                                     "hbm_frac": nbytes / (per / 1e3) / 1e9 / HBM_PEAK_GBS,
                                     "tflops": flops / (per / 1e3) / 1e12}
                if w == 8:
                    r["precond_pass"]["fp64_frac"] = r["precond_pass"]["tflops"] / FP64_PEAK_TFLOPS
                r["phases_ms_per_iter"] = {k: v[0] / 20 for k, v in prof.items() if v[1] > 0}
            row[name] = r
        row["speedup"] = row["identity"]["time_ms"] / row["jacobi"]["time_ms"]
        out.append(row)
        Mj.close()
        op.close()
        del B
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "BCG time to tolerance, point Jacobi vs M = I (device time)",
                      "results": out}))


def run_one_reduction(args):
    """Alg. "1R-CG" against Alg. "2R-CG" on one GPU: device time to tolerance (the smaller
    of two runs after a warm-up), iterations, and time per iteration (23 minus 3
    iterations, over 20)."""
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    build()
    h = Handle(0)
    # variants: (name, one_reduction, replace_every)
    std = (("two_reductions", False, 0), ("one_reduction", True, 0), ("one_reduction_replace10", True, 10))
    ir = (("two_reductions", False, 0), ("one_reduction", True, 0), ("one_reduction_replace1", True, 1))
    cases = [
        ("poisson2d 64^2 5-point CSR, s=4, FP64 BCG eta=inf, 1e-8", "poisson2d", "csr", None, 4, False,
         dict(tol=1e-8, eta=math.inf), std),
        ("laplace3d 128^3 stencil, s=8, FP64 BCG eta=inf, 1e-8", "laplace3d", "stencil", None, 8, False,
         dict(tol=1e-8, eta=math.inf), std),
        ("vardiff3d 128^3 var7 stencil, s=8, FP64 BCG eta=1e4, Jacobi, 1e-8", "vardiff3d", "stencil", 128, 8,
         True, dict(tol=1e-8, eta=1e4), std),
        ("vardiff3d 128^3 var7 stencil, s=16, FP32 BCG + FP64 refinement, Jacobi, eta=1, 1e-10", "vardiff3d",
         "stencil", 128, 16, True, dict(tol=1e-10, eta=1.0, prec="fp32_ir"), ir),
    ]
    out = []
    for label, wl, use, grid, s, jac, kw, variants in cases:
        prob = W.problem(wl, s=s, grid=grid, with_csr=(use == "csr"))
        op = operator_from_problem(h, prob, use)
        M = h.op_jacobi(op) if jac else None
        B = torch.from_numpy(prob.B).cuda()
        row = {"case": label}
        for name, one, rep in variants:
            h.solve("bcg", op, B, maxit=3, record=False, precond=M, one_reduction=one, replace_every=rep, **kw)
            times = []
            for _ in range(2):
                _, info = h.solve("bcg", op, B, maxit=20000, record=False, precond=M, one_reduction=one,
                                  replace_every=rep, **kw)
                times.append(info.elapsed_ms)
            pk = dict(kw, tol=0.0)
            if kw.get("prec") == "fp32_ir":
                pk["ir_max_outer"] = 1
            _, i23 = h.solve("bcg", op, B, maxit=23, record=False, precond=M, one_reduction=one, replace_every=rep,
                             **pk)
            _, i3 = h.solve("bcg", op, B, maxit=3, record=False, precond=M, one_reduction=one, replace_every=rep,
                            **pk)
            row[name] = {"time_ms": min(times), "iters": info.iters, "converged": info.converged,
                         "status": info.status_name, "replacements": info.replacements,
                         "relres_max": info.relres_max, "ms_per_iter": (i23.elapsed_ms - i3.elapsed_ms) / 20}
        out.append(row)
        if M is not None:
            M.close()
        op.close()
        del B
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "BCG time to tolerance, one vs two reductions per iteration (device time)",
                      "results": out}))


def _flush_timer(torch):
    """Device time (ms) of one call after an L2 flush (512 MB written twice, so that the
    host has enqueued the call before the start event is reached), CUDA events."""
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timeit(fn, reps=10, warm=3):
        for _ in range(warm):
            fn()
        tot = 0.0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            flush.zero_()
            flush.zero_()          # keeps the device busy while the host enqueues fn
            e0.record(); fn(); e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps
    return timeit


def run_sweep(h, args, prob, torch):
    """The s in {1, 4, 8, 16, 32} half of the metric on the 128^3 Laplacian, stencil and CSR:
    FP64 BCG (eta = inf) RHS*iter/s over 10 steady-state iterations (after 3), the FP64 rate
    of the iteration against the FP64 peak, and the fused operator + Gram pass (Q = A P with
    alpha = P^T Q, bkrylov_spmm_gram) in FP32 against the measured HBM copy bandwidth
    (algorithmic bytes: P read, Q written, plus the CSR arrays)."""
    import workloads as W
    from paper_2104_02494_gb300.api import operator_from_problem
    n = prob.B.shape[0]
    B32 = W.normal_block(n, 32, 0)               # the Laplacian's B is the first s columns of this draw
    timeit = _flush_timer(torch)
    out = {}
    for use in ("stencil", "csr"):
        op = operator_from_problem(h, prob, use)
        for ss in (1, 4, 8, 16, 32):
            B2 = torch.from_numpy(np.ascontiguousarray(B32[:, :ss])).cuda()
            kk = 10
            m2 = time_iters(h, op, B2, ss, 3, kk, torch)
            fl = iteration_flops(n, ss)
            by_it = iteration_bytes(n, ss) + (prob.A.nnz * 12 + 4 * (n + 1) if use == "csr" else 0)
            e = {"rhs_iter_per_s": ss * kk / (m2 / 1000.0), "ms_per_iter": m2 / kk,
                 "fp64_tflops": fl / (m2 / kk / 1000.0) / 1e12}
            e["fp64_frac"] = e["fp64_tflops"] / FP64_PEAK_TFLOPS
            e["hbm_frac"] = by_it / (m2 / kk / 1000.0) / 1e9 / HBM_PEAK_GBS
            P32 = B2.float()
            Q32 = torch.empty_like(P32)
            G = torch.empty(ss, ss, dtype=torch.float64, device="cuda")
            t = timeit(lambda: h.spmm_gram(op, P32, Q32, G=G))
            by = 2 * 4 * n * ss + (prob.A.nnz * 8 + 4 * (n + 1) if use == "csr" else 0)
            e["spmm_bdot_fp32"] = {"ms": t, "gbs": by / (t / 1000.0) / 1e9,
                                   "hbm_frac": by / (t / 1000.0) / 1e9 / HBM_PEAK_GBS}
            out[f"{use}_s{ss}"] = e
            del B2, P32, Q32
        op.close()
    torch.cuda.empty_cache()
    return out


def run_scalar_cg(h, args, prob, torch):
    """Block CG against s independent scalar CG solves on the 128^3 Laplacian stencil (FP64,
    max-column relative residual 1e-8), s in {1, 4, 8, 16, 32}: the block solve with QR
    stabilisation (eta = inf); the s columns solved one after another by CG (s = 1, eta = 0:
    no normaliser after the first); and the s scalar CGs run side by side as one block in the
    block-parallel subalgebra with p = 1 (every s x s quantity diagonal, eta = 0).  Device time
    of each solve call, one untimed 3-iteration solve of each shape first.  The columns are the
    first s of one seeded N(0, 1) draw, so the sequential time of s columns is a prefix sum."""
    import workloads as W
    from paper_2104_02494_gb300.api import operator_from_problem
    n = prob.B.shape[0]
    B32 = W.normal_block(n, 32, 0)
    op = operator_from_problem(h, prob, "stencil")
    widths = (1, 4, 8, 16, 32)
    col_ms, col_it = [], []
    for j in range(max(widths)):
        b = torch.from_numpy(np.ascontiguousarray(B32[:, j:j + 1])).cuda()
        if j == 0:
            h.solve("bcg", op, b, tol=1e-8, maxit=3, eta=0.0, record=False)
        _, info = h.solve("bcg", op, b, tol=1e-8, maxit=20000, eta=0.0, record=False)
        col_ms.append(info.elapsed_ms)
        col_it.append(info.iters)
    out = {"workload": "laplace3d 128^3 7-point stencil, FP64, to 1e-8"}
    for ss in widths:
        Bs = torch.from_numpy(np.ascontiguousarray(B32[:, :ss])).cuda()
        e = {}
        for name, kw in (("block", dict(eta=math.inf)), ("batched_scalar", dict(eta=0.0, p=1))):
            if name == "batched_scalar" and ss == 1:
                continue
            h.solve("bcg", op, Bs, tol=1e-8, maxit=3, record=False, **kw)
            _, info = h.solve("bcg", op, Bs, tol=1e-8, maxit=20000, record=False, **kw)
            e[name] = {"ms": info.elapsed_ms, "iters": info.iters, "converged": bool(info.converged)}
        e["sequential_scalar"] = {"ms": float(sum(col_ms[:ss])), "iters_max": int(max(col_it[:ss])),
                                  "iters_sum": int(sum(col_it[:ss]))}
        e["block_speedup_vs_sequential"] = e["sequential_scalar"]["ms"] / e["block"]["ms"]
        if "batched_scalar" in e:
            e["block_speedup_vs_batched"] = e["batched_scalar"]["ms"] / e["block"]["ms"]
        out[f"s{ss}"] = e
        del Bs
    op.close()
    torch.cuda.empty_cache()
    return out


def run_ir_pair(h, args, torch):
    """The FP32+IR vs FP64 half of the metric: time to a max-column relative residual of 1e-10
    on the 192^3 log-normal diffusion workload (s = 16), both with point Jacobi: FP64 BCG with
    the adaptive criterion at eta = 1e4 against FP32 inner BCG (to 1e-5, eta = 1) inside FP64
    refinement.  Device time of the solve call; the true residual is recomputed in FP64 by the
    library.  One untimed 3-iteration solve of each first."""
    import workloads as W
    from paper_2104_02494_gb300.api import operator_from_problem
    prob = W.problem("vardiff3d", s=16, with_csr=False)
    op = operator_from_problem(h, prob, "stencil")
    M = h.op_jacobi(op)
    Bd = torch.from_numpy(prob.B).cuda()
    nb = torch.linalg.vector_norm(Bd, dim=0)
    out = {"workload": "vardiff3d 192^3 var7 stencil, s=16, point Jacobi, to 1e-10"}
    for name, prec, eta in (("fp64", "fp64", 1e4), ("fp32_ir", "fp32_ir", 1.0)):
        h.solve("bcg", op, Bd, tol=1e-10, maxit=3, eta=eta, prec=prec, record=False, precond=M,
                ir_max_outer=1)
        X = torch.zeros_like(Bd)
        X, info = h.solve("bcg", op, Bd, X, tol=1e-10, maxit=20000, eta=eta, prec=prec, record=False,
                          precond=M)
        R = h.residual(op, Bd, X)
        out[name] = {"seconds": info.elapsed_ms / 1000.0, "iters": info.iters, "outer": info.outer,
                     "reorths": info.reorths, "converged": bool(info.converged), "eta": eta,
                     "true_relres_max": float((torch.linalg.vector_norm(R, dim=0) / nb).max())}
    out["speedup_fp32_ir_vs_fp64"] = out["fp64"]["seconds"] / out["fp32_ir"]["seconds"]
    M.close()
    op.close()
    del Bd
    torch.cuda.empty_cache()
    return out



def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ir:
        return run_ir(args)
    if args.probe:
        return run_probe(args)
    if args.phases:
        return run_phases(args)
    if args.micro:
        return run_micro(args)
    if args.tt:
        return run_tt(args)
    if args.subalgebra:
        return run_subalgebra(args)
    if args.precond:
        return run_precond(args)
    if args.one_reduction:
        return run_one_reduction(args)
    rank, world, dist = dist_init(args)
    import torch
    import workloads as W
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle, operator_from_problem
    from paper_2104_02494_gb300 import _lib

    build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    s, Wm, K = args.s, max(3, args.warmup), max(1, args.steps)
    prob = W.problem("laplace3d", s=s, grid=args.grid, with_csr=(args.op == "csr" or rank == 0))
    n = prob.B.shape[0]
    h = Handle(dev)
    op = operator_from_problem(h, prob, args.op)
    Bd = torch.from_numpy(prob.B).cuda()
    torch.cuda.synchronize()

    # warm up the library (workspace, module load)
    h.solve("bcg", op, Bd, tol=0.0, maxit=Wm, eta=math.inf, record=False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = Clocks(dev).__enter__()
    ms = time_iters(h, op, Bd, s, Wm, K, torch)
    torch.cuda.synchronize()
    ms, value = aggregate(ms, s * K, dist)
    if dist:
        dist.barrier()

    # per-phase device times (profiled solve, events around every phase)
    h.profile_reset()
    h.solve("bcg", op, Bd, tol=0.0, maxit=K, eta=math.inf, record=False, profile=True)
    prof = [(nm, t, nl) for nm, t, nl in h.profile() if nl > 0]
    tot = sum(t for _, t, _ in prof)
    phases = {nm: {"ms_per_launch": t / max(nl, 1), "ms_per_iter": t / K, "share": t / tot,
                   "launches": nl} for nm, t, nl in prof}
    # the dominant kernel phase, per iteration (a phase whose launches include kernels that
    # return at once on a device decision counts the working kernel), against whichever of
    # the FP64 pipe and HBM it comes closer to
    dom = max((p for p in prof if p[0] in PHASE_FLOPS), key=lambda p: p[1])
    dom_ms = dom[1] / K
    tfl = PHASE_FLOPS[dom[0]](n, s) / (dom_ms / 1000.0) / 1e12
    gbs = PHASE_BYTES[dom[0]](n, s) / (dom_ms / 1000.0) / 1e9
    traffic = NCU_TRAFFIC.get((dom[0], args.grid, s, args.op))
    if gbs / HBM_PEAK_GBS >= tfl / FP64_PEAK_TFLOPS:
        roofline = {"bound": "hbm", "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                    "frac": gbs / HBM_PEAK_GBS, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "fp64_tflops": tfl, "fp64_frac": tfl / FP64_PEAK_TFLOPS}
    else:
        roofline = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tfl / FP64_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 2.07 GHz x 2 DFMA/clk/SM x 2 flop",
                    "hbm_achieved_gbs": gbs, "hbm_frac": gbs / HBM_PEAK_GBS}
    roofline.update({"kernel": dom[0], "ms_per_launch": dom_ms, "launches_per_iter": dom[2] / K, "traffic": traffic,
                     "traffic_unit": "bytes per launch (ncu dram read + write)" if traffic else None})
    for nm, t_ms, nl in prof:
        if nm in PHASE_ITER_BYTES and nm in phases:
            per_it = t_ms / K
            phases[nm]["ms_per_iter"] = per_it
            phases[nm]["hbm_frac"] = PHASE_ITER_BYTES[nm](n, s) / (per_it / 1000.0) / 1e9 / HBM_PEAK_GBS
    iteration = {"ms": ms / K, "fp64_tflops": iteration_flops(n, s) / (ms / K / 1000.0) / 1e12,
                 "hbm_gbs": iteration_bytes(n, s) / (ms / K / 1000.0) / 1e9}
    iteration["fp64_frac"] = iteration["fp64_tflops"] / FP64_PEAK_TFLOPS
    iteration["hbm_frac"] = iteration["hbm_gbs"] / HBM_PEAK_GBS

    # end to end through the C ABI with host buffers
    Bh = np.ascontiguousarray(prob.B)
    Xh = np.zeros_like(Bh)
    t0 = time.perf_counter()
    _, ie = h.solve("bcg", op, Bh, Xh, tol=0.0, maxit=K, eta=math.inf, record=False)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": s * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * Bh.nbytes / K,
           "d2h_bytes_per_step": Xh.nbytes / K, "note": "setup (residual, first QR) included"}

    sweep = ir = scalar = None
    if rank == 0 and not args.no_extra:
        sweep = run_sweep(h, args, prob, torch)
        scalar = run_scalar_cg(h, args, prob, torch)
        ir = run_ir_pair(h, args, torch)
    clk.__exit__(None, None, None)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, s, iters=3)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}

    launches = _lib.load().bkrylov_bcg_launches_per_iteration(n, s, None) * K
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"laplace3d {args.grid}^3 7-point, {args.op}, s={s}, BCG eta=inf",
                           "n": n, "s": s, "l2": "inputs larger than L2 (each n x s block 134 MB)",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "normaliser": "CholeskyQR2 (Householder TSQR for declined blocks)"},
                "iteration": iteration, "roofline": roofline, "phases": phases, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk.summary(), "gpu_launches": launches}
        if sweep:
            line["sweep"] = sweep
        if scalar:
            line["scalar_cg"] = scalar
        if ir:
            line["ir"] = ir
        print(json.dumps(line))
    h.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
