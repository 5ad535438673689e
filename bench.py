#!/usr/bin/env python3
"""Benchmark of the GB300 AF-IETI solver; by default on the C3 workload.

Workload (C3, the largest of the paper-shaped configurations whose stored
stiffness fits one GPU): 3D compressible elasticity (E = 1, nu = 0.3) on a
thick quarter annulus (radii 1..2, height 1) split into 6x4x3 = 72 patches
of uneven sizes: degree p = 4 (the seed-0 draw from {2,3,4,5}), C^3 splines,
element counts per patch column drawn from {12,16,24,32,48} (seed 0: 12/16/32
x 12/24/48 x 32, nine distinct patch shapes, 6.59 M DoF), all-floating with
Dirichlet conditions on the whole outer boundary, body force with
uniform[-1,1] nodal coefficients (seeded), preconditioned MINRES to 1e-8
relative residual (estimate and true residual).  `--workload C2|C4|C5-mid`
selects another configuration.  `--workload C5` runs the metric's own
configuration, whose stored stiffness would need 1.9 TB, on the matrix-free
operator (run_matrix_free; about ten minutes with three warm-up solves), and
`--fd-only --workload C5` its local solvers alone.

One step = one complete AF-IETI solve (lambda_0, MINRES, recovery) with the
load vector resident in HBM.  The per-step inputs are larger than L2: every
iteration streams the stiffness stencil (each FP64 coefficient held as a
pair of FP32 numbers and applied in double-FP32 arithmetic; 106 GB for C3).
As in the paper's INEXACT timings, the reported solve time includes the
local-solver setup (Algorithm 1 step 1, timed once by the library and added
to the measured solve); the stiffness assembly and constraint setup are
reported as setup_s.

Beside the headline the line reports the plain FP64 form (FP64 local solvers
and FP64 stencil), the mixed form with the FP64 stencil, eight right-hand
sides solved together (multi_rhs), the geometry-inclusion local solvers of
Section 5.2.3 on the same problem (geometry_inclusion), FD-apply rates, the
rooflines of the dominant kernels, and the metric's own configuration C5 on
the matrix-free stiffness (matrix_free_C5: its products and a bounded run of
its iterations).  The contexts are built one after the
other, each freed before the next, so that the largest workload fits.

  python bench.py [--gpus N --steps K --warmup W --prec fp32|fp64|tf32|bf16 --workload C2]
  python bench.py --impl reference ...   (the CPU oracle as the reference arm)

With N > 1 (torchrun) every rank solves its own seeded right-hand side on its
own GPU (replicas, weak scaling); the solve has no cross-GPU exchange.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
_CORES = len(os.sched_getaffinity(0))
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(_CORES))

METRIC = "AF-IETI solve time and FD-apply DoF/s, mixed vs FP64 plain, at 1e-8 residual"
_COMMON = ("E=1 nu=0.3, Dirichlet outer boundary, seeded uniform[-1,1] body-force coefficients, "
           "MINRES tol 1e-8")
WORKLOADS = {
    "C3": "C3: thick quarter annulus (radii 1..2, height 1), 6x4x3 = 72 uneven patches, p=4 "
          "(seed-0 draw from {2,3,4,5}), C^3, element counts per patch column drawn from "
          "{12,16,24,32,48} (seed 0: 12/16/32 x 12/24/48 x 32), " + _COMMON,
    "C2": "C2: unit cube, 4x4x4 patches, p=3, C^2, 16^3 elements/patch, 10% interior jitter, "
          + _COMMON,
    "C4": "C4: thick quarter annulus, 6x4x3 patches, p=3, C^2, 24^3 elements/patch, " + _COMMON,
    "C5-mid": "C5-mid: 2x2x2 patches of the C5 twisted box (45-degree twist), p=4, C^3, "
              "48^3 elements/patch, " + _COMMON,
    "C5": "C5: twisted box (unit cube, 45-degree twist about z), 8x8x4 = 256 patches, p=4, C^3, "
          "48^3 elements/patch (108 M DoF), matrix-free stiffness, " + _COMMON,
}
# workloads whose stored stiffness exceeds device memory: matrix-free operator
MATRIX_FREE_WORKLOADS = ("C5",)
# oracle samples: same geometry kind and degree as the workload, oracle-sized
SAMPLES = {"C3": ("C3-mid", "2x2x1 uneven quarter-annulus patches, p=4, element columns "
                            "4/6 x 4/6 x 4"),
           "C2": ("C2-mid", "3x3x3 jittered cube patches, p=3, 6^3 elements"),
           "C5": ("C5-small", "2x2x2 twisted-box patches, p=4, 3^3 elements")}


def workload_label(name):
    return WORKLOADS.get(name, name)


def sample_for(workload):
    return SAMPLES.get(workload, SAMPLES["C2"])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", default="tf32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--workload", default="C3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fd-only", action="store_true",
                    help="time only the FD local solvers (P_A^{-1} and the interior solves) "
                         "on a local-solvers-only context of --workload")
    ap.add_argument("--nrhs", type=int, default=8, help="batch size of the --fd-only batched line")
    ap.add_argument("--fd-slab", action="store_true",
                    help="--fd-only: send every tensor through the three-pass kernels")
    ap.add_argument("--precs", default="fp64,fp32,tf32,bf16", help="--fd-only: precisions to time")
    ap.add_argument("--plain-iters", type=int, default=6,
                    help="matrix-free workloads: iterations of the bounded plain FP64 run")
    ap.add_argument("--fd-fixed", action="store_true",
                    help="--fd-only: the fixed FD work split instead of the timed one")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(x, world, device="cuda"):
    """Max of a per-rank scalar over all ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Each rank solves its own right-hand side: body-force seed = rank."""
    return rank


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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
                 "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
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
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle arm
def oracle_sample_time(workload, steps=1, warmup=0):
    """Time the CPU oracle's complete AF-IETI solve on the bounded sample of
    `workload` (same geometry kind and degree, oracle-sized) and its
    per-iteration components on that sample.  Returns (measured seconds per
    sample solve, details); details["projection_s"] scales the sample to the
    workload by the DoF ratio (iteration counts of the method do not depend
    on h or H, Theorem 1, and the oracle's per-iteration work is linear in
    the DoF count), and is labelled as a projection wherever used."""
    import numpy as np
    import afi_workloads as W
    from oracle.ieti import AFIETI
    name, desc = sample_for(workload)
    t = time.time()
    P = W.config(name)
    s = AFIETI(P)
    s.assemble()
    s._local()
    f = s.load(W.body_force_coeffs(P))
    prep = time.time() - t
    n_full = W.config(workload).ndof
    times, iters = [], 0
    for i in range(warmup + steps):
        t0 = time.time()
        _, _, info = s.solve(f, tol=1e-8)
        if i >= warmup:
            times.append(time.time() - t0)
        iters = info["iters"]
    per = sum(times) / len(times)
    scale = n_full / s.ndof
    # per-iteration components on the sample (one of each, median of 5)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, s.ndof)
    lam = rng.uniform(-1, 1, s.nc)

    def med(fn):
        ts = []
        for _ in range(5):
            t0 = time.time()
            fn()
            ts.append(time.time() - t0)
        return sorted(ts)[2] * 1e3
    comp = {"stiffness_matvec_ms": med(lambda: s.A @ x),
            "fd_PA_inv_ms": med(lambda: s.PA_inv(x)),
            "P_S_ms": med(lambda: s.P_S(lam)),
            "saddle_op_ms": med(lambda: s.op(x, lam)),
            "preconditioner_ms": med(lambda: s.precond_apply(x, lam))}
    return per, {"sample": f"{name} ({desc}, {s.ndof} DoF, same geometry kind as {workload}): "
                           f"full oracle AF-IETI solve to 1e-8, {iters} iterations, "
                           f"{per:.2f} s measured",
                 "sample_name": name, "sample_dofs": s.ndof, "iterations": iters,
                 "prep_s": round(prep, 1), "sample_s": round(per, 3), "cores": _CORES,
                 "projection_s": round(per * scale, 3), "projection_scale": round(scale, 2),
                 "per_iteration_on_sample": {k: round(v, 2) for k, v in comp.items()}}


def oracle_fd_rate(workload="C2", max_tensors=12, seconds=3.0):
    """The CPU oracle's FD apply (Algorithm 1 by tensordot, FP64, the host's
    BLAS threads) on a bounded sample of the workload's (patch, component)
    tensors: DoF/s of P_A^{-1}, the same quantity as fd_apply_dofs_per_s."""
    import numpy as np
    import afi_workloads as W
    from oracle import fd as ofd
    P = W.config(workload)
    tensors = []
    for k in range(min(P.npatch, max_tensors)):
        p = int(P.degree[k])
        Ks, Ms = ofd.patch_1d(P.nel[k], p)
        U = [ofd.gen_eig(K, M)[1] for K, M in zip(Ks, Ms)]
        D = [ofd.gen_eig(K, M)[0] for K, M in zip(Ks, Ms)]
        lam, mu = P.lame[k]
        diag = ofd.Lambda(D, P.dim, 0, lam, mu, 1.0)
        r = np.random.default_rng(k).standard_normal(diag.shape)
        tensors.append((r, U, diag))
    dofs, t0, reps = 0, time.time(), 0
    while True:
        for r, U, diag in tensors:
            ofd.fd_solve(r, U, diag)
            dofs += r.size
        reps += 1
        if time.time() - t0 >= seconds:
            break
    el = time.time() - t0
    return {"value": round(dofs / el, 1), "unit": "DoF/s", "cores": _CORES, "kind": "oracle",
            "sample": f"{workload}: P_A^-1 FD (tensordot, FP64) on {len(tensors)} patch tensors, "
                      f"{reps} sweeps in {el:.1f} s"}


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the host cores.
    Each step is one complete oracle solve of the bounded sample of the
    workload, and the line reports that measured time; the DoF-scaled figure
    for the workload itself is a separate, labelled projection."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    per, det = oracle_sample_time(args.workload, steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": round(per, 3), "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(per * 1e3, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{det['sample_name']}: bounded sample of the {args.workload} "
                                   f"workload ({det['sample']})",
                       "same_config_as_gpu_line": False},
            "projection": {"value": det["projection_s"], "unit": "s",
                           "to": workload_label(args.workload),
                           "method": f"measured sample time x {det['projection_scale']} "
                                     f"(DoF ratio {args.workload} / sample; iteration counts are "
                                     "mesh- and patch-count independent)"},
            "per_iteration_ms": det["per_iteration_on_sample"],
            "cpu_baseline": {"value": round(per, 3), "unit": "s", "cores": det["cores"],
                             "kind": "oracle", "sample": det["sample"]},
            "e2e": {"value": round(per, 3), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- our arm
def pair_copy_bytes(prob):
    """Bytes of the row-compressed pair copy of the stencil (8 B per
    coefficient whose neighbour lies in its row, sub-planes padded to even)."""
    d = prob.dim
    total = 0
    for k in range(prob.npatch):
        p = int(prob.degree[k])
        ns = prob.n(k)
        rows = 1
        for n in ns[1:]:
            rows *= n
        stride = 0
        for o1 in range(2 * p + 1):
            sz = rows * (ns[0] - abs(o1 - p))
            stride += sz + (sz & 1)
        total += d * d * (2 * p + 1) ** (d - 1) * stride
    return 8 * total


def stencil_stats(prob):
    """Algorithmic FLOPs (2 per structural nonzero of A) and stored bytes
    (every stencil coefficient, 8 B, plus x and y) of one stiffness matvec."""
    d = prob.dim
    nnz, stored, ndof = 0, 0, 0
    for k in range(prob.npatch):
        p = int(prob.degree[k])
        ns = prob.n(k)
        rows = 1
        for n in ns:
            rows *= n * (2 * p + 1) - p * (p + 1)
        nnz += d * d * rows
        N = 1
        for n in ns:
            N *= n
        NP = N // ns[0] * (ns[0] + ns[0] % 2)     # rows padded to even length
        stored += d * d * (2 * p + 1) ** d * NP
        ndof += d * N
    return 2 * nnz, stored * 8 + 2 * ndof * 8


def traffic_record(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (lines `kernel@workload bytes source md5`), if it was taken on
    the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 3 and parts[0] == f"{kernel}@{workload}":
            src = os.path.join(ROOT, "paper_2001_09626_gb300", "csrc", parts[2])
            if len(parts) >= 4 and os.path.exists(src):
                h = hashlib.md5(open(src, "rb").read()).hexdigest()[:12]
                if h != parts[3]:
                    return None
            return float(parts[1])
    return None


def fp64_peak_tflops():
    """FP64 throughput of this GPU, measured in the run: cuBLAS DGEMM 4096^3
    through torch.matmul, best of 5 (the FP64 peak is not among the
    measured peaks)."""
    import torch
    n = 4096
    a = torch.rand(n, n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def dtype_label(prec, stencil_f64=False):
    stiff = "f64 stiffness" if stencil_f64 else "double-f32 stiffness (f32 pairs)"
    return f"mixed: f64 Krylov/residual/jumps, {prec} local solvers, {stiff} in the iterations"


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    import afi_workloads as W
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    prob = W.config(args.workload)
    coeffs = W.body_force_coeffs(prob, seed=replica_seed(rank))
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # ---- 1. the mixed form (the headline), its end-to-end form, eight
    # right-hand sides together, FD rates and the stiffness roofline
    t0 = time.time()
    s = Solver(prob, prec=args.prec, tol=1e-8, maxit=5000, use_graph=True)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    f = s.load_vector(coeffs)
    n_dof, n_c = s.n_dof, s.n_c
    for _ in range(args.warmup):
        s.solve(f)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    L0 = A.afi_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        u, lam = s.solve(f)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = (A.afi_kernel_launches() - L0) // args.steps
    clocks = sampler.stop()
    ms_solve = reduce_max(e0.elapsed_time(e1) / args.steps, world)
    info = dict(s.last_info)
    # one solve as the paper times INEXACT: MINRES plus the local-solver setup
    # (Algorithm 1 step 1: univariate matrices, eigensolves, operand tables)
    fd_setup_ms = reduce_max(float(info["t_fd_setup_ms"]), world)
    ms = ms_solve + fd_setup_ms

    # end to end through the C ABI with host buffers (pinned), copies timed
    f_h = f.cpu().pin_memory()
    u_h = torch.empty_like(f_h).pin_memory()
    f_d = torch.empty_like(f)
    u_d = torch.empty_like(f)
    lam_d = s.zeros(s.n_c)

    def e2e_step():
        f_d.copy_(f_h, non_blocking=True)
        A.ieti_solve(s.ctx, f_d, u_d, lam_d, 1)
        u_h.copy_(u_d, non_blocking=True)
    # secondary measurements: fewer repetitions when one solve takes seconds
    reps2 = max(1, min(args.steps, 3)) if ms < 3000 else 1
    e2e_step()
    barrier()
    ms_e2e = reduce_max(timed(e2e_step, args.steps if ms < 3000 else 2), world)
    del f_d, u_d, lam_d

    # the batched stiffness on eight vectors (its first call also picks the
    # launch width by timing)
    X8 = torch.rand(8, s.n_dof, dtype=torch.float64, device="cuda")
    Y8 = torch.empty_like(X8)
    for _ in range(2):
        A.afi_apply_batch(s.ctx, A.AFI_OP_STIFFNESS, X8, Y8, 8)
    mv8_ms = timed(lambda: A.afi_apply_batch(s.ctx, A.AFI_OP_STIFFNESS, X8, Y8, 8), 5)
    del X8, Y8
    # eight seeded right-hand sides solved together (lockstep MINRES, one
    # batched stiffness launch per iteration) against one at a time
    # (timed on its first call when a solve takes seconds: the one-time
    # capture of the batched iteration graph is then below 0.1% of it)
    F8 = torch.stack([s.load_vector(W.body_force_coeffs(prob, seed=100 + j)) for j in range(8)])
    if ms < 3000:
        s.solve(F8)
    ms_multi = timed(lambda: s.solve(F8), 1)
    info_multi = dict(s.last_info)
    del F8

    # FD apply throughput (P_A^{-1} on every patch and component), one
    # right-hand side and a batch of 8 in one launch
    r = torch.rand(s.n_dof, dtype=torch.float64, device="cuda")
    r8 = torch.rand(8, s.n_dof, dtype=torch.float64, device="cuda")
    fd_ms, fd8_ms = {}, {}
    for prec in ("fp64", args.prec):
        s.set_precision(prec)
        for _ in range(3):
            s.fd(r)
            s.fd(r8)
        fd_ms[prec] = timed(lambda: s.fd(r), 20)
        fd8_ms[prec] = timed(lambda: s.fd(r8), 10)
    s.set_precision(args.prec)
    del r, r8

    # dominant kernel: the iterations' double-FP32 stiffness matvec (x split,
    # then one stencil launch per apply), timed on the launching stream
    x = torch.rand(s.n_dof, dtype=torch.float64, device="cuda")
    for _ in range(3):
        s.apply(A.AFI_OP_STIFFNESS, x)
    mv_ms = timed(lambda: s.apply(A.AFI_OP_STIFFNESS, x), 20)
    s.close()
    del s
    torch.cuda.empty_cache()

    # ---- 2. the plain FP64 form, same right-hand side: FP64 local solvers
    # and the FP64 stiffness stencil (a second context, built after the
    # first is freed)
    s64 = Solver(prob, prec="fp64", tol=1e-8, maxit=5000, use_graph=True, stencil_f64=True)
    s64.solve(f)
    ms_plain = timed(lambda: s64.solve(f), reps2)
    info_plain = dict(s64.last_info)
    # the mixed solve with the FP64 stencil, for the effect of the stencil form
    s64.set_precision(args.prec)
    s64.solve(f)
    ms_mixed64 = timed(lambda: s64.solve(f), reps2)
    info_mixed64 = dict(s64.last_info)
    for _ in range(3):
        s64.apply(A.AFI_OP_STIFFNESS, x)
    mv64_ms = timed(lambda: s64.apply(A.AFI_OP_STIFFNESS, x), 20)
    s64.close()
    del s64
    torch.cuda.empty_cache()
    fp64_peak = fp64_peak_tflops()

    # ---- 3. the paper's geometry-inclusion local solvers (Section 5.2.3) on
    # the same problem and right-hand side: fit, tables and scalings are
    # local-solver setup and are counted in the solve time
    try:
        t0g = time.time()
        sg = Solver(prob, prec=args.prec, tol=1e-8, maxit=5000, use_graph=True, geo=True)
        torch.cuda.synchronize()
        setup_geo = time.time() - t0g
        sg.solve(f)
        ms_geo = timed(lambda: sg.solve(f), reps2)
        info_geo = dict(sg.last_info)
        sg.close()
        geometry_inclusion = {"solve_s": round((ms_geo + info_geo["t_fd_setup_ms"]) / 1e3, 4),
                              "iterations": info_geo["iters"], "relres_true": info_geo["relres_true"],
                              "fit_and_tables_s": round(info_geo["t_fd_setup_ms"] / 1e3, 4),
                              "setup_s": round(setup_geo, 3)}
    except A.AfiError as e:
        geometry_inclusion = {"skipped": str(e)}

    # ---- 4. the metric's own configuration, C5 (108 M DoF, stored stencil
    # 1.9 TB), on the matrix-free stiffness: its products and a bounded run of
    # the mixed iterations (the full solve is `--workload C5`)
    matrix_free_c5 = None
    if world == 1 and args.workload == "C3":
        try:
            matrix_free_c5 = matrix_free_probe(args, timed)
        except Exception as e:   # a failure here must not lose the headline line
            matrix_free_c5 = {"skipped": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()

    multi_rhs = {"nrhs": 8, "solve_s": round((ms_multi + fd_setup_ms) / 1e3, 4),
                 "per_rhs_s": round((ms_multi / 8 + fd_setup_ms) / 1e3, 4),
                 "iterations_max": info_multi["iters"], "relres_true_max": info_multi["relres_true"],
                 "one_at_a_time_s": round(8 * ms_solve / 1e3, 4),
                 "speedup_vs_one_at_a_time": round(8 * ms_solve / ms_multi, 3),
                 "stiffness_8_vectors_ms": round(mv8_ms, 3),
                 "stiffness_1_vector_ms": round(mv_ms, 4)}
    flops, stored_bytes = stencil_stats(prob)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # algorithmic bytes: 8 B per structural nonzero of A, x read, y written
    alg_bytes = 8 * (flops // 2) + 16 * n_dof
    gbs = alg_bytes / (mv_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs / hbm, 3), "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "traffic": traffic_record("k_stencil_mv_rows", args.workload),
                "kernel": "k_split_x + k_stencil_mv_rows<3,3> (double-FP32 stiffness matvec on the "
                          "row-compressed pair copy, bulk-copy pipeline)",
                "bytes_per_launch": alg_bytes, "launch_ms": round(mv_ms, 4),
                "pair_copy_bytes": pair_copy_bytes(prob),
                "fp64_stencil_bytes": stored_bytes,
                "fp64_form": {"kernel": "k_stencil_mv<3,3> (FP64 FMAs)", "launch_ms": round(mv64_ms, 4),
                              "TFLOPs": round(flops / (mv64_ms * 1e-3) / 1e12, 4),
                              "frac_of_fp64_peak": round(flops / (mv64_ms * 1e-3) / 1e12 / fp64_peak, 3),
                              "fp64_peak_tflops": round(fp64_peak, 3),
                              "fp64_peak_source": "cuBLAS DGEMM 4096^3 measured in this run "
                                                  "(not in MEASURED_PEAKS.json)",
                              "GBs": round(stored_bytes / (mv64_ms * 1e-3) / 1e9, 1)}}
    fd_bytes = 16 * n_dof
    fd_kernel = ("k_fd_tc / k_fd_plane + k_fd_line (tcgen05)" if args.prec in ("tf32", "bf16")
                 else "k_fd (SIMT)")
    roofline_fd = {"bound": "hbm", "kernel": f"{fd_kernel}, {args.prec}",
                   "achieved": round(fd_bytes / (fd_ms[args.prec] * 1e-3) / 1e9, 1),
                   "peak": hbm, "unit": "GB/s",
                   "frac": round(fd_bytes / (fd_ms[args.prec] * 1e-3) / 1e9 / hbm, 4),
                   "traffic": traffic_record("k_fd", args.workload),
                   "bytes_per_launch": fd_bytes,
                   "nrhs8": {"achieved": round(8 * fd_bytes / (fd8_ms[args.prec] * 1e-3) / 1e9, 1),
                             "frac": round(8 * fd_bytes / (fd8_ms[args.prec] * 1e-3) / 1e9 / hbm, 4),
                             "launch_ms": round(fd8_ms[args.prec], 4),
                             "traffic": (traffic_record("k_fd_nrhs8", args.workload)
                                         if args.prec == "tf32" else None)}}

    line = {"metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_label(args.prec), "data": "synthetic",
            "config": {"workload": workload_label(args.workload),
                       "n_dof": n_dof, "n_c": n_c,
                       "local_solver_precision": args.prec,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 ({pair_copy_bytes(prob) / 1e9:.1f} GB pair stencil "
                             "streamed each iteration)"},
            "iterations": info["iters"], "relres_true": info["relres_true"],
            "fp64_restarts": info["fp64_restarts"],
            "setup_s": round(setup_s, 3),
            "solve_s_without_fd_setup": round(ms_solve / 1e3, 4),
            "fd_setup_s": round(fd_setup_ms / 1e3, 4),
            "plain_fp64": {"solve_s": round((ms_plain + info_plain["t_fd_setup_ms"]) / 1e3, 4),
                           "form": "FP64 local solvers and FP64 stiffness stencil",
                           "iterations": info_plain["iters"],
                           "relres_true": info_plain["relres_true"]},
            "mixed_fp64_stencil": {"solve_s": round((ms_mixed64 + info_mixed64["t_fd_setup_ms"]) / 1e3, 4),
                                   "iterations": info_mixed64["iters"],
                                   "relres_true": info_mixed64["relres_true"]},
            "multi_rhs": multi_rhs, "geometry_inclusion": geometry_inclusion,
            "fd_apply_dofs_per_s": {k: round(n_dof / (v * 1e-3), 1) for k, v in fd_ms.items()},
            "fd_apply_dofs_per_s_nrhs8": {k: round(8 * n_dof / (v * 1e-3), 1)
                                          for k, v in fd8_ms.items()},
            "e2e": {"value": round((ms_e2e + fd_setup_ms) / 1e3, 4), "unit": "s",
                    "h2d_bytes_per_step": 8 * n_dof, "d2h_bytes_per_step": 8 * n_dof},
            "gpu_launches": int(launches), "roofline": roofline, "roofline_fd": roofline_fd,
            "clocks": clocks}
    if matrix_free_c5 is not None:
        line["matrix_free_C5"] = matrix_free_c5
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per, det = oracle_sample_time(args.workload, steps=1, warmup=0)
        line["cpu_baseline"] = {"value": det["projection_s"], "unit": "s", "cores": det["cores"],
                                "kind": "oracle", "projection": True,
                                "sample": det["sample"] + f"; value = sample time x "
                                          f"{det['projection_scale']} (DoF ratio to "
                                          f"{args.workload})",
                                "measured_sample_s": det["sample_s"],
                                "per_iteration_ms_on_sample": det["per_iteration_on_sample"]}
        line["cpu_baseline_fd"] = oracle_fd_rate(args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_fd_only(args):
    """FD-apply throughput on a local-solvers-only context (no stiffness, no
    constraints): DoF/s and the HBM roofline of the 16 B/DoF algorithmic
    traffic, for one right-hand side and a batch, every precision."""
    import torch
    import __graft_entry__ as g
    g.build()
    import afi_workloads as W
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config(args.workload)
    s = Solver(prob, prec=args.prec, tol=1e-8, local_only=True, fd_slab=args.fd_slab,
               fd_fixed=args.fd_fixed)
    stream = torch.cuda.current_stream()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    n_int = 0
    for k in range(prob.npatch):
        m = 1
        for n in prob.n(k):
            m *= n - 2
        n_int += prob.dim * m
    out = {}
    gen = torch.Generator(device="cuda").manual_seed(0)
    for prec in args.precs.split(","):
        s.set_precision(prec)
        row = {}
        for interior, n in ((False, s.n_dof), (True, n_int)):
            for nrhs in (1, args.nrhs):
                r = torch.rand((nrhs, n) if nrhs > 1 else (n,), dtype=torch.float64,
                               device="cuda", generator=gen)
                for _ in range(max(3, args.warmup)):
                    s.fd(r, interior=interior)
                ms = timed(lambda: s.fd(r, interior=interior), max(5, args.steps))
                dofs = nrhs * n
                row[f"{'interior' if interior else 'PA_inv'}_nrhs{nrhs}"] = {
                    "ms": round(ms, 4), "dofs_per_s": round(dofs / (ms * 1e-3), 1),
                    "GBs": round(16 * dofs / (ms * 1e-3) / 1e9, 1),
                    "frac_hbm": round(16 * dofs / (ms * 1e-3) / 1e9 / hbm, 4)}
        out[prec] = row
    line = {"metric": "FD-apply DoF/s", "unit": "DoF/s", "workload": args.workload,
            "path": ("three-pass (forced)" if args.fd_slab else
                     ("fixed split" if args.fd_fixed else "timed split")),
            "n_dof": s.n_dof, "n_int": n_int, "hbm_peak_GBs": hbm, "fd": out}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_fd_rate(args.workload)
    print(json.dumps(line), flush=True)
    s.close()


def mf_flops_per_element(p):
    """FLOPs of one element in the matrix-free stiffness kernel, as it runs
    (k_mf in csrc/mf.cu): six fields through three forward direction passes
    (2 + 3 + 3 table contractions of (p+1)^4 FMAs each), three components
    through three back passes (3 + 3 + 2), two FLOPs per FMA, plus the
    pointwise Jacobian inverse, stress and flux (168 FLOPs per Gauss point)."""
    nb = p + 1
    return 2 * (6 * 8 + 3 * 8) * nb ** 4 + 168 * nb ** 3


def fp32_peak_tflops(sm_mhz=2070.0, sms=152):
    """FP32 FMA peak from the unit counts: 128 FP32 lanes per SM, 2 FLOPs
    per FMA, at the given SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def matrix_free_probe(args, timed, iters=12):
    """C5 on the matrix-free stiffness, within the default run's budget: the
    FP32 and FP64 products (the FP32 one against the FP32 rate from the unit
    counts) and a bounded run of `iters` mixed MINRES iterations, whose time
    less its final FP64 true residual gives the time per iteration."""
    import numpy as np
    import torch
    import afi_workloads as W
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config("C5")
    p = int(prob.degree[0])
    ne = sum(int(np.prod(prob.nel[k])) for k in range(prob.npatch))
    t0 = time.time()
    s = Solver(prob, prec=args.prec, tol=1e-8, maxit=iters, use_graph=True, matrix_free=True)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    try:
        x = torch.rand(s.n_dof, dtype=torch.float64, device="cuda")
        s.apply(A.AFI_OP_STIFFNESS, x)
        mv_ms = timed(lambda: s.apply(A.AFI_OP_STIFFNESS, x), 3)
        f = s.load_vector(W.body_force_coeffs(prob))
        s.solve(f, allow_not_converged=True)
        ms_run = timed(lambda: s.solve(f, allow_not_converged=True), 1)
        info = dict(s.last_info)
    finally:
        s.close()
    torch.cuda.empty_cache()
    s64 = Solver(prob, prec="fp64", tol=1e-8, maxit=iters, matrix_free=True, stencil_f64=True)
    try:
        x = torch.rand(s64.n_dof, dtype=torch.float64, device="cuda")
        mv64_ms = timed(lambda: s64.apply(A.AFI_OP_STIFFNESS, x), 1)
    finally:
        s64.close()
    flops = mf_flops_per_element(p) * ne
    peak = fp32_peak_tflops(2070.0)
    achieved = flops / (mv_ms * 1e-3) / 1e12
    return {"workload": workload_label("C5"), "n_dof": int(prob.ndof), "setup_s": round(setup_s, 2),
            "fp32_product_ms": round(mv_ms, 2), "fp64_product_ms": round(mv64_ms, 1),
            "bounded_run": {"iterations": info["iters"], "ms": round(ms_run, 1),
                            "per_iteration_ms": round(max(0.0, info["t_solve_ms"] - mv64_ms)
                                                      / max(1, info["iters"]), 2),
                            "method": "mixed MINRES (TF32 local solvers, FP32 products, CUDA "
                                      "graph) capped at the iteration count, less its final "
                                      "FP64 true residual; the full solve is bench.py "
                                      "--workload C5"},
            "roofline": {"bound": "alu", "kernel": f"k_mf<float,{p}>", "achieved": round(achieved, 2),
                         "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                         "peak_source": "FP32 FMA peak from the unit counts (152 SMs x 128 lanes "
                                        "x 2 FLOP x 2070 MHz), not measured",
                         "flops_per_launch": flops, "traffic": None}}


def run_matrix_free(args):
    """The metric's own configuration on the matrix-free operator (C5: 256
    twisted-box patches, p = 4, 48^3 elements, 108 M DoF; the stored stencil
    would need 1.9 TB).  One step = one complete solve of one seeded
    right-hand side: MINRES with TF32 local solvers and FP32 matrix-free
    products, refined against the FP64 true residual to 1e-8, plus the
    local-solver setup.  Beside it: the plain FP64 form's per-iteration time
    on a bounded run (its full solve would take tens of minutes, so its solve
    time is a labelled projection), eight right-hand sides (solved one after
    the other: a labelled projection), FD rates and the roofline of the
    FP32 matrix-free kernel (FP32-pipe bound)."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import afi_workloads as W
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    torch.cuda.set_device(0)
    prob = W.config(args.workload)
    p = int(prob.degree[0])
    ne = sum(int(np.prod(prob.nel[k])) for k in range(prob.npatch))
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t0 = time.time()
    s = Solver(prob, prec=args.prec, tol=1e-8, maxit=5000, use_graph=True, matrix_free=True)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    f = s.load_vector(W.body_force_coeffs(prob))
    n_dof, n_c = s.n_dof, s.n_c
    for _ in range(args.warmup):
        s.solve(f)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    L0 = A.afi_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        u, lam = s.solve(f)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = (A.afi_kernel_launches() - L0) // args.steps
    clocks = sampler.stop()
    ms_solve = e0.elapsed_time(e1) / args.steps
    info = dict(s.last_info)
    fd_setup_ms = float(info["t_fd_setup_ms"])
    ms = ms_solve + fd_setup_ms
    # end to end through the C ABI with pinned host buffers
    f_h = f.cpu().pin_memory()
    u_h = torch.empty_like(f_h).pin_memory()
    f_d, u_d, lam_d = torch.empty_like(f), torch.empty_like(f), s.zeros(s.n_c)

    def e2e_step():
        f_d.copy_(f_h, non_blocking=True)
        A.ieti_solve(s.ctx, f_d, u_d, lam_d, 1)
        u_h.copy_(u_d, non_blocking=True)
    ms_e2e = timed(e2e_step, 1)
    del f_d, u_d, lam_d
    # the FP32 matrix-free product (dominant kernel) and the FD rates
    x = torch.rand(n_dof, dtype=torch.float64, device="cuda")
    for _ in range(2):
        s.apply(A.AFI_OP_STIFFNESS, x)
    mv_ms = timed(lambda: s.apply(A.AFI_OP_STIFFNESS, x), 5)
    r8 = torch.rand(8, n_dof, dtype=torch.float64, device="cuda")
    fd_ms, fd8_ms = {}, {}
    for prec in ("fp64", args.prec):
        s.set_precision(prec)
        for _ in range(2):
            s.fd(x)
            s.fd(r8)
        fd_ms[prec] = timed(lambda: s.fd(x), 10)
        fd8_ms[prec] = timed(lambda: s.fd(r8), 5)
    s.set_precision(args.prec)
    del r8
    s.close()
    del s
    torch.cuda.empty_cache()
    # the plain FP64 form (FP64 local solvers, FP64 matrix-free products):
    # a bounded run of its iterations, per-iteration time measured
    s64 = Solver(prob, prec="fp64", tol=1e-8, maxit=args.plain_iters, use_graph=True,
                 matrix_free=True, stencil_f64=True)
    s64.solve(f, allow_not_converged=True)
    ms_plain_run = timed(lambda: s64.solve(f, allow_not_converged=True), 1)
    info_plain = dict(s64.last_info)
    for _ in range(1):
        s64.apply(A.AFI_OP_STIFFNESS, x)
    mv64_ms = timed(lambda: s64.apply(A.AFI_OP_STIFFNESS, x), 2)
    s64.close()
    del s64, x
    torch.cuda.empty_cache()
    # the bounded run also takes one FP64 true residual after its last
    # iteration: one FP64 product, taken out of the per-iteration time
    plain_iter_ms = max(0.0, info_plain["t_solve_ms"] - mv64_ms) / max(1, info_plain["iters"])
    fp64_peak = fp64_peak_tflops()
    flops = mf_flops_per_element(p) * ne
    clock = float(clocks.get("sm_mhz") or 2070.0) if isinstance(clocks, dict) else 2070.0
    fp32_peak = fp32_peak_tflops(2070.0)
    achieved = flops / (mv_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(fp32_peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4),
                "peak_source": "FP32 FMA peak from the unit counts: 152 SMs x 128 lanes x 2 FLOP "
                               "x 2070 MHz (not measured)",
                "traffic": None,
                "kernel": f"k_mf<float,{p}> (matrix-free FP32 stiffness: element-wise sum "
                          "factorisation, Jacobian from the control points), with its FP64->FP32 "
                          "input and FP32->FP64 output passes",
                "flops_per_launch": flops, "flops_per_element": mf_flops_per_element(p),
                "elements": ne, "launch_ms": round(mv_ms, 3),
                "sm_mhz_median_in_solve": clock,
                "fp64_form": {"kernel": f"k_mf<double,{p}>", "launch_ms": round(mv64_ms, 2),
                              "TFLOPs": round(flops / (mv64_ms * 1e-3) / 1e12, 4),
                              "frac_of_fp64_peak": round(flops / (mv64_ms * 1e-3) / 1e12 / fp64_peak, 3),
                              "fp64_peak_tflops": round(fp64_peak, 3),
                              "fp64_peak_source": "cuBLAS DGEMM 4096^3 measured in this run"}}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    fd_bytes = 16 * n_dof
    roofline_fd = {"bound": "hbm", "kernel": f"k_fd_plane + k_fd_line (tcgen05), {args.prec}",
                   "achieved": round(fd_bytes / (fd_ms[args.prec] * 1e-3) / 1e9, 1), "peak": hbm,
                   "unit": "GB/s", "frac": round(fd_bytes / (fd_ms[args.prec] * 1e-3) / 1e9 / hbm, 4),
                   "traffic": None, "bytes_per_launch": fd_bytes,
                   "nrhs8": {"achieved": round(8 * fd_bytes / (fd8_ms[args.prec] * 1e-3) / 1e9, 1),
                             "frac": round(8 * fd_bytes / (fd8_ms[args.prec] * 1e-3) / 1e9 / hbm, 4),
                             "launch_ms": round(fd8_ms[args.prec], 4)}}
    line = {"metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": f"mixed: f64 Krylov/residual/jumps, {args.prec} local solvers, "
                     "f32 matrix-free stiffness in the iterations (refined against the f64 "
                     "matrix-free true residual)",
            "data": "synthetic",
            "config": {"workload": workload_label(args.workload), "n_dof": n_dof, "n_c": n_c,
                       "local_solver_precision": args.prec, "stiffness": "matrix-free",
                       "parallelism": "single GPU",
                       "l2": "inputs larger than L2 (108 M DoF: 0.86 GB per vector; every "
                             "product reads the control points and the input)"},
            "iterations": info["iters"], "relres_true": info["relres_true"],
            "refinement_runs": info["fp64_restarts"], "setup_s": round(setup_s, 3),
            "solve_s_without_fd_setup": round(ms_solve / 1e3, 4),
            "fd_setup_s": round(fd_setup_ms / 1e3, 4),
            "plain_fp64": {"form": "FP64 local solvers and FP64 matrix-free products",
                           "measured_iterations": info_plain["iters"],
                           "measured_s": round(ms_plain_run / 1e3, 3),
                           "per_iteration_ms": round(plain_iter_ms, 2),
                           "projection": True,
                           "solve_s": round((plain_iter_ms * info["iters"] +
                                             info_plain["t_fd_setup_ms"]) / 1e3, 2),
                           "method": "(bounded FP64 run - one FP64 product for its final true "
                                     "residual) / its iterations, x the mixed solve's iteration "
                                     "count"},
            "multi_rhs": {"nrhs": 8, "projection": True,
                          "solve_s": round(8 * ms_solve / 1e3 + fd_setup_ms / 1e3, 2),
                          "method": "matrix-free products share no coefficient stream: eight "
                                    "solves one after the other, 8 x the measured solve"},
            "fd_apply_dofs_per_s": {k: round(n_dof / (v * 1e-3), 1) for k, v in fd_ms.items()},
            "fd_apply_dofs_per_s_nrhs8": {k: round(8 * n_dof / (v * 1e-3), 1)
                                          for k, v in fd8_ms.items()},
            "e2e": {"value": round((ms_e2e + fd_setup_ms) / 1e3, 4), "unit": "s",
                    "h2d_bytes_per_step": 8 * n_dof, "d2h_bytes_per_step": 8 * n_dof},
            "gpu_launches": int(launches), "roofline": roofline, "roofline_fd": roofline_fd,
            "clocks": clocks}
    if not args.no_cpu_baseline:
        per, det = oracle_sample_time(args.workload, steps=1, warmup=0)
        line["cpu_baseline"] = {"value": det["projection_s"], "unit": "s", "cores": det["cores"],
                                "kind": "oracle", "projection": True,
                                "sample": det["sample"] + f"; value = sample time x "
                                          f"{det['projection_scale']} (DoF ratio to "
                                          f"{args.workload})",
                                "measured_sample_s": det["sample_s"],
                                "per_iteration_ms_on_sample": det["per_iteration_on_sample"]}
        line["cpu_baseline_fd"] = oracle_fd_rate(args.workload)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.fd_only:
        run_fd_only(args)
    elif args.workload in MATRIX_FREE_WORKLOADS:
        run_matrix_free(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
