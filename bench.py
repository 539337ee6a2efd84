"""Benchmark: Calderón-preconditioned PMCHWT solves on one GB300 (or N replicas).

Workload (default): dielectric sphere of radius 1, icosphere with 5120
triangles (7680 RWG/BC functions, 15360 PMCHWT unknowns), k_e = 5,
eps_r = 3.17 + 0.01i, x-polarised plane wave along +z; A on RWG with the
paper's default quadrature orders (q_near, q_medium, q_far, q_singular) =
(4, 3, 2, 6): 36 / 16 / 9 evaluations per regular pair by its near / medium /
far class and order-4 Sauter–Schwab singular rules; the full block-diagonal
Calderón preconditioner D on the barycentric mesh (dense, same rules);
FP32-bulk assembly and complex64 matvecs with FP64 GMRES recurrences and FP64
iterative refinement, tol 1e-5, restart 200.

One step = one complete solve through the C ABI (spaces, assembly of A and P,
Gram matrix, right-hand side, GMRES, far field on 362 directions). The FP64
GPU path is timed on the same workload for comparison, and the FP32 far field
is compared against it. With --gpus N (torchrun) every rank solves its own
replica of the workload: there is no exchange step.

--impl reference times the CPU oracle (plain FP64, test infrastructure) on a
bounded sample of the same workload and extrapolates to solves/s.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"name": "sphere5120_k5_D_dense", "level": 4, "k": 5.0, "eps": 3.17 + 0.01j,
            "tol": 1e-5, "restart": 200, "q_regular": 0}
# regular rules of every workload: 0 = near / medium / far classes at the paper's
# default orders (4, 3, 2); 6 = the 6-point rule for every regular pair
Q = dict(q_regular_A=0, q_regular_P=0)
METRIC = "PMCHWT solves/s (FP32 bulk, full Calderon D, 5120-triangle sphere, k=5)"
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the float32 BC-pair
# kernel (exterior pass of the workload) from one ncu capture; None once the kernel
# has changed since the counters were taken
BC_TILE_TRAFFIC = 4.253343e9 + 3.534395e9


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def _alu_peak(n_sm, sm_max_mhz):
    """Point-pair evaluations/s bound of the FP32 pipe for the regular rule.

    Per evaluation the formulation needs 42 FP32 instructions (distance 6,
    phase and Cody–Waite reduction 5, amplitude and G 4, g 7, weights 4,
    moment sums 16) and 3 XU instructions (rsqrt, sin, cos); an SM issues
    128 FP32 and 16 XU thread-instructions per clock, so the FP32 pipe binds:
    128/42 = 3.05 evaluations per SM clock.
    """
    per_sm_clk = min(128.0 / 42.0, 16.0 / 3.0)
    return per_sm_clk * n_sm * sm_max_mhz * 1e6


def max_over_ranks(vals):
    """Each value's maximum over the ranks of the process group (the values
    themselves without one). The tensor lives where the backend reduces: on
    the rank's GPU for NCCL, on the host for gloo."""
    import torch
    import torch.distributed as tdist
    vals = [float(v) for v in vals]
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return vals
    dev = torch.device("cuda", torch.cuda.current_device()) if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def run_ours(args, rank, world):
    import torch

    from paper_2008_04772_gb300 import build as libbuild
    from paper_2008_04772_gb300 import cal, meshgen

    libbuild.build()
    dev = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)
    L = cal.lib()
    ctx = cal.Context(dev)
    stream = torch.cuda.ExternalStream(L.cal_ctx_stream(ctx.h), device=dev)
    W = WORKLOAD
    m = meshgen.icosphere(W["level"])
    inc = meshgen.plane_wave_x_along_z()
    dirs = meshgen.sphere_cut_directions(181)
    opts32 = cal.solve_opts(precond="D", precision=cal.FP32, tol=W["tol"], restart=W["restart"], **Q)
    opts64 = cal.solve_opts(precond="D", precision=cal.FP64, tol=W["tol"], restart=W["restart"], **Q)
    opts32all = cal.solve_opts(precond="D", precision=cal.FP32_ALL, tol=W["tol"], restart=W["restart"], **Q)

    def one_step(opts, mesh=None, e2e=False):
        """One solve; returns (solution info, far field). e2e: mesh from host arrays each step."""
        if e2e:
            mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
        sol = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], inc, opts=opts)
        F = sol.far_field(dirs)
        return sol.info(), F

    mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    for _ in range(args.warmup):
        one_step(opts32, mesh)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
    # timed region: K device-timed steps (inputs resident: mesh created before)
    L.cal_profile_enable(1)
    n0 = L.cal_kernel_launches()
    lat = []
    infos = []
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            info, F32 = one_step(opts32, mesh)
            ev1.record(stream)
            ev1.synchronize()
            lat.append(ev0.elapsed_time(ev1))
            infos.append(info)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t0
    if dist:
        tdist.barrier()
    n_launch = L.cal_kernel_launches() - n0
    prof = {}
    for name in ("bc_tile", "rwg_regular", "singular", "pair_gemv", "bicgstab", "gram"):
        import ctypes
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        u = ctypes.c_double()
        L.cal_profile_read(name.encode(), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(u))
        prof[name] = {"launches": n.value, "ms": ms.value, "units": u.value}
    L.cal_profile_enable(0)
    t_dev, t_wall = max_over_ranks([sum(lat) / 1e3, t_wall])
    # e2e through host buffers: mesh arrays in, far field out, every step
    t_e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        a = time.perf_counter()
        one_step(opts32, e2e=True)
        torch.cuda.synchronize()
        t_e2e.append(time.perf_counter() - a)
    # FP64 GPU path on the same workload, and the FP32 vs FP64 far-field error
    a = time.perf_counter()
    info64, F64 = one_step(opts64, mesh)
    t64 = time.perf_counter() - a
    err = float(np.linalg.norm(F32 - F64) / np.linalg.norm(F64))
    # the same comparison with the stopping error taken out: a converged float64
    # solve (tol 1e-10) against float32 bulk at tol 1e-5 and at tol 1e-9
    _, F64c = one_step(cal.solve_opts(precond="D", precision=cal.FP64, tol=1e-10, restart=W["restart"],
                                      maxit=2000, **Q), mesh)
    _, F32c = one_step(cal.solve_opts(precond="D", precision=cal.FP32, tol=1e-9, restart=W["restart"],
                                      maxit=2000, **Q), mesh)
    rel_c = lambda F: float(np.linalg.norm(F - F64c) / np.linalg.norm(F64c))  # noqa: E731
    err_detail = {"fp32_tol1e-5_vs_converged_fp64": rel_c(F32), "fp64_tol1e-5_vs_converged_fp64": rel_c(F64),
                  "fp32_tol1e-9_vs_converged_fp64": rel_c(F32c),
                  "note": "at tol 1e-5 both solves carry their GMRES stopping error (~1e-5..1e-4); "
                          "the float32 floor is the tol-1e-9 line"}
    # variant: float32 singular pairs as well
    one_step(opts32all, mesh)
    torch.cuda.synchronize()
    a = time.perf_counter()
    reps = max(1, min(args.steps, 3))
    for _ in range(reps):
        info_all, F32all = one_step(opts32all, mesh)
    t_all = (time.perf_counter() - a) / reps
    err_all = float(np.linalg.norm(F32all - F64) / np.linalg.norm(F64))
    if rank != 0:
        return None
    info = infos[-1]
    ms_step = 1e3 * t_dev / args.steps
    value = world * args.steps / t_dev
    N = int(info.n_unknowns)
    entries = 2 * (N // 2) ** 2 * 2 * 2   # S, C at k_e and k_m on RWG and on BC (dense D)
    bc = prof["bc_tile"]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = _measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    achieved = bc["units"] / (bc["ms"] / 1e3) if bc["ms"] > 0 else 0.0
    peak = _alu_peak(n_sm, sm_max)
    clocks = clk.summary()
    h2d = m.verts.nbytes + m.tris.nbytes + m.domain.nbytes + inc.nbytes
    d2h = int(np.prod(F32.shape)) * 16
    out = {
        "metric": "PMCHWT solves/s",
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 bulk (singular static sums and refinement residuals in double-float, GMRES recurrences f64)",
        "data": "synthetic (seeded icosphere, plane wave)",
        "config": {"workload": W["name"], "triangles": int(len(m.tris)), "unknowns": N,
                   "k_ext": W["k"], "eps_r": [W["eps"].real, W["eps"].imag],
                   "preconditioner": "D (full block-diagonal Calderon, dense BC)",
                   "rules": "A and P: paper default orders (4,3,2,6): regular 6/4/3-point rules by "
                            "near/medium/far class (relative distance 2, 4), Sauter-Schwab 4^4 singular",
                   "tol": W["tol"], "restart": W["restart"], "parallelism": f"replicas{world}",
                   "l2": "working set > L2 (each step writes ~2.4 GB of operators)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "iterations": int(info.iterations),
        "matvecs": int(info.matvecs),
        "phase_s": {"setup": info.t_setup, "assemble_A": info.t_assemble_A,
                    "assemble_P": info.t_assemble_P, "solve": info.t_solve},
        "entries_per_s": entries / (ms_step / 1e3),
        "fp64_gpu": {"solves_per_s": 1.0 / t64, "iterations": int(info64.iterations)},
        "err_farfield_fp32_vs_fp64": err,
        "err_detail": err_detail,
        "fp32_all_variant": {"solves_per_s": 1.0 / t_all, "err_farfield_vs_fp64": err_all,
                             "iterations": int(info_all.iterations),
                             "note": "singular pairs also in float32 (CAL_FP32_ALL)"},
        "gpu_launches": int(n_launch),
        "kernels_ms": {k: v["ms"] / args.steps for k, v in prof.items()},
        "roofline": {"bound": "alu", "kernel": "bc_owner_kernel<0,128,true>",
                     "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Geval/s",
                     "frac": achieved / peak if peak else None, "traffic": BC_TILE_TRAFFIC,
                     "traffic_note": "dram read+write bytes of one exterior launch, one ncu capture; "
                                     "the per-launch work is "
                                     f"{bc['units'] / max(bc['launches'], 1) / 1e9:.1f} G evaluations",
                     "peak_source": f"derived: {n_sm} SMs x 3.05 eval/clk x {sm_max:.0f} MHz"},
        "clocks": clocks,
        "e2e": {"value": 1.0 / statistics.median(t_e2e), "unit": "solves/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
    }
    if args.multirhs:
        out["multi_rhs"] = run_multirhs(dev)
    if args.matrix_free:
        out["matrix_free_vs_stored"] = run_matrix_free(dev)
    if args.serving:
        out["serving"] = run_serving(dev)
    if args.variants:
        out["preconditioners"] = run_variants(dev, dirs)
    if args.table2:
        out["three_cubes_table2"] = run_table2(dev)
    if args.near_field:
        out["near_field"] = run_near_field(dev)
    if args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample)
    return out


# Preconditioner variants of the headline sphere (full vs reduced vs near-field-only,
# and the bi-parametric cheaper rules for P of Section 3.2): name, options
VARIANTS = [
    ("none", dict(precond="none", maxit=2000, **Q)),
    ("D", dict(precond="D", **Q)),
    ("D_uniform6", dict(precond="D", q_regular_A=6, q_regular_P=6)),
    ("De", dict(precond="De", **Q)),
    ("Di", dict(precond="Di", **Q)),
    ("Se", dict(precond="Se", **Q)),
    ("Si", dict(precond="Si", **Q)),
    ("Di_near2h", dict(precond="Di", near_cutoff_P=2.0, **Q)),
    ("Di_near4h", dict(precond="Di", near_cutoff_P=4.0, **Q)),
    ("Si_near2h_bp_q11", dict(precond="Si", near_cutoff_P=2.0, q_regular_A=0, q_regular_P=1, q_singular_P=1)),
    ("Si_near4h_bp_q11", dict(precond="Si", near_cutoff_P=4.0, q_regular_A=0, q_regular_P=1, q_singular_P=1)),
    ("D_bp_q11", dict(precond="D", q_regular_A=0, q_regular_P=1, q_singular_P=1)),
    ("Si_near0_bp_q11", dict(precond="Si", near_cutoff_P=0.0, q_regular_A=0, q_regular_P=1, q_singular_P=1)),
]


def run_variants(dev, dirs):
    """Every preconditioner of the headline workload: solves/s (median of 3 solves
    after one warm-up), GMRES iterations, stored P bytes and assembly times, and the
    float32 error of each: against the float64 GPU solve with the same
    preconditioner and tolerance, and its floor (float32 at tol 1e-9) against a
    converged float64 solve (tol 1e-10; the discrete solution does not depend on
    the preconditioner)."""
    import ctypes

    import torch

    from paper_2008_04772_gb300 import cal, meshgen
    W = WORKLOAD
    L = cal.lib()
    ctx = cal.Context(dev)
    m = meshgen.icosphere(W["level"])
    mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    inc = meshgen.plane_wave_x_along_z()
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
    conv = {}  # converged float64 far field per rule of A (the discrete solution's only dependence)

    def converged(qa):
        if qa not in conv:
            conv[qa] = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], inc, opts=cal.solve_opts(
                precond="D", precision=cal.FP64, tol=1e-10, restart=W["restart"], maxit=2000, q_regular_A=qa,
                q_regular_P=0)).far_field(dirs)[0]
        return conv[qa]
    out = {"workload": W["name"],
           "reference": "err_fp32_vs_fp64: float64 GPU solve with the same preconditioner and tol 1e-5; "
                        "fp32_floor: float32 at tol 1e-9 against a converged float64 solve (tol 1e-10) with the "
                        "same rules for A; err_vs_converged: the timed float32 solve (tol 1e-5) against it",
           "rules": "q_regular 0 = near/medium/far classes at the paper's default orders (4,3,2) for A and P, "
                    "6 = the 6-point rule for all regular pairs (D_uniform6), bi-parametric P (1, 1) (the *_bp_q11 lines)"}
    for name, o in VARIANTS:
        opts = cal.solve_opts(precision=cal.FP32, tol=W["tol"], restart=W["restart"], **o)
        ts = []
        for rep in range(4):
            if rep == 3:
                L.cal_profile_enable(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], inc, opts=opts, allow_not_converged=True)
            F = sol.far_field(dirs)
            torch.cuda.synchronize()
            if rep:
                ts.append(time.perf_counter() - t0)
        fam = {}
        for kn in ("bc_tile", "rwg_regular", "singular", "pair_gemv", "pair_spmv", "bicgstab", "gmres_cgs"):
            n_, ms_, u_ = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            L.cal_profile_read(kn.encode(), ctypes.byref(n_), ctypes.byref(ms_), ctypes.byref(u_))
            if n_.value:
                fam[kn] = round(ms_.value, 3)
        L.cal_profile_enable(0)
        info = sol.info()
        o64 = dict(o, precision=cal.FP64, tol=W["tol"], restart=W["restart"])
        F64 = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], inc, opts=cal.solve_opts(**o64),
                               allow_not_converged=True).far_field(dirs)
        Fc = converged(o.get("q_regular_A", 0))
        res = {"solves_per_s": 1.0 / statistics.median(ts), "iterations": int(info.iterations),
               "converged": int(info.converged), "bytes_P_mb": info.bytes_P / 1e6,
               "assemble_P_s": info.t_assemble_P, "solve_s": info.t_solve,
               "err_fp32_vs_fp64": rel(F[0], F64[0]), "err_vs_converged": rel(F[0], Fc), "kernels_ms": fam}
        if info.converged:  # the floor of a solve that stops at maxit says nothing about float32
            o9 = dict(o, precision=cal.FP32, tol=1e-9, restart=W["restart"], maxit=2000)
            F9 = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], inc, opts=cal.solve_opts(**o9),
                                  allow_not_converged=True).far_field(dirs)
            res["fp32_floor"] = rel(F9[0], Fc)
        out[name] = res
    return out


MULTI_RHS = {"name": "aggregate8x2500_kD20_Di_near2h_32rhs", "prisms": 8, "tris_per_prism": 2500, "seed": 0,
             "k": 20.0, "eps": 3.17 + 0.01j, "nrhs": 32, "precond": "Di", "near_cutoff_P": 2.0, "tol": 1e-5}


def run_multirhs(dev):
    """The 32-direction aggregate: FP32-bulk solve whose GMRES applies the stored
    blocks to all 32 columns at once through the tcgen05 3xTF32 product."""
    import ctypes

    import torch

    from paper_2008_04772_gb300 import cal, meshgen
    W = MULTI_RHS
    L = cal.lib()
    ctx = cal.Context(dev)
    m = meshgen.prism_aggregate(W["prisms"], W["tris_per_prism"], seed=W["seed"], diameter=1.0, gap=0.05)
    mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    d = meshgen.fibonacci_directions(W["nrhs"])
    inc = np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)
    opts = cal.solve_opts(precond=W["precond"], precision=cal.FP32, tol=W["tol"], near_cutoff_P=W["near_cutoff_P"], **Q)
    L.cal_profile_enable(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sol = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], inc, opts=opts)
    sol.far_field(meshgen.fibonacci_directions(64))
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    fam = {}
    for name in ("gemm_tc", "pair_gemv", "pair_spmv", "bicgstab", "gmres_cgs", "bc_tile", "rwg_regular", "singular"):
        n_, ms_, u_ = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        L.cal_profile_read(name.encode(), ctypes.byref(n_), ctypes.byref(ms_), ctypes.byref(u_))
        fam[name] = {"launches": n_.value, "ms": round(ms_.value, 3)}
    n, ms, u = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    L.cal_profile_read(b"gemm_tc", ctypes.byref(n), ctypes.byref(ms), ctypes.byref(u))
    L.cal_profile_enable(0)
    info = sol.info()
    peaks = _measured_peaks()
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25  # nominal dense TF32 / BF16 ratio
    achieved = u.value / (ms.value / 1e3) / 1e12 if ms.value > 0 else 0.0
    N = int(info.n_unknowns) // 2
    return {
        "workload": W["name"], "triangles": int(len(m.tris)), "unknowns": int(info.n_unknowns),
        "k_ext": W["k"], "nrhs": W["nrhs"], "preconditioner": f"{W['precond']} near-field {W['near_cutoff_P']}h",
        "seconds": t, "solves_per_s": W["nrhs"] / t, "iterations": int(info.iterations),
        "phase_s": {"setup": info.t_setup, "assemble_A": info.t_assemble_A, "assemble_P": info.t_assemble_P,
                    "solve": info.t_solve},
        "bytes_A_gb": info.bytes_A / 1e9, "bytes_P_gb": info.bytes_P / 1e9,
        "gemm_tc": {"launches": n.value, "ms": ms.value,
                    "roofline": {"bound": "tensor", "achieved": achieved, "peak": tf32_peak, "unit": "TFLOP/s",
                                 "frac": achieved / tf32_peak,
                                 "flops": "executed TF32 flops, 3 products x 2 M K NB per launch",
                                 "peak_source": "measured bf16 burst x 1.1/2.25 (nominal TF32/BF16)"}},
        "columns_N": N,
        "kernels": fam,
    }


MATRIX_FREE = {"name": "aggregate8x4000_kD40_Di_near3h", "prisms": 8, "tris_per_prism": 4000, "seed": 0,
               "k": 40.0, "eps": 3.17 + 0.01j, "precond": "Di", "near_cutoff_P": 3.0, "tol": 1e-5}


def run_matrix_free(dev):
    """The largest single-GPU aggregate (8 prisms, ~32k triangles, ~96k unknowns,
    kD = 40): stored dense complex64 A versus matrix-free A, the same FP32-bulk
    solve with float64 refinement both ways, the time per operator application,
    the HBM fraction of the stored product and the ALU fraction of the
    matrix-free kernel, and the far-field difference between the two."""
    import ctypes

    import torch

    from paper_2008_04772_gb300 import cal, meshgen
    W = MATRIX_FREE
    L = cal.lib()
    ctx = cal.Context(dev)
    m = meshgen.prism_aggregate(W["prisms"], W["tris_per_prism"], seed=W["seed"], diameter=1.0, gap=0.05)
    mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    inc = meshgen.plane_wave_x_along_z()
    dirs = meshgen.fibonacci_directions(64)
    out = {"workload": W["name"], "triangles": int(len(m.tris)), "unknowns": 2 * mesh.info().n_edges,
           "k_ext": W["k"], "preconditioner": f"{W['precond']} near-field {W['near_cutoff_P']}h"}
    far = {}
    for free in (0, 1):
        opts = cal.solve_opts(precond=W["precond"], precision=cal.FP32, tol=W["tol"],
                              near_cutoff_P=W["near_cutoff_P"], matrix_free=free, **Q)
        L.cal_profile_enable(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], inc, opts=opts)
        far[free] = sol.far_field(dirs)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        fam = {}
        for name in ("rwg_free", "pair_gemv", "pair_spmv", "rwg_regular", "singular"):
            n_, ms_, u_ = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            L.cal_profile_read(name.encode(), ctypes.byref(n_), ctypes.byref(ms_), ctypes.byref(u_))
            fam[name] = (n_.value, ms_.value, u_.value)
        L.cal_profile_enable(0)
        info = sol.info()
        key = "matrix_free" if free else "stored"
        out[key] = {"seconds": t, "iterations": int(info.iterations), "matvecs": int(info.matvecs),
                    "bytes_A_gb": info.bytes_A / 1e9, "phase_s": {"assemble_A": info.t_assemble_A,
                                                                 "assemble_P": info.t_assemble_P,
                                                                 "solve": info.t_solve},
                    "kernels_ms": {k: round(v[1], 3) for k, v in fam.items() if v[0]}}
        apps = max(1, int(info.matvecs) // (4 * W["prisms"] ** 2 + 4 * W["prisms"]))
        out[key]["operator_applications"] = apps
        if free and fam["rwg_free"][0]:
            n_, ms_, u_ = fam["rwg_free"]
            n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
            peak = _alu_peak(n_sm, _measured_peaks().get("sm_max_mhz", 2070.0))
            out[key]["rwg_free"] = {"launches": n_, "ms_per_launch": ms_ / n_,
                                    "roofline": {"bound": "alu", "achieved": u_ / (ms_ / 1e3) / 1e9,
                                                 "peak": peak / 1e9, "unit": "Geval/s",
                                                 "frac": u_ / (ms_ / 1e3) / peak,
                                                 "note": "evaluations counted on the device; class rules put 9 "
                                                         "evaluations on a far pair, so the per-pair work (moments, "
                                                         "the 3 x 3 local S and C, their application) dominates"}}
        if not free and fam["pair_gemv"][0]:
            n_, ms_, u_ = fam["pair_gemv"]
            hbm = _measured_peaks().get("hbm_gbs", 6783.5)
            out[key]["pair_gemv"] = {"launches": n_, "ms_per_launch": ms_ / n_,
                                     "roofline": {"bound": "hbm", "achieved": u_ / (ms_ / 1e3) / 1e9, "peak": hbm,
                                                  "unit": "GB/s", "frac": u_ / (ms_ / 1e3) / 1e9 / hbm}}
    out["far_field_rel_diff"] = float(np.linalg.norm(far[1] - far[0]) / np.linalg.norm(far[0]))
    return out


# Section 4 Table table:multiple_particle: the three cubes (side 0.4, corners at x =
# -1, 0, 1), n = 1.311 + 2.289e-9 i, E^inc = z e^{ik_e x}, 10 elements per
# wavelength; P = D with (chi_P, nu_P, q_P) per row, P's blocks as H-matrices with
# ACA to nu_P and the block-level cutoff chi_P. Printed values per row: iterations
# (matvecs) and Mem(P) relative to row 1, for k_e = 2.1 and 11.4 (the "7 (582)"
# rows read as 528, Table tab:matvecs).
TABLE2 = {"n": 1.311 + 2.289e-9j, "k": (2.1, 11.4), "tol": 1e-5, "restart": 200,
          "rows": [(math.inf, 0.001, (0, 4), ((6, 456, 1.0), (9, 672, 1.0))),
                   (math.inf, 0.001, (1, 1), ((7, 528, 1.0), (9, 672, 1.0))),
                   (math.inf, 0.01, (0, 4), ((6, 456, 0.78), (9, 672, 0.70))),
                   (math.inf, 0.01, (1, 1), ((7, 528, 0.78), (9, 672, 0.71))),
                   (math.inf, 0.1, (1, 1), ((7, 528, 0.57), (9, 672, 0.44))),
                   (math.inf, 0.5, (1, 1), ((9, 672, 0.41), (11, 816, 0.31))),
                   (1.0, 0.1, (1, 1), ((7, 528, 0.57), (9, 672, 0.44))),
                   (0.1, 0.1, (1, 1), ((84, 6072, 0.41), (16, 1176, 0.29))),
                   (0.0, 0.1, (1, 1), ((198, 14280, 0.36), (36, 2616, 0.18)))]}


def run_table2(dev):
    """The three-cube benchmark of Section 4 on the GPU (float64, the paper's
    scattered-trace right-hand side, P's blocks as H-matrices with ACA), every
    row of Table 2 with its iterations, matvecs and Mem(P) relative to row 1
    beside the printed values, and the real-index rerun of row 1."""
    from paper_2008_04772_gb300 import cal, meshgen
    T = TABLE2
    ctx = cal.Context(dev)
    inc = np.array([[1.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    out = {"workload": "three cubes of side 0.4, n = 1.311 + 2.289e-9i, E^inc = z e^{ik x}, h = 2 pi / (10 k)",
           "precision": "float64", "rhs": "scattered traces (rhs_mode 1)", "tol": T["tol"],
           "note": "A is dense (the paper's A is an H-matrix with nu_A = 0.001); P = D as H-matrices (ACA to nu_P, "
                   "admissible leaves beyond chi_P dropped); q_P (4,3,2,6) = class rules and order-4 singular rules",
           "rows": {}}
    for ki, k in enumerate(T["k"]):
        m = meshgen.three_cubes(2 * math.pi / (10 * k))
        mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
        h = mesh.info().h
        key = f"k={k}"
        out[key] = {"triangles": int(len(m.tris)), "unknowns": 2 * int(mesh.info().n_edges)}
        mem1 = None
        for chi, nu, (qr, qs), printed in T["rows"]:
            name = f"chi={chi}, nu={nu}, q={'(4,3,2,6)' if qr == 0 else '(1,1,1,1)'}"
            opts = cal.solve_opts(precond="D", precision=cal.FP64, tol=T["tol"], restart=T["restart"], maxit=2000,
                                  rhs_mode=1, q_regular_A=0, q_singular_A=4, q_regular_P=qr, q_singular_P=qs,
                                  aca_nu_P=nu, near_cutoff_P=(chi / h if math.isfinite(chi) else math.inf))
            t0 = time.perf_counter()
            info = cal.pmchwt_solve(ctx, mesh, k, T["n"] ** 2, inc, opts=opts, allow_not_converged=True).info()
            mem1 = mem1 or info.bytes_P
            out["rows"].setdefault(name, {})[key] = {
                "iterations": int(info.iterations), "matvecs": int(info.matvecs),
                "mem_P_rel": info.bytes_P / mem1, "bytes_P_mb": info.bytes_P / 1e6,
                "paper": {"iterations": printed[ki][0], "matvecs": printed[ki][1], "mem_P_rel": printed[ki][2]},
                "seconds": time.perf_counter() - t0}
        opts = cal.solve_opts(precond="D", precision=cal.FP64, tol=T["tol"], restart=T["restart"], maxit=2000,
                              rhs_mode=1, q_regular_A=0, q_regular_P=0, aca_nu_P=0.001)
        info = cal.pmchwt_solve(ctx, mesh, k, T["n"].real ** 2, inc, opts=opts, allow_not_converged=True).info()
        out[key]["real_index_row1"] = {"iterations": int(info.iterations), "matvecs": int(info.matvecs)}
        # the last row: the mixed discretisation (P = D from A's blocks, dense, total traces)
        t0 = time.perf_counter()
        opts = cal.solve_opts(precond="D", precision=cal.FP64, tol=T["tol"], restart=T["restart"], maxit=2000,
                              q_regular_A=0, discretisation=1)
        info = cal.pmchwt_solve(ctx, mesh, k, T["n"] ** 2, inc, opts=opts, allow_not_converged=True).info()
        out["rows"].setdefault("mixed discretisation, P = D", {})[key] = {
            "iterations": int(info.iterations), "matvecs": int(info.matvecs),
            "paper": {"iterations": (5, 9)[ki], "matvecs": (384, 672)[ki]},
            "bytes_A_plus_P_mb": (info.bytes_A + info.bytes_P) / 1e6, "seconds": time.perf_counter() - t0}
    return out


NEAR_FIELD = {"plane": "z = 0", "extent": 2.0, "grid": 128, "levels": 2}


def run_near_field(dev):
    """|E|^2 on a plane through the headline sphere (the maps of Section 5): the
    float32 near-field kernel over the solved traces, timed, with its rate in
    point-source interactions per second against the FP32-pipe bound."""
    import ctypes

    import torch

    from paper_2008_04772_gb300 import cal, meshgen
    W, NF = WORKLOAD, NEAR_FIELD
    L = cal.lib()
    ctx = cal.Context(dev)
    m = meshgen.icosphere(W["level"])
    mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    sol = cal.pmchwt_solve(ctx, mesh, W["k"], W["eps"], meshgen.plane_wave_x_along_z(),
                           opts=cal.solve_opts(precond="D", precision=cal.FP32, tol=W["tol"], **Q))
    g = np.linspace(-NF["extent"], NF["extent"], NF["grid"])
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    sol.near_field(pts[:64], levels=NF["levels"])  # warm-up
    L.cal_profile_enable(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, reg = sol.near_field(pts, levels=NF["levels"])
    t = time.perf_counter() - t0
    n_, ms_, u_ = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    L.cal_profile_read(b"near_field", ctypes.byref(n_), ctypes.byref(ms_), ctypes.byref(u_))
    L.cal_profile_enable(0)
    nsrc = len(m.tris) * 6 * 4 ** NF["levels"]
    n_in = int(np.sum(reg >= 0))
    inter = (len(pts) - n_in) * nsrc + n_in * nsrc  # one scatterer: all sources either way
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = _measured_peaks().get("sm_max_mhz", 2070.0)
    # per interaction ~76 FP32-pipe instructions (distance 7, phase with Cody-Waite 8,
    # amplitude and G 5, g 10, sums: G u_2 12, g div u_2 (x - y) 10, curl 24) and
    # 3 XU (rsqrt, sin, cos): the FP32 pipe binds
    peak = n_sm * 128.0 / 76.0 * sm_max * 1e6
    rate = inter / (ms_.value / 1e3) if ms_.value > 0 else 0.0
    I2 = np.sum(np.abs(E[0]) ** 2, 1)
    return {"workload": f"{W['name']} |E|^2 on the plane {NF['plane']}, {NF['grid']}^2 points in "
                        f"[-{NF['extent']}, {NF['extent']}]^2, 6-point rule on 4^{NF['levels']} sub-triangles",
            "points": len(pts), "inside": n_in, "sources": nsrc, "seconds": t, "kernel_ms": ms_.value,
            "interactions_per_s": rate, "max_E2": float(I2.max()), "mean_E2_outside": float(I2[reg < 0].mean()),
            "roofline": {"bound": "alu", "achieved": rate / 1e9, "peak": peak / 1e9, "unit": "Ginteractions/s",
                         "frac": rate / peak, "peak_source": f"derived: {n_sm} SMs x 128/76 per clk x {sm_max:.0f} MHz"}}


SERVING = {"name": "aggregate_requests_scaled", "requests": 64, "seed": 0, "prisms": (1, 8),
           "tris_per_prism": (250, 2000), "k": (1.0, 10.0), "eps_re": (2.5, 3.5), "eps_im": 0.01,
           "nrhs": (1, 16), "ndir": 64, "precond": "D", "near_cutoff_P": math.inf, "tol": 1e-5,
           "slots": 4, "load": 0.8}


def serving_requests(n, seed):
    """Seeded request mix shaped like the aggregate serving workload, scaled down
    in requests and triangles per prism (see SERVING) so that it fits the bench."""
    from paper_2008_04772_gb300 import meshgen
    S = SERVING
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        npr = int(rng.integers(S["prisms"][0], S["prisms"][1] + 1))
        tpp = [int(t) for t in rng.integers(S["tris_per_prism"][0], S["tris_per_prism"][1] + 1, npr)]
        m = meshgen.prism_aggregate(npr, tpp, seed=1000 * seed + i, diameter=1.0, gap=0.05)
        k = float(rng.uniform(*S["k"]))
        eps = complex(rng.uniform(*S["eps_re"]), S["eps_im"])
        nrhs = int(rng.integers(S["nrhs"][0], S["nrhs"][1] + 1))
        d = rng.normal(size=(nrhs, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        inc = np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)
        out.append((m, k, eps, inc))
    return out


def run_serving(dev):
    """Closed-loop saturation run, then Poisson arrivals at `load` x that rate."""
    from paper_2008_04772_gb300 import cal, meshgen
    S = SERVING
    opts = cal.solve_opts(precond=S["precond"], precision=cal.FP32, tol=S["tol"],
                          near_cutoff_P=S["near_cutoff_P"], **Q)
    dirs = meshgen.fibonacci_directions(S["ndir"])
    reqs = serving_requests(S["requests"], S["seed"])
    q = cal.Queue(dev, slots=S["slots"])

    def submit(r):
        m, k, eps, inc = r
        return q.submit(m.verts, m.tris, m.domain, k, eps, inc, dirs, opts=opts)

    # warm-up on requests of another seed (kernels, memory pool)
    for t in [submit(r) for r in serving_requests(4, S["seed"] + 1)]:
        q.wait(t)
    # closed loop: every request submitted at once
    t0 = time.perf_counter()
    tickets = [submit(r) for r in reqs]
    res = [q.wait(t)[0] for t in tickets]
    t_closed = time.perf_counter() - t0
    ok = sum(r.status == 0 for r in res)
    cols = sum(len(r[3]) for r in reqs)
    rate = S["load"] * len(reqs) / t_closed
    # open loop: Poisson arrivals at `load` x the saturated rate
    rng = np.random.default_rng(S["seed"] + 2)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    tk = [None] * len(reqs)

    def feeder():
        start = time.perf_counter()
        for i, r in enumerate(reqs):
            dt = arrivals[i] - (time.perf_counter() - start)
            if dt > 0:
                time.sleep(dt)
            tk[i] = submit(r)

    th = threading.Thread(target=feeder)
    t1 = time.perf_counter()
    th.start()
    lat = []
    statuses = []
    detail = []
    for i in range(len(reqs)):
        while tk[i] is None:
            time.sleep(0.001)
        r = q.wait(tk[i])[0]
        lat.append(1e3 * (r.t_done - r.t_submit))
        statuses.append(r.status)
        detail.append((len(reqs[i][0].tris), round(reqs[i][1], 2), len(reqs[i][3]), r.status, r.iterations,
                       round(1e3 * (r.t_done - r.t_start))))
    th.join()
    t_open = time.perf_counter() - t1
    st = q.stats()
    q.close()
    tri = [len(r[0].tris) for r in reqs]
    return {
        "workload": S["name"],
        "requests": len(reqs),
        "scale": "the serving configuration states 512 requests with 500-4000 triangles per prism; this run "
                 f"takes {len(reqs)} requests (1/{512 // len(reqs)}) with {S['tris_per_prism'][0]}-"
                 f"{S['tris_per_prism'][1]} triangles per prism (half the stated range) so that both loops fit the "
                 "bench's minutes",
        "mix": {"prisms": list(S["prisms"]), "tris_per_prism": list(S["tris_per_prism"]),
                "triangles": [int(min(tri)), int(max(tri))], "k": list(S["k"]),
                "eps_r": f"U{list(S['eps_re'])} + {S['eps_im']}i", "nrhs": list(S["nrhs"]),
                "columns": cols, "far_field_dirs": S["ndir"],
                "preconditioner": S["precond"] + (f" near-field {S['near_cutoff_P']}h"
                                                  if math.isfinite(S["near_cutoff_P"]) else " dense"),
                "tol": S["tol"]},
        "slots": S["slots"],
        "closed_loop": {"solves_per_s": len(reqs) / t_closed, "columns_per_s": cols / t_closed,
                        "seconds": t_closed, "ok": ok},
        "open_loop": {"arrival_rate_per_s": rate, "solves_per_s": len(reqs) / t_open,
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                      "ok": sum(s == 0 for s in statuses)},
        "latency": "arrival (submit) to far field ready, queue clock",
        "slowest": sorted(detail, key=lambda x: -x[5])[:6],
        "statuses": {str(k): statuses.count(k) for k in set(statuses)},
        "queue": {"peak_running": st.peak_running, "merged": st.merged, "problems_created": st.problems_created,
                  "evictions": st.evictions, "peak_reserved_gb": st.peak_reserved_bytes / 1e9,
                  "budget_gb": st.budget_bytes / 1e9},
    }


def _host_cores() -> int:
    """Cores this process may run on (what nproc prints)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(sample_tris: int, seed: int = 0):
    """The oracle's local blocks for `sample_tris` test triangles against all trial
    triangles, barycentric (P) and primal (A), at k_e and k_i on the headline
    workload. Returns (measured seconds, seconds extrapolated by triangle-pair
    count to the assembly of one solve: P 2 passes over 30720^2 barycentric
    pairs, A 2 passes over 5120^2 primal pairs, description)."""
    from oracle import bem, spaces
    from paper_2008_04772_gb300 import meshgen
    W = WORKLOAD
    m = meshgen.icosphere(W["level"])
    topo = spaces.Topology(m.verts, m.tris, m.domain)
    rwg, bc = spaces.rwg_space(topo), spaces.bc_space(topo)
    rules = bem.Rules(W["q_regular"], 4)
    km = W["k"] * np.sqrt(W["eps"])
    rng = np.random.default_rng(seed)
    t_meas = t_extra = 0.0
    desc = []
    for sp, name in ((bc, "barycentric"), (rwg, "primal")):
        X, ids = bem._space_tri_arrays(sp)
        nt = sp.tri_xyz.shape[0]
        test = rng.choice(nt, size=min(sample_tris, nt), replace=False)
        trial = np.arange(nt)
        t = 0.0
        for k in (W["k"], km):
            a = time.perf_counter()
            bem.local_blocks(X, ids, test, trial, k, rules)
            t += time.perf_counter() - a
        t_meas += t
        t_extra += t / (2 * len(test) * nt) * 2 * nt * nt
        desc.append(f"{len(test)} {name} test triangles x {nt}")
    return t_meas, t_extra, " and ".join(desc)


def oracle_c1_solve():
    """One complete oracle solve of the 320-triangle sphere (k = 2, full D, 6-point
    and order-4 rules, GMRES to 1e-6, far field on 362 directions): phase times."""
    from oracle import bem, pmchwt
    from paper_2008_04772_gb300 import meshgen
    bem.build()
    m = meshgen.icosphere(2)
    inc = meshgen.plane_wave_x_along_z()
    t0 = time.perf_counter()
    pb = pmchwt.PMCHWT(m.verts, m.tris, m.domain, 2.0, 3.17 + 0.01j, precond="D")
    pb.assemble()
    t1 = time.perf_counter()
    x, info = pb.solve(inc[0], tol=1e-6)
    t2 = time.perf_counter()
    pb.far_field(x, meshgen.sphere_cut_directions(181))
    t3 = time.perf_counter()
    return {"assemble_s": t1 - t0, "gmres_s": t2 - t1, "far_field_s": t3 - t2, "total_s": t3 - t0,
            "iterations": int(info["iterations"]), "solves_per_s": 1.0 / (t3 - t0)}


def _one_core(args):
    """Run `bench.py <args>` with one thread for OpenMP and the BLAS; its JSON line."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), *args], env=env, capture_output=True, text=True,
                       timeout=600)
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(sample_tris: int):
    """The oracle (plain FP64 C + numpy) on the host cores, reported beside the GPU.

    value: the headline workload (5120-triangle sphere), extrapolated from a
    sample of the oracle's assembly (`oracle_sample`; GMRES and far field are
    excluded there: on the complete 320-triangle solve below they are a few % of
    the time). Also: the complete 320-triangle solve on all cores, and the same
    sample on one core.
    """
    from oracle import bem
    bem.build()
    cores = _host_cores()
    t_meas, t_extra, desc = oracle_sample(sample_tris)
    c1 = oracle_c1_solve()
    one = _one_core(["--oracle-sample", str(max(2, sample_tris // 4))])
    return {"value": 1.0 / t_extra, "unit": "solves/s", "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": f"oracle local blocks for {desc} at k_e and k_i ({t_meas:.2f} s measured), extrapolated by "
                      "triangle-pair count to the assembly of one solve; GMRES and far field excluded",
            "c1_full_solve_all_cores": c1,
            "one_core": {"value": 1.0 / one["extrapolated_s"], "unit": "solves/s", "cores": 1,
                         "sample": one["sample"], "measured_s": one["measured_s"]}}


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores (rank 0 only): each step is the
    bounded sample of the headline workload's assembly, the value its
    extrapolation to one solve (labelled), ms_per_step the time each step took."""
    if rank != 0:
        return None
    from oracle import bem
    bem.build()
    for _ in range(args.warmup):
        oracle_sample(2)
    meas, vals = [], []
    desc = ""
    for q in range(args.steps):
        t_meas, t_extra, desc = oracle_sample(args.cpu_sample, seed=q)
        meas.append(t_meas)
        vals.append(1.0 / t_extra)
    v = statistics.median(vals)
    cores = _host_cores()
    return {"metric": "PMCHWT solves/s", "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(meas),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded icosphere, plane wave)", "impl": "reference",
            "config": {"workload": WORKLOAD["name"], "parallelism": f"host cores ({cores})"},
            "extrapolated": True,
            "note": "each step times the oracle's assembly of a sample of test triangles (ms_per_step); value is "
                    "that sample extrapolated by triangle-pair count to one solve of the workload",
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"oracle local blocks for {desc} at k_e and k_i per step, extrapolated"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_case(which: str) -> None:
    """One profiling case on the 5120-triangle sphere (k = 5), with the bench's
    regular rules (near / medium / far classes at the paper's default orders 4, 3, 2):
      bc    one dense FP32 assembly of S and C on the Buffa–Christiansen space
            (the BC-pair kernel and the split Sauter–Schwab kernel);
      gemv  an unpreconditioned FP32 solve capped at 3 GMRES iterations (the PMCHWT
            GEMV launches on the stored A blocks);
      gemm  the tensor-core product of the stored 7680 x 7680 complex64 S block with
            32 vectors (cal_matvec, 3xTF32 on tcgen05), three times;
      free  three FP32 GMRES iterations with the matrix-free PMCHWT operator;
      solve one complete solve of the bench workload (FP32 bulk, full D, tol 1e-5);
      multi one FP32 solve of 32 incident directions with the near-field reduced
            preconditioner Di (chi = 2h);
      near  one FP32 solve, then |E|^2 on a 64^2 grid of the plane z = 0 (composite level 2).
    """
    import torch

    from paper_2008_04772_gb300 import build, cal, meshgen
    build.build()
    ctx = cal.Context(0)
    m = meshgen.icosphere(4)
    mesh = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    k, eps, inc = 5.0, 3.17 + 0.01j, meshgen.plane_wave_x_along_z()
    if which == "bc":
        bc = cal.Space(mesh, cal.BC)
        cal.assemble(ctx, cal.OP_S | cal.OP_C, k, bc, q_regular=0, precision=cal.FP32)
    elif which == "gemm":
        op = cal.assemble(ctx, cal.OP_S, k, cal.Space(mesh, cal.RWG), precision=cal.FP32)
        n = op.info().cols
        x = torch.randn((32, 2 * n), dtype=torch.float32, device="cuda")
        y = torch.zeros((32, 2 * n), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for _ in range(3):
            op.matvec(cal.OP_S, x.data_ptr(), y.data_ptr(), nrhs=32)
        torch.cuda.synchronize()
    elif which == "free":
        cal.pmchwt_solve(ctx, mesh, k, eps, inc, allow_not_converged=True,
                         opts=cal.solve_opts(precond="none", precision=cal.FP32, maxit=3, refine=0,
                                             matrix_free=1, q_regular_A=0))
    elif which == "gemv":
        cal.pmchwt_solve(ctx, mesh, k, eps, inc, allow_not_converged=True,
                         opts=cal.solve_opts(precond="none", precision=cal.FP32, maxit=3, refine=0))
    elif which == "multi":
        d = meshgen.fibonacci_directions(32)
        cal.pmchwt_solve(ctx, mesh, k, eps, np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1),
                         opts=cal.solve_opts(precond="Di", near_cutoff_P=2.0, precision=cal.FP32, tol=1e-5, **Q))
    elif which == "near":
        sol = cal.pmchwt_solve(ctx, mesh, k, eps, inc, opts=cal.solve_opts(precond="D", precision=cal.FP32, **Q))
        g = np.linspace(-2.0, 2.0, 64)
        X, Y = np.meshgrid(g, g, indexing="ij")
        sol.near_field(np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1), levels=2)
    elif which == "solve":
        sol = cal.pmchwt_solve(ctx, mesh, k, eps, inc,
                               opts=cal.solve_opts(precond="D", precision=cal.FP32, tol=1e-5, **Q))
        sol.far_field(meshgen.sphere_cut_directions(181))
    else:
        raise SystemExit(f"unknown case {which!r}")
    torch.cuda.synchronize()
    print("case done:", which)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default=None, choices=["bc", "gemv", "gemm", "free", "solve", "multi", "near"],
                    help="run one profiling case and exit (no JSON line)")
    ap.add_argument("--cpu-sample", type=int, default=24, help="test triangles per space for the oracle sample")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="skip the request-queue (continuous batching) run")
    ap.add_argument("--no-multirhs", dest="multirhs", action="store_false",
                    help="skip the 32-direction aggregate run")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the preconditioner variants of the headline workload")
    ap.add_argument("--no-table2", dest="table2", action="store_false",
                    help="skip the three-cube benchmark of Section 4")
    ap.add_argument("--no-near-field", dest="near_field", action="store_false",
                    help="skip the |E|^2 plane map")
    ap.add_argument("--no-matrix-free", dest="matrix_free", action="store_false",
                    help="skip the stored versus matrix-free comparison")
    args = ap.parse_args()
    if args.oracle_sample:  # one oracle sample, as one JSON line (the one-core baseline runs this)
        from oracle import bem
        bem.build()
        t_meas, t_extra, desc = oracle_sample(args.oracle_sample)
        print(json.dumps({"measured_s": t_meas, "extrapolated_s": t_extra, "sample": desc}))
        return
    if args.case:
        run_case(args.case)
        return
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
        tdist.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
