#!/usr/bin/env python
"""Benchmark of the aSP-AMG hot path on one GB300 (or N independent replicas).

One step = the whole path for one synthetic problem already resident in HBM:
rebuild the hierarchy from K (aFSAI smoother with Lanczos omega, SRQCG test
space, affinity coarsening, DPLS prolongation, Galerkin products, the coarse
level's explicit inverse) and solve K u = f by PCG with one V(1,1)-cycle per iteration to
||r|| <= 1e-8 ||f||.  The default workload is the 128 x 32 x 32 cantilever
beam with lognormal Young's moduli and an FP64 V-cycle; the FP32 V-cycle of the
same configuration is measured next to it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(plain C, OpenMP over its row loops on all host cores) on the same workload:
each step one whole set-up + PCG solve of the 128 x 32 x 32 beam.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 residual & V-cycles/s (FP64 vs mixed/batched), SpMV %HBM peak"
UNIT = "solutions/s"
RTOL = 1e-8
# FP64 arithmetic peak for FMA-bound kernels: the nominal 1.25 TFLOP/s of this
# GPU (152 SMs x 2 FP64 FMA per clock x 2 flop x ~2.06 GHz); a chain-of-FMA
# probe on the same GPUs measured 6.28e11 FMA/s (1.256 TFLOP/s)
FP64_TFLOPS = 1.25
FP64_PEAK_SOURCE = "nominal FP64 rate (1.25 TFLOP/s); FMA-chain probe measured 1.256"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
# ncu captures summarised under profiles/; a kernel whose code changed since its
# capture has no entry
TRAFFIC: dict = {
    # level-0 K of the 128x32x32 beam, two warps per slice (here
    # k_sellmv<double, double, 3, 0, 2, 2>): 278.63 MB read + 4.44 MB written
    # (profiles/k_sellmv_level0_beam.md)
    "k_sellmv_fp64_level0": 283.07e6,
    # det::k_spmv_cols<3, 1>, level-0 A times 10 columns: 307.19 MB read +
    # 28.07 MB written (profiles/k_spmv_cols_beam.md)
    "k_spmv_cols": 335.27e6,
}
# aFSAI kernel: fraction of the FP64 FMA lane peak in its ncu capture
# (profiles/k_fsai_beam96x24x24.md); None once the kernel changed
FSAI_LANE_FRAC = 0.251


def workload_config(n3=None):
    """The bench workload's config, the same for both arms."""
    import workloads as W
    if n3 is None:
        n3 = 3 * W.beam().free_nodes()
    return {"workload": "cantilever beam 128x32x32 Q1 hex (%d dofs), x=0 clamped, tip shear, lognormal E "
                        "(mu 0, sigma 1), nu 0.3; set-up + PCG to 1e-8, FP64" % n3,
            "l2": "inputs larger than L2 (fine K alone 259 MB)"}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                    "sw_power_cap"), f[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def max_over_ranks(v, ws):
    """Largest value over the ranks (the slowest replica's time)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as td
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def aggregate(ms_local, ws):
    """(ms per step of the slowest rank, whole-job solutions per second): every
    rank solves its own replica of the workload in each step."""
    ms = max_over_ranks(ms_local, ws)
    return ms, ws * 1e3 / ms


def gpu_problem(A, p):
    d = A.fe_assemble(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.nu, p.E, p.clamp_axis)
    n = d["nfree"]
    d["V0"] = A.fe_rbm(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, n)
    if p.load == "end_shear":
        d["f"] = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "end_shear",
                           g=[p.shear_total], nfree=n)
    elif p.load == "top_pressure":
        d["f"] = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "top_pressure",
                           p=p.pressure, nfree=n)
    else:
        d["f"] = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "body", g=p.body, nfree=n)
    return d


def _timed(fn, reps=1):
    """(result, ms) of fn() timed with CUDA events on the current stream,
    after one untimed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / reps


def extra_slab(A, W):
    """The 256x256x4 layered slab: FP64, FP32 and FP32 with bf16-stored G, P
    V-cycles inside FP64 CG to 1e-8 (set-up + solve per step)."""
    import torch
    p = W.slab()
    d = gpu_problem(A, p)
    out = {"workload": "slab 256x256x4 (%d dofs), E 1/1e4 layers, nu 0.45, h_z 0.05" % (3 * d["nfree"])}
    x64 = None
    for prec in ("fp64", "fp32", "bf16gp"):
        S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec=prec)

        def step():
            S.update_values(d["vals"])
            return S.solve(d["f"], RTOL)
        (x, its, rel, rc), ms = _timed(step)
        st = S.stats()
        r = {"ms_per_solution": ms, "n_it": its[0], "setup_ms": st["T_p"] * 1e3, "solve_ms": st["T_s"] * 1e3}
        if x64 is None:
            x64 = x
        else:
            r["rel_diff_vs_fp64_solution"] = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
        out[prec] = r
        S.close()
    return out


def run_extra(fn, *args):
    """fn(*args), or {"error": ...} when it raises: the extra workloads are
    reported beside the headline, and a failing one must not take the
    headline line with it."""
    try:
        return fn(*args)
    except Exception as e:  # noqa: BLE001 -- recorded in the JSON line
        return {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}


def batched_problem(A, p):
    """K, V0 of the cube recipe p on the device and its load cases as the
    columns of one (3 nfree, k) FP64 right-hand side."""
    import torch
    d = gpu_problem(A, p)
    k = p.nodal.shape[0]
    F = torch.empty((3 * d["nfree"], k), dtype=torch.float64, device="cuda")
    for c in range(k):
        F[:, c] = A.fe_load(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, "top_nodal",
                            p=p.nodal[c].reshape(-1), nfree=d["nfree"])
    return d, F


def extra_batched(A, W):
    """The 96^3 cube with 64 load cases: one block solve (FP32 V-cycle, FP64
    CG, per-column masks) against solving the cases one at a time in FP64."""
    import torch
    p = W.cube_batched()
    d, F = batched_problem(A, p)
    k = F.shape[1]
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec="fp32")
    (X, its, rel, rc), ms_b = _timed(lambda: S.solve(F, RTOL))
    S64 = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"])
    (x1, it1, rel1, rc1), ms_1 = _timed(lambda: S64.solve(F[:, 0].contiguous(), RTOL))
    out = {"workload": "cube 96^3 (%d dofs), 64 load cases N(0,1) on the top face" % (3 * d["nfree"]),
           "k": k, "batched_fp32_ms": ms_b, "batched_solutions_per_s": k * 1e3 / ms_b,
           "n_it_max": max(its), "n_it_min": min(its), "single_fp64_ms": ms_1, "single_fp64_n_it": it1[0],
           "speedup_per_solution_vs_single_fp64": ms_1 * k / ms_b,
           "setup_ms": S.stats()["T_p"] * 1e3,
           "rel_diff_col0_vs_fp64": float(torch.linalg.norm(X[:, 0] - x1) / torch.linalg.norm(x1))}
    S.close()
    S64.close()
    return out


def extra_adjoint(A, W):
    """The 128^3 SIMP cube: compliance, its gradient for every element by one
    forward and one adjoint solve (FP32 V-cycle, FP64 CG) and the element
    gather kernel."""
    import torch
    p = W.cube_simp()
    d = gpu_problem(A, p)
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec="fp32")
    conn = A.fe_conn(p.nx, p.ny, p.nz, p.clamp_axis)
    rho = torch.tensor(p.rho, device="cuda")

    def step():
        r = rho.clone().requires_grad_(True)
        u = A.LinearSolve.apply(S, d["f"], r ** 3, d["Ke0"], conn, RTOL)
        L = torch.dot(d["f"], u)
        L.backward()
        return r.grad
    g, ms = _timed(step)
    st = S.stats()
    out = {"workload": "SIMP cube 128^3 (%d dofs, %d elements), rho ~ U(0.1, 1), E = rho^3"
                       % (3 * d["nfree"], p.ne),
           "forward_adjoint_gradient_ms": ms, "setup_ms": st["T_p"] * 1e3, "n_it": st["n_it"],
           "grad_abs_sum": float(g.abs().sum())}
    S.close()
    return out


def extra_scalar_vs_block(A, W):
    """The bench beam with the paper's scalar method (block size 1: every dof
    its own node, the per-dof defaults of Table "TestParam") against the
    3x3-block form: iterations, complexities, set-up and solve time (FP64)."""
    import torch
    p = W.beam()
    d = gpu_problem(A, p)
    out = {"workload": "cantilever beam 128x32x32 (%d dofs), FP64 V-cycle, rtol 1e-8" % (3 * d["nfree"])}
    srp, scol, sval = A.bsr_to_scalar(d["rowptr"], d["col"], d["vals"])
    for name, args, kw in (("block3", (d["rowptr"], d["col"], d["vals"]), {}),
                           ("scalar", (srp, scol, sval), {"block": 1})):
        S = A.Solver(*args, d["V0"], **kw)
        vals = args[2]

        def step():
            S.update_values(vals)
            return S.solve(d["f"], RTOL)
        (x, its, rel, rc), ms = _timed(step)
        st = S.stats()
        out[name] = {"ms_per_solution": ms, "n_it": its[0], "setup_ms": st["T_p"] * 1e3, "solve_ms": st["T_s"] * 1e3,
                     "levels": st["nlev"], "C_gd": st["C_gd"], "C_op": st["C_op"], "C_fs": st["C_fs"],
                     "true_relres": rel[0],
                     "setup_phases_ms": {q: 1e3 * st[q] for q in ("T_sm", "T_ts", "T_cs", "T_pl", "T_rap")}}
        S.close()
    return out


def extra_beam6502k(A, W):
    """The paper's beam6502k shape (App. A.6): 512 x 64 x 64 two-material
    cantilever, right-hand side of ones, FP32 V-cycle inside FP64 CG to 1e-8,
    one set-up and one solve.  The paper reports 87 iterations, T_p = 115.1 s,
    T_s = 53.6 s on one KNL with its real matrix (App. A.6, default
    parameters): context only.  The material jump slows this solver down (its
    iteration count grows with the mesh on this shape), hence the higher
    iteration limit."""
    import torch
    p = W.beam6502k()
    vals = None
    for nu in np.unique(p.nu_elem):
        Em = np.where(p.nu_elem == nu, p.E, 0.0)
        dm = A.fe_assemble(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, float(nu), Em, p.clamp_axis)
        if vals is None:
            d, vals = dm, dm["vals"].clone()
        else:
            vals += dm["vals"]
    n = d["nfree"]
    V0 = A.fe_rbm(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.clamp_axis, n)
    f = torch.ones(3 * n, dtype=torch.float64, device="cuda")
    out = {"workload": "beam6502k-like 512x64x64 (%d dofs, %d blocks), E 1e4/1e7, nu 0.2/0.4, b = ones"
                       % (3 * n, d["col"].numel()),
           "paper_context": {"n_it": 87, "T_p_s": 115.1, "T_s_s": 53.6, "hardware": "1x Xeon Phi 7250 (68 cores)"}}
    S = A.Solver(d["rowptr"], d["col"], vals, V0, vcycle_prec="fp32", maxit=4000)
    x, its, rel, rc = S.solve(f, RTOL)
    st = S.stats()
    # rc follows the recurrence rule (Sec. 4); the FP64 true residual can stay
    # above rtol on this shape, so both residuals are reported
    out["fp32"] = {"n_it": its[0], "rc": rc, "setup_ms": st["T_p"] * 1e3, "solve_ms": st["T_s"] * 1e3,
                   "levels": st["nlev"], "C_op": st["C_op"], "true_relres": rel[0],
                   "rec_relres": st["relres_rec"], "restarts": st["restarts"],
                   "true_residual_met": bool(rel[0] <= RTOL)}
    S.close()
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_full():
    """One whole oracle solution of the bench workload: FE assembly, set-up
    (Algorithm 1) and PCG to 1e-8; (seconds of set-up + solve, iterations).
    The oracle's row loops run on all host cores (OpenMP)."""
    import oracle as orc
    import workloads as W
    p = W.beam()
    K, nm = orc.assemble(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.nu, p.E, p.clamp_axis)
    V0 = orc.rbm(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, nm)
    f = orc.load_end_shear(p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, p.shear_total, nm)
    t0 = time.perf_counter()
    H = orc.Hierarchy(K, V0)
    x, it, rr, rc = H.pcg(f, RTOL)
    sec = time.perf_counter() - t0
    del H
    if rc != 0:
        raise RuntimeError("oracle PCG did not converge: %s" % rc)
    return sec, it


def oracle_baseline():
    """cpu_baseline of the GPU arm: the oracle on the whole workload, run in a
    child process (its OpenMP threads stay out of the GPU process)."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-once"], capture_output=True,
                       text=True, timeout=1800, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / d["sec"], "unit": UNIT, "cores": d["cores"], "kind": "oracle",
            "sample": "the whole workload: oracle set-up + PCG to 1e-8 on the 128x32x32 beam (%d its), "
                      "%.2f s, OpenMP on %d host cores" % (d["it"], d["sec"], d["cores"])}


def run_oracle_once(args):
    sec, it = oracle_full()
    print(json.dumps({"sec": sec, "it": it, "cores": host_cores()}), flush=True)


def run_reference(args):
    ws, rank, local = dist()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_full()
    t0 = time.perf_counter()
    secs, its = [], []
    for _ in range(args.steps):
        sec, it = oracle_full()
        secs.append(sec)
        its.append(it)
    wall = time.perf_counter() - t0
    ms = 1e3 * sum(secs) / len(secs)
    value = 1e3 / ms
    cores = host_cores()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "each step the whole workload: oracle set-up + PCG to 1e-8 on the "
                                      "128x32x32 beam (%d its), OpenMP on %d host cores" % (its[-1], cores)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": wall}
    print(json.dumps(out), flush=True)


def level_sizes(S):
    """Per level: (block rows, nnzb A, nnzb G, nnzb P, coarse block rows)."""
    out = []
    for k in range(S.nlev):
        i = S.level_info(k)
        out.append((i["nr"], i["nnzb_A"], i["nnzb_G"], i["nnzb_P"], i["nc"]))
    return out


def vcycle_work(levels, prec):
    """Algorithmic bytes and fused multiply-adds of one PCG iteration: the FP64
    CG operator product and vector kernels, plus one V(1,1)-cycle (per level:
    G, G^T, A twice each, R and P once, every matrix streamed once per product
    with its column indices, row pointers and slice offsets, every vector read
    or written once per product; the coarse level one dense product).  Values
    8 B (FP64), 4 B (FP32) or 2 B (bf16 G, G^T, P, R); V-cycle vectors 8 or 4 B."""
    sv_a = 8 if prec == "fp64" else 4
    sv_g = {"fp64": 8, "fp32": 4, "bf16gp": 2}[prec]
    w = 8 if prec == "fp64" else 4

    def mat(nr, nnzb, sv):
        return nnzb * (9 * sv + 4) + 4 * (nr + 1) + 4 * ((nr + 31) // 32 + 1)

    nr0, nnzb0 = levels[0][0], levels[0][1]
    n0 = 3 * nr0
    by = mat(nr0, nnzb0, 8) + 16 * n0            # CG operator q = K p
    fma = 9 * nnzb0
    mixed = prec != "fp64"
    by += 16 * n0                                 # p.q
    by += (48 + (4 if mixed else 0)) * n0         # x, r updates, r.r (+ FP32 copy of r)
    by += (28 if mixed else 16) * n0              # r.z (+ FP64 copy of z, r.z_old)
    by += (32 if mixed else 24) * n0              # p = z + beta p (+ z_old)
    for k, (nr, na, ng, npb, nc) in enumerate(levels):
        n = 3 * nr
        if k == len(levels) - 1:
            by += 8 * n * n + 2 * w * n
            fma += n * n
            continue
        by += 2 * mat(nr, ng, sv_g) + 2 * mat(nr, ng, sv_g) + 2 * mat(nr, na, sv_a)
        by += mat(nr, npb, sv_g) + mat(nc, npb, sv_g)
        by += w * (18 * n + 2 * 3 * nc)
        fma += 9 * (4 * ng + 2 * na + 2 * npb)
    return by, fma


def run_ours(args):
    import torch

    import paper_1902_01715_gb300 as A
    import workloads as W

    ws, rank, local = dist()
    if ws > 1:
        import torch.distributed as td
        torch.cuda.set_device(local)
        td.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    A.build()
    A.lib()
    p = W.beam()
    d = gpu_problem(A, p)
    n3 = 3 * d["nfree"]
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec=args.prec)
    vals, f = d["vals"], d["f"]

    def step(solver):
        solver.update_values(vals)
        x, it, rr, rc = solver.solve(f, RTOL)
        if rc != 0:
            raise RuntimeError("solve did not converge: %s" % rc)
        return x, it[0]

    for _ in range(args.warmup):
        step(S)
    torch.cuda.synchronize()
    barrier(ws)
    l0 = A.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st_setup, st_solve, its = [], [], []
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            x, it = step(S)
            s = S.stats()
            st_setup.append(s["T_p"])
            st_solve.append(s["T_s"])
            its.append(it)
        e1.record()
        torch.cuda.synchronize()
    barrier(ws)
    launches = A.launch_count() - l0
    ms, value = aggregate(e0.elapsed_time(e1) / args.steps, ws)
    stats = S.stats()
    clocks = clk.summary()

    pk = peaks()
    hbm = pk.get("hbm_gbs")
    hpk = hbm if hbm else 6800.0
    hsrc = "measured" if hbm else "fallback"
    levels = level_sizes(S)
    nnzb0 = levels[0][1]
    # dominant kernel of the step: the solve phase's sparse product k_sellmv
    # (all its launches together hold the largest share of the step's launch
    # time), measured on its largest launch, the FP64 product with the level-0
    # K.  A 3x3 FP64 block brings 76 B for 9 FMAs (8.4 B per FMA), less than
    # the 10.7 B per FMA at which HBM and the FP64 pipe balance: its roof is
    # the FP64 pipe ("alu"); the HBM fraction is reported beside it
    spmv_ms, spmv_bytes = S.bench_spmv(0, "A", a64=True, reps=50)
    gbps = spmv_bytes / (spmv_ms * 1e-3) / 1e9
    spmv_flops = 18.0 * nnzb0
    spmv_tf = spmv_flops / (spmv_ms * 1e-3) / 1e12
    roofline = {"kernel": "amg::k_sellmv (solve-phase sparse product; level-0 K x, FP64)", "bound": "alu",
                "achieved": spmv_tf, "peak": FP64_TFLOPS, "unit": "TFLOP/s", "frac": spmv_tf / FP64_TFLOPS,
                "traffic": TRAFFIC.get("k_sellmv_fp64_level0"), "peak_source": FP64_PEAK_SOURCE,
                "ms_per_launch": spmv_ms, "flops_per_launch": spmv_flops, "bytes_per_launch": spmv_bytes,
                "hbm": {"achieved": gbps, "peak": hpk, "unit": "GB/s", "frac": gbps / hpk, "peak_source": hsrc}}
    # the set-up's FP64 product of A_0 with the n_tv test-space columns (the
    # S = G A G^T products of Algorithm 4)
    t_tv = S.params.n_tv
    ms_c, by_c = S.bench_spmv(0, "A_cols", reps=20)
    flops_c = 18.0 * nnzb0 * t_tv
    ach = flops_c / (ms_c * 1e-3) / 1e12
    roofline_cols = {"kernel": "det::k_spmv_cols (set-up product A_0 X, %d FP64 columns)" % t_tv, "bound": "alu",
                     "achieved": ach, "peak": FP64_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_TFLOPS,
                     "traffic": TRAFFIC.get("k_spmv_cols"), "peak_source": FP64_PEAK_SOURCE,
                     "ms_per_launch": ms_c, "flops_per_launch": flops_c, "bytes_per_launch": by_c}
    # the largest set-up kernel: the first aFSAI pass on A_0 (FP64 issue bound;
    # dense row systems of varying size, so no byte or flop count per unit)
    fsai_ms, _ = S.bench_spmv(0, "fsai", reps=3)
    setup_ms = 1e3 * sum(st_setup) / len(st_setup)
    roofline_fsai = {"kernel": "det::k_fsai (first aFSAI pass on A_0, Algorithm 3)", "bound": "alu",
                     "ms_per_launch": fsai_ms, "share_of_setup": fsai_ms / setup_ms, "share_of_step": fsai_ms / ms,
                     "fp64_lane_frac_ncu": FSAI_LANE_FRAC}
    # the whole PCG iteration (CG operator, vector kernels and one V-cycle)
    # against its algorithmic bytes and FMAs, from the per-level sizes
    sol_ms = 1e3 * sum(st_solve) / len(st_solve)
    it_avg = sum(its) / len(its)

    def vc_line(prec, ms_it):
        by, fm = vcycle_work(levels, prec)
        d = {"bytes_per_it": by, "fma_per_it": fm, "ms_per_it": ms_it, "GBps": by / (ms_it * 1e-3) / 1e9}
        d["hbm_frac"] = d["GBps"] / hpk
        if prec == "fp64":
            d["fp64_tflops"] = 2.0 * fm / (ms_it * 1e-3) / 1e12
            d["fp64_frac"] = d["fp64_tflops"] / FP64_TFLOPS
        return d

    roofline_vcycle = {"note": "solve time / iterations (includes the first V-cycle and the true-residual check)",
                       args.prec: vc_line(args.prec, sol_ms / it_avg)}
    # FP32 V-cycle of the same configuration (not part of value)
    fp32 = None
    if args.prec == "fp64" and not args.no_compare:
        S32 = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec="fp32")
        for _ in range(2):
            step(S32)
        torch.cuda.synchronize()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record()
        for _ in range(args.steps):
            x32, it32 = step(S32)
        e3.record()
        torch.cuda.synchronize()
        s32 = S32.stats()
        err = float(torch.linalg.norm(x32 - x) / torch.linalg.norm(x))
        ms32, by32 = S32.bench_spmv(0, "A", a64=False, reps=50)
        levels32 = level_sizes(S32)
        by32it, fm32it = vcycle_work(levels32, "fp32")
        ms32it = s32["T_s"] * 1e3 / it32
        roofline_vcycle["fp32"] = {"bytes_per_it": by32it, "fma_per_it": fm32it, "ms_per_it": ms32it,
                                   "GBps": by32it / (ms32it * 1e-3) / 1e9,
                                   "hbm_frac": by32it / (ms32it * 1e-3) / 1e9 / hpk}
        fp32 = {"ms_per_step": e2.elapsed_time(e3) / args.steps, "n_it": it32,
                "solve_ms": s32["T_s"] * 1e3, "vcycles_per_s": it32 / s32["T_s"],
                "restarts": s32["restarts"], "true_relres": s32["relres_true"],
                "rel_diff_vs_fp64_solution": err,
                "spmv_level0": {"kernel": "amg::k_sellmv (level-0 K x, FP32)", "ms_per_launch": ms32,
                                "bytes_per_launch": by32, "GBps": by32 / (ms32 * 1e-3) / 1e9,
                                "frac": by32 / (ms32 * 1e-3) / 1e9 / hpk}}
        S32.close()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        vh = torch.empty(vals.shape, dtype=torch.float64, pin_memory=True)
        vh.copy_(vals)
        fh = torch.empty(f.shape, dtype=torch.float64, pin_memory=True)
        fh.copy_(f)
        xh = torch.empty(f.shape, dtype=torch.float64, pin_memory=True)
        import ctypes as C
        L = A.lib()
        iters = (C.c_int * 1)()
        rel = (C.c_double * 1)()

        def host_step():
            A.check(L.amg_update_values(S._h, C.c_void_p(vh.data_ptr()), A.AMG_MEM_HOST))
            rc = L.amg_solve(S._h, 1, C.c_void_p(fh.data_ptr()), C.c_void_p(xh.data_ptr()), RTOL,
                             iters, rel, A.AMG_MEM_HOST)
            A.check(rc)

        host_step()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        torch.cuda.synchronize()
        t = max_over_ranks((time.perf_counter() - t0) / args.steps, ws)
        e2e = {"value": ws / t, "unit": UNIT, "h2d_bytes_per_step": int(vh.numel() * 8 + fh.numel() * 8),
               "d2h_bytes_per_step": int(xh.numel() * 8), "ms_per_step": t * 1e3}

    extras = None
    if not args.no_extras:
        extras = {name: run_extra(fn, A, W) for name, fn in (
            ("mixed_precision", extra_slab), ("batched", extra_batched), ("adjoint", extra_adjoint),
            ("scalar_vs_block", extra_scalar_vs_block), ("beam6502k", extra_beam6502k))}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_baseline()

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "f32",
        "data": "synthetic",
        "config": workload_config(n3) if args.prec == "fp64" else
                  dict(workload_config(n3), workload=workload_config(n3)["workload"] + " CG, %s V-cycle"
                       % args.prec.upper()),
        "parallelism": "%d independent replicas" % ws if ws > 1 else "single GPU",
        "solve": {"n_it": int(round(sum(its) / len(its))), "setup_ms": 1e3 * sum(st_setup) / len(st_setup),
                  "solve_ms": 1e3 * sum(st_solve) / len(st_solve), "true_relres": stats["relres_true"],
                  "rec_relres": stats["relres_rec"], "restarts": stats["restarts"],
                  "vcycles_per_s": sum(its) / sum(st_solve),
                  "levels": stats["nlev"], "C_gd": stats["C_gd"], "C_op": stats["C_op"],
                  "C_fs": stats["C_fs"],
                  "setup_phases_ms": {k: 1e3 * stats[k] for k in ("T_sm", "T_ts", "T_cs", "T_pl", "T_rap")}},
        "fp32_vcycle": fp32,
        "roofline": roofline,
        "roofline_vcycle": roofline_vcycle,
        "roofline_setup_cols": roofline_cols,
        "roofline_fsai": roofline_fsai,
        "configs": extras,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


def run_micro(args):
    """Per-level solve-phase sparse products of the default workload, each
    timed with CUDA events (the kernel-level view behind the step time)."""
    import torch

    import paper_1902_01715_gb300 as A
    import workloads as W
    torch.cuda.set_device(0)
    A.build()
    A.lib()
    d = gpu_problem(A, W.beam())
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec=args.prec)
    hbm = peaks().get("hbm_gbs", 6800.0)
    rows = []
    torch.cuda.nvtx.range_push("spmv_A0_fp64")
    ms, by = S.bench_spmv(0, "A", a64=True, reps=args.reps)
    torch.cuda.nvtx.range_pop()
    rows.append({"level": 0, "matrix": "A(fp64, CG)", "ms": ms, "GBps": by / ms / 1e6,
                 "frac": by / ms / 1e6 / hbm})
    for k in range(S.nlev - 1):
        for which in ("A", "G", "GT", "P", "R"):
            if k == 0 and which == "A":
                torch.cuda.nvtx.range_push("spmv_A0_vcycle")
            ms, by = S.bench_spmv(k, which, a64=False, reps=args.reps)
            if k == 0 and which == "A":
                torch.cuda.nvtx.range_pop()
            rows.append({"level": k, "matrix": which, "prec": args.prec, "ms": ms, "GBps": by / ms / 1e6,
                         "frac": by / ms / 1e6 / hbm, "nnzb": S.level_info(k)["nnzb_" + ("A" if which == "A" else "G" if which in ("G", "GT") else "P")]})
    print(json.dumps({"micro": rows}), flush=True)


def run_batched(args):
    """One batched solve of the cube recipe at n^3 with its 64 load cases
    (FP32 V-cycle, FP64 CG, per-column masks) after a warm-up solve, inside
    the NVTX range "batched" (the case the batched-product profiles capture)."""
    import torch

    import paper_1902_01715_gb300 as A
    import workloads as W
    torch.cuda.set_device(0)
    A.build()
    A.lib()
    d, F = batched_problem(A, W.cube_batched(args.batched, 64))
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec="fp32")
    S.solve(F, RTOL)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("batched")
    e0.record()
    X, its, rel, rc = S.solve(F, RTOL)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"batched": {"n": args.batched, "k": F.shape[1], "rc": rc, "n_it_max": max(its),
                                  "ms": e0.elapsed_time(e1), "max_true_relres": max(rel)}}), flush=True)
    S.close()
    if rc != 0:
        sys.exit(1)


def run_sweep(args):
    """Parameter sensitivity on the default beam (GPU timings): one JSON line
    per setting of the coarsening threshold theta, the prolongation limits
    (n_max, kappa_p) and the smoother growth (k_g, rho_g), the other
    parameters at their defaults; FP64 V-cycle, set-up + solve to 1e-8."""
    import torch

    import paper_1902_01715_gb300 as A
    import workloads as W
    torch.cuda.set_device(0)
    A.build()
    A.lib()
    p = W.beam(*args.dims) if args.dims else W.beam()
    d = gpu_problem(A, p)
    grid = [("theta", {"theta": v}) for v in (2, 3, 4, 5, 6, 8, 10)]
    grid += [("n_max", {"n_max": v}) for v in (1, 2, 3, 4, 5)]
    grid += [("kappa_p", {"kappa_p": v}) for v in (10.0, 50.0, 100.0)]
    grid += [("k_g x rho_g", {"k_g": k, "rho_g": r, "k_i": k, "rho_i": r}) for k, r in ((2, 1), (2, 2), (4, 2), (6, 2), (4, 3))]
    for name, over in grid:
        S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], **over)

        def step():
            S.update_values(d["vals"])
            return S.solve(d["f"], RTOL)
        (x, its, rel, rc), ms = _timed(step)
        st = S.stats()
        print(json.dumps({"sweep": name, "params": over, "ms_per_solution": ms, "n_it": its[0], "rc": rc,
                          "setup_ms": st["T_p"] * 1e3, "solve_ms": st["T_s"] * 1e3, "levels": st["nlev"],
                          "C_gd": st["C_gd"], "C_op": st["C_op"], "C_fs": st["C_fs"]}), flush=True)
        S.close()


def run_single(args):
    """One set-up + solve of the workload with no warm-up (the command the
    kernel launch lists under profiles/ are taken from); prints a summary, not
    a bench line."""
    import torch

    import paper_1902_01715_gb300 as A
    import workloads as W
    torch.cuda.set_device(0)
    A.build()
    A.lib()
    p = W.beam(*args.dims) if args.dims else W.beam()
    d = gpu_problem(A, p)
    l0 = A.launch_count()
    S = A.Solver(d["rowptr"], d["col"], d["vals"], d["V0"], vcycle_prec=args.prec)
    x, it, rr, rc = S.solve(d["f"], RTOL)
    torch.cuda.synchronize()
    st = S.stats()
    print(json.dumps({"single": {"dims": [p.nx, p.ny, p.nz], "n_it": it[0], "rc": rc, "setup_ms": st["T_p"] * 1e3,
                                 "solve_ms": st["T_s"] * 1e3, "launches": A.launch_count() - l0}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--micro", action="store_true", help="per-level sparse-product timings only")
    ap.add_argument("--single", action="store_true", help="one set-up + solve, no warm-up (for profilers)")
    ap.add_argument("--sweep", action="store_true", help="parameter sensitivity on the beam (one line per setting)")
    ap.add_argument("--dims", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    help="beam size nx,ny,nz for --single (default 128,32,32)")
    ap.add_argument("--batched", type=int, default=0, metavar="N",
                    help="one batched solve of the N^3 cube with 64 load cases (for profilers)")
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "bf16gp"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the slab, batched and adjoint runs")
    ap.add_argument("--oracle-once", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.oracle_once:
        run_oracle_once(args)
    elif args.single:
        run_single(args)
    elif args.sweep:
        run_sweep(args)
    elif args.micro:
        run_micro(args)
    elif args.batched:
        run_batched(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
