#!/usr/bin/env python3
"""Time to 1e-10 relative residual for cascading-smoother multigrid.

Workload (default): 3D Poisson, 7-point FD on a 256^3 interior grid,
homogeneous Dirichlet, RHS ~ U[-1,1] (seeded); Galerkin hierarchy down to
4^3; additive cascade of depth 3; V(2,2) with reverse pre- / forward
post-smoothing.  One step = setup_hierarchy + setup_cascade + solve from
x = 0 until ||b - A x|| / ||b|| <= 1e-10, inputs resident in HBM.

The chosen form (``value``) keeps the FP64 setup (its least squares in
FP64) and runs the cycle in FP32 inside FP64 iterative refinement; the
plain FP64 form (stationary FP64 V-cycle iteration) is timed
beside it.  Also reported: the sweep kernel's achieved HBM bandwidth
against the measured copy peak, the same step end to end through the C ABI
with host buffers, and the FP64 CPU oracle on the whole workload (all host
threads) and on a one-thread sample.

``--impl reference`` times the oracle alone (the baseline arm).
Multi-GPU (torchrun): independent replicas, one problem per rank.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "time-to-1e-10 residual & smoother GB/s vs HBM peak: chosen vs plain FP64"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "ncu_traffic.json")
FALLBACK_HBM = 6800.0


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256, help="interior nodes per side")
    p.add_argument("--kind", default="additive", choices=["additive", "multiplicative"])
    p.add_argument("--nu", type=int, default=3)
    p.add_argument("--mu", type=int, default=2)
    p.add_argument("--order", default="RF")
    p.add_argument("--cpu-n", type=int, default=128, help="side of the oracle's one-thread sample")
    p.add_argument("--no-extras", action="store_true", help="time the chosen form only")
    p.add_argument("--learned-meshes", type=int, default=2000, help="training meshes of the learned setup")
    p.add_argument("--learned-n", type=int, default=511, help="interior nodes per side of a training mesh")
    p.add_argument("--learned-steps", type=int, default=20000, help="Adam steps")
    p.add_argument("--interface-maxit", type=int, default=300, help="GMRES steps allowed on the interface workload")
    p.add_argument("--interface-precision", default="fp64", choices=["fp32", "fp64"],
                   help="cycle and Krylov precision of the batched interface solve (FP32 Krylov vectors resolve "
                        "~1e-6 of ||r|| per GMRES cycle and restart, which the 1e8-contrast modes punish)")
    p.add_argument("--interface-restart", type=int, default=160,
                   help="GMRES restart of the interface workload (the oracle needs 149 steps at 1023^2 without restart)")
    p.add_argument("--general-n", type=int, default=1535, help="interior nodes per side of the general-path mesh")
    p.add_argument("--stokes-n", type=int, default=256, help="cells per side of the MAC Stokes problem")
    p.add_argument("--overlap-n", type=int, default=767, help="interior nodes per side of the overlapping-block mesh")
    p.add_argument("--overlap-mult-n", type=int, default=255,
                   help="mesh of the multiplicative overlapping-block line (its exact setup fills E along colour chains)")
    p.add_argument("--batch-count", type=int, default=512, help="problems of the batched workload timed")
    p.add_argument("--batch-fp64-count", type=int, default=32,
                   help="problems on which FP32 and FP64 cycles are compared")
    p.add_argument("--krylov", default="gmres_right", choices=["gmres", "gmres_right"],
                   help="GMRES form of the interface and batched workloads (cycle applied left or right)")
    p.add_argument("--batch-maxit", type=int, default=400, help="GMRES steps allowed per problem")
    p.add_argument("--batch-single", type=int, default=4, help="problems also solved on the single-problem path")
    p.add_argument("--batch-profile-count", type=int, default=16, help="problems in the batch profile case")
    p.add_argument("--profile", default="",
                   choices=["", "setup", "step", "step16", "sweep", "multirhs", "blocksetup", "batch", "general",
                            "overlap", "sketch", "mlp", "tcgemm"],
                   help="run one untimed setup (or setup + solve) and exit: the case ncu captures")
    return p.parse_args()


def csrc_hash() -> str:
    """Hash of the sources the sweep kernel is built from (its traffic record
    is void once they change)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2606_12577_gb300", "csrc")
    for f in ("cs_internal.cuh", "cs_stencil.cu"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            t = [v.strip() for v in line.split(",")]
            if len(t) >= 9:
                rows.append(t)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- the oracle
def oracle_step(n, kind, nu, mu, order):
    import oracle
    import problems
    A, b = problems.poisson3d(n)
    t0 = time.perf_counter()
    h = oracle.Hierarchy(A)
    c = oracle.Cascade(h, kind, nu=nu)
    x, it, hist, fin = oracle.solve(h, c, b, method="stationary", mu_pre=mu, mu_post=mu, rf=order == "RF",
                                    tol=1e-10)
    dt = time.perf_counter() - t0
    return dt, it, fin


def cpu_model() -> str:
    """The host CPU's model name (lscpu; /proc/cpuinfo; the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(a, n_full):
    """The FP64 oracle on the host cores: the whole workload on every host
    thread (OpenMP over rows and blocks; results are bitwise those of one
    thread), and one thread on a --cpu-n^3 sample of the same family.
    Measured, not scaled."""
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    dt, it, fin = oracle_step(n_full, a.kind, a.nu, a.mu, a.order)
    oracle.set_threads(1)
    dt1, it1, _ = oracle_step(a.cpu_n, a.kind, a.nu, a.mu, a.order)
    oracle.set_threads(ncores)
    return {"value": dt * 1e3, "unit": "ms", "cores": ncores, "threads": ncores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"the whole workload: FP64 oracle, {n_full}^3, setup + stationary solve to 1e-10 "
                      f"({it} cycles, final {fin:.2e}) on {ncores} host threads; measured, not scaled",
            "one_thread": {"value": dt1 * 1e3, "unit": "ms", "threads": 1,
                           "workload": f"the same family at {a.cpu_n}^3 (setup + solve, {it1} cycles), "
                                       f"one thread, measured, not scaled"}}


def run_reference(a):
    """The baseline arm: each step is the whole workload (setup + solve to
    1e-10) in the FP64 oracle on every host thread."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cfg = config(a)
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    for _ in range(a.warmup):
        oracle_step(a.n, a.kind, a.nu, a.mu, a.order)
    ts = []
    for _ in range(a.steps):
        dt, it, fin = oracle_step(a.n, a.kind, a.nu, a.mu, a.order)
        ts.append(dt)
    v = statistics.mean(ts) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "ms", "cores": ncores, "threads": ncores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"each step: the whole workload in the FP64 oracle ({a.n}^3, setup + "
                                       f"stationary solve to 1e-10, {it} cycles) on {ncores} host threads; "
                                       f"measured, not scaled"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value: float, world: int, device) -> float:
    """The largest of every rank's value (all ranks receive it): the job's
    time is its slowest replica's.  One rank: the value itself."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config(a):
    return {"workload": f"3D Poisson 7-point FD {a.n}^3 interior, Dirichlet, RHS U[-1,1] seed 2002; "
                        f"{a.kind} cascade nu={a.nu}, V({a.mu},{a.mu}) {a.order}, Galerkin to 4^3, "
                        f"setup + solve to 1e-10",
            "global_batch": 1, "unknowns": a.n ** 3, "parallelism": f"replicas x{a.gpus}",
            "l2": "inputs larger than L2 (A alone is 0.94 GB)"}


def learned_section(a, cmg, problems, dev):
    """Learned setup (workload 5): Q1 elements on jittered meshes, log-normal
    coefficients (sigma 2, correlation 16 elements), 3x3-node blocks,
    additive nu = 3.  The network is trained on labels of the exact setup of
    seeded training meshes, then the exact and learned setups of a 511^2
    evaluation mesh are compared (setup time, GMRES iterations to 1e-10,
    convergence factor)."""
    import numpy as np
    import torch

    import oracle
    from paper_2606_12577_gb300 import learned
    import multiprocessing as mpc
    nb_side = -(-a.learned_n // 3)
    nproc = max(1, min(16, os.cpu_count() or 1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # the meshes stream from a spawn pool of host processes (the parent holds
    # a CUDA context) while the GPU labels the ones that have arrived
    with mpc.get_context("spawn").Pool(nproc) as pool:
        stream_in = pool.imap(_q1_mesh, [(a.learned_n, 50000 + k) for k in range(a.learned_meshes)], chunksize=2)
        X, T = learned.make_dataset(stream_in, total=a.learned_meshes * nb_side * nb_side)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    mdl = cmg.MLP(X.shape[1], 128, T.shape[1], max_batch=8192, seed=1)
    t0 = time.perf_counter()
    hist = learned.train(mdl, X, T, steps=a.learned_steps, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    A5 = problems.q1_jittered(511, 10000)
    learned.setup_pair(A5, mdl)  # warm-up (graph capture, pool)
    h5, res = learned.setup_pair(A5, mdl)
    b5 = torch.tensor(problems.rhs(A5.N, 10000), dtype=torch.float64, device=dev)
    out = {"workload": "Q1 FE, jittered 512^2-element mesh (511^2 unknowns), log-normal kappa (sigma 2, corr 16h), "
                       "3x3-node blocks (9x9 Lambda), additive nu=3, GMRES V(1,1) RF to 1e-10",
           "training": {"meshes": a.learned_meshes, "mesh_unknowns": a.learned_n ** 2, "samples": int(X.shape[0]),
                        "dataset_gb": (X.numel() + T.numel()) * 4 / 1e9, "steps": a.learned_steps, "batch": 4096,
                        "epochs": a.learned_steps * 4096 / int(X.shape[0]), "loss_first": float(np.mean(hist[:10])),
                        "loss_last": float(np.mean(hist[-50:])), "generate_and_label_s": t_label,
                        "host_processes": nproc, "train_s": t_train,
                        "gemm": "tcgen05 BF16 (FP32 factors as hi + lo pairs), FP32 accumulation in TMEM"}}
    del X, T
    torch.cuda.empty_cache()
    used, ratio = cmg.learned_status(res["learned"][0])
    out["predicted_blocks_in_use"] = bool(used == 1)
    out["level1_objective_ratio_predicted"] = ratio
    out["blocks"] = cmg.learned_stats(res["learned"][0])
    # the method without the network at the learned path's setup cost: the
    # exact level-1 blocks repeated nu = 3 times (a nu = 1 cascade applied
    # mu = 3 times per smoothing: the same sweeps per cycle)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cmg.setup_cascade(h5, "additive", nu=1)
    torch.cuda.synchronize()
    e0.record(s)
    c1 = cmg.setup_cascade(h5, "additive", nu=1)
    e1.record(s)
    torch.cuda.synchronize()
    res["level1_repeated"] = (c1, e0.elapsed_time(e1), None)
    for name in ("exact", "learned", "level1_repeated"):
        c, setup_ms, wall_ms = res[name]
        mu = 3 if name == "level1_repeated" else 1
        x = torch.zeros(A5.N, dtype=torch.float64, device=dev)
        cmg.solve(h5, c, b5, x, method="gmres", tol=1e-10, maxit=300, mu_pre=mu, mu_post=mu,
                  raise_on_error=False)  # warm-up (graph capture of the cycle)
        x.zero_()
        torch.cuda.synchronize()
        e0.record(s)
        info = cmg.solve(h5, c, b5, x, method="gmres", tol=1e-10, maxit=300, mu_pre=mu, mu_post=mu,
                         raise_on_error=False)
        e1.record(s)
        torch.cuda.synchronize()
        solve_ms = e0.elapsed_time(e1)
        x = torch.zeros(A5.N, dtype=torch.float64, device=dev)
        st = cmg.solve(h5, c, b5, x, method="stationary", tol=1e-10, maxit=40, mu_pre=mu, mu_post=mu,
                       raise_on_error=False)
        out[name] = {"setup_ms": setup_ms, "gmres_solve_ms": solve_ms, "total_ms": setup_ms + solve_ms,
                     "gmres_iterations": info.iterations, "converged": info.converged,
                     "rho_gmres": oracle.rho_from_history(info.history) if len(info.history) > 2 else None,
                     "rho_stationary": oracle.rho_from_history(st.history) if len(st.history) > 2 else None}
    return out


def small_2d_section(a, cmg, problems, dev):
    """The small latency-bound case: 2D Poisson 5-point 64^2, Dirichlet, point
    blocks, additive nu = 3, V(1,1) RF, Galerkin levels to 4^2 and the dense
    coarsest solve, FP64 throughout, RHS U[-1,1] (seed 1000): setup + solve
    to 1e-10 per step (CUDA events, 20 steps after 3 warm-up), stationary and
    right-preconditioned GMRES; the V-cycle is graph-captured."""
    import torch
    A = problems.poisson(2, 64)
    coeff = torch.tensor(A.coeff, dtype=torch.float64, device=dev)
    b = torch.tensor(problems.rhs(A.N, 1000), dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream()
    out = {"workload": "2D Poisson 5-point 64^2, additive nu=3, V(1,1) RF, FP64 setup + solve to 1e-10"}
    for method in ("stationary", "gmres_right"):
        info = [None]

        def one():
            h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff)
            c = cmg.setup_cascade(h, "additive", nu=3)
            x = torch.zeros(A.N, dtype=torch.float64, device=dev)
            info[0] = cmg.solve(h, c, b, x, method=method, tol=1e-10, mu_pre=1, mu_post=1, order="RF")
            return h, c

        for _ in range(3):
            h, c = one()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(20):
            one()
        e1.record(s)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / 20
        x = torch.zeros(A.N, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(20):
            x.zero_()
            cmg.solve(h, c, b, x, method=method, tol=1e-10, mu_pre=1, mu_post=1, order="RF")
        e1.record(s)
        torch.cuda.synchronize()
        out[method] = {"setup_plus_solve_ms": step_ms, "solve_ms": e0.elapsed_time(e1) / 20,
                       "iterations": info[0].iterations, "final_rel_residual": float(info[0].final_rel_residual)}
    return out


def tensor_core_section(a, cmg, dev):
    """The learned setup's tcgen05 BF16 GEMM (C = A B^T, FP32 accumulation in
    tensor memory) on an 8192^3 problem, against the measured cuBLAS BF16
    burst peak, and the network's training step at batch 4096 (nine GEMMs,
    every FP32 factor as a BF16 hi + lo pair)."""
    import torch
    try:
        with open(PEAKS) as f:
            peak = float(json.load(f)["bf16_tflops"])
        src = "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except Exception:
        peak, src = 1900.0, "fallback"
    n = 8192
    g = torch.Generator(device=dev).manual_seed(3)
    A = torch.randn(n, n, device=dev, generator=g).to(torch.bfloat16)
    B = torch.randn(n, n, device=dev, generator=g).to(torch.bfloat16)
    for _ in range(3):
        cmg.tc_gemm_bf16(A, B)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        C = cmg.tc_gemm_bf16(A, B)
    e1.record(s)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / reps * 1e-3
    tf = 2.0 * n ** 3 / t / 1e12
    ref = (A[:64].float() @ B[:64].float().T)
    err = float((C[:64, :64] - ref).abs().max() / ref.abs().max())
    del A, B, C
    m = cmg.MLP(225, 128, 243, max_batch=4096, seed=1)
    Xm = torch.randn(4096, 225, device=dev, generator=g) * 0.3
    Tm = torch.randn(4096, 243, device=dev, generator=g) * 0.1
    for _ in range(3):
        m.train_step(Xm, Tm, 1e-3, with_loss=True)
    torch.cuda.synchronize()
    e0.record(s)
    for k in range(50):
        m.train_step(Xm, Tm, 1e-3, with_loss=(k == 49))
    e1.record(s)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return {"gemm_8192": {"bound": "tensor", "kernel": "k_tc_gemm_persistent (tcgen05.mma kind::f16, 128x256 tiles, TMA 128B "
                                                        "swizzle, 4 stages, two TMEM accumulators)", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                          "frac": tf / peak, "launch_ms": t * 1e3, "peak_source": src, "max_rel_err_64x64": err},
            "mlp_train_step_ms_b4096": e0.elapsed_time(e1) / 50}


def interface_section(a, cmg, problems, dev):
    """Elliptic interface workload: 1024^2, ~200 inclusions (contrast
    1e-4..1e4), 2x2-node blocks, additive nu = 3, 32 seeded RHS, GMRES(30)
    (--krylov: the cycle applied on the right by default) with V(1,1)-RF FP32
    cycles to 1e-10 per RHS (at most --interface-maxit steps).  The 32 RHS
    are solved together in one batched launch (RHS contiguous per node,
    block steps over (block, RHS) items); the single-RHS path solves the
    first RHS for comparison."""
    import torch
    Ai = problems.interface2d(1024)
    m = 32
    B = problems.rhs(Ai.N, problems.config_seed(3), m)
    s = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    bd = torch.tensor(B.reshape(-1), dtype=torch.float64, device=dev)
    cmg.setup_many([Ai], kind="additive", nu=3, lowp=True, block=2)  # warm-up
    torch.cuda.synchronize()
    e[0].record(s)
    hs, cs = cmg.setup_many([Ai], kind="additive", nu=3, lowp=True, block=2)
    e[1].record(s)
    bt = cmg.Batch(hs, cs, [m], precision=a.interface_precision, method=a.krylov, autotune=True,
                   restart=a.interface_restart)
    x = torch.zeros_like(bd)
    bt.solve([bd], [x], tol=1e-10, maxit=2, raise_on_error=False)  # warm-up (graph)
    x.zero_()
    torch.cuda.synchronize()
    l0 = cmg.kernel_launches()
    e[2].record(s)
    info = bt.solve([bd], [x], tol=1e-10, maxit=a.interface_maxit, raise_on_error=False)[0]
    e[3].record(s)
    torch.cuda.synchronize()
    launches = cmg.kernel_launches() - l0
    rel = []
    Xm = x.view(Ai.N, m)
    out = {"workload": "elliptic interface 1024^2, 200 inclusions (contrast 1e-4..1e4), 2x2-node blocks, additive "
                       f"nu=3, 32 RHS, {a.krylov}({a.interface_restart}) V(1,1) RF {a.interface_precision} cycles and "
                       "Krylov vectors to 1e-10, the 32 RHS in one batched launch",
           "precision": a.interface_precision,
           "krylov": a.krylov,
           "setup_ms": e[0].elapsed_time(e[1]), "solve_ms": e[2].elapsed_time(e[3]),
           "gmres_steps": info.iterations, "all_converged": bool(info.converged),
           "worst_rel_residual": float(info.final_rel_residual), "gpu_launches": int(launches),
           "schedule": {k: v for k, v in bt.config().items() if k != "tuned"}}
    # the single-RHS path on the first RHS, for comparison
    x1 = torch.zeros(Ai.N, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    e[2].record(s)
    i1 = cmg.solve(hs[0], cs[0], bd.view(Ai.N, m)[:, 0].contiguous(), x1, method=a.krylov, precision="fp32",
                   tol=1e-10, maxit=a.interface_maxit, restart=a.interface_restart, raise_on_error=False)
    e[3].record(s)
    torch.cuda.synchronize()
    out["single_rhs_path_first_rhs"] = {"solve_ms": e[2].elapsed_time(e[3]), "gmres_steps": i1.iterations,
                                        "converged": bool(i1.converged),
                                        "rel_residual": float(i1.final_rel_residual)}
    del bt, hs, cs, Xm, rel
    return out


def stencil_rel_residual(A, x, b, m, dev):
    """max over right-hand sides of ||b - A x|| / ||b|| for a 2D stencil
    operator (RHS-contiguous vectors), in FP64 torch arithmetic."""
    import torch
    nx, ny = A.n[0], A.n[1]
    X = x.view(ny, nx, m)
    Bm = b.view(ny, nx, m)
    C = torch.tensor(A.coeff, dtype=torch.float64, device=dev).view(-1, ny, nx, 1)
    Y = torch.zeros_like(X)
    for s_, (dx, dy, _) in enumerate(A.offsets):
        sh = torch.zeros_like(X)
        sh[max(-dy, 0):ny + min(-dy, 0), max(-dx, 0):nx + min(-dx, 0)] = \
            X[max(dy, 0):ny + min(dy, 0), max(dx, 0):nx + min(dx, 0)]
        Y += C[s_] * sh
    r = (Bm - Y).reshape(-1, m).norm(dim=0) / Bm.reshape(-1, m).norm(dim=0).clamp_min(1e-300)
    return float(r.max())


def _batch_problem(k):
    import problems
    return problems.batch_problem(k)


def _q1_mesh(args):
    """One training mesh of the learned setup (runs in a pool worker)."""
    import problems as pr
    n, seed = args
    return pr.q1_jittered(n, seed)


def make_batch_problems(K):
    """The first K problems of the batched workload, generated on the host
    cores (a spawn pool: the parent already holds a CUDA context)."""
    import multiprocessing as mpc
    nproc = max(1, min(16, (os.cpu_count() or 1), K // 8))
    if nproc == 1:
        return [_batch_problem(k) for k in range(K)]
    with mpc.get_context("spawn").Pool(nproc) as pool:
        return pool.map(_batch_problem, range(K), chunksize=4)


def batch_section(a, cmg, problems, dev):
    """Batched solve (many uneven problems): the first ``--batch-count``
    problems (default all 512) of the batched workload (2D
    variable-coefficient Poisson, sides U{33..513}, 1..8 RHS each,
    correlated log-uniform coefficients on [1e-3, 1e3]), red-black
    multiplicative nu = 3, V(1,1) RF, GMRES(30) (--krylov) to 1e-10 per RHS
    with FP32 cycles: one persistent cooperative launch per solve (autotuned
    schedule).  On the first ``--batch-fp64-count`` problems FP32 and FP64
    cycles are compared, and the single-problem path solves each RHS of the
    first problems in turn."""
    import numpy as np
    import torch
    K = a.batch_count
    t0 = time.perf_counter()
    P = make_batch_problems(K)
    t_gen = time.perf_counter() - t0
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"first {K} problems of the 512-problem batch: 2D variable-coefficient Poisson, sides "
                       "U{33..513}, 1..8 RHS, log-uniform coefficients [1e-3,1e3] (correlation 8h); multiplicative "
                       f"nu=3 red-black, V(1,1) RF, {a.krylov}(30) to 1e-10 per RHS",
           "krylov": a.krylov, "problems": K, "unknowns": int(sum(A.N for A, _, _ in P)),
           "rhs_unknowns": int(sum(A.N * m for A, m, _ in P)), "generate_s": t_gen}
    cmg.setup_many([A for A, _, _ in P[:2]], kind="multiplicative", nu=3, lowp=True)  # warm-up
    torch.cuda.synchronize()
    e0.record(s)
    hs, cs = cmg.setup_many([A for A, _, _ in P], kind="multiplicative", nu=3, lowp=True)
    e1.record(s)
    torch.cuda.synchronize()
    out["setup_ms"] = e0.elapsed_time(e1)
    bs = [torch.tensor(b, device=dev) for _, _, b in P]

    def run(nprob, prec, tune):
        t0 = time.perf_counter()
        bt = cmg.Batch(hs[:nprob], cs[:nprob], [m for _, m, _ in P[:nprob]], precision=prec, method=a.krylov,
                       autotune=tune)
        plan_s = time.perf_counter() - t0
        xs = [torch.zeros_like(b) for b in bs[:nprob]]
        torch.cuda.synchronize()
        l0 = cmg.kernel_launches()
        e0.record(s)
        infos = bt.solve(bs[:nprob], xs, tol=1e-10, maxit=a.batch_maxit, raise_on_error=False)
        e1.record(s)
        torch.cuda.synchronize()
        its = [i.iterations for i in infos]
        res = {"problems": nprob, "solve_ms": e0.elapsed_time(e1), "converged": int(sum(i.converged for i in infos)),
               "all_converged": bool(all(i.converged for i in infos)),
               "iterations_min_median_max": [int(np.min(its)), int(np.median(its)), int(np.max(its))],
               "worst_rel_residual": float(max(i.final_rel_residual for i in infos)),
               "gpu_launches": int(cmg.kernel_launches() - l0), "plan_s": plan_s,
               "plan_bytes": int(bt.nbytes())}
        if tune:
            res["schedule"] = bt.config()
        # the true residual of every problem and RHS, recomputed here from the
        # stencil in FP64 with plain tensor arithmetic (a check beside the
        # solver's own residual, outside the timed region)
        res["checked_worst_rel_residual"] = max(
            stencil_rel_residual(P[p][0], xs[p], bs[p], P[p][1], dev) for p in range(nprob))
        del bt, xs
        torch.cuda.empty_cache()
        return res

    out["gmres_fp32_cycles"] = run(K, "fp32", True)
    nsub = min(K, a.batch_fp64_count)
    out[f"first_{nsub}"] = {"gmres_fp32_cycles": run(nsub, "fp32", False), "gmres_fp64_cycles": run(nsub, "fp64", False)}
    # the single-problem path on the first problems, one RHS at a time
    nsub = min(K, a.batch_single)
    torch.cuda.synchronize()
    e0.record(s)
    l0 = cmg.kernel_launches()
    conv = 0
    for p in range(nsub):
        A, m, _ = P[p]
        B = bs[p].view(A.N, m)
        for r in range(m):
            x1 = torch.zeros(A.N, dtype=torch.float64, device=dev)
            conv += cmg.solve(hs[p], cs[p], B[:, r].contiguous(), x1, method=a.krylov, precision="fp32", tol=1e-10,
                              maxit=a.batch_maxit, raise_on_error=False).converged
    e1.record(s)
    torch.cuda.synchronize()
    out["single_problem_path"] = {"problems": nsub, "rhs_unknowns": int(sum(P[p][0].N * P[p][1] for p in range(nsub))),
                                  "solve_ms": e0.elapsed_time(e1), "rhs_converged": int(conv),
                                  "gpu_launches": int(cmg.kernel_launches() - l0)}
    del hs, cs, bs
    return out


def cascade_forms_section(a, cmg, A, coeff, bd, dev):
    """The headline workload (3D Poisson 256^3, V(2,2) RF, FP32 cycles in FP64
    refinement to 1e-10) with other cascades: multiplicative red-black
    nu = 2 and 3 (exact setup), and the sketched setup (32 Rademacher
    columns, FP32 sketch vectors) for multiplicative nu = 3 and 4 and additive
    nu = 3.  The exact multiplicative nu = 4 setup would keep radius-8 residual
    rows (about 94 GB in FP64 at 256^3); the sketched one keeps two N x 32
    arrays.  Each form: one untimed run, then one run timed with events
    around the setup and the solve."""
    import torch
    forms = [("multiplicative", 2, {}), ("multiplicative", 3, {}),
             ("multiplicative", 3, {"sketch": 32, "setup_precision": "fp32"}),
             ("multiplicative", 4, {"sketch": 32, "setup_precision": "fp32"}),
             ("additive", 3, {"sketch": 32, "setup_precision": "fp32"})]
    s = torch.cuda.current_stream()
    out = {}
    for kind, nu, kw in forms:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        res = None
        for rep in range(2):
            torch.cuda.synchronize()
            ev[0].record(s)
            h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff)
            c = cmg.setup_cascade(h, kind, nu=nu, lowp=True, sketch_seed=2024, **kw)
            ev[1].record(s)
            x = torch.zeros(A.N, dtype=torch.float64, device=dev)
            info = cmg.solve(h, c, bd, x, method="refine", precision="fp32", tol=1e-10, mu_pre=a.mu,
                             mu_post=a.mu, order=a.order, maxit=100, raise_on_error=False)
            ev[2].record(s)
            torch.cuda.synchronize()
            res = {"setup_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
                   "total_ms": ev[0].elapsed_time(ev[2]), "iterations": info.iterations,
                   "converged": bool(info.converged), "final_rel_residual": float(info.final_rel_residual),
                   "cascade_bytes": int(c.nbytes()) if hasattr(c, "nbytes") else None}
            del h, c, x
            torch.cuda.empty_cache()
        name = f"{kind}_nu{nu}" + ("_sketch32" if kw.get("sketch") else "_exact")
        out[name] = res
    return out


def general_section(a, cmg, problems, dev):
    """The general sparse path (CSR operator, user transfers, index-driven
    kernels) on the jittered Q1 mesh of --general-n interior nodes per side
    in grid order (the operator larger than L2): hierarchy and additive
    nu = 2 cascade setup times, the roofline of the point-block cascade step
    (one thread per row reading its CSR row), and right-preconditioned
    GMRES V(1,1) to 1e-10."""
    import torch
    t0 = time.perf_counter()
    u = problems.unstructured_q1(a.general_n, 7, renumber=False)
    t_gen = time.perf_counter() - t0
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev[0].record(s)
    hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, seed=3)
    ev[1].record(s)
    cg = cmg.gsetup_cascade(hg, "additive", nu=2)
    ev[2].record(s)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lev = hg.level(0)
    N, nnz = lev["N"], lev["nnz"]
    b = torch.rand(N, dtype=torch.float64, device=dev)
    xs = [torch.rand(N, dtype=torch.float64, device=dev) for _ in range(2)]
    for k in range(3):
        cmg.gsweep(hg, cg, 0, k % 2, b, xs[k % 2], xs[(k + 1) % 2])
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for k in range(reps):
        cmg.gsweep(hg, cg, 0, k % 2, b, xs[k % 2], xs[(k + 1) % 2])
    e1.record(s)
    torch.cuda.synchronize()
    t_sweep = e0.elapsed_time(e1) / reps * 1e-3
    # algorithmic bytes: values and column indices of A, row pointers,
    # Lambda, b, x read, x written
    nbytes = nnz * 12 + (N + 1) * 8 + 4 * 8 * N
    peak, src = peaks()
    bd = torch.tensor(problems.rhs(N, 3), dtype=torch.float64, device=dev)
    x = torch.zeros(N, dtype=torch.float64, device=dev)
    cmg.gsolve(hg, cg, bd, x, method="gmres_right", tol=1e-10, maxit=100)  # warm-up
    x.zero_()
    torch.cuda.synchronize()
    e0.record(s)
    info = cmg.gsolve(hg, cg, bd, x, method="gmres_right", tol=1e-10, maxit=100, raise_on_error=False)
    e1.record(s)
    torch.cuda.synchronize()
    return {"workload": f"jittered Q1 {a.general_n}^2 interior nodes (grid order) as a general CSR operator "
                        f"({N} unknowns, {nnz} entries), user bilinear transfers, Galerkin levels, greedy colouring, "
                        "additive nu=2 point-block cascade, right GMRES V(1,1) RF to 1e-10",
            "generate_s": t_gen, "hierarchy_ms": ev[0].elapsed_time(ev[1]), "cascade_ms": ev[1].elapsed_time(ev[2]),
            "setup_wall_s": wall, "levels": hg.nlevels,
            "colours": [hg.level(l)["ncolours"] for l in range(hg.nlevels)],
            "sweep_roofline": {"bound": "hbm", "kernel": "k_gsweep_point (CSR row per thread, additive step)",
                               "achieved": nbytes / t_sweep / 1e9, "peak": peak, "unit": "GB/s",
                               "frac": nbytes / t_sweep / 1e9 / peak, "algorithmic_bytes_per_launch": nbytes,
                               "launch_ms": t_sweep * 1e3, "peak_source": src},
            "solve_ms": e0.elapsed_time(e1), "iterations": info.iterations, "converged": bool(info.converged),
            "final_rel_residual": float(info.final_rel_residual)}


def stokes_section(a, cmg, problems, dev):
    """Stokes prescaling on a synthetic saddle-point problem: the MAC
    staggered-grid steady Stokes operator on --stokes-n^2 cells with no-slip
    walls, (d+1)-DOF cell blocks on every level, staggered transfers,
    Galerkin levels, additive nu = 3, right GMRES V(1,1) to 1e-10, with the
    Stokes prescaling (q = 1 and q = infinity) and without prescaling."""
    import torch
    t0 = time.perf_counter()
    u = problems.mac_stokes_2d(a.stokes_n)
    t_gen = time.perf_counter() - t0
    hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=u["blocks"], fields=u["fields"], seed=3)
    N = u["A"].shape[0]
    bd = torch.tensor(problems.rhs(N, 5), dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream()
    out = {"workload": f"MAC staggered-grid steady Stokes, {a.stokes_n}^2 cells, no-slip walls ({N} unknowns), "
                       "cell blocks of pressure + right and top faces, Galerkin levels, additive nu=3, right GMRES "
                       "V(1,1) RF to 1e-10", "generate_s": t_gen, "levels": hg.nlevels}
    for mode in ("stokes1", "stokesinf", "none"):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record(s)
        cg = cmg.gsetup_cascade(hg, "additive", nu=3, prescale=mode)
        ev[1].record(s)
        x = torch.zeros(N, dtype=torch.float64, device=dev)
        info = cmg.gsolve(hg, cg, bd, x, method="gmres_right", tol=1e-10, maxit=300, raise_on_error=False)
        ev[2].record(s)
        torch.cuda.synchronize()
        out[mode] = {"cascade_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
                     "iterations": info.iterations, "converged": bool(info.converged),
                     "final_rel_residual": float(info.final_rel_residual)}
        del cg
    return out


def overlap_section(a, cmg, problems, dev):
    """Overlapping blocks (Sec. 3.6.2) and PCG (SM "On preconditioned
    conjugate gradient") on the jittered Q1 mesh of --overlap-n interior
    nodes per side: the nodes of every element form a block (an interior
    node lies in 4), additive nu = 2 with theta-averaged fusion and right
    GMRES, the same with the SPD projection and PCG, and the multiplicative
    form (colours separate blocks sharing a node) with right GMRES on the
    smaller --overlap-mult-n mesh (its 19 colours let a node's row of E grow
    along chains of colour steps, so its exact setup costs far more than the
    additive one); all V(1,1) RF to 1e-10."""
    import torch
    t0 = time.perf_counter()
    u = problems.unstructured_q1(a.overlap_n, 7, renumber=False)
    t_gen = time.perf_counter() - t0
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=u["cells"], seed=3)
    t_h = time.perf_counter() - t0
    N = u["A"].shape[0]
    bd = torch.tensor(problems.rhs(N, 5), dtype=torch.float64, device=dev)
    out = {"workload": f"jittered Q1 {a.overlap_n}^2 interior nodes ({N} unknowns), element blocks of up to 4 "
                       f"nodes overlapping ({hg.level(0)['nblocks']} blocks), Galerkin levels, V(1,1) RF to 1e-10",
           "generate_s": t_gen, "hierarchy_s": t_h, "levels": hg.nlevels, "colours_level0": hg.level(0)["ncolours"]}
    um = problems.unstructured_q1(a.overlap_mult_n, 7, renumber=False)
    hm = cmg.gsetup_hierarchy(um["A"], um["Ps"], rscale=0.25, blocks=um["cells"], seed=3)
    bm = torch.tensor(problems.rhs(um["A"].shape[0], 5), dtype=torch.float64, device=dev)
    for name, kind, spd, method in (("additive_nu2_gmres_right", "additive", False, "gmres_right"),
                                    ("additive_nu2_spd_pcg", "additive", True, "pcg"),
                                    (f"multiplicative_nu2_gmres_right_{a.overlap_mult_n}", "multiplicative", False,
                                     "gmres_right")):
        if kind == "multiplicative":
            hg, bd, N = hm, bm, um["A"].shape[0]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record(s)
        cg = cmg.gsetup_cascade(hg, kind, nu=2, spd=spd)
        ev[1].record(s)
        x = torch.zeros(N, dtype=torch.float64, device=dev)
        info = cmg.gsolve(hg, cg, bd, x, method=method, tol=1e-10, maxit=300, raise_on_error=False)
        ev[2].record(s)
        torch.cuda.synchronize()
        out[name] = {"unknowns": N, "cascade_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
                     "iterations": info.iterations, "converged": bool(info.converged),
                     "final_rel_residual": float(info.final_rel_residual)}
        del cg
    return out


# ------------------------------------------------------------------- ours
def main():
    a = args_()
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    if world > 1:
        dist.barrier()
    ge.build()
    import paper_2606_12577_gb300 as cmg
    import problems

    if a.profile == "multirhs":  # the multi-RHS block steps the bench times (interface problem, n^2)
        Ai = problems.interface2d(a.n)
        hb = cmg.setup_hierarchy(Ai.dim, Ai.n, Ai.offsets, torch.tensor(Ai.coeff, device=dev), block=2)
        cb = cmg.setup_cascade(hb, "additive", nu=3, lowp=True)
        Xb = [torch.rand(Ai.N * 32, device=dev, dtype=torch.float32) for _ in range(2)]
        Bb = torch.rand(Ai.N * 32, device=dev, dtype=torch.float32)
        for k in range(5):
            cmg.sweep_rhs(hb, cb, 0, k % 3, Bb, Xb[k % 2], Xb[(k + 1) % 2], 32)
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "n": a.n}), flush=True)
        return

    if a.profile == "batch":  # one batched GMRES solve of the first problems of the batched workload, 3 steps
        P = [problems.batch_problem(k) for k in range(a.batch_profile_count)]
        hs, cs = cmg.setup_many([A for A, _, _ in P], kind="multiplicative", nu=3, lowp=True)
        bt = cmg.Batch(hs, cs, [m for _, m, _ in P], precision="fp32", method="gmres", threads=256, tiles_per_cta=4)
        bs = [torch.tensor(b, device=dev) for _, _, b in P]
        xs = [torch.zeros_like(b) for b in bs]
        bt.solve(bs, xs, tol=1e-300, maxit=3, raise_on_error=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "problems": len(P), "launches": cmg.kernel_launches()}), flush=True)
        return

    if a.profile in ("general", "overlap"):  # general-path setup and five additive steps on a jittered Q1 mesh
        nq = a.general_n if a.profile == "general" else a.overlap_n
        u = problems.unstructured_q1(nq, 7, renumber=False)
        hg = cmg.gsetup_hierarchy(u["A"], u["Ps"], rscale=0.25, blocks=u["cells"] if a.profile == "overlap" else None,
                                  seed=3)
        cg = cmg.gsetup_cascade(hg, "additive", nu=2)
        N = hg.N(0)
        bg = torch.rand(N, dtype=torch.float64, device=dev)
        xg = [torch.rand(N, dtype=torch.float64, device=dev) for _ in range(2)]
        for k in range(5):
            cmg.gsweep(hg, cg, 0, k % 2, bg, xg[k % 2], xg[(k + 1) % 2])
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "n": nq, "launches": cmg.kernel_launches()}), flush=True)
        return

    if a.profile == "tcgemm":  # three 8192^3 BF16 products on the tensor cores (the persistent kernel)
        g = torch.Generator(device=dev).manual_seed(3)
        At = torch.randn(8192, 8192, device=dev, generator=g).to(torch.bfloat16)
        Bt = torch.randn(8192, 8192, device=dev, generator=g).to(torch.bfloat16)
        for _ in range(3):
            cmg.tc_gemm_bf16(At, Bt)
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "launches": cmg.kernel_launches()}), flush=True)
        return

    if a.profile == "mlp":  # five training steps of the learned-setup network at batch 4096 (tensor-core GEMMs)
        m = cmg.MLP(225, 128, 243, max_batch=4096, seed=1)
        g = torch.Generator(device=dev).manual_seed(5)
        Xm = torch.randn(4096, 225, device=dev, generator=g) * 0.3
        Tm = torch.randn(4096, 243, device=dev, generator=g) * 0.1
        for k in range(5):
            m.train_step(Xm, Tm, 1e-3, with_loss=(k == 4))
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "launches": cmg.kernel_launches()}), flush=True)
        return

    if a.profile == "sketch":  # the sketched multiplicative setup (s = 32 columns) on the 3D Poisson problem
        As, _ = problems.poisson3d(a.n)
        hs = cmg.setup_hierarchy(As.dim, As.n, As.offsets, torch.tensor(As.coeff, dtype=torch.float64, device=dev))
        cmg.setup_cascade(hs, "multiplicative", nu=a.nu, sketch=32, sketch_seed=2024, setup_precision="fp32")
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "n": a.n, "launches": cmg.kernel_launches()}), flush=True)
        return

    if a.profile == "blocksetup":  # the exact 3x3-block setup of the learned-setup workload (Q1, n^2)
        Aq = problems.q1_jittered(a.n, 10000)
        hq = cmg.setup_hierarchy(Aq.dim, Aq.n, Aq.offsets, torch.tensor(Aq.coeff, device=dev), block=3)
        cmg.setup_cascade(hq, "additive", nu=3)
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "n": a.n, "launches": cmg.kernel_launches()}), flush=True)
        return

    A, b = problems.poisson3d(a.n)
    coeff = torch.tensor(A.coeff, dtype=torch.float64, device=dev)
    bd = torch.tensor(b, dtype=torch.float64, device=dev)
    mu = a.mu

    def step(precision, method, lowp, out=None, setup="fp64"):
        h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff)
        c = cmg.setup_cascade(h, a.kind, nu=a.nu, lowp=lowp, setup_precision=setup)
        x = torch.zeros(A.N, dtype=torch.float64, device=dev)
        info = cmg.solve(h, c, bd, x, method=method, precision=precision, tol=1e-10, mu_pre=mu, mu_post=mu,
                         order=a.order, raise_on_error=precision != "bf16")
        if out is not None:
            out.append(info)
        return h, c, x

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        barrier()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)

    if a.profile:
        h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff)
        c = cmg.setup_cascade(h, a.kind, nu=a.nu, lowp=2 if a.profile == "step16" else True,
                              setup_precision="fp32" if a.profile in ("setup", "step") else "fp64")
        if a.profile in ("step", "step16"):
            x = torch.zeros(A.N, dtype=torch.float64, device=dev)
            cmg.solve(h, c, bd, x, method="refine", precision="bf16" if a.profile == "step16" else "fp32",
                      tol=1e-10, mu_pre=mu, mu_post=mu, order=a.order)
        if a.profile == "sweep":  # the FP32 finest-level steps the roofline loop times
            xb = [torch.rand(A.N, device=dev, dtype=torch.float32) for _ in range(2)]
            b32 = torch.rand(A.N, device=dev, dtype=torch.float32)
            for k in range(5):
                cmg.sweep(h, c, 0, k % a.nu, b32, xb[k % 2], xb[(k + 1) % 2],
                          colour=-1 if a.kind == "additive" else 0)
        torch.cuda.synchronize()
        print(json.dumps({"profile": a.profile, "n": a.n, "launches": cmg.kernel_launches()}), flush=True)
        return

    infos = []
    # ---- chosen form: the setup's products R = A~ E and the E rows in FP32
    # (inner products summed in FP64 over FP32 chunks, every lambda solved
    # and stored in FP64), FP32 cycles in FP64 iterative refinement
    for _ in range(a.warmup):
        step("fp32", "refine", True, setup="fp32")
    clk = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    l0 = cmg.kernel_launches()
    clk.start()
    ms = timed(lambda: step("fp32", "refine", True, infos, setup="fp32"), a.steps, 0)
    clocks = clk.stop()
    launches = cmg.kernel_launches() - l0
    it_chosen = infos[-1].iterations
    res_chosen = infos[-1].final_rel_residual

    result = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
              "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
              "dtype": "f32 cycle + f64 refinement; f32 setup products, f64 least squares", "data": "synthetic",
              "config": config(a),
              "iterations": it_chosen, "final_rel_residual": res_chosen, "gpu_launches": launches,
              "clocks": clocks, "solves_per_s_all_gpus": world * 1e3 / ms}

    if not a.no_extras:
        # split: setup vs solve (events around each phase, one extra run)
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(s)
        h = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff)
        c = cmg.setup_cascade(h, a.kind, nu=a.nu, lowp=True, setup_precision="fp32")
        ev[1].record(s)
        x = torch.zeros(A.N, dtype=torch.float64, device=dev)
        cmg.solve(h, c, bd, x, method="refine", precision="fp32", tol=1e-10, mu_pre=mu, mu_post=mu, order=a.order)
        ev[2].record(s)
        torch.cuda.synchronize()
        result["setup_ms"] = ev[0].elapsed_time(ev[1])
        result["solve_ms"] = ev[1].elapsed_time(ev[2])
        # the same setup computing every row (no repeated-row reuse): the cost
        # on operators without a constant-coefficient interior
        ev[0].record(s)
        h0 = cmg.setup_hierarchy(A.dim, A.n, A.offsets, coeff, reuse=False)
        c0 = cmg.setup_cascade(h0, a.kind, nu=a.nu, lowp=True, reuse=False)
        ev[1].record(s)
        torch.cuda.synchronize()
        result["setup_every_row_ms"] = ev[0].elapsed_time(ev[1])
        del c0, h0
        # ---- roofline of the sweep kernel (FP32 additive step, finest level)
        N = A.N
        lvl = cmg.query_level(h, 0)
        nst = lvl["nst"]
        xb = [torch.rand(N, device=dev, dtype=torch.float32) for _ in range(2)]
        b32 = torch.rand(N, device=dev, dtype=torch.float32)
        reps = 20
        for k in range(3):
            cmg.sweep(h, c, 0, k % a.nu, b32, xb[k % 2], xb[(k + 1) % 2], colour=-1 if a.kind == "additive" else 0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for k in range(reps):
            cmg.sweep(h, c, 0, k % a.nu, b32, xb[k % 2], xb[(k + 1) % 2], colour=-1 if a.kind == "additive" else 0)
        e1.record(s)
        torch.cuda.synchronize()
        t_sweep = e0.elapsed_time(e1) / reps * 1e-3
        bytes_sweep = (nst + 4) * 4 * N  # A (nst), Lambda, b, x read, x written: FP32
        peak, src = peaks()
        achieved = bytes_sweep / t_sweep / 1e9
        traffic = None
        try:
            with open(TRAFFIC) as f:
                tr = json.load(f)
            if tr.get("csrc_hash") == csrc_hash() and tr.get("n") == a.n:
                traffic = tr["sweep_fp32_bytes_per_launch"]
        except Exception:
            traffic = None
        result["roofline"] = {"bound": "hbm", "kernel": "k_sweep_f32x2 (additive step, FP32, two nodes per thread, finest level)",
                              "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                              "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                              "traffic": traffic, "algorithmic_bytes_per_launch": bytes_sweep,
                              "launch_ms": t_sweep * 1e3}
        result["smoother_gbs"] = achieved
        # ---- multiplicative red-black colour step (in place, FP32, finest level): the
        # colours interleave, so A, Lambda, b and x are read for every node
        # (sector granularity) and x is written for the colour's half
        cm = cmg.setup_cascade(h, "multiplicative", nu=a.nu, lowp=True)
        xr = xb[0]
        for k in range(3):
            cmg.sweep(h, cm, 0, k % a.nu, b32, xr, xr, colour=k % 2)
        torch.cuda.synchronize()
        e0.record(s)
        for k in range(reps):
            cmg.sweep(h, cm, 0, k % a.nu, b32, xr, xr, colour=k % 2)
        e1.record(s)
        torch.cuda.synchronize()
        t_col = e0.elapsed_time(e1) / reps * 1e-3
        bytes_col = (nst + 3) * 4 * N + 4 * (N // 2)
        result["colour_step_roofline"] = {
            "bound": "hbm", "kernel": "k_sweep<3,STAR,float,COLOURED> (multiplicative colour step, in place, finest level)",
            "achieved": bytes_col / t_col / 1e9, "peak": peak, "unit": "GB/s",
            "frac": bytes_col / t_col / 1e9 / peak, "algorithmic_bytes_per_launch": bytes_col, "launch_ms": t_col * 1e3}
        # ---- BF16-storage additive step (FP32 arithmetic, finest level): (nst + 4) x 2 B per node
        c16 = cmg.setup_cascade(h, a.kind, nu=a.nu, lowp=2)
        x16 = [t.to(torch.bfloat16) for t in xb]
        b16 = b32.to(torch.bfloat16)
        for k in range(3):
            cmg.sweep(h, c16, 0, k % a.nu, b16, x16[k % 2], x16[(k + 1) % 2], colour=-1 if a.kind == "additive" else 0)
        torch.cuda.synchronize()
        e0.record(s)
        for k in range(reps):
            cmg.sweep(h, c16, 0, k % a.nu, b16, x16[k % 2], x16[(k + 1) % 2], colour=-1 if a.kind == "additive" else 0)
        e1.record(s)
        torch.cuda.synchronize()
        t16 = e0.elapsed_time(e1) / reps * 1e-3
        bytes16 = (nst + 4) * 2 * N
        result["bf16_step_roofline"] = {
            "bound": "hbm", "kernel": "k_sweep_bf16x2 (additive step, BF16 storage, FP32 arithmetic, finest level)",
            "achieved": bytes16 / t16 / 1e9, "peak": peak, "unit": "GB/s", "frac": bytes16 / t16 / 1e9 / peak,
            "algorithmic_bytes_per_launch": bytes16, "launch_ms": t16 * 1e3}
        del h, c, x, cm, c16, x16, b16
        torch.cuda.empty_cache()
        # ---- multi-RHS block step (the block product X_b -= Lambda_b R_b):
        # elliptic interface 1024^2, 200 inclusions, 2x2-node blocks, 32 RHS, FP32
        Ai = problems.interface2d(1024)
        ci = torch.tensor(Ai.coeff, dtype=torch.float64, device=dev)
        hb = cmg.setup_hierarchy(Ai.dim, Ai.n, Ai.offsets, ci, block=2)
        cb = cmg.setup_cascade(hb, "additive", nu=3, lowp=True)
        m, Ni = 32, Ai.N
        Xb = [torch.rand(Ni * m, device=dev, dtype=torch.float32) for _ in range(2)]
        Bb = torch.rand(Ni * m, device=dev, dtype=torch.float32)
        for k in range(3):
            cmg.sweep_rhs(hb, cb, 0, k % 3, Bb, Xb[k % 2], Xb[(k + 1) % 2], m)
        torch.cuda.synchronize()
        e0.record(s)
        for k in range(reps):
            cmg.sweep_rhs(hb, cb, 0, k % 3, Bb, Xb[k % 2], Xb[(k + 1) % 2], m)
        e1.record(s)
        torch.cuda.synchronize()
        t_m = e0.elapsed_time(e1) / reps * 1e-3
        bytes_m = (5 + 4 + 3 * m) * 4 * Ni  # A, Lambda (16 per 4-node block), B, X read, X written
        result["multi_rhs_block_step"] = {
            "workload": "elliptic interface 1024^2, 200 inclusions (contrast 1e-4..1e4), 2x2-node blocks "
                        "(4x4 Lambda), 32 RHS, FP32, finest level",
            "launch_ms": t_m * 1e3, "achieved_gbs": bytes_m / t_m / 1e9, "frac_of_peak": bytes_m / t_m / 1e9 / peak,
            "algorithmic_bytes_per_launch": bytes_m, "bound": "hbm"}
        del hb, cb, ci, Xb, Bb
        torch.cuda.empty_cache()
        result["small_2d_poisson_64"] = small_2d_section(a, cmg, problems, dev)
        result["tensor_core_gemm"] = tensor_core_section(a, cmg, dev)
        result["learned_setup"] = learned_section(a, cmg, problems, dev)
        torch.cuda.empty_cache()
        result["interface_solve"] = interface_section(a, cmg, problems, dev)
        torch.cuda.empty_cache()
        result["batched_solve"] = batch_section(a, cmg, problems, dev)
        torch.cuda.empty_cache()
        result["cascade_forms"] = cascade_forms_section(a, cmg, A, coeff, bd, dev)
        torch.cuda.empty_cache()
        result["general_path"] = general_section(a, cmg, problems, dev)
        torch.cuda.empty_cache()
        result["stokes_prescaling"] = stokes_section(a, cmg, problems, dev)
        torch.cuda.empty_cache()
        result["overlapping_blocks"] = overlap_section(a, cmg, problems, dev)
        torch.cuda.empty_cache()
        # ---- plain FP64 path (stationary V-cycle iteration)
        pinfo = []
        ms64 = timed(lambda: step("fp64", "stationary", False, pinfo), max(2, a.steps // 2), 1)
        result["plain_fp64"] = {"ms_per_step": ms64, "iterations": pinfo[-1].iterations,
                                "final_rel_residual": pinfo[-1].final_rel_residual,
                                "speedup_chosen_vs_plain": ms64 / ms}
        # ---- the chosen form with every setup product in FP64
        sinfo = []
        ms_s64 = timed(lambda: step("fp32", "refine", True, sinfo, setup="fp64"), max(2, a.steps // 2), 1)
        result["chosen_with_fp64_setup_products"] = {"ms_per_step": ms_s64, "iterations": sinfo[-1].iterations,
                                                     "final_rel_residual": sinfo[-1].final_rel_residual}
        # ---- BF16 storage (FP32 arithmetic) cycles inside FP64 refinement
        binfo = []
        ms16 = timed(lambda: step("bf16", "refine", 2, binfo), max(2, a.steps // 2), 1)
        result["bf16_cycles"] = {"ms_per_step": ms16, "iterations": binfo[-1].iterations,
                                 "final_rel_residual": binfo[-1].final_rel_residual,
                                 "converged": bool(binfo[-1].converged)}
        # ---- end to end through the C ABI with host buffers (pinned)
        pin_coeff = torch.tensor(A.coeff, dtype=torch.float64).pin_memory()
        pin_b = torch.tensor(b, dtype=torch.float64).pin_memory()
        pin_x = torch.zeros(A.N, dtype=torch.float64).pin_memory()
        cn = pin_coeff.numpy()

        def e2e_step():
            h2 = cmg.setup_hierarchy(A.dim, A.n, A.offsets, cn)
            c2 = cmg.setup_cascade(h2, a.kind, nu=a.nu, lowp=True, setup_precision="fp32")
            pin_x.zero_()
            cmg.solve(h2, c2, pin_b, pin_x, method="refine", precision="fp32", tol=1e-10, mu_pre=mu, mu_post=mu,
                      order=a.order, host_buffers=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        # host wall clock per step (the host-side setup and copies are part of
        # it); the median of the steps, so that one slow host step does not set it
        times = []
        for _ in range(max(3, a.steps)):
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
        e2e_ms = max_over_ranks(float(np.median(times)), world, dev)
        result["e2e"] = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(A.coeff.nbytes + 2 * 8 * A.N),
                         "d2h_bytes_per_step": int(8 * A.N), "steps_ms": [round(t, 2) for t in times]}
        if rank == 0 and world == 1:
            result["cpu_baseline"] = cpu_baseline(a, a.n)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
