#!/usr/bin/env python
"""Time-to-solution and DOF/s of the GenEO hot path on one GB300.

A step is one pass of the whole path on the 3D Darcy workload (Q1, 128^3
elements, 2,146,689 dofs, 8x8x8 subdomains of 16^3 elements grown by two
element layers, kappa = exp(Gaussian field) with 1e6-contrast slabs, at most
20 eigenvectors per subdomain below tau = 0.3, PCG to relative residual
1e-8): geneo_setup (partition of unity, local matrices, factorisations,
eigensolves, coarse space) + geneo_pcg_solve + geneo_destroy, inputs resident
in device memory.  value = dofs solved per second over the timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Under torchrun (N > 1) every rank solves its own copy of the workload
(replicas: the hot path has no cross-GPU exchange on one box); the reported
value is the dofs of all ranks over the slowest rank's time.
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

METRIC = "time-to-solution & DOF/s at rel-res 1e-8, mixed vs FP64; serve p50/p99 latency"
UNIT = "DOF/s"

WORKLOADS = {
    "darcy3d_128": dict(nel=(128, 128, 128), parts=(8, 8, 8), overlap=2, nev=20, tau=0.3,
                        desc="3D Darcy Q1 128^3 elements (2,146,689 dofs), 8x8x8 subdomains of "
                             "16^3 elements, overlap 2, kappa=exp(GRF l=0.1 s2=4) x 1e6 slabs, "
                             "nev<=20, tau=0.3, PCG rel-res 1e-8"),
    "darcy3d_64": dict(nel=(64, 64, 64), parts=(4, 4, 4), overlap=2, nev=20, tau=0.3,
                       desc="3D Darcy Q1 64^3 elements (274,625 dofs), 4x4x4 subdomains of 16^3 "
                            "elements, overlap 2, kappa=exp(GRF) x 1e6 slabs, nev<=20, tau=0.3 "
                            "(profiling case: same subdomain size as the 128^3 workload)"),
    "darcy2d_64": dict(nel=(64, 64), parts=(4, 4), overlap=1, nev=10, tau=0.3,
                       desc="2D Darcy Q1 64^2 (4,225 dofs), 4x4 subdomains, overlap 1, channels "
                            "1e6, nev<=10, tau=0.3, PCG rel-res 1e-8"),
}


def make_problem(name):
    import gen
    w = WORKLOADS[name]
    if len(w["nel"]) == 3:
        kap = gen.kappa_grf_layers_3d(w["nel"], seed=1)
    else:
        kap = gen.kappa_channels_2d(w["nel"], seed=0)
    return gen.darcy_problem(w["nel"], kap, w["parts"], w["overlap"])


def fp64_peak():
    """FP64 ALU peak: 152 SMs x 4 flop/clk (2 DFMA) x 2070 MHz."""
    return 152 * 4 * 2070e6


def fp32_peak():
    """FP32 ALU peak: 152 SMs x 256 flop/clk (128 FFMA) x 2070 MHz."""
    return 152 * 256 * 2070e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(prob, nev, tau, n_sample, pcg_iters):
    """Time the oracle on a sample of interior subdomains (local Dirichlet
    matrix + LU, Neumann/overlap assembly, ARPACK shift-invert eigensolve,
    coarse vectors, one local solve) on one core, then extrapolate to the
    whole workload: setup = mean per-subdomain time x N; solve = pcg_iters x
    (N local solves + one SpMV); the coarse factorisation is timed at full
    size when its dimension is known from the GPU run."""
    import numpy as np
    import scipy.sparse.linalg as spla
    import oracle
    t0 = time.perf_counter()
    sets = oracle.subdomain_sets(prob)
    e_tau = oracle.element_multiplicity(prob)
    c, xs = oracle.partition_of_unity(prob, sets)
    t_struct = time.perf_counter() - t0
    N = prob.n_sub
    # interior subdomains (largest, most expensive)
    sizes = np.array([s["N"].size for s in sets])
    order = np.argsort(-sizes, kind="stable")
    pick = order[:n_sample]
    t_setup, t_solve = [], []
    for j in pick:
        t1 = time.perf_counter()
        Aj = oracle.dirichlet_matrix(prob.A, sets[j]["D"])
        lu = spla.splu(Aj.tocsc())
        At, B = oracle.geneo_pencil(prob, j, sets, xs, e_tau)
        lam, P = oracle.local_eigenpairs(At, B, nev + min(10, nev), -0.01, 2500, 1e-12)
        m = oracle.select_count(lam, tau, nev)
        oracle.coarse_vectors(P, xs[j], m)
        t_setup.append(time.perf_counter() - t1)
        r = np.ones(sets[j]["D"].size)
        t2 = time.perf_counter()
        lu.solve(r)
        t_solve.append(time.perf_counter() - t2)
    x = np.ones(prob.n)
    t3 = time.perf_counter()
    prob.A @ x
    t_spmv = time.perf_counter() - t3
    total = t_struct + float(np.mean(t_setup)) * N + pcg_iters * (float(np.mean(t_solve)) * N + 2 * t_spmv)
    return {"seconds": total, "sample_s": t_struct + sum(t_setup) + sum(t_solve) + t_spmv,
            "n_sample": int(len(pick))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    w = WORKLOADS[args.workload]
    prob = make_problem(args.workload)
    iters = args.ref_pcg_iters
    vals = []
    for step in range(args.warmup + args.steps):
        r = oracle_sample(prob, w["nev"], w["tau"], args.ref_sample, iters)
        if step >= args.warmup:
            vals.append(prob.n / r["seconds"])
    value = statistics.median(vals)
    sample = ("oracle (numpy/scipy FP64, ARPACK shift-invert) on %d largest subdomains per step, "
              "1 core; extrapolated: setup x %d subdomains + %d PCG iterations x (%d local LU "
              "solves + SpMV)" % (args.ref_sample, prob.n_sub, iters, prob.n_sub))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="darcy3d_128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=3)
    ap.add_argument("--ref-pcg-iters", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-8)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10944_gb300 import geneo as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = WORKLOADS[args.workload]
    prob = make_problem(args.workload)
    host = G.problem_arrays(prob)
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    b_dev = torch.from_numpy(prob.b).cuda()
    x_dev = torch.zeros_like(b_dev)
    prec = G.GENEO_PREC_FP32 if args.precision == "fp32" else G.GENEO_PREC_FP64
    opts = G.geneo_default_options(nev_max=w["nev"], tau=w["tau"], precision=prec)
    problem = G.make_problem(dev, prob.n, prob.n_sub, prob.elem_dofs.shape[1], prob.ndn,
                             G.GENEO_MEM_DEVICE)
    stream = torch.cuda.current_stream()

    def step():
        h = G.geneo_setup(problem, opts, stream)
        try:
            info = G.geneo_pcg_solve(h, b_dev, x_dev, 1, args.tol, 2000, G.GENEO_MEM_DEVICE,
                                     stream=stream)
            q = G.geneo_query(h)
        finally:
            G.geneo_destroy(h)
        return info, q

    for _ in range(args.warmup):
        info, q = step()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    launches0 = G.geneo_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    infos, qs = [], []
    for _ in range(args.steps):
        info, q = step()
        infos.append(info)
        qs.append(q)
    ev1.record(stream)
    barrier()
    launches = G.geneo_launch_count() - launches0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    t_max = ms
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = prob.n * args.steps * world / (t_max / 1e3)
    res = float(np.linalg.norm(prob.b - prob.A @ x_dev.cpu().numpy()) / np.linalg.norm(prob.b))

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
        hp = G.make_problem(pinned, prob.n, prob.n_sub, prob.elem_dofs.shape[1], prob.ndn,
                            G.GENEO_MEM_HOST)
        b_h = torch.from_numpy(prob.b).pin_memory()
        x_h = torch.zeros_like(b_h).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in pinned.values()) + b_h.numel() * 8
        d2h = x_h.numel() * 8
        times = []
        for _ in range(max(1, min(args.steps, 2))):
            barrier()
            t0 = time.perf_counter()
            h = G.geneo_setup(hp, opts, stream)
            try:
                G.geneo_pcg_solve(h, b_h, x_h, 1, args.tol, 2000, G.GENEO_MEM_HOST, stream=stream)
            finally:
                G.geneo_destroy(h)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        e2e = {"value": prob.n / statistics.median(times), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # roofline of the dominant kernel (largest share of the step's device time)
    qm = qs[-1]
    step_ms = t_max / args.steps
    cands = {
        "band_potrf (batched Cholesky of A_j, K_j)": (qm["factor_flops"], qm["factor_event_ms"]),
        "band_solve (eigensolver K_j^{-1} blocks)": (qm["eigsolve_flops"], qm["eigsolve_event_ms"]),
    }
    dom = max(cands, key=lambda k: cands[k][1])
    fl, kms = cands[dom]
    peak = fp32_peak() if args.precision == "fp32" else fp64_peak()
    achieved = fl / (kms / 1e3) if kms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "share_of_step": kms / step_ms,
                "peak_source": "derived: 152 SMs x %d flop/clk x 2070 MHz (%s ALU)"
                               % (256 if args.precision == "fp32" else 4, args.precision.upper())}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r = oracle_sample(prob, w["nev"], w["tau"], args.ref_sample, infos[-1]["iterations"])
        cpu = {"value": prob.n / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d largest subdomains (setup incl. ARPACK) + one local solve each, "
                         "1 core, %.1f s of CPU work; extrapolated to %d subdomains and %d PCG "
                         "iterations" % (r["n_sample"], r["sample_s"], prob.n_sub,
                                         infos[-1]["iterations"])}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32-factors/f64",
            "data": "synthetic",
            "config": {"workload": w["desc"], "precision": args.precision,
                       "l2": "inputs larger than L2 (2.1M-dof CSR and 1.07 GB of element matrices); no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
            "cpu_baseline": cpu,
            "detail": {"pcg_iterations": infos[-1]["iterations"], "rel_residual_true": res,
                       "kappa_estimate": infos[-1]["kappa_estimate"], "dim_coarse": qm["dim_coarse"],
                       "eig_iterations": qm["eig_iterations"], "block_size": qm["block_size"],
                       "setup_ms": dict(zip(["structure", "assembly", "factor", "eigensolve", "basis",
                                             "coarse_matrix", "coarse_factor", "total"],
                                            [round(v, 3) for v in qm["setup_ms"]])),
                       "device_gb": qm["device_bytes"] / 1e9},
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
