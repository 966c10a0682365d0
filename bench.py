"""Benchmark of the GB300 oblique-projection FEAST hot path.

A step is one pass of GFEAST lines 5-17 (projection, projected QZ, Ritz
residuals and stopping test, then the contour-integral subspace build with
one shifted multi-right-hand-side solve per node, the node sum and the two
orthonormalisations) on the dense prescribed-spectrum pencil
n = 4096, m0 = 1280, 32 trapezoid nodes on |z| = 1.  The LU set-up is timed
separately.  One JSON line is printed by rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload NAME] [--prec fp64]

--impl reference times the FP64 oracle (the plain CPU restatement of the
method) on the host cores on a bounded sample of the same workload.
N > 1 (launched by torchrun): independent replicas, one per GPU, no
collective on the data path; value = iterations of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
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

from paper_1404_1768_gb300 import inputs  # noqa: E402

METRIC = "FEAST iters/s & eigpairs/s vs plain FP64 GPU at resid≤1e-10; % TC/HBM peak"
# FP64 pipe of a GB300: 152 SMs x 2 DFMA/clock x 2 flop x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 pipe: 152 SMs x 128 FFMA/clock x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="dense_n4096_m1280_q32", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--prec", default="fp64", choices=["fp64", "c64r"],
                    help="fp64: every step in FP64; c64r: complex64 factors and solves with "
                         "refinement (residual in double-single arithmetic)")
    ap.add_argument("--no-converge", action="store_true",
                    help="skip the untimed run to convergence (parity / eigpairs/s)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU baseline sample")
    return ap.parse_args()


# ----------------------------------------------------------------------- dist
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------- inputs
def make_problem(cfg):
    return inputs.prescribed_pencil(cfg["n"], cfg["m0"], seed=cfg["seed"], center=cfg["center"],
                                    radius=cfg["radius"])


def feast_kwargs(cfg):
    return dict(contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"],
                a=cfg["radius"], eps=cfg.get("eps", 1e-12), eta=1e-3, max_iter=50)


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------- CPU baseline
def cpu_baseline(cfg, p, budget_s: float = 20.0):
    """The oracle, as it stands, on a bounded sample of one iteration of the
    workload, scaled to iterations/s.  Small workloads run whole iterations."""
    import oracle
    threads = oracle.num_threads()
    n, m0, q = cfg["n"], cfg["m0"], cfg["q"]
    if n * n * m0 * q <= 5e8:
        fe = oracle.Feast(p.A, p.B, p.Y, **feast_kwargs(cfg))
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < budget_s and k < 50:
            it = fe.iterate()
            k += 1
            if it["flag"] != 2:
                break
        dt = time.perf_counter() - t0
        fe.close()
        return {"value": k / dt, "unit": "iters/s", "cores": threads, "kind": "oracle",
                "sample": f"{k} whole GFEAST iterations (lines 5-17) of the oracle"}
    # large: solve step sampled on a subset of columns of one node, QZ on a
    # smaller pencil (cubic scaling), the n x m0 x m0 products on a subset
    rng = np.random.default_rng(1)
    # a well-conditioned stand-in for one node's LU factors (the substitution
    # cost does not depend on the values): unit-lower part small, dominant
    # diagonal, identity pivots
    f = np.asfortranarray(0.01 * inputs.complex_normal(rng, (n, n)) + 4.0 * np.eye(n))
    piv = np.arange(n, dtype=np.int32)
    ncol = max(threads, 16)
    b = inputs.complex_normal(rng, (n, ncol))
    t0 = time.perf_counter()
    oracle.lu_solve_cols(f, piv, b)
    t_col = (time.perf_counter() - t0) / ncol
    mq = 256
    Aq = inputs.complex_normal(rng, (mq, mq))
    Bq = np.triu(inputs.complex_normal(rng, (mq, mq))) + 2 * np.eye(mq)
    t0 = time.perf_counter()
    oracle.ggev(Aq, Bq)
    t_qz = (time.perf_counter() - t0) * (m0 / mq) ** 3
    kk = 128
    U = inputs.complex_normal(rng, (n, kk))
    t0 = time.perf_counter()
    oracle.gemm(U, U, conj_a=True)
    t_prod = (time.perf_counter() - t0) * (m0 / kk) ** 2
    # per iteration: q*m0 column solves, one QZ, ~6 n x m0 x m0 products
    # (projection pair, Ritz vectors, A x / B x, two QRs), two n x n x m0
    # operator products (= 2 n/m0 units of n x m0 x m0)
    t_iter = q * m0 * t_col + t_qz + (6 + 2 * n / m0) * t_prod
    return {"value": 1.0 / t_iter, "unit": "iters/s", "cores": threads, "kind": "oracle",
            "sample": (f"oracle substitution on {ncol} columns of one n={n} factor "
                       f"(x{q * m0 // ncol} to q*m0 columns), oracle QZ on a {mq}x{mq} pencil "
                       f"(x{(m0 / mq) ** 3:.0f}), oracle n x {kk} x {kk} product "
                       f"(x{(6 + 2 * n / m0) * (m0 / kk) ** 2:.0f}); iteration time "
                       f"{t_iter:.1f} s")}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cfg = inputs.WORKLOADS[args.workload]
    p = make_problem(cfg)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(cfg, p, budget_s=5.0)
    for _ in range(args.steps):
        vals.append(cpu_baseline(cfg, p, budget_s=10.0))
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": config_dict(cfg, args, world),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(cfg, args, world):
    return {"workload": args.workload, "n": cfg["n"], "m0": cfg["m0"], "q": cfg["q"],
            "rule": "trapezoid" if cfg["rule"] == 0 else "gauss-legendre",
            "contour": f"circle center {cfg['center']} radius {cfg['radius']}",
            "pencil": "A = P diag(lam) Q, B = P Q, lam uniform in |z| <= 2 (seeded)",
            "precision": args.prec, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (per-node LU factors)"}


# ----------------------------------------------------------------------- GPU arm
def gpu_arm(args):
    import torch
    import paper_1404_1768_gb300 as fg

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fg.load()
    cfg = inputs.WORKLOADS[args.workload]
    p = make_problem(cfg)
    n, m0, q = cfg["n"], cfg["m0"], cfg["q"]
    kw = feast_kwargs(cfg)
    if args.prec == "c64r":
        kw.update(prec=fg.FEAST_C64_REFINE, refine_tol=1e-13, max_refine=4)
    stream = torch.cuda.current_stream()

    # pinned host inputs (column-major) for the end-to-end leg
    hA = torch.from_numpy(np.ascontiguousarray(p.A.ravel(order="F"))).pin_memory()
    hB = torch.from_numpy(np.ascontiguousarray(p.B.ravel(order="F"))).pin_memory()
    hY = torch.from_numpy(np.ascontiguousarray(p.Y.ravel(order="F"))).pin_memory()
    h2d_bytes = (hA.numel() + hB.numel() + hY.numel()) * 16

    barrier(world)
    torch.cuda.synchronize()
    # ---- end-to-end: host inputs -> set-up -> W + K passes -> host outputs
    t_e2e0 = time.perf_counter()
    dA = hA.to(dev, non_blocking=True)
    dB = hB.to(dev, non_blocking=True)
    dY = hY.to(dev, non_blocking=True)
    fe = fg.Feast(dA.view(n, n).t(), dB.view(n, n).t(), dY.view(m0, n).t(), no_stop=True,
                  device=dev, **kw)
    setup_ms = fe.setup_info["ms_lu"] + fe.setup_info["ms_solve"]
    log(f"setup: LU {fe.setup_info['ms_lu']:.1f} ms, first subspace {fe.setup_info['ms_solve']:.1f} ms")
    for _ in range(args.warmup):
        it = fe.iterate()
        log("warmup", {k: (round(v, 3) if isinstance(v, float) else v) for k, v in it.items()})
    torch.cuda.synchronize()
    barrier(world)
    launches0 = fg.kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    infos = [fe.iterate() for _ in range(args.steps)]
    ev1.record(stream)
    for it in infos:
        log("timed", {k: (round(v, 3) if isinstance(v, float) else v) for k, v in it.items()})
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = fg.kernel_launches() - launches0
    t_dev = ev0.elapsed_time(ev1) / 1e3
    # the result read back to the host (status scalars are read every pass)
    d2h_bytes = 64 * (args.warmup + args.steps)
    t_e2e1 = time.perf_counter()
    t_e2e = t_e2e1 - t_e2e0
    barrier(world)
    t_dev_max = max_over_ranks(t_dev, world, dev)
    t_e2e_max = max_over_ranks(t_e2e, world, dev)

    value = world * args.steps / t_dev_max
    e2e_value = world * (args.warmup + args.steps) / t_e2e_max
    ms_solve = statistics.mean(i["ms_solve"] for i in infos)
    solve_flops = 8.0 * q * n * n * m0          # complex MAC = 8 flops, a4
    if args.prec == "fp64":
        t_solve = ms_solve
        peak, peak_src = FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"
        kern = "subspace-build solves (k_gemm + k_trsv_diag), FP64 pipe"
    else:
        # the complex64 solve of the pass (refinement sweeps timed separately)
        t_solve = max(ms_solve - statistics.mean(i["ms_refine"] for i in infos), 1e-6)
        peak, peak_src = FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz"
        kern = "subspace-build complex64 solves (k_gemm<float2> + k_trsv_diag), FP32 pipe"
    achieved = solve_flops / (t_solve / 1e3) / 1e12

    # ---- untimed: continue to convergence for parity and eigpairs/s
    parity = None
    eig_rate = None
    if not args.no_converge:
        k_stop = None
        for i in infos:
            if i["flag"] != 2:
                k_stop = i["k"]
                break
        it = infos[-1]
        while k_stop is None and it["k"] < kw["max_iter"]:
            it = fe.iterate()
            if it["flag"] != 2:
                k_stop = it["k"]
        if k_stop is not None:
            r = fe.eigs(want_vectors=False)
            ref = p.lam[np.abs(p.lam - cfg["center"]) < cfg["radius"]]
            errs = []
            pool = list(ref)
            for x in r["lam"]:
                j = int(np.argmin([abs(x - y) for y in pool]))
                errs.append(abs(x - pool[j]) / max(abs(pool[j]), 1e-300))
                pool.pop(j)
            parity = {"flag": r["flag"], "count": r["count"], "exact_count": int(len(ref)),
                      "k_stop": k_stop, "max_rel_eig_err_vs_prescribed": max(errs) if errs else 0.0,
                      "max_resid_eq_5_1": float(np.max(r["res"])) if r["count"] else 0.0}
            t_total = setup_ms / 1e3 + k_stop * (t_dev / args.steps)
            eig_rate = r["count"] / t_total
    fe.close()

    if rank == 0:
        cb = None
        if not args.no_baseline:
            cb = cpu_baseline(cfg, p)
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if args.prec == "fp64" else "c64+c128 refine",
            "data": "synthetic", "config": config_dict(cfg, args, world),
            "setup_ms": setup_ms, "eigpairs_per_s": eig_rate, "parity": parity,
            "phase_ms": {k: statistics.mean(i[k] for i in infos)
                         for k in ("ms_proj", "ms_qz", "ms_solve", "ms_qr", "ms_refine")},
            "refine_sweeps": [i["refine_sweeps_max"] for i in infos],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": kern, "peak_source": peak_src},
            "cpu_baseline": cb,
            "e2e": {"value": e2e_value, "unit": "iters/s",
                    "h2d_bytes_per_step": h2d_bytes / (args.warmup + args.steps),
                    "d2h_bytes_per_step": d2h_bytes / (args.warmup + args.steps)},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
