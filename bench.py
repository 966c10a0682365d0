"""Benchmark of the GB300 oblique-projection FEAST hot path.

A step is one pass of GFEAST lines 5-17 (projection, projected QZ, Ritz
residuals and stopping test, then the contour-integral subspace build with
one shifted multi-right-hand-side solve per node, the node sum and the two
orthonormalisations) on the dense prescribed-spectrum pencil
n = 4096, m0 = 1280, 32 trapezoid nodes on |z| = 1, in the precision form
(complex64 factors and solves with FP64-accurate refinement; --prec fp64
for the plain FP64 path, which the precision form's line also times for
comparison).  The LU set-up is timed separately.  One JSON line is printed
by rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload NAME] [--prec c64r|fp64] [--no-fp64]

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
    ap.add_argument("--prec", default="c64r", choices=["fp64", "c64r"],
                    help="c64r (precision form): complex64 factors and solves on the tensor cores "
                         "with FP64-accurate refinement; fp64: the plain FP64 path")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain-FP64 comparison passes of the precision form")
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
def parity_report(fe, p, cfg):
    r = fe.eigs(want_vectors=True)
    ref = p.lam[np.abs(p.lam - cfg["center"]) < cfg["radius"]]
    errs = []
    pool = list(ref)
    for x in r["lam"]:
        if not pool:
            break
        j = int(np.argmin([abs(x - y) for y in pool]))
        errs.append(abs(x - pool[j]) / max(abs(pool[j]), 1e-300))
        pool.pop(j)
    return r, {"flag": r["flag"], "count": r["count"], "exact_count": int(len(ref)),
               "max_rel_eig_err_vs_prescribed": max(errs) if errs else 0.0,
               "max_resid_eq_5_1": float(np.max(r["res"])) if r["count"] else 0.0}


def timed_run(fg, torch, dev, stream, host, n, m0, kw, steps, warmup, converge, world):
    """One whole solve through the public API from pinned host buffers:
    host -> device copies, set-up, `warmup` passes, `steps` passes timed with
    CUDA events on the library's stream, then (if converge) passes until a
    stop fires and the eigenpairs back to the host.  Returns the timings."""
    hA, hB, hY = host
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dA = hA.to(dev, non_blocking=True)
    dB = hB.to(dev, non_blocking=True)
    dY = hY.to(dev, non_blocking=True)
    fe = fg.Feast(dA.view(n, n).t(), dB.view(n, n).t(), dY.view(m0, n).t(), no_stop=True,
                  device=dev, stream=stream, **kw)
    setup_ms = fe.setup_info["ms_lu"] + fe.setup_info["ms_solve"]
    infos = []
    for _ in range(warmup):
        infos.append(fe.iterate())
    torch.cuda.synchronize()
    launches0 = fg.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    timed = [fe.iterate() for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    launches = fg.kernel_launches() - launches0
    infos += timed
    k_stop = None
    for it in infos:
        if it["flag"] != 2:
            k_stop = it["k"]
            break
    res = None
    if converge:
        it = infos[-1]
        while k_stop is None and it["k"] < kw["max_iter"]:
            it = fe.iterate()
            infos.append(it)
            if it["flag"] != 2:
                k_stop = it["k"]
        if k_stop is not None:
            res = fe.eigs(want_vectors=True)   # device -> host: values, residuals, vectors
    torch.cuda.synchronize()
    t_job = time.perf_counter() - t0
    return dict(fe=fe, setup_ms=setup_ms, infos=infos, timed=timed, t_dev=t_dev, launches=launches,
                k_stop=k_stop, t_job=t_job, res=res)


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
    kw_prec = dict(kw)
    if args.prec == "c64r":
        kw_prec.update(prec=fg.FEAST_C64_REFINE, refine_tol=1e-13, max_refine=4)
    stream = torch.cuda.current_stream()

    # pinned host inputs (column-major)
    hA = torch.from_numpy(np.ascontiguousarray(p.A.ravel(order="F"))).pin_memory()
    hB = torch.from_numpy(np.ascontiguousarray(p.B.ravel(order="F"))).pin_memory()
    hY = torch.from_numpy(np.ascontiguousarray(p.Y.ravel(order="F"))).pin_memory()
    h2d_bytes = (hA.numel() + hB.numel() + hY.numel()) * 16

    clocks = ClockSampler(local)
    clocks.start()
    run = timed_run(fg, torch, dev, stream, (hA, hB, hY), n, m0, kw_prec, args.steps, args.warmup,
                    not args.no_converge, world)
    clk = clocks.stop()
    for it in run["infos"]:
        log("pass", {k: (round(v, 3) if isinstance(v, float) else v) for k, v in it.items()})
    t_dev_max = max_over_ranks(run["t_dev"], world, dev)
    value = world * args.steps / t_dev_max
    infos = run["timed"]
    setup_ms, launches = run["setup_ms"], run["launches"]
    parity, eig_rate, e2e = None, None, None
    d2h_bytes = 0
    if run["res"] is not None:
        r = run["res"]
        _, parity = parity_report(run["fe"], p, cfg)
        parity["k_stop"] = run["k_stop"]
        # eigpairs/s over the device work of the whole solve: set-up + every pass
        t_total = (run["setup_ms"] + sum(
            i["ms_proj"] + i["ms_qz"] + i["ms_solve"] + i["ms_qr"] for i in run["infos"])) / 1e3
        eig_rate = r["count"] / t_total
        d2h_bytes = 16 * m0 + 8 * m0 + 16 * n * m0 + 64 * run["k_stop"]
        t_job = max_over_ranks(run["t_job"], world, dev)
        e2e = {"value": world * run["k_stop"] / t_job, "unit": "iters/s",
               "h2d_bytes_per_step": h2d_bytes / run["k_stop"],
               "d2h_bytes_per_step": d2h_bytes / run["k_stop"],
               "what": "whole solve through the public API: pinned host A, B, Y -> device, set-up, "
                       "passes until the stop fires, eigenpairs back to the host; iterations / wall time"}
    run["fe"].close()
    del run

    # the plain FP64 path on the same pencil, for the comparison the metric names
    fp64 = None
    if args.prec != "fp64" and not args.no_fp64:
        r64 = timed_run(fg, torch, dev, stream, (hA, hB, hY), n, m0, kw, 2, 1, False, world)
        fp64 = {"iters_per_s": 2 / r64["t_dev"], "ms_per_iter": 1e3 * r64["t_dev"] / 2,
                "setup_ms": r64["setup_ms"], "warmup": 1, "steps": 2,
                "phase_ms": {k: statistics.mean(i[k] for i in r64["timed"])
                             for k in ("ms_proj", "ms_qz", "ms_solve", "ms_qr")}}
        r64["fe"].close()
        del r64

    # roofline of the dominant phase: the kernel behind it and its algorithmic work
    ph = {k: statistics.mean(i[k] for i in infos)
          for k in ("ms_proj", "ms_qz", "ms_solve", "ms_qr", "ms_refine")}
    solve_flops = 8.0 * q * n * n * m0          # complex MAC = 8 flops, a4
    if args.prec == "fp64":
        t_solve = ph["ms_solve"]
        roof = {"bound": "alu", "achieved": solve_flops / (t_solve / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "kernel": "subspace-build solves (k_gemm<double2> + k_trsv_diag), FP64 pipe",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    else:
        t_solve = max(ph["ms_solve"] - ph["ms_refine"], 1e-6)
        roof = {"bound": "alu", "achieved": solve_flops / (t_solve / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s",
                "kernel": "subspace-build complex64 solves (k_gemm<float2> + k_trsv_diag), FP32 pipe",
                "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None

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
            "setup_ms": setup_ms,
            "eigpairs_per_s": eig_rate, "parity": parity,
            "phase_ms": ph,
            "refine_sweeps": [i["refine_sweeps_max"] for i in infos],
            "fp64_path": fp64,
            "roofline": roof,
            "cpu_baseline": cb,
            "e2e": e2e,
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
