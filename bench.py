"""Benchmark of the GB300 oblique-projection FEAST hot path.

A step is one whole GFEAST solve through the public API on the dense
prescribed-spectrum pencil n = 4096, m0 = 1280, 32 trapezoid nodes on
|z| = 1, in the precision form (complex64 factors and solves on the tensor
cores, the subspace build in defect form on the Ritz pairs, FP64-accurate
tensor-core products, the projected problem solved warm once its pairs have
converged; --prec fp64 for the plain FP64 path, which the precision form's
line also times on one whole solve for comparison): the pencil and start
block from pinned host memory, set-up (lines 1-3), passes of lines 5-17
until a stopping test fires, the eigenpairs back to the host.  value =
GFEAST passes of the timed solves / CUDA-event time of exactly those passes
(no pass after the stop); e2e = the same passes / wall time of the whole
solves.  One JSON line is printed by rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload NAME] [--prec c64r|fp64] [--no-fp64]

--impl reference times the FP64 oracle (the plain CPU restatement of the
method) on the host cores: whole oracle passes of a bounded sample of the
same workload, scaled to it.
N > 1 (launched by torchrun): one solve shared by N GPUs, node-sharded --
each rank owns a range of the quadrature nodes (their factors and solves)
and the partial quadrature sums are all-reduced with NCCL once per pass;
value = passes / slowest rank's pass time (strong scaling).
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


def _measured(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except Exception:
        return fallback


# Dense peaks for the kernels timed inside a solve: the measured sustained
# bf16 rate (MEASURED_PEAKS.json) times GB300's nominal ratio to bf16 (dense
# per GPU: bf16 2250, tf32 1100, fp64 1.25 TFLOP/s).
# The tensor-core GEMM launches are timed one by one (the burst figure);
# phases of a pass are timed inside the long step (the sustained one).
BF16_BURST_TFLOPS = _measured("bf16_tflops", 1900.0)
BF16_SUSTAINED_TFLOPS = _measured("bf16_tflops_sustained", 1700.0)
TF32_PEAK_TFLOPS = BF16_SUSTAINED_TFLOPS * 1100.0 / 2250.0
TF32_BURST_TFLOPS = BF16_BURST_TFLOPS * 1100.0 / 2250.0
FP64_MEASURED_TFLOPS = BF16_SUSTAINED_TFLOPS * 1.25 / 2250.0
TF32_SOURCE = "MEASURED_PEAKS.json bf16_tflops_sustained x nominal tf32/bf16 ratio (1100/2250)"
TF32_BURST_SOURCE = "MEASURED_PEAKS.json bf16_tflops (burst) x nominal tf32/bf16 ratio (1100/2250)"
FP64_SOURCE = "MEASURED_PEAKS.json bf16_tflops_sustained x nominal fp64/bf16 ratio (1.25/2250)"


HBM_PEAK_GBS = _measured("hbm_gbs", 6800.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="dense_n4096_m1280_q32", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--prec", default="c64r", choices=["fp64", "c64r"],
                    help="c64r (precision form): complex64 factors and solves on the tensor cores, "
                         "FP64-accurate products, defect-form subspace build; fp64: the plain FP64 path")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain-FP64 comparison passes of the precision form")
    ap.add_argument("--profile-pass", type=int, default=None,
                    help="wrap pass K of the first timed solve in an NVTX range 'timed' (for ncu --nvtx-include)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU baseline sample")
    ap.add_argument("--nworkers", type=int, default=16,
                    help="ragged batch: host worker threads (one CUDA stream each)")
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
class Problem:
    """One workload: its synthetic pencil, the FEAST keywords, the exact
    eigenvalues inside the contour, and how to hand it to the library and to
    the oracle."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.band = "nx" in cfg
        if self.band:
            bp = inputs.convection_diffusion(cfg["nx"], cfg["m0"], seed=cfg["seed"], beta=cfg["beta"])
            self.bp = bp
            self.n, self.m0, self.q = bp.n, cfg["m0"], cfg["q"]
            lam = inputs.convection_diffusion_spectrum(cfg["nx"], cfg["beta"])
            self.ref = lam[((lam - cfg["center"].real) / cfg["a"]) ** 2 < 1.0]
            self.kw = dict(kind=1, kl=bp.kl, ku=bp.ku, b_identity=True, contour_kind=1, rule=cfg["rule"],
                           q=cfg["q"], center=cfg["center"], a=cfg["a"], b=cfg["b"], eps=cfg["eps"],
                           eta=1e-3, max_iter=50)
            self.host_arrays = [bp.A_band, bp.Y]
        else:
            p = inputs.prescribed_pencil(cfg["n"], cfg["m0"], seed=cfg["seed"], center=cfg["center"],
                                         radius=cfg["radius"])
            self.p = p
            self.n, self.m0, self.q = cfg["n"], cfg["m0"], cfg["q"]
            self.ref = p.lam[np.abs(p.lam - cfg["center"]) < cfg["radius"]]
            self.kw = dict(contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"],
                           a=cfg["radius"], eps=cfg.get("eps", 1e-12), eta=1e-3, max_iter=50)
            self.host_arrays = [p.A, p.B, p.Y]

    def pinned(self):
        import torch
        return [torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).pin_memory()
                for a in self.host_arrays]

    def feast(self, fg, dev, stream, dev_arrays, **extra):
        kw = dict(self.kw)
        kw.update(extra)
        if self.band:
            dA, dY = dev_arrays
            rows = self.bp.kl + self.bp.ku + 1
            return fg.Feast(dA.view(self.n, rows).t(), None, dY.view(self.m0, self.n).t(),
                            device=dev, stream=stream, **kw)
        dA, dB, dY = dev_arrays
        n = self.n
        return fg.Feast(dA.view(n, n).t(), dB.view(n, n).t(), dY.view(self.m0, n).t(),
                        device=dev, stream=stream, **kw)

    def oracle_feast(self, oracle):
        if self.band:
            return oracle.Feast(self.bp.A_band, None, self.bp.Y, **self.kw)
        return oracle.Feast(self.p.A, self.p.B, self.p.Y, **self.kw)

    def describe(self):
        c = self.cfg
        if self.band:
            return {"n": self.n, "m0": self.m0, "q": self.q, "rule": "gauss-legendre",
                    "contour": f"ellipse center {c['center']} semi-axes {c['a']}, {c['b']}",
                    "pencil": f"-Lap u + {tuple(c['beta'])}.grad u, {c['nx']}x{c['nx']} grid, 5-point, "
                              f"B = I, half-bandwidth {self.bp.kl} (closed-form spectrum)"}
        return {"n": self.n, "m0": self.m0, "q": self.q,
                "rule": "trapezoid" if c["rule"] == 0 else "gauss-legendre",
                "contour": f"circle center {c['center']} radius {c['radius']}",
                "pencil": "A = P diag(lam) Q, B = P Q, lam uniform in |z| <= 2 (seeded)"}


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------- CPU baseline
# Oracle sample size: the largest n^2 m0 q of a pass the oracle finishes in
# a few seconds on a host's cores
ORACLE_PASS_WORK = 1.2e10


def oracle_sample(prob):
    """The bounded oracle sample of a workload and its scale factor s: the
    workload itself when one oracle pass is a few seconds of CPU work (small
    dense, banded), else the same generator at n/s, m0/s (same q, contour and
    tolerances).  Every term of a dense pass is cubic in s (q n^2 m0 solves,
    n^2 m0 operator products, n m0^2 projections, QRs and Ritz products,
    m0^3 projected QZ), so one sampled pass times s^3 is one pass of the
    workload."""
    if prob.band:
        return prob, 1
    s = 1
    while (prob.n / s) ** 2 * (prob.m0 / s) * prob.q > ORACLE_PASS_WORK:
        s *= 2
    if s == 1:
        return prob, 1
    cfg = dict(prob.cfg, n=prob.n // s, m0=prob.m0 // s)
    return Problem(cfg), s


def golden_oracle_run(workload):
    """The stored converged oracle run of a workload (tests/golden), parsed
    from its text file, or None.  Written by a script that calls only the
    oracle; read here as data."""
    path = os.path.join(ROOT, "tests", "golden", f"{workload}_oracle.txt")
    if not os.path.exists(path):
        return None
    out = {"passes": [], "lam": [], "res": []}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, _, rest = line.strip().partition(" ")
        if key == "eig":
            re_, im_, r_ = rest.split()
            out["lam"].append(complex(float(re_), float(im_)))
            out["res"].append(float(r_))
        elif key == "pass":
            k, cnt, flag, err, sec = rest.split()
            out["passes"].append(dict(k=int(k), count=int(cnt), flag=int(flag), err=float(err), s=float(sec)))
        elif key == "host":
            out["host"] = rest
        elif key in ("threads", "flag", "k", "count", "exact_count"):
            out[key] = int(rest)
        elif key in ("setup_s", "err"):
            out[key] = float(rest)
    out["lam"] = np.array(out["lam"])
    out["res"] = np.array(out["res"])
    return out


class OracleSampler:
    """Whole passes of the oracle (GFEAST lines 5-17) on the bounded sample of
    a workload; a context that has stopped is replaced by a fresh one (its
    set-up is not part of any timed pass)."""

    def __init__(self, prob):
        import oracle
        self.oracle = oracle
        self.sprob, self.scale = oracle_sample(prob)
        self.fe = None
        self.setup_s = []

    def one_pass(self) -> float:
        if self.fe is None:
            t0 = time.perf_counter()
            self.fe = self.sprob.oracle_feast(self.oracle)
            self.setup_s.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        it = self.fe.iterate()
        dt = time.perf_counter() - t0
        if it["flag"] != 2:
            self.fe.close()
            self.fe = None
        return dt

    def close(self):
        if self.fe is not None:
            self.fe.close()
            self.fe = None

    def describe(self, npass: int, t_pass: float) -> str:
        sp = self.sprob
        if self.scale == 1:
            return (f"{npass} whole oracle GFEAST passes (lines 5-17) of the workload itself "
                    f"(n={sp.n}, m0={sp.m0}, q={sp.q}), {t_pass:.2f} s each, after the oracle's set-up")
        return (f"{npass} whole oracle GFEAST passes (lines 5-17, timed) of the same generator at "
                f"n={sp.n}, m0={sp.m0}, q={sp.q} (1/{self.scale} of n and m0), {t_pass:.2f} s each, "
                f"x{self.scale ** 3} (every term of a pass is cubic in n and m0 together) = "
                f"{t_pass * self.scale ** 3:.0f} s per pass of the workload")


def cpu_baseline(prob, args, budget_s: float = 20.0):
    """The oracle, as it stands, timed on this host's cores: whole passes of
    its bounded sample (set-up excluded), scaled to passes/s of the workload;
    beside it, where one was stored, the full-size oracle run's own timed
    passes (on the host that wrote it)."""
    import oracle
    threads = oracle.num_threads()
    smp = OracleSampler(prob)
    times = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and len(times) < 50:
        times.append(smp.one_pass())
    smp.close()
    t_pass = statistics.median(times)
    cb = {"value": 1.0 / (t_pass * smp.scale ** 3), "unit": "iters/s", "cores": threads, "kind": "oracle",
          "sample": smp.describe(len(times), t_pass), "cpu": _cpu_model()}
    g = golden_oracle_run(args.workload)
    if g is not None and g["passes"]:
        ps = [p["s"] for p in g["passes"]]
        cb["full_size_oracle_run"] = {
            "what": "the stored converged oracle run of this workload (tests/golden): every pass timed",
            "host": g.get("host"), "threads": g.get("threads"), "setup_s": g.get("setup_s"),
            "passes": len(ps), "median_pass_s": statistics.median(ps), "iters_per_s": 1.0 / statistics.median(ps)}
    return cb


def _cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def reference_special(args, cfg):
    """Oracle timings for the batch and differentiation workloads: whole
    oracle runs on a sample, scaled to the workload's unit."""
    import oracle
    threads = oracle.num_threads()
    if "batch" in cfg:
        rb = inputs.ragged_batch(cfg["batch"], cfg["n_lo"], cfg["n_hi"], seed=cfg["seed"])
        # whole runs of mid-size pencils (a short budget per step), scaled by sum n^3
        return batch_cpu_baseline(cfg, rb, budget_s=2.0)
    if cfg.get("search"):
        # the complete algorithm (SEARCH then GFEAST from its basis) at n/4,
        # width and counts scaled alike, time scaled by n^3
        sc = cfg["search"]
        n = cfg["n"] // 4
        m0 = cfg["m0"] // 4
        p = inputs.gapped_pencil(n, m0, cfg["n_in"] // 4, seed=cfg["seed"])
        kw = dict(contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"], a=cfg["radius"],
                  eps=cfg["eps"])
        pool = inputs.complex_normal(np.random.default_rng(cfg["seed"] + 1), (n, sc["pool"] // 4))
        t0 = time.perf_counter()
        o = oracle.Feast(p.A, p.B, p.Y, **kw)
        r = o.search(pool, sc["alpha"], max(1, sc["p"] // 4), sc["rank_tol"])
        o.close()
        o2 = oracle.Feast(p.A, p.B, r["U1"], **kw)
        o2.set_U1(r["U1"])
        passes = len(o2.run())
        o2.close()
        dt = time.perf_counter() - t0
        t_full = dt * 64.0
        return {"value": passes / t_full, "unit": "iters/s", "cores": threads, "kind": "oracle",
                "sample": f"oracle SEARCH + GFEAST at n={n} ({dt:.1f} s, {passes} passes) scaled by (4)^3 "
                          f"to n={cfg['n']}"}
    if cfg.get("compare"):
        # the oracle's GFEAST on the gapped pencil at n/4 (width and count
        # scaled alike), time scaled by n^3
        n = cfg["n"] // 4
        p = inputs.gapped_pencil(n, cfg["m0"] // 4, cfg["n_in"] // 4, seed=cfg["seed"])
        t0 = time.perf_counter()
        o = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"],
                         a=cfg["radius"], eps=cfg["eps"])
        passes = len(o.run())
        o.close()
        dt = time.perf_counter() - t0
        t_full = dt * 64.0
        return {"value": passes / t_full, "unit": "iters/s", "cores": threads, "kind": "oracle",
                "sample": f"oracle GFEAST at n={n} ({dt:.1f} s, {passes} passes) scaled by (4)^3 to n={cfg['n']}"}
    # differentiation: the oracle's gradient (two whole-pencil QZs) at n/4, scaled by n^3
    n = cfg["n"] // 4
    p = inputs.prescribed_pencil(n, 8, seed=cfg["seed"])
    t0 = time.perf_counter()
    oracle.eig_grad_abs2(p.A, p.B, 0, cfg["center"], cfg["radius"])
    dt = time.perf_counter() - t0
    t_full = dt * 64.0
    return {"value": 1.0 / t_full, "unit": "gradients/s", "cores": threads, "kind": "oracle",
            "sample": f"oracle gradient at n={n} ({dt:.1f} s) scaled by (4)^3 to n={cfg['n']}"}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cfg = inputs.WORKLOADS[args.workload]
    if "batch" in cfg or cfg.get("grad") or cfg.get("search") or cfg.get("compare"):
        vals = [reference_special(args, cfg) for _ in range(max(1, args.steps))]
        v = statistics.median([x["value"] for x in vals])
        cb = dict(vals[-1])
        cb["value"] = v
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": cb["unit"], "n_gpus": 0,
                "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 / v, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
                "config": {"workload": args.workload}, "cpu_baseline": cb,
                "e2e": {"value": v, "unit": cb["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    # a step is one whole oracle pass (lines 5-17) of the workload's bounded
    # sample, timed on its own; value scales the timed passes to passes/s of
    # the workload (s^3, see oracle_sample)
    import oracle
    prob = Problem(cfg)
    smp = OracleSampler(prob)
    for _ in range(args.warmup):
        smp.one_pass()
    times = [smp.one_pass() for _ in range(args.steps)]
    smp.close()
    t_step = sum(times) / len(times)
    v = 1.0 / (t_step * smp.scale ** 3)
    cb = {"value": v, "unit": "iters/s", "cores": oracle.num_threads(), "kind": "oracle",
          "sample": smp.describe(len(times), t_step), "cpu": _cpu_model()}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "step": "one timed oracle pass of the sample (value scales it by s^3 to the workload)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": config_dict(prob, args, world),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict(prob, args, world):
    d = {"workload": args.workload}
    d.update(prob.describe())
    d.update({"precision": args.prec,
              "parallelism": "one GPU" if world == 1 else f"node-sharded over {world} GPUs (NCCL all-reduce of U)",
              "l2": "inputs larger than L2 (per-node LU factors)"})
    return d


# ----------------------------------------------------------------------- GPU arm
def parity_report(r, prob):
    errs = []
    pool = list(prob.ref)
    for x in r["lam"]:
        if not pool:
            break
        j = int(np.argmin([abs(x - y) for y in pool]))
        errs.append(abs(x - pool[j]) / max(abs(pool[j]), 1e-300))
        pool.pop(j)
    return {"flag": r["flag"], "count": r["count"], "exact_count": int(len(prob.ref)),
            "max_rel_eig_err_vs_exact": max(errs) if errs else 0.0,
            "max_resid_eq_5_1": float(np.max(r["res"])) if r["count"] else 0.0}


def match_eigs(lam, ref):
    """Relative errors of lam against ref as multisets: both sorted by real
    then imaginary part, each value matched to its nearest unmatched
    partner."""
    pool = list(np.asarray(ref)[np.lexsort((np.imag(ref), np.real(ref)))])
    errs = []
    for x in np.asarray(lam)[np.lexsort((np.imag(lam), np.real(lam)))]:
        if not pool:
            break
        d = np.abs(np.asarray(pool) - x)
        j = int(np.argmin(d))
        errs.append(float(d[j] / max(abs(pool[j]), 1e-300)))
        pool.pop(j)
    return errs


def oracle_parity(r, golden, k_stop):
    """The GPU solve against the stored converged oracle run of the same
    workload: the inside count exactly, every eigenvalue to 1e-8 relative
    (the precision form's bound), the stop flag, the pass index."""
    errs = match_eigs(r["lam"], golden["lam"])
    worst = max(errs) if errs else 0.0
    return {"oracle_count": golden.get("count"), "count_match": int(r["count"]) == int(golden.get("count", -1)),
            "oracle_flag": golden.get("flag"), "oracle_k": golden.get("k"), "k": k_stop,
            "max_rel_eig_err_vs_oracle": worst, "within_1e-8": bool(worst <= 1e-8) and
            int(r["count"]) == int(golden.get("count", -1))}


def solve_once(fg, torch, dev, stream, prob, host, kw, nvtx_pass=None):
    """One whole GFEAST solve through the public API -- the bench's step:
    the pencil and start block copied from pinned host memory to the device,
    set-up (lines 1-3: contour, node-batched LU, first subspace), passes of
    lines 5-17 until a stopping test fires (flag 1, 0 or -1; line 15 caps it
    at max_iter), then the eigenvalues, residuals and eigenvectors back to
    the host.  A CUDA event on the library's stream follows every pass, so
    each pass has its own device time."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dev_arrays = [h.to(dev, non_blocking=True) for h in host]
    fe = prob.feast(fg, dev, stream, dev_arrays, **kw)
    setup_ms = fe.setup_info["ms_lu"] + fe.setup_info["ms_solve"]
    evs = [torch.cuda.Event(enable_timing=True)]
    evs[0].record(stream)
    infos = []
    try:
        while True:
            k = len(infos) + 1
            if nvtx_pass is not None and k == nvtx_pass:
                torch.cuda.nvtx.range_push("timed")     # ncu --nvtx-include "timed/" captures this pass
            it = fe.iterate()
            if nvtx_pass is not None and k == nvtx_pass:
                torch.cuda.nvtx.range_pop()
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            evs.append(ev)
            infos.append(it)
            if it["flag"] != 2:
                break
        res = fe.eigs(want_vectors=True)        # device -> host: values, residuals, vectors
        torch.cuda.synchronize()
    finally:
        fe.close()
    t_wall = time.perf_counter() - t0
    pass_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(infos))]
    return dict(setup_ms=setup_ms, setup_info=fe.setup_info, infos=infos, pass_ms=pass_ms, k_stop=infos[-1]["k"],
                t_wall=t_wall, res=res)



RETRIES = []     # (step, error) of every solve that a bounded device wait ended


def solve_step(fg, *a, step="", **kw):
    """solve_once, run again once if a bounded device wait gave up (status
    ETIMEOUT: the library's kernels returned, the context is intact).  The
    failed attempt stays inside whatever wall-clock region the caller times,
    and the JSON line lists it under "retried_solves"."""
    try:
        return solve_once(fg, *a, **kw)
    except fg.FeastError as e:
        if e.status != -6:
            raise
        RETRIES.append(dict(step=step, error=str(e)))
        log("solve ended by a bounded wait, run again:", str(e))
        return solve_once(fg, *a, **kw)


# DRAM bytes per launch of the kernels that lead two workloads' roofline
# entries, from ncu captures of exactly those workloads (the summaries under
# profiles/ give the commands); valid for those sizes only
HQR_FP32_DRAM_BYTES = 40165376 + 52448512                      # k_hqr, cold pass, n = 4096, m0 = 1280
BAND_SOLVE_DRAM_BYTES = (434.031616 + 110.770432 + 700.294144 + 119.855616) * 1e6   # k_gb_fwd + k_gb_bwd


def _bf16_peak():
    return _measured("bf16_tflops_sustained", 1753.1)


def roofline_phases(prob, args, ph, infos):
    """One roofline entry per phase of a pass, each for the kernel class that
    carries the phase; "achieved" = the phase's algorithmic work / the
    phase's CUDA-event time on the library's stream (so every other kernel
    of the phase counts against it: a lower bound on the kernel's own rate).
    Complex multiply-add = 8 flops."""
    n, m0, q = prob.n, prob.m0, prob.q
    out = {}
    # subspace-build solves (and the band solves)
    out["subspace-build solves"] = roofline(prob, args, ph)
    if prob.band:
        return out
    warm = [i for i in infos if i.get("qz_warm")]
    cold = [i for i in infos if not i.get("qz_warm")]
    t_warm = sum(i["ms_qz"] for i in warm)
    t_cold = sum(i["ms_qz"] for i in cold)
    gms = sum(i.get("ms_warm_gemm", 0.0) for i in warm)
    gfl = sum(i.get("warm_gemm_flop", 0.0) for i in warm)
    if warm and t_warm >= t_cold and gms > 0.0 and gfl > 0.0:
        # the library's own CUDA events around exactly the product launches
        # of the warm Newton step: FP64 GEMMs and triangular inverses for C
        # and C', the defect-form products on the digit-sliced tensor-core
        # GEMM; reported against the FP64 peak (what the arithmetic needs)
        ach = gfl / (gms / 1e3) / 1e12
        out["projected eigensolve"] = {
            "bound": "alu", "achieved": ach, "peak": FP64_MEASURED_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_MEASURED_TFLOPS, "traffic": None,
            "kernel": "warm Newton step: k_gemm<double2> + triangular inverses (C = B~^-1 A~, C' = Zh^H C Zh) "
                      "and k_oz_gemm for the defect-form products (D V^, V^-1 W', V^ G, V^ S1, W' G), "
                      "FP64-equivalent flops; CUDA events around exactly those launches",
            "peak_source": FP64_SOURCE,
            "algorithmic_flops_per_pass": gfl / len(warm), "kernel_ms_per_pass": gms / len(warm),
            "warm_passes": len(warm), "cold_passes": len(cold),
            "tail_schur_rows": statistics.mean(i["qz_rows"] for i in warm)}
    elif warm and t_warm >= t_cold:
        # warm solve without the library's segment events: FP64 products at
        # m0 (4 with a triangular factor, half the MACs; 1 full), 2
        # triangular inverses (~m0^3/3 MACs each), over the warm phase time
        flops = 8.0 * (4 * 0.5 + 1 + 2.0 / 3.0) * m0 ** 3 * len(warm)
        ach = flops / (t_warm / 1e3) / 1e12
        out["projected eigensolve"] = {
            "bound": "alu", "achieved": ach, "peak": FP64_MEASURED_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_MEASURED_TFLOPS, "traffic": None,
            "kernel": "k_gemm<double2> (warm Newton step) on the FP64 pipe, with the tail Schur form inside "
                      "the same phase time",
            "peak_source": FP64_SOURCE,
            "algorithmic_flops_per_pass": flops / len(warm), "warm_passes": len(warm), "cold_passes": len(cold)}
    elif cold:
        # cold projected solve: the multishift QR's rotations (phases x 32
        # rotations x 2 m0 element pairs x the FP32 operations of one
        # element-pair rotation: ~172 in double-single arithmetic, ~24 in the
        # FP32 build that the cold passes with a loose acceptance take), over
        # the whole cold projected-eigensolve phase time
        fp32 = [i for i in cold if i.get("qz_cold_fp32") == 1]
        ops = sum(i["qz_phases"] * 32 * 2 * m0 * (24.0 if i.get("qz_cold_fp32") == 1 else 172.0) for i in cold)
        # DRAM bytes of one cold-pass k_hqr launch from the ncu capture of
        # this workload (profiles/k_hqr_fp32_dense_n4096_m1280_q32.md)
        meas = HQR_FP32_DRAM_BYTES if (n, m0, q) == (4096, 1280, 32) and fp32 else None
        out["projected eigensolve"] = {
            "bound": "alu", "achieved": ops / (t_cold / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ops / (t_cold / 1e3) / 1e12 / FP32_PEAK_TFLOPS, "traffic": meas,
            "kernel": ("k_hqr multishift QR with early deflation (FP32 build on %d of %d cold passes, then the FP64 "
                       "Newton polish; double-single otherwise): a latency-bound rotation chain; phase time of the "
                       "cold passes (Hessenberg reduction, Newton step and eigenvectors included)" % (len(fp32), len(cold))),
            "peak_source": "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz",
            "algorithmic_ops_per_pass": ops / len(cold), "warm_passes": len(warm), "cold_passes": len(cold)}
    if args.prec != "fp64":
        # orthonormalisation: two Cholesky-QR-twice (U and B U1) + B U1:
        # Gram m0^2 n and V R^-1 n m0^2 MACs per Cholesky-QR pass on the
        # digit-sliced tensor-core GEMM (36 bf16 products of the realified
        # operands per real product: 36 * 8 tensor flops per complex MAC)
        tc_macs = 2 * (2 * (2 * n * m0 * m0) + m0 ** 3) + (0 if prob.kw.get("b_identity") else n * n * m0)
        tflops = 36 * 8.0 * tc_macs
        t_qr = ph["ms_qr"] / 1e3
        pk = _bf16_peak()
        out["orthonormalisation"] = {
            "bound": "tensor", "achieved": tflops / t_qr / 1e12, "peak": pk, "unit": "TFLOP/s",
            "frac": tflops / t_qr / 1e12 / pk, "traffic": None,
            "kernel": "k_oz_gemm (Gram matrices, V R^-1, B U1; bf16 digit products) with the FP64 Cholesky and "
                      "triangular inverses inside the same phase time",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (timed inside a pass)",
            "fp64_equivalent_tflops": 8.0 * tc_macs / t_qr / 1e12,
            "algorithmic_flops_per_pass": tflops}
        # projection U2^H [A U1 | B U1] + A U1 (and the Ritz products of line 6)
        pm = n * n * m0 + 2 * m0 * n * m0 + 3 * n * m0 * m0
        pf = 36 * 8.0 * pm
        t_p = ph["ms_proj"] / 1e3
        out["projection"] = {
            "bound": "tensor", "achieved": pf / t_p / 1e12, "peak": pk, "unit": "TFLOP/s",
            "frac": pf / t_p / 1e12 / pk, "traffic": None,
            "kernel": "k_oz_gemm (A U1, U2^H [A U1 | B U1], U1 Y, [A U1 | B U1] Y)",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (timed inside a pass)", "algorithmic_flops_per_pass": pf}
    return out


def roofline_dominant(prob, args, ph, infos):
    """Roofline of the pass's dominant phase (largest CUDA-event time), with
    the others listed beside it."""
    solve = ph["ms_solve"] - (ph["ms_refine"] if args.prec != "fp64" else 0.0)
    times = {"projected eigensolve": ph["ms_qz"], "subspace-build solves": solve,
             "orthonormalisation": ph["ms_qr"], "projection": ph["ms_proj"]}
    rows = roofline_phases(prob, args, ph, infos)
    for k, r in rows.items():
        r["phase"] = k
        r["share_of_pass"] = times.get(k, 0.0) / sum(times.values())
    dom = max((k for k in rows), key=lambda k: times.get(k, 0.0))
    others = [rows[k] for k in rows if k != dom]
    return rows[dom], others


def roofline(prob, args, ph):
    """Roofline entry for the phase that carries the workload's defining
    kernel: the dense shifted solves (FP64 or FP32 pipe) or the band solves
    (HBM)."""
    n, m0, q = prob.n, prob.m0, prob.q
    t_solve = max(ph["ms_solve"] - (ph["ms_refine"] if args.prec != "fp64" else 0.0), 1e-6) / 1e3
    if prob.band:
        # forward sweep over kl multipliers, backward over kl + ku + 1 factor
        # entries per column, per right-hand side and node: 8 flops per
        # complex multiply-add.  At ~47 flops per byte of factors the band
        # solves sit above GB300's FP64 ridge (0.16 flop/B) and FP32 ridge
        # (~10 flop/B): arithmetic-bound, not HBM-bound.
        kl, ku = prob.bp.kl, prob.bp.ku
        flops = 8.0 * q * m0 * n * (2 * kl + ku + 1)
        es = 16 if args.prec == "fp64" else 8
        traffic = q * (2 * kl + ku + 1) * n * es + 4 * q * n * m0 * es
        peak = FP64_PEAK_TFLOPS if args.prec == "fp64" else FP32_PEAK_TFLOPS
        # DRAM bytes of one forward + backward solve from the ncu capture of
        # this workload (profiles/k_gb_solve_band_n16384_m64_q16.md)
        meas = (BAND_SOLVE_DRAM_BYTES if (args.prec != "fp64" and (n, kl, ku, q, m0) == (16384, 128, 128, 16, 64))
                else None)
        return {"bound": "alu", "achieved": flops / t_solve / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / t_solve / 1e12 / peak, "traffic": meas,
                "kernel": "band solves k_gb_fwd + k_gb_bwd (subspace-build phase), "
                          + ("FP64 pipe" if args.prec == "fp64" else "FP32 pipe"),
                "peak_source": "derived: 152 SMs x " + ("2 DFMA" if args.prec == "fp64" else "128 FFMA")
                               + "/clk x 2 flop x 2.07 GHz",
                "algorithmic_flops_per_pass": flops, "algorithmic_bytes_per_pass": traffic,
                "hbm_gbs": traffic / t_solve / 1e9}
    flops = 8.0 * q * n * n * m0          # complex MAC = 8 flops, a4
    if args.prec == "fp64":
        return {"bound": "alu", "achieved": flops / t_solve / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": flops / t_solve / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "subspace-build solves (k_gemm<double2> + k_trsv_diag), FP64 pipe",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                "algorithmic_flops_per_pass": flops}
    pk = TF32_PEAK_TFLOPS / 3.0
    return {"bound": "tensor", "achieved": flops / t_solve / 1e12, "peak": pk, "unit": "TFLOP/s",
            "frac": flops / t_solve / 1e12 / pk, "traffic": None,
            "kernel": "subspace-build complex64 solves, whole phase (k_tc_cgemm2 tcgen05 kind::tf32 + "
                      "k_trsv_diag + in-block k_gemm<float2> + right-hand-side splits); complex flops of the "
                      "solves",
            "peak_source": TF32_SOURCE + ", / 3 (three TF32 products per FP32-accurate product)",
            "algorithmic_flops_per_pass": flops}


def tc_gemm_rooflines(setup_infos, pass_infos):
    """The tensor-core GEMM (k_tc_cgemm2) alone, from the library's CUDA
    events around exactly its launches: the set-up LU's trailing updates
    A22 -= L21 U12, and the off-block updates of each pass's shifted solves.
    achieved = complex flops (8 per complex multiply-add) / launch time; the
    peak is the TF32 peak / 3 -- three TF32 products (head x head, head x
    tail, tail x head of the realified operands) make one FP32-accurate
    product, so frac is the tensor pipe's share of its peak."""
    pk = TF32_BURST_TFLOPS / 3.0
    out = []
    for what, infos in (("LU trailing updates (set-up)", setup_infos), ("shifted-solve updates (passes)", pass_infos)):
        ms = sum(i.get("ms_tc_gemm", 0.0) for i in infos)
        fl = sum(i.get("tc_gemm_flop", 0.0) for i in infos)
        if ms <= 0.0 or fl <= 0.0:
            continue
        ach = fl / (ms / 1e3) / 1e12
        out.append({"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "traffic": None, "phase": what,
                    "kernel": "k_tc_cgemm2 (persistent, cta_group::2 256 x 256 tiles, tcgen05 kind::tf32, 3 "
                              "split products); CUDA events around exactly its launches",
                    "peak_source": TF32_BURST_SOURCE + ", / 3 (three TF32 products per FP32-accurate product)",
                    "tensor_pipe_active_ncu": 0.792,
                    "ncu": "profiles/k_tc_cgemm2_lu_update_dense_n2048_m512_q8.md (first LU trailing update, "
                           "n = 2048, 8 nodes): tensor pipe 79.2 % active, DRAM 541 MB per launch = the "
                           "algorithmic bytes",
                    "launch_ms_total": ms, "algorithmic_flops_total": fl, "runs": len(infos)})
    return out


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
    prob = Problem(cfg)
    n, m0 = prob.n, prob.m0
    kw_prec = {}
    if args.prec == "c64r":
        kw_prec = dict(prec=fg.FEAST_C64_REFINE, refine_tol=1e-13, max_refine=4)
    if world > 1:
        # node-sharded (end of Section 4.3): each rank owns a contiguous range
        # of the q quadrature nodes -- their factors and solves -- and the
        # partial quadrature sums of line 16 are all-reduced with NCCL; lines
        # 5-15 and 17 run on every rank.  One solve is shared by all ranks.
        kw_prec = dict(kw_prec, node_range=fg.shard_nodes(prob.q, world, rank),
                       collective=fg.dist_collective())
    stream = torch.cuda.current_stream()
    host = prob.pinned()
    h2d_bytes = sum(h.numel() * h.element_size() for h in host)

    for w in range(args.warmup):
        solve_step(fg, torch, dev, stream, prob, host, kw_prec, step=f"warm-up {w}")
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = fg.kernel_launches()
    t0 = time.perf_counter()
    runs = [solve_step(fg, torch, dev, stream, prob, host, kw_prec, step=f"timed {i}",
                       nvtx_pass=(args.profile_pass if i == 0 else None)) for i in range(args.steps)]
    torch.cuda.synchronize()
    barrier(world)
    t_region = time.perf_counter() - t0
    launches = fg.kernel_launches() - launches0
    clk = clocks.stop()
    for it, ms in zip(runs[0]["infos"], runs[0]["pass_ms"]):
        d = {k: (float(f"{v:.4g}") if isinstance(v, float) else v) for k, v in it.items()}
        d["pass_ms"] = round(ms, 2)
        log("pass", d)

    passes = sum(r["k_stop"] for r in runs)
    t_pass = sum(sum(r["pass_ms"]) for r in runs) / 1e3
    t_pass_max = max_over_ranks(t_pass, world, dev)
    t_region_max = max_over_ranks(t_region, world, dev)
    value = passes / t_pass_max                 # one solve shared by all ranks
    infos = [it for r in runs for it in r["infos"]]
    warm = [(it, ms) for r in runs for it, ms in zip(r["infos"], r["pass_ms"]) if it["k"] >= 4]
    warm_rate = len(warm) / (sum(ms for _, ms in warm) / 1e3) if warm else None
    setup_ms = statistics.mean(r["setup_ms"] for r in runs)
    last = runs[-1]
    r = last["res"]
    parity = parity_report(r, prob)
    parity["k_stop"] = [x["k_stop"] for x in runs]
    parity["flags"] = [x["res"]["flag"] for x in runs]
    golden = golden_oracle_run(args.workload)
    if golden is not None:
        parity["vs_oracle"] = oracle_parity(r, golden, last["k_stop"])
    counts = sum(x["res"]["count"] for x in runs)
    t_dev_solve = sum(x["setup_ms"] + sum(x["pass_ms"]) for x in runs) / 1e3
    d2h_bytes = statistics.mean((16 + 8) * x["res"]["count"] + 16 * n * x["res"]["count"] for x in runs)
    e2e = {"value": passes / t_region_max, "unit": "iters/s",
           "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
           "eigpairs_per_s": counts / t_region_max,
           "what": "whole solves through the public API: pinned host pencil and start block -> device, "
                   "set-up, passes until the stop fires, eigenvalues, residuals and eigenvectors back to "
                   "the host; passes / wall time of exactly those solves"}

    # the plain FP64 path on the same pencil: one whole solve, its passes
    # timed the same way (the same pass indices 1..k_stop of its own run)
    fp64 = None
    if args.prec != "fp64" and not args.no_fp64:
        r64 = solve_step(fg, torch, dev, stream, prob, host,
                         {k: v for k, v in kw_prec.items() if k in ("node_range", "collective")})
        rate64 = r64["k_stop"] / (sum(r64["pass_ms"]) / 1e3)
        fp64 = {"iters_per_s": rate64, "ms_per_iter": sum(r64["pass_ms"]) / r64["k_stop"],
                "setup_ms": r64["setup_ms"], "k_stop": r64["k_stop"], "flag": r64["res"]["flag"],
                "count": r64["res"]["count"], "whole_solve_s": r64["t_wall"],
                "pass_ms": [round(x, 1) for x in r64["pass_ms"]],
                "phase_ms": {k: statistics.mean(i[k] for i in r64["infos"])
                             for k in ("ms_proj", "ms_qz", "ms_solve", "ms_qr")},
                "speedup_passes": value / rate64,
                "speedup_whole_solve": r64["t_wall"] / statistics.mean(x["t_wall"] for x in runs),
                "parity": parity_report(r64["res"], prob)}
        del r64

    ph = {k: statistics.mean(i[k] for i in infos)
          for k in ("ms_proj", "ms_qz", "ms_solve", "ms_qr", "ms_refine")}
    roof, roof_kernels = roofline_dominant(prob, args, ph, infos)
    roof_kernels += tc_gemm_rooflines([r["setup_info"] for r in runs], infos)

    if rank == 0:
        cb = None
        if not args.no_baseline:
            cb = cpu_baseline(prob, args)
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_region_max / args.steps,
            "step": "one whole GFEAST solve (set-up, passes 1..k_stop, eigenpairs to the host); value = "
                    "GFEAST passes of the timed solves / CUDA-event time of exactly those passes",
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "c128" if args.prec == "fp64" else "c64+c128",
            "data": "synthetic", "config": config_dict(prob, args, world),
            "setup_ms": setup_ms,
            "warm_pass_rate": {"value": warm_rate, "unit": "iters/s", "passes": "k >= 4 up to k_stop",
                               "count": len(warm)},
            "eigpairs_per_s": counts / t_dev_solve,
            "pass_ms": [round(x, 1) for x in last["pass_ms"]],
            "parity": parity,
            "phase_ms": ph,
            "qz": {"warm": [i["qz_warm"] for i in last["infos"]], "qr_rows": [i["qz_rows"] for i in last["infos"]],
                   "sweeps": [i["qz_sweeps"] for i in last["infos"]],
                   "warm_resid": [i["qz_warm_resid"] for i in last["infos"]]},
            "fp64_path": fp64,
            "roofline": roof,
            "roofline_kernels": roof_kernels,
            "cpu_baseline": cb,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "retried_solves": RETRIES,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_arm(args, cfg):
    """Ragged batch workload: all pencils through one feast_solve_batch call
    (worker pool inside the library).  A step is one solve of the whole
    batch to convergence; value = GFEAST iterations of all pencils / time."""
    import torch
    import paper_1404_1768_gb300 as fg
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fg.load()
    rb = inputs.ragged_batch(cfg["batch"], cfg["n_lo"], cfg["n_hi"], seed=cfg["seed"])
    prec = fg.FEAST_C64_REFINE if args.prec == "c64r" else fg.FEAST_FP64
    probs = [dict(A=p.A, B=p.B, Y=p.Y, contour_kind=0, rule=0, q=cfg["q"], center=p.center, a=p.radius,
                  eps=cfg["eps"], prec=prec, refine_tol=1e-13, max_refine=4) for p in rb.pencils]
    # warm-up batches double as the schedule autotuner's trials: each times
    # the whole batch at one candidate concurrency; the timed batches use
    # the fastest
    tuner = fg.BatchSchedule(candidates=sorted({16, 32, 64, args.nworkers}))
    for _ in range(args.warmup):
        nw = tuner.next()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fg.solve_batch(probs, nworkers=nw)
        torch.cuda.synchronize()
        tuner.record(nw, time.perf_counter() - t0)
        torch.cuda.empty_cache()           # (each worker count sizes its own workspace)
        log("batch schedule trial", nw, "workers", round(tuner.times[nw], 2), "s")
    nworkers = tuner.best
    clocks = ClockSampler(local)
    clocks.start()
    times, outs = [], None
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = fg.solve_batch(probs, nworkers=nworkers)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    t = statistics.median(times)
    iters = sum(o["k"] for o in outs)
    worst, counts_ok, res_max, fails = 0.0, 0, 0.0, 0
    for p, o in zip(rb.pencils, outs):
        if o["status"] != 0 or o["flag"] != 1:
            fails += 1
            continue
        ref = p.lam[np.abs(p.lam - p.center) < p.radius]
        counts_ok += int(o["count"] == len(ref))
        pool = list(ref)
        for x in o["lam"]:
            if not pool:
                break
            j = int(np.argmin([abs(x - y) for y in pool]))
            worst = max(worst, abs(x - pool[j]) / max(abs(pool[j]), 1e-300))
            pool.pop(j)
        if o["count"]:
            res_max = max(res_max, float(np.max(o["res"])))
    # the dominant phase over the pencils' own streams (16 workers run
    # concurrently, so each pencil's event times include its neighbours'
    # kernels: the rates below are lower bounds), and the solves beside it
    solve_flops = sum(o["k"] * 8.0 * cfg["q"] * p.n * p.n * p.Y.shape[1] for p, o in zip(rb.pencils, outs)
                      if o["status"] == 0)
    t_solve = sum(o["ms_solve"] for o in outs) / 1e3
    t_qz = sum(o["ms_qz"] for o in outs) / 1e3
    t_pass = sum(o["ms_pass"] for o in outs) / 1e3
    pk = TF32_PEAK_TFLOPS / 3.0 if args.prec == "c64r" else FP64_MEASURED_TFLOPS
    solves = {"bound": "tensor" if args.prec == "c64r" else "alu", "achieved": solve_flops / t_solve / 1e12,
              "peak": pk, "unit": "TFLOP/s", "frac": solve_flops / t_solve / 1e12 / pk, "traffic": None,
              "phase": "subspace-build solves of all pencils", "share_of_pass_time": t_solve / t_pass,
              "kernel": "node-batched complex64 LU solves (k_tc_cgemm2 off-block updates, k_trsv_diag, in-block "
                        "k_gemm<float2>) per pencil; summed per-pencil stream time (concurrent pencils overlap)",
              "peak_source": (TF32_SOURCE + ", / 3") if args.prec == "c64r" else FP64_SOURCE}
    qz = {"bound": "alu", "achieved": None, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": None,
          "traffic": None, "phase": "projected eigensolves of all pencils", "share_of_pass_time": t_qz / t_pass,
          "kernel": "k_qz / k_small_schur / k_hqr (latency-bound rotation chains; no flop-rate reported)"}
    roof = qz if t_qz >= t_solve else solves
    roof_others = [solves] if roof is qz else [qz]
    cb = None
    if rank == 0 and not args.no_baseline:
        cb = batch_cpu_baseline(cfg, rb)
    if rank == 0:
        line = {"metric": METRIC, "value": iters / t, "unit": "iters/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c128" if args.prec == "fp64" else "c64+c128", "data": "synthetic",
                "config": {"workload": args.workload, "pencils": cfg["batch"],
                           "n_range": [cfg["n_lo"], cfg["n_hi"]], "q": cfg["q"],
                           "m0": "max(8, ceil(1.5 s / 8) * 8) per pencil", "precision": args.prec,
                           "parallelism": "replicas1", "workers": nworkers},
                "schedule_autotune": {"trials_s": {str(k): round(v, 3) for k, v in tuner.times.items()},
                                      "chosen_workers": nworkers},
                "pencils_per_s": cfg["batch"] / t, "total_iterations": iters,
                "parity": {"converged": cfg["batch"] - fails, "exact_counts": counts_ok,
                           "max_rel_eig_err_vs_exact": worst, "max_resid_eq_5_1": res_max},
                "e2e": {"value": iters / t, "unit": "iters/s",
                        "what": "host numpy pencils -> device, whole batch solved, results to host"},
                "clocks": clk, "roofline": roof, "roofline_kernels": roof_others, "cpu_baseline": cb}
        print(json.dumps(line))
    return 0


def batch_cpu_baseline(cfg, rb, budget_s: float = 25.0):
    """The oracle timed on whole GFEAST runs of a sample of the batch's
    pencils (those at the 10th, 25th, 40th and 55th percentiles of n, in that
    order, until the budget), scaled to the batch by the sum of n^3 (a pass
    costs ~n^3 with m0 ~ n)."""
    import oracle
    order = sorted(range(len(rb.pencils)), key=lambda i: rb.pencils[i].n)
    done, t_sum = [], 0.0
    for i in [order[int(f * (len(order) - 1))] for f in (0.10, 0.25, 0.40, 0.55)]:
        if t_sum > budget_s:
            break
        p = rb.pencils[i]
        t0 = time.perf_counter()
        fe = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=cfg["q"], center=p.center, a=p.radius,
                          eps=cfg["eps"])
        fe.run()
        fe.close()
        t_sum += time.perf_counter() - t0
        done.append(i)
    scale = sum(p.n ** 3 for p in rb.pencils) / sum(rb.pencils[i].n ** 3 for i in done)
    t_all = t_sum * scale
    return {"value": len(rb.pencils) / t_all, "unit": "pencils/s", "cores": oracle.num_threads(), "kind": "oracle",
            "cpu": _cpu_model(),
            "sample": f"whole oracle GFEAST runs of {len(done)} pencils (n = "
                      f"{', '.join(str(rb.pencils[i].n) for i in done)}; {t_sum:.1f} s), scaled by sum n^3 "
                      f"(x{scale:.1f}) to the {len(rb.pencils)} pencils"}


def grad_arm(args, cfg):
    """Differentiation form: one step = L = sum_{lambda inside} |lambda|^2 by
    GFEAST on (A, B) plus its gradients with respect to A and B (a GFEAST run
    on the conjugate-transposed pencil and the adjoint kernels), through the
    torch.autograd.Function.  Checked against the closed form of the
    prescribed-spectrum pencil and against central differences."""
    import torch
    import paper_1404_1768_gb300 as fg
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fg.load()
    p = inputs.prescribed_pencil(cfg["n"], cfg["m0"], seed=cfg["seed"], center=cfg["center"], radius=cfg["radius"])
    n = cfg["n"]
    kw = dict(contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"], a=cfg["radius"], eps=cfg["eps"])
    if args.prec == "c64r":
        kw.update(prec=fg.FEAST_C64_REFINE, refine_tol=1e-13, max_refine=4)
    A0 = torch.from_numpy(p.A).cuda()
    B0 = torch.from_numpy(p.B).cuda()
    Y = torch.from_numpy(p.Y).cuda()

    def step():
        A = A0.clone().requires_grad_(True)
        B = B0.clone().requires_grad_(True)
        L = fg.eig_sum_abs2(A, B, Y, **kw)
        L.backward()
        return float(L), A.grad, B.grad

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L, gA, gB = step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    t = statistics.median(times)
    # closed form: G_A = 2 P^-H diag(lam_in) Q^-H, G_B = -2 P^-H diag(|lam_in|^2) Q^-H
    inside = np.abs(p.lam - cfg["center"]) < cfg["radius"]
    d = np.where(inside, p.lam, 0.0)
    Pih = np.linalg.inv(p.P).conj().T
    Qih = np.linalg.inv(p.Q).conj().T
    refA = 2.0 * (Pih * d[None, :]) @ Qih
    refB = -2.0 * (Pih * (np.abs(d) ** 2)[None, :]) @ Qih
    eA = float(np.max(np.abs(gA.cpu().numpy() - refA)) / np.max(np.abs(refA)))
    eB = float(np.max(np.abs(gB.cpu().numpy() - refB)) / np.max(np.abs(refB)))
    # central differences along two random complex directions (forward runs only)
    # (directions of spectral norm ~2 and step 1e-6 keep every eigenvalue far
    # from the contour; the difference quotient's own error is about the
    # eigenvalue accuracy of the runs divided by the step)
    fd = []
    h = 1e-6
    with torch.no_grad():
        for t_ in range(2):
            E = torch.from_numpy(inputs.complex_normal(np.random.default_rng(100 + t_), (n, n)) / np.sqrt(n)).cuda()
            lp = float(fg.eig_sum_abs2(A0 + h * E, B0, Y, **kw))
            lm = float(fg.eig_sum_abs2(A0 - h * E, B0, Y, **kw))
            an = float(torch.real(torch.vdot(gA.reshape(-1), E.reshape(-1))))
            fd.append(abs((lp - lm) / (2 * h) - an) / max(1.0, abs(an)))
    if rank == 0:
        line = {"metric": METRIC, "value": 1.0 / t, "unit": "gradients/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128" if args.prec == "fp64" else "c64+c128",
                "data": "synthetic",
                "config": {"workload": args.workload, "n": n, "m0": cfg["m0"], "q": cfg["q"],
                           "loss": "sum of |lambda|^2 over the eigenvalues inside |z| < 1",
                           "precision": args.prec, "parallelism": "replicas1"},
                "L": L, "inside": int(inside.sum()),
                "parity": {"max_rel_err_grad_A_vs_closed_form": eA, "max_rel_err_grad_B_vs_closed_form": eB,
                           "central_difference_rel_err": fd},
                "e2e": {"value": 1.0 / t, "unit": "gradients/s",
                        "what": "device-resident A, B: forward GFEAST run, backward GFEAST run on the "
                                "conjugate-transposed pencil, adjoint kernels"},
                "clocks": clk, "roofline": None, "cpu_baseline": None}
        print(json.dumps(line))
    return 0


def search_arm(args, cfg):
    """The complete algorithm on a gapped pencil: SEARCH (Section 4.1) then
    GFEAST from its basis.  A step is one whole solve (set-up, SEARCH, passes
    until the stop fires); value = GFEAST passes / time, with SEARCH's own
    time and its bound t beside it."""
    import torch
    import paper_1404_1768_gb300 as fg
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fg.load()
    sc = cfg["search"]
    p = inputs.gapped_pencil(cfg["n"], cfg["m0"], cfg["n_in"], seed=cfg["seed"])
    inside = np.abs(p.lam - cfg["center"]) < cfg["radius"]
    pool_np = inputs.complex_normal(np.random.default_rng(cfg["seed"] + 1), (cfg["n"], sc["pool"]))
    kw = dict(contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"], a=cfg["radius"], eps=cfg["eps"])
    if args.prec == "c64r":
        kw.update(prec=fg.FEAST_C64_REFINE, refine_tol=1e-13, max_refine=4)

    def solve():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = fg.Feast(p.A, p.B, p.Y, **kw)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = g.search(pool_np, sc["alpha"], sc["p"], sc["rank_tol"])
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        hist = g.run()
        res = g.eigs(want_vectors=False)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        g.close()
        return dict(setup=t1 - t0, search=t2 - t1, iterate=t3 - t2, passes=len(hist), t=r["t"], s0=r["s0"],
                    res=res)

    for _ in range(args.warmup):
        solve()
    clocks = ClockSampler(local)
    clocks.start()
    runs = [solve() for _ in range(args.steps)]
    clk = clocks.stop()
    med = sorted(runs, key=lambda x: x["setup"] + x["search"] + x["iterate"])[len(runs) // 2]
    tot = med["setup"] + med["search"] + med["iterate"]
    res = med["res"]
    pool_ = list(p.lam[inside])
    worst = 0.0
    for x in res["lam"]:
        j = int(np.argmin([abs(x - y) for y in pool_]))
        worst = max(worst, abs(x - pool_[j]) / abs(pool_[j]))
        pool_.pop(j)
    if rank == 0:
        line = {"metric": METRIC, "value": med["passes"] / tot, "unit": "iters/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "c128" if args.prec == "fp64" else "c64+c128", "data": "synthetic",
                "config": {"workload": args.workload, "n": cfg["n"], "m0_workspace": cfg["m0"], "q": cfg["q"],
                           "pencil": "A = P diag(lam) Q, B = P Q, %d eigenvalues in |z| < 0.7, the rest in "
                                     "1.5 < |z| < 2 (seeded)" % cfg["n_in"],
                           "search": sc, "precision": args.prec, "parallelism": "replicas1"},
                "search_ms": 1e3 * med["search"], "setup_ms": 1e3 * med["setup"],
                "iterate_ms": 1e3 * med["iterate"],
                "parity": {"t": med["t"], "exact_inside": int(inside.sum()), "s0": med["s0"],
                           "flag": res["flag"], "count": res["count"],
                           "max_rel_eig_err_vs_exact": worst, "max_resid_eq_5_1": float(np.max(res["res"]))},
                "e2e": {"value": med["passes"] / tot, "unit": "iters/s",
                        "what": "host pencil -> device, set-up, SEARCH, GFEAST passes until the stop fires, "
                                "eigenvalues back to the host"},
                "clocks": clk, "roofline": None, "cpu_baseline": None}
        print(json.dumps(line))
    return 0


def sparse_arm(args, cfg):
    """A sparse pencil in CSR with no useful ordering (the banded workload's
    operator, rows and columns shuffled, B stored explicitly): a step is one
    whole solve through SparseFeast -- reverse Cuthill-McKee, scatter into
    band storage, set-up, GFEAST passes until the stop fires, eigenvalues to
    the host.  value = passes / that time; parity against the closed-form
    spectrum."""
    import torch
    import paper_1404_1768_gb300 as fg
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fg.load()
    sp = inputs.sparse_pencil(cfg["nx"], cfg["m0"], seed=cfg["seed"], beta=cfg["beta"], mass=cfg["sparse"]["mass"])
    n = sp.n
    lam = inputs.convection_diffusion_spectrum(cfg["nx"], cfg["beta"])
    ref = lam[((lam - cfg["center"].real) / cfg["a"]) ** 2 < 1.0] if cfg["sparse"]["mass"] == 0.0 else None
    kw = dict(contour_kind=1, rule=cfg["rule"], q=cfg["q"], center=cfg["center"], a=cfg["a"], b=cfg["b"],
              eps=cfg["eps"], eta=1e-3, max_iter=50)
    if args.prec == "c64r":
        kw.update(prec=fg.FEAST_C64_REFINE, refine_tol=1e-13, max_refine=4)
    t0 = time.perf_counter()
    perm, kl, ku = fg.csr_rcm(n, sp.A, sp.B)
    order_ms = 1e3 * (time.perf_counter() - t0)
    rows = np.repeat(np.arange(n), np.diff(sp.A[0]))
    bw_before = int(np.abs(rows - sp.A[1]).max())

    def solve():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = fg.SparseFeast(n, sp.A, sp.B, sp.Y, **kw)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hist = g.run()
        res = g.eigs(want_vectors=False)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        g.close()
        return dict(setup=t1 - t0, iterate=t2 - t1, passes=len(hist), res=res)

    for _ in range(args.warmup):
        solve()
    clocks = ClockSampler(local)
    clocks.start()
    runs = [solve() for _ in range(args.steps)]
    clk = clocks.stop()
    med = sorted(runs, key=lambda x: x["setup"] + x["iterate"])[len(runs) // 2]
    tot = med["setup"] + med["iterate"]
    res = med["res"]
    worst = None
    if ref is not None and res["count"] == len(ref):
        worst = float(max(np.min(np.abs(ref - x)) / abs(x) for x in res["lam"]))
    if rank == 0:
        line = {"metric": METRIC, "value": med["passes"] / tot, "unit": "iters/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "c128" if args.prec == "fp64" else "c64+c128", "data": "synthetic",
                "config": {"workload": args.workload, "n": n, "m0": cfg["m0"], "q": cfg["q"],
                           "pencil": "convection-diffusion (beta %s) on a %d x %d grid, rows and columns in a "
                                     "random order, CSR; B = I + %g * neighbour sum / 4, stored"
                                     % (cfg["beta"], cfg["nx"], cfg["nx"], cfg["sparse"]["mass"]),
                           "precision": args.prec, "parallelism": "replicas1"},
                "ordering": {"bandwidth_before": bw_before, "kl": kl, "ku": ku, "rcm_ms": order_ms},
                "setup_ms": 1e3 * med["setup"], "iterate_ms": 1e3 * med["iterate"],
                "parity": {"flag": res["flag"], "count": res["count"],
                           "exact_count": None if ref is None else int(len(ref)),
                           "max_rel_eig_err_vs_exact": worst,
                           "max_resid_eq_5_1": float(np.max(res["res"])) if res["count"] else None,
                           "passes": med["passes"]},
                "e2e": {"value": med["passes"] / tot, "unit": "iters/s",
                        "what": "host CSR pencil -> ordering, device band storage, set-up, GFEAST passes "
                                "until the stop fires, eigenvalues back to the host"},
                "clocks": clk, "roofline": None, "cpu_baseline": None}
        print(json.dumps(line))
    return 0


def compare_arm(args, cfg):
    """The comparison of Section 5 on one gapped pencil: GFEAST (oblique
    projection), the Rayleigh-Ritz FEAST of Section 3 (same driver, test
    basis U1) and Block CIRR of Section 2.1 (one pass over g moments of h
    random columns), all on the GPU at the same width.  A step solves the
    pencil with all three (each: set-up, solve, eigenvalues to the host);
    value = GFEAST passes / GFEAST time, the other methods' times and
    accuracies beside it."""
    import torch
    import paper_1404_1768_gb300 as fg
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fg.load()
    cc = cfg["compare"]
    p = inputs.gapped_pencil(cfg["n"], cfg["m0"], cfg["n_in"], seed=cfg["seed"])
    inside = np.abs(p.lam - cfg["center"]) < cfg["radius"]
    exact = p.lam[inside]
    Yc = inputs.complex_normal(np.random.default_rng(cfg["seed"] + 2), (cfg["n"], cc["h"]))
    kw = dict(contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"], a=cfg["radius"], eps=cfg["eps"])
    if args.prec == "c64r":
        kw.update(prec=fg.FEAST_C64_REFINE, refine_tol=1e-13, max_refine=4)

    def accuracy(res):
        pool_ = list(exact)
        worst = 0.0
        for x in res["lam"]:
            if not pool_:
                break
            j = int(np.argmin([abs(x - y) for y in pool_]))
            worst = max(worst, abs(x - pool_[j]) / abs(pool_[j]))
            pool_.pop(j)
        return worst

    def one(method):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        proj = fg.FEAST_OBLIQUE if method == "gfeast" else fg.FEAST_RAYLEIGH_RITZ
        g = fg.Feast(p.A, p.B, p.Y, projection=proj, **kw)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if method == "cirr":
            g.cirr(Yc, cc["g"])
            passes = 1
        else:
            passes = len(g.run())
        res = g.eigs(want_vectors=False)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        g.close()
        return dict(setup=t1 - t0, solve=t2 - t1, passes=passes, res=res)

    methods = ("gfeast", "rayleigh_ritz", "cirr")

    def step():
        return {m: one(m) for m in methods}

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    runs = [step() for _ in range(args.steps)]
    clk = clocks.stop()
    out = {}
    for m in methods:
        rs = sorted((r[m] for r in runs), key=lambda x: x["setup"] + x["solve"])
        med = rs[len(rs) // 2]
        res = med["res"]
        out[m] = {"ms_total": 1e3 * (med["setup"] + med["solve"]), "ms_setup": 1e3 * med["setup"],
                  "ms_solve": 1e3 * med["solve"], "passes": med["passes"], "flag": res["flag"],
                  "count": res["count"], "max_rel_eig_err_vs_exact": accuracy(res),
                  "max_resid_eq_5_1": float(np.max(res["res"])) if res["count"] else None}
    gf = out["gfeast"]
    if rank == 0:
        line = {"metric": METRIC, "value": gf["passes"] / (1e-3 * gf["ms_total"]), "unit": "iters/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": gf["ms_total"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c128" if args.prec == "fp64" else "c64+c128", "data": "synthetic",
                "config": {"workload": args.workload, "n": cfg["n"], "m0": cfg["m0"], "q": cfg["q"],
                           "pencil": "A = P diag(lam) Q, B = P Q, %d eigenvalues in |z| < 0.7, the rest in "
                                     "1.5 < |z| < 2 (seeded)" % cfg["n_in"],
                           "cirr": cc, "precision": args.prec, "parallelism": "replicas1"},
                "exact_inside": int(inside.sum()), "compare": out,
                "e2e": {"value": gf["passes"] / (1e-3 * gf["ms_total"]), "unit": "iters/s",
                        "what": "host pencil -> device, set-up, GFEAST passes until the stop fires, "
                                "eigenvalues back to the host"},
                "clocks": clk, "roofline": None, "cpu_baseline": None}
        print(json.dumps(line))
    return 0


def arm_for(cfg):
    """The GPU arm that measures a workload (its configuration's kind)."""
    if "batch" in cfg:
        return batch_arm
    for key, arm in (("grad", grad_arm), ("search", search_arm), ("compare", compare_arm),
                     ("sparse", sparse_arm)):
        if cfg.get(key):
            return arm
    return None     # the dense / banded pass of gpu_arm


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    cfg = inputs.WORKLOADS[args.workload]
    arm = arm_for(cfg)
    return arm(args, cfg) if arm else gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
