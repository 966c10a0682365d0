"""Writes dense_n4096_m1280_q32_oracle.txt: one converged run of the FP64
oracle (Algorithm GFEAST, lines 1-17 with the seeded start block in place of
SEARCH) on the dense n = 4096 workload of the precision form.

The workload: A = P diag(lam) Q, B = P Q (seed 0, lam uniform in |z| <= 2),
m0 = 1280, 32 trapezoid nodes on the circle |z| = 1, eps = 1e-10,
eta = 1e-3, max_iter = 50.  The script calls only the oracle and the seeded
input generator; nothing here comes from the CUDA library.  It records the
stop (flag, pass index, count), every accepted eigenvalue with its eq. 5.1
residual, and the wall time of the oracle's set-up and of each pass with the
host's CPU model and thread count, so the per-pass CPU time is a timing, not
a model.

    python tests/golden/make_dense_n4096_oracle.py      # ~1-2 h on 8 cores
"""
from __future__ import annotations

import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1404_1768_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "dense_n4096_m1280_q32_oracle.txt")
WORKLOAD = "dense_n4096_m1280_q32"


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def main(out: str = OUT) -> None:
    cfg = inputs.WORKLOADS[WORKLOAD]
    n, m0, q = cfg["n"], cfg["m0"], cfg["q"]
    p = inputs.prescribed_pencil(n, m0, seed=cfg["seed"], center=cfg["center"], radius=cfg["radius"])
    kw = dict(contour_kind=0, rule=cfg["rule"], q=q, center=cfg["center"], a=cfg["radius"],
              eps=cfg["eps"], eta=1e-3, max_iter=50)
    threads = oracle.num_threads()
    t0 = time.perf_counter()
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    t_setup = time.perf_counter() - t0
    print(f"set-up {t_setup:.1f} s", flush=True)
    passes = []
    while True:
        t0 = time.perf_counter()
        it = o.iterate()
        dt = time.perf_counter() - t0
        passes.append((it, dt))
        print(f"pass {it['k']}: count {it['count']} flag {it['flag']} err {it['err']:.3e} ({dt:.1f} s)",
              flush=True)
        if it["flag"] != 2:
            break
    r = o.result()
    o.close()
    order = np.lexsort((r["lam"].imag, r["lam"].real))
    lines = [
        "# One converged run of the FP64 oracle (Algorithm GFEAST, Section 4.3) on the dense",
        f"# workload {WORKLOAD}: A = P diag(lam) Q, B = P Q, seed {cfg['seed']},",
        f"# n = {n}, m0 = {m0}, {q} trapezoid nodes on |z| = {cfg['radius']}, eps = {cfg['eps']}, eta = 1e-3.",
        "# Written by tests/golden/make_dense_n4096_oracle.py (calls only the oracle and the",
        "# seeded generator).  Timings are wall-clock seconds of the oracle on this host.",
        f"host {cpu_model()}",
        f"threads {threads}",
        f"setup_s {t_setup:.3f}",
        "# pass k count flag err seconds",
    ]
    for it, dt in passes:
        lines.append(f"pass {it['k']} {it['count']} {it['flag']} {it['err']:.6e} {dt:.3f}")
    lines += [
        f"flag {r['flag']}",
        f"k {r['k']}",
        f"count {r['count']}",
        f"exact_count {int(np.sum(np.abs(p.lam - cfg['center']) < cfg['radius']))}",
        f"err {r['err']:.6e}",
        "# accepted eigenvalues (sorted by real, then imaginary part): re im residual_eq_5_1",
    ]
    for i in order:
        lines.append(f"eig {r['lam'][i].real:.17e} {r['lam'][i].imag:.17e} {r['res'][i]:.6e}")
    with open(out + ".tmp", "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(out + ".tmp", out)
    print("wrote", out, flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else OUT)
