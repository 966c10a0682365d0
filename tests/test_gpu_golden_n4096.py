"""The precision form at the n = 4096 workload (A = P diag(lam) Q, B = P Q,
seed 0, m0 = 1280, 32 trapezoid nodes on |z| = 1, eps = 1e-10) against the
stored converged run of the FP64 oracle on the same inputs
(tests/golden/dense_n4096_m1280_q32_oracle.txt, written by the script beside
it, which calls only the oracle): the inside count exactly, every eigenvalue
to 1e-8 relative (the precision form's bound), the same stop (flag 1 within
one pass of the oracle's), residuals of eq. 5.1 at most 1e-10."""
import os

import numpy as np
import pytest

from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dense_n4096_m1280_q32_oracle.txt")


def _read_golden(path):
    out = {"lam": [], "res": []}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, _, rest = line.strip().partition(" ")
        if key == "eig":
            re_, im_, r_ = rest.split()
            out["lam"].append(complex(float(re_), float(im_)))
            out["res"].append(float(r_))
        elif key in ("flag", "k", "count", "exact_count"):
            out[key] = int(rest)
    out["lam"] = np.array(out["lam"])
    return out


def test_precision_form_n4096_matches_the_stored_oracle_run():
    import paper_1404_1768_gb300 as fg
    gold = _read_golden(GOLDEN)
    cfg = inputs.WORKLOADS["dense_n4096_m1280_q32"]
    p = inputs.prescribed_pencil(cfg["n"], cfg["m0"], seed=cfg["seed"], center=cfg["center"], radius=cfg["radius"])
    g = fg.Feast(p.A, p.B, p.Y, contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"],
                 a=cfg["radius"], eps=cfg["eps"], eta=1e-3, max_iter=50, prec=fg.FEAST_C64_REFINE,
                 refine_tol=1e-13, max_refine=4)
    hist = g.run()
    r = g.eigs(want_vectors=False)
    g.close()
    assert gold["flag"] == 1 and r["flag"] == 1
    assert r["count"] == gold["count"] == gold["exact_count"] == p.inside_count()
    assert abs(hist[-1]["k"] - gold["k"]) <= 1
    # eigenvalues as multisets, both sorted, each matched to its nearest
    pool = list(gold["lam"])
    worst = 0.0
    for x in sorted(r["lam"], key=lambda v: (v.real, v.imag)):
        d = np.abs(np.asarray(pool) - x)
        j = int(np.argmin(d))
        worst = max(worst, d[j] / abs(pool[j]))
        pool.pop(j)
    assert worst <= 1e-8, worst
    assert np.max(r["res"]) <= 1e-10
