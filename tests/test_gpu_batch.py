"""Ragged batch: many independent pencils of uneven size, each with its own
circle, solved concurrently by the library's worker pool; every pencil's
result must equal what the single-pencil oracle finds for it."""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu


def _match(a, b):
    b = list(b)
    worst = 0.0
    for x in sorted(a, key=lambda v: (v.real, v.imag)):
        j = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[j]))
        b.pop(j)
    return worst


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_batch_matches_oracle(prec):
    import paper_1404_1768_gb300 as fg
    rb = inputs.ragged_batch(6, 48, 140, seed=11)
    probs = []
    for p, m0 in zip(rb.pencils, rb.m0):
        probs.append(dict(A=p.A, B=p.B, Y=p.Y, contour_kind=0, rule=0, q=16, center=p.center,
                          a=p.radius, eps=1e-10, prec=prec, refine_tol=1e-14))
    out = fg.solve_batch(probs, nworkers=4)
    for p, o, pr in zip(rb.pencils, out, probs):
        assert o["status"] == 0 and o["flag"] == 1
        ref = p.lam[np.abs(p.lam - p.center) < p.radius]
        assert o["count"] == len(ref)
        if len(ref):
            assert _match(o["lam"], ref) < 1e-8
            assert np.all(o["res"] < 1e-10)
        orc = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=16, center=p.center,
                           a=p.radius, eps=1e-10)
        orc.run()
        ro = orc.result()
        assert ro["count"] == o["count"]
        orc.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_batch_mixed_paths(prec):
    """Pencils large enough that their projected problems take both
    eigensolver paths (m0 <= 64: one-CTA QZ with a size-dependent shared
    memory request; m0 > 64: the cooperative QR), solved by 8 concurrent
    workers: every pencil converges to its exact inside count."""
    import paper_1404_1768_gb300 as fg
    rb = inputs.ragged_batch(12, 64, 480, seed=5)
    assert min(rb.m0) <= 64 < max(rb.m0)
    probs = [dict(A=p.A, B=p.B, Y=p.Y, contour_kind=0, rule=0, q=16, center=p.center, a=p.radius, eps=1e-10,
                  prec=prec, refine_tol=1e-13, max_refine=4) for p in rb.pencils]
    out = fg.solve_batch(probs, nworkers=8)
    for p, o in zip(rb.pencils, out):
        assert o["status"] == 0 and o["flag"] == 1
        ref = p.lam[np.abs(p.lam - p.center) < p.radius]
        assert o["count"] == len(ref)
        if len(ref):
            assert _match(o["lam"], ref) / max(1.0, np.max(np.abs(ref))) < 1e-8
