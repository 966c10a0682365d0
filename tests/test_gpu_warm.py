"""The warm-started projected eigensolve (line 6 from the second pass on,
m0 >= 96): the Ritz pairs of each pass are ordered by their expected
residual after filtering, r_i / |rho(lambda_i)|, line 16
filters the Ritz vectors, and the next projected matrix is solved as a
block-triangular perturbation (QR of the unconverged trailing block only, one
Newton step for the rest).  Cold passes whose pairs are needed only to 1e-3 of the accuracy reached so
far take the FP32 QR's Schur form polished by the same Newton step.  The
run must end where the cold solve ends: the prescribed eigenvalues, the
oracle's count, and -- pass by pass -- Ritz values equal to a library
eigensolver's on the GPU's own projected pencil."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fg():
    import paper_1404_1768_gb300 as fg
    return fg


def _match(a, b):
    b = list(b)
    worst = 0.0
    for x in a:
        j = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[j]) / max(abs(b[j]), 1e-300))
        b.pop(j)
    return worst


@pytest.mark.parametrize("prec", [0, 1])
def test_warm_solve_end_to_end(prec):
    fg = _fg()
    n, m0 = 640, 208
    p = inputs.prescribed_pencil(n, m0, seed=21)
    kw = dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0, eps=1e-11)
    g = fg.Feast(p.A, p.B, p.Y, prec=prec, refine_tol=1e-14, **kw)
    warm_seen = fp32_seen = 0
    while True:
        it = g.iterate()
        if it["flag"] != 2:
            break
        if it["qz_cold_fp32"] == 1:
            # a cold pass whose pairs were needed to 1e-3 eta: the FP32 QR's
            # Schur form polished by the Newton step
            fp32_seen += 1
            assert it["qz_rows"] == m0 and it["qz_warm_resid"] <= 1e-6
        if it["qz_warm"] or it["qz_cold_fp32"] == 1:
            warm_seen += it["qz_warm"]
            assert it["qz_rows"] < m0 or it["qz_cold_fp32"] == 1
            assert it["qz_warm_resid"] <= max(1e-13, 1e-3 * 1e-3)
            # every Ritz value of this pass against a library eigensolver on
            # the projected pencil the GPU formed
            At, Bt = g.get("At"), g.get("Bt")
            ref = sl.eig(At, Bt, right=False)
            lam = g.get("lam")
            scale = np.abs(ref).max()
            tol = (1e-9 + 100 * it["qz_warm_resid"]) * scale
            pool = list(ref)
            for x in lam:
                j = int(np.argmin([abs(x - y) for y in pool]))
                assert abs(x - pool[j]) <= tol, (x, pool[j])
                pool.pop(j)
    assert warm_seen >= 1 and fp32_seen >= 1
    r = g.eigs()
    ref = p.lam[np.abs(p.lam) < 1.0]
    assert r["flag"] == 1 and r["count"] == len(ref)
    assert _match(r["lam"], ref) < 1e-9
    assert np.all(r["res"] < 1e-11)
    # both forms against the FP64 oracle's run on the same pencil and start
    # block: the count exactly, the eigenvalues to 1e-10 (FP64) or 1e-8
    # (precision form) relative, the stop within one pass
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    o.run()
    ro = o.result()
    o.close()
    assert ro["flag"] == 1 and ro["count"] == r["count"]
    assert _match(r["lam"], ro["lam"]) < (1e-10 if prec == 0 else 1e-8)
    assert abs(ro["k"] - it["k"]) <= 1
    g.close()


def test_ritz_pairs_ordered_by_expected_residual():
    """From m0 = 96 on, a pass leaves its pairs in increasing r_i / |rho(lambda_i)|
    (r_i of eq. 5.1, rho the filter of eq. 4.1 with the GPU's own nodes and
    weights): the order in which line 16 filters them."""
    fg = _fg()
    p = inputs.prescribed_pencil(400, 128, seed=3)
    g = fg.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=16, center=0j, a=1.0, eps=1e-11)
    for _ in range(2):
        g.iterate()
        z, w, lam, res = g.get("z"), g.get("w"), g.get("lam"), g.get("res")
        rho = np.abs([(w / (z - x)).sum() for x in lam])
        key = res / rho
        assert np.all(np.diff(key) >= -1e-12 * np.abs(key).max())
        # the Ritz vectors were permuted with their values: A x = lambda B x
        # to the reported residual
        X = g.get("X")
        for i in (0, len(lam) // 2, len(lam) - 1):
            x = X[:, i]
            r = np.linalg.norm(p.A @ x - lam[i] * (p.B @ x)) / (np.linalg.norm(p.A @ x) + np.linalg.norm(p.B @ x))
            assert abs(r - res[i]) <= 1e-6 * max(res[i], 1e-12) + 1e-14
    g.close()
