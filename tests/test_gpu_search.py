"""SEARCH on the GPU (Section 4.1, Algorithm SEARCH) against the oracle's
SEARCH on the same pencil and the same random columns: the same bound t and
trace estimate s0, the same subspace, and GFEAST started from it finds the
inside eigenvalues (a gap around the contour makes the numerical rank
unambiguous)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec,p_start", [(0, 10), (0, 60), (1, 10)])
def test_search_then_gfeast(prec, p_start):
    fg = _fg()
    n, cap, n_in = 300, 96, 41
    p = inputs.gapped_pencil(n, cap, n_in, seed=11)
    inside = np.abs(p.lam) < 1.0
    # 32 nodes: the filter leaves < 3e-6 of the outside part, so the rank
    # at 1e-4 is unambiguous (the inside singular values stay above 1e-1
    # of the largest for this pool)
    kw = dict(contour_kind=0, rule=0, q=32, center=0j, a=1.0, eps=1e-11)
    pool = inputs.complex_normal(np.random.default_rng(12), (n, 400))
    g = fg.Feast(p.A, p.B, p.Y, prec=prec, refine_tol=1e-14, **kw)
    r = g.search(pool, 1.5, p_start, 1e-4)
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    ro = o.search(pool, 1.5, p_start, 1e-4)
    assert r["t"] == ro["t"] == n_in
    assert r["s0"] == ro["s0"]
    # the same subspace: the GPU basis lies in the oracle's span
    U1 = g.get("U1")
    Uo = ro["U1"]
    assert np.abs(U1.conj().T @ U1 - np.eye(n_in)).max() < 1e-12
    # (the two pivot orders may differ where column norms nearly tie; the
    # spans then differ by the filter's leak of the outside part, < 1e-5)
    assert np.abs(U1 - Uo @ (Uo.conj().T @ U1)).max() < 1e-4
    # GFEAST from the search's basis, width t
    g.run()
    res = g.eigs()
    assert res["flag"] == 1 and res["count"] == n_in
    assert _match(res["lam"], p.lam[inside]) < 1e-10
    g.close()
    o.close()


def test_search_reports_a_too_small_workspace():
    """With the context's m0 below the inside count the search cannot grow
    far enough: FEAST_ENOCONV, not a wrong bound."""
    fg = _fg()
    n, cap, n_in = 200, 24, 40
    p = inputs.gapped_pencil(n, cap, n_in, seed=13)
    g = fg.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=16, center=0j, a=1.0)
    pool = inputs.complex_normal(np.random.default_rng(14), (n, 300))
    with pytest.raises(fg.FeastError) as ei:
        g.search(pool, 1.5, 8, 0.1)
    assert ei.value.status == -7
    g.close()
