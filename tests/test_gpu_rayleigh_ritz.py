"""The Rayleigh-Ritz projection option (Algorithm FEAST, Section 3) on the
GPU against the oracle's: the same projected matrices in the first pass, the
same stop, count and eigenvalues on Hermitian / Hermitian-positive-definite
pencils (through the one-CTA QZ at m0 <= 64 and the triangularised large
solver above), and the failure of Example 3.1 (no pair is ever accepted)."""
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
        worst = max(worst, abs(x - b[j]))
        b.pop(j)
    return worst


KW = dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0, eps=1e-10)


@pytest.mark.parametrize("n,m0,seed,lam_radius,prec", [(160, 48, 0, 4.0, 0), (120, 80, 1, 2.0, 0),
                                                       (120, 80, 1, 2.0, 1)])
def test_rayleigh_ritz_hermitian_matches_oracle(n, m0, seed, lam_radius, prec):
    fg = _fg()
    p = inputs.hermitian_pencil(n, m0, seed=seed, lam_radius=lam_radius)
    inside = np.abs(p.lam) < 1.0
    g = fg.Feast(p.A, p.B, p.Y, projection=fg.FEAST_RAYLEIGH_RITZ, prec=prec, **KW)
    o = oracle.Feast(p.A, p.B, p.Y, projection=1, **KW)
    g.iterate(); o.iterate()
    # (the precision form's first subspace comes from complex64 solves, so
    # its projected matrices agree to the single-precision filter's error)
    for name in ("At", "Bt"):
        a, b = g.get(name), o.get(name)
        assert np.abs(a - b).max() < (1e-4 if prec else 1e-11) * np.abs(b).max(), name
    hg, ho = g.run(), o.run()
    rg, ro = g.eigs(), o.result()
    assert rg["flag"] == ro["flag"] == 1
    assert rg["count"] == ro["count"] == inside.sum()
    assert _match(rg["lam"], p.lam[inside]) < 1e-11
    assert _match(rg["lam"], ro["lam"]) < 1e-11
    assert np.all(rg["res"] < 1e-10)
    g.close(); o.close()


def test_rayleigh_ritz_example_3_1_accepts_nothing():
    from test_oracle_pins import load_example_3_1
    fg = _fg()
    A, B, eig, inside = load_example_3_1()
    Y = inputs.complex_normal(np.random.default_rng(0), (4, 2))
    kw = dict(contour_kind=0, rule=1, q=16, center=0j, a=1.0, eps=1e-13, max_iter=6)
    g = fg.Feast(A, B, Y, projection=fg.FEAST_RAYLEIGH_RITZ, **kw)
    hist = g.run()
    assert all(h["count"] == 0 for h in hist)
    r = g.eigs()
    assert r["flag"] == -1 and r["count"] == 0
    g.close()
    # the same pencil, oblique: 0.2 and 0.5
    g = fg.Feast(A, B, Y, projection=fg.FEAST_OBLIQUE, **kw)
    g.run()
    r = g.eigs()
    assert r["flag"] == 1 and r["count"] == 2
    assert _match(r["lam"], [v for v, _ in inside]) < 1e-13
    g.close()


def test_projection_option_validated():
    fg = _fg()
    p = inputs.hermitian_pencil(40, 8, seed=2)
    with pytest.raises(fg.FeastError) as ei:
        fg.Feast(p.A, p.B, p.Y, projection=2, **KW)
    assert ei.value.status == -1
