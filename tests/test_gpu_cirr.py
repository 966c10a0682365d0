"""Block CIRR (Section 2.1, Algorithm Block_CIRR) on the GPU against the
oracle's on the same pencil, contour and random block: the same selected
count, eigenvalues that agree to the rounding of the (full-rank) moment
block's basis, the prescribed spectrum where the quadrature is fine enough,
and the Example 3.1 failure (nothing accepted)."""
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


@pytest.mark.parametrize("prec", [0, 1])
def test_cirr_fine_quadrature_matches_oracle_and_spectrum(prec):
    fg = _fg()
    p = inputs.gapped_pencil(120, 24, 12, seed=6, r_out=2.0, lam_radius=3.0)
    inside = np.abs(p.lam) < 1.0
    Y = inputs.complex_normal(np.random.default_rng(5), (120, 4))
    kw = dict(contour_kind=0, rule=1, q=64, center=0j, a=1.0)
    g = fg.Feast(p.A, p.B, p.Y[:, :16], projection=fg.FEAST_RAYLEIGH_RITZ, prec=prec, **kw)
    info = g.cirr(Y, 4)
    r = g.eigs()
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    ro = o.cirr(Y, 4)
    assert info["flag"] == r["flag"] == -1
    assert r["count"] == ro["count"] == inside.sum() == 12
    assert _match(r["lam"], ro["lam"]) < 1e-11
    assert _match(r["lam"], p.lam[inside]) < 1e-11
    assert np.all(r["res"] < 1e-10)
    g.close(); o.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_cirr_coarse_quadrature_matches_oracle(prec):
    """q = 32 on a narrower gap: the one-shot method is accurate to ~1e-6 only,
    and both sides must land on the same approximations."""
    fg = _fg()
    p = inputs.gapped_pencil(200, 32, 20, seed=3)
    Y = inputs.complex_normal(np.random.default_rng(5), (200, 8))
    kw = dict(contour_kind=0, rule=0, q=32, center=0j, a=1.0)
    g = fg.Feast(p.A, p.B, p.Y, projection=fg.FEAST_RAYLEIGH_RITZ, prec=prec, **kw)
    g.cirr(Y, 4)
    r = g.eigs()
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    ro = o.cirr(Y, 4)
    assert r["count"] == ro["count"] == 20
    assert _match(r["lam"], ro["lam"]) < 1e-8
    np.testing.assert_allclose(np.sort(r["res"]), np.sort(ro["res"]), rtol=1e-4)
    g.close(); o.close()


def test_cirr_example_3_1_accepts_nothing():
    from test_oracle_pins import load_example_3_1
    fg = _fg()
    A, B, eig, inside = load_example_3_1()
    Y0 = inputs.complex_normal(np.random.default_rng(0), (4, 2))
    g = fg.Feast(A, B, Y0, projection=fg.FEAST_RAYLEIGH_RITZ, contour_kind=0, rule=1, q=16, center=0j, a=1.0)
    g.cirr(inputs.complex_normal(np.random.default_rng(1), (4, 1)), 2)
    r = g.eigs()
    assert r["count"] == 0 and r["flag"] == -1
    g.close()


def test_cirr_arguments_checked():
    fg = _fg()
    p = inputs.gapped_pencil(60, 8, 4, seed=1)
    Y = inputs.complex_normal(np.random.default_rng(2), (60, 4))
    g = fg.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=16, center=0j, a=1.0)   # oblique
    with pytest.raises(fg.FeastError) as ei:
        g.cirr(Y, 2)
    assert ei.value.status == -1
    g.close()
    g = fg.Feast(p.A, p.B, p.Y, projection=fg.FEAST_RAYLEIGH_RITZ, contour_kind=0, rule=0, q=16, center=0j, a=1.0)
    with pytest.raises(fg.FeastError) as ei:
        g.cirr(Y, 3)        # t = 12 > m0 = 8
    assert ei.value.status == -1
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_cirr_and_rayleigh_ritz_on_a_banded_pencil(prec):
    """The comparison methods on the banded path (12 x 12 convection-diffusion
    grid, ellipse around its lowest 5 eigenvalues): Block CIRR and the
    Rayleigh-Ritz FEAST against the oracle's on the same band storage, and
    both against the closed-form spectrum."""
    fg = _fg()
    nx = 12
    bp = inputs.convection_diffusion(nx, 12, seed=1)
    lam = inputs.convection_diffusion_spectrum(nx)
    lo, hi = lam[0] * 0.5, 0.5 * (lam[4] + lam[5])
    cen, a = 0.5 * (lo + hi), 0.5 * (hi - lo)
    kw = dict(kind=1, kl=bp.kl, ku=bp.ku, b_identity=True, contour_kind=1, rule=1, q=32,
              center=complex(cen), a=a, b=a / 4)
    Y = inputs.complex_normal(np.random.default_rng(3), (bp.n, 4))
    g = fg.Feast(bp.A_band, None, bp.Y, projection=fg.FEAST_RAYLEIGH_RITZ, prec=prec, refine_tol=1e-14, **kw)
    g.cirr(Y, 3)
    r = g.eigs()
    o = oracle.Feast(bp.A_band, None, bp.Y, **kw)
    ro = o.cirr(Y, 3)
    assert r["count"] == ro["count"] == 5
    assert _match(r["lam"], ro["lam"]) < 1e-9 * lam[4]
    assert _match(r["lam"], lam[:5]) < 1e-9 * lam[4]
    g.close(); o.close()
    # (the precision form's residual floor on this pencil is ~1e-11: eps sits
    # a decade above it, so that the stop is line 13's, not line 14's)
    eps = 1e-11 if prec == 0 else 1e-10
    g = fg.Feast(bp.A_band, None, bp.Y, projection=fg.FEAST_RAYLEIGH_RITZ, prec=prec, refine_tol=1e-14,
                 eps=eps, **kw)
    g.run()
    r = g.eigs()
    o = oracle.Feast(bp.A_band, None, bp.Y, projection=1, eps=eps, **kw)
    o.run()
    ro = o.result()
    assert r["flag"] == ro["flag"] == 1
    assert r["count"] == ro["count"] == 5
    assert _match(r["lam"], lam[:5]) < 1e-9 * lam[4]
    g.close(); o.close()
