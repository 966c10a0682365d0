"""Banded pencils on the GPU: band LU (unblocked-convention multipliers in
LAPACK band storage) and band solves against the oracle's band LU, and the
whole method on the convection-diffusion operator against its closed-form
spectrum, up to the full 128 x 128 grid."""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fg():
    import paper_1404_1768_gb300 as fg
    return fg


def _match_rel(a, b):
    b = list(b)
    worst = 0.0
    for x in sorted(a, key=lambda v: (v.real, v.imag)):
        j = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[j]) / abs(b[j]))
        b.pop(j)
    return worst


def _random_band(n, kl, ku, seed):
    rng = np.random.default_rng(seed)
    ab = np.zeros((kl + ku + 1, n), complex, order="F")
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[ku + i - j, j] = complex(rng.standard_normal(), rng.standard_normal())
    return ab


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,kl,ku,m0,q", [(100, 10, 10, 8, 8), (77, 3, 5, 13, 5), (300, 40, 33, 9, 6)])
def test_band_filter_matches_oracle(prec, n, kl, ku, m0, q):
    """U = sum_j w_j (z_j B - A)^{-1} B V with band A and band B (kl, ku not
    multiples of the 32-wide panels, n with ragged tails)."""
    fg = _fg()
    A = _random_band(n, kl, ku, n)
    B = _random_band(n, kl, ku, n + 1)
    B[ku, :] += 6.0                      # keep B well conditioned
    Y = inputs.complex_normal(np.random.default_rng(3), (n, m0))
    kw = dict(contour_kind=1, rule=1, q=q, center=0.5 + 0.2j, a=1.5, b=0.8, kind=1, kl=kl, ku=ku)
    g = fg.Feast(A, B, Y, prec=prec, refine_tol=1e-14, max_refine=6, **kw)
    o = oracle.Feast(A, B, Y, **kw)
    V = inputs.complex_normal(np.random.default_rng(4), (n, m0))
    Ug, Uo = g.filter(V), o.filter(V)
    err = np.abs(Ug - Uo).max() / np.abs(Uo).max()
    assert err < (1e-11 if prec == 0 else 1e-10), err
    g.close(); o.close()


def _fast_band(n, kl, ku, seed):
    """Like _random_band, a column at a time (for the wide bands)."""
    rng = np.random.default_rng(seed)
    ab = np.zeros((kl + ku + 1, n), complex, order="F")
    for j in range(n):
        i0, i1 = max(0, j - ku), min(n, j + kl + 1)
        ab[ku + i0 - j:ku + i1 - j, j] = rng.standard_normal(i1 - i0) + 1j * rng.standard_normal(i1 - i0)
    return ab


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,kl,ku,q,b_identity", [(1900, 900, 900, 4, False), (2000, 1500, 1400, 3, True),
                                                  (3064, 3000, 2800, 2, True)])
def test_wide_band_filter_matches_oracle(prec, n, kl, ku, q, b_identity):
    """Bands too wide for the full solve staging (8 right-hand sides x 16
    factor columns per CTA): the solves stage fewer of each, down to one
    right-hand side and one factor column per CTA for kl + ku = 5800 in FP64.
    13 right-hand sides leave a ragged last chunk at every staging width."""
    fg = _fg()
    m0 = 13
    A = _fast_band(n, kl, ku, 11 * n)
    A[ku, :] += 60.0
    B = None
    if not b_identity:
        B = _fast_band(n, kl, ku, 11 * n + 1)
        B[ku, :] += 90.0
    Y = inputs.complex_normal(np.random.default_rng(5), (n, m0))
    kw = dict(contour_kind=1, rule=1, q=q, center=0.5 + 0.2j, a=1.5, b=0.8, kind=1, kl=kl, ku=ku,
              b_identity=b_identity)
    g = fg.Feast(A, B, Y, prec=prec, refine_tol=1e-14, max_refine=8, **kw)
    o = oracle.Feast(A, B, Y, **kw)
    V = inputs.complex_normal(np.random.default_rng(6), (n, m0))
    Ug, Uo = g.filter(V), o.filter(V)
    err = np.abs(Ug - Uo).max() / np.abs(Uo).max()
    assert err < (1e-11 if prec == 0 else 1e-10), err
    g.close(); o.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,kl,ku,m0,q", [(100, 10, 10, 8, 8), (333, 37, 21, 11, 6)])
def test_band_filter_identity_b_matches_oracle(prec, n, kl, ku, m0, q):
    """B = I: the precision form's refinement residual takes its band product
    A X in double-single arithmetic; the filtered block still agrees with the
    oracle's to 1e-10."""
    fg = _fg()
    A = _random_band(n, kl, ku, 5 * n)
    A[ku, :] *= 4.0
    Y = inputs.complex_normal(np.random.default_rng(7), (n, m0))
    kw = dict(contour_kind=1, rule=1, q=q, center=0.3 - 0.4j, a=2.5, b=1.2, kind=1, kl=kl, ku=ku,
              b_identity=True)
    g = fg.Feast(A, None, Y, prec=prec, refine_tol=1e-14, max_refine=8, **kw)
    o = oracle.Feast(A, None, Y, **kw)
    V = inputs.complex_normal(np.random.default_rng(8), (n, m0))
    Ug, Uo = g.filter(V), o.filter(V)
    err = np.abs(Ug - Uo).max() / np.abs(Uo).max()
    assert err < (1e-11 if prec == 0 else 1e-10), err
    g.close(); o.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_band_gfeast_small_grid_closed_form(prec):
    """12 x 12 grid, ellipse around the lowest 5 eigenvalues: exact count,
    closed-form eigenvalues, and agreement with the oracle's run."""
    fg = _fg()
    nx = 12
    bp = inputs.convection_diffusion(nx, 12, seed=1)
    lam = inputs.convection_diffusion_spectrum(nx)
    lo, hi = lam[0] * 0.5, 0.5 * (lam[4] + lam[5])
    cen, a = 0.5 * (lo + hi), 0.5 * (hi - lo)
    kw = dict(kind=1, kl=bp.kl, ku=bp.ku, b_identity=True, contour_kind=1, rule=1, q=16,
              center=complex(cen), a=a, b=a / 4, eps=1e-11)
    g = fg.Feast(bp.A_band, None, bp.Y, prec=prec, refine_tol=1e-14, **kw)
    g.run()
    r = g.eigs()
    o = oracle.Feast(bp.A_band, None, bp.Y, **kw)
    o.run()
    ro = o.result()
    assert r["flag"] == 1 and r["count"] == ro["count"] == 5
    assert _match_rel(r["lam"], lam[:5]) < 1e-9
    assert _match_rel(r["lam"], ro["lam"]) < 1e-9
    g.close(); o.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_band_full_grid_n16384(prec):
    """The 128 x 128 workload (n = 16384, half-bandwidth 128, 16 nodes,
    m0 = 64): the 41 eigenvalues inside the ellipse, each within 1e-8
    relative of the closed form, residuals of eq. 5.1 below 1e-10."""
    fg = _fg()
    c = inputs.WORKLOADS["band_n16384_m64_q16"]
    bp = inputs.convection_diffusion(c["nx"], c["m0"], seed=c["seed"], beta=c["beta"])
    lam = inputs.convection_diffusion_spectrum(c["nx"], c["beta"])
    inside = lam[((lam - c["center"].real) / c["a"]) ** 2 < 1.0]
    assert len(inside) == 41
    g = fg.Feast(bp.A_band, None, bp.Y, kind=1, kl=bp.kl, ku=bp.ku, b_identity=True,
                 contour_kind=1, rule=c["rule"], q=c["q"], center=c["center"], a=c["a"], b=c["b"],
                 eps=c["eps"], prec=prec, refine_tol=1e-13, max_iter=30)
    g.run()
    r = g.eigs(want_vectors=False)
    assert r["flag"] == 1 and r["count"] == 41
    assert _match_rel(r["lam"], inside) < 1e-8
    assert np.all(r["res"] < 1e-10)
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_band_non_regular_pencil_reports_singular(prec):
    """Tridiagonal A and B sharing a zero row: det(z B - A) = 0 for every
    z, so every shifted band matrix has an exact zero pivot -> FEAST_ESINGULAR
    at set-up (the complex64 band LU of the precision form included)."""
    fg = _fg()
    n, kl, ku = 70, 1, 1
    A = _random_band(n, kl, ku, 3)
    B = _random_band(n, kl, ku, 4)
    B[ku, :] += 5.0
    for M in (A, B):
        for j in range(max(0, 37 - ku), min(n, 37 + kl + 1)):
            M[ku + 37 - j, j] = 0.0          # row 37 of both is zero
    Y = inputs.complex_normal(np.random.default_rng(2), (n, 4))
    with pytest.raises(fg.FeastError) as ei:
        fg.Feast(A, B, Y, prec=prec, contour_kind=0, rule=1, q=8, center=0j, a=1.0, kind=1, kl=kl, ku=ku)
    assert ei.value.status == -4


def test_band_lu_complex64_without_refinement():
    """The complex64 band LU on its own (no refinement sweeps: every digit of
    the filtered block comes from the factors and one solve each): n = 3000
    with kl = 120, ku = 90 (94 panels of the one-launch factorisation, a
    ragged last one), a diagonally dominant band, so the complex64 solve is
    good to ~1e-6 of the oracle's FP64 one; a factor entry off by a race or a
    misplaced interchange would show as O(1)."""
    fg = _fg()
    n, kl, ku, m0, q = 3000, 120, 90, 12, 4
    A = _fast_band(n, kl, ku, 21)
    A[ku, :] += 4.0 * (kl + ku)
    B = _fast_band(n, kl, ku, 22)
    B[ku, :] += 4.0 * (kl + ku)
    Y = inputs.complex_normal(np.random.default_rng(9), (n, m0))
    kw = dict(contour_kind=1, rule=1, q=q, center=0.5 + 0.2j, a=1.5, b=0.8, kind=1, kl=kl, ku=ku)
    g = fg.Feast(A, B, Y, prec=1, refine_tol=1e-14, max_refine=0, **kw)
    o = oracle.Feast(A, B, Y, **kw)
    V = inputs.complex_normal(np.random.default_rng(10), (n, m0))
    Ug, Uo = g.filter(V), o.filter(V)
    err = np.abs(Ug - Uo).max() / np.abs(Uo).max()
    assert err < 1e-4, err
    g.close(); o.close()
