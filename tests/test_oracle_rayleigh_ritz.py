"""Pins of the oracle's Rayleigh-Ritz option (the projection of Algorithm
FEAST, Section 3, kept as a comparison to GFEAST's oblique projection):

* on a Hermitian / Hermitian-positive-definite pencil the Rayleigh-Ritz
  matrices are Hermitian with B~ positive definite (a property of the
  projection with test space = search space; the oblique B~ is the
  triangular R2 instead), and the run finds the prescribed real eigenvalues;
* on Example 3.1 the Rayleigh-Ritz matrices vanish (to the filter's leak,
  which shrinks every pass) and no eigenpair is ever accepted, while the
  oblique projection recovers 0.2 and 0.5 -- the failure the paper shows;
* on a general (non-Hermitian) pencil with a clean gap both projections
  reach the prescribed eigenvalues (the projection is exact on an invariant
  subspace as long as U1^H B U1 is nonsingular).
"""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs
from test_oracle_pins import load_example_3_1


def _match(a, b):
    b = list(b)
    worst = 0.0
    for x in a:
        j = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[j]))
        b.pop(j)
    return worst


KW = dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0)


def test_rayleigh_ritz_hermitian_pencil():
    p = inputs.hermitian_pencil(120, 80, seed=1)
    inside = np.abs(p.lam) < 1.0
    # the generator: A Hermitian, B Hermitian positive definite
    assert np.array_equal(p.A, p.A.conj().T) and np.array_equal(p.B, p.B.conj().T)
    assert np.linalg.eigvalsh(p.B).min() > 0
    o = oracle.Feast(p.A, p.B, p.Y, eps=1e-10, projection=1, **KW)
    o.iterate(); o.iterate()
    At, Bt = o.get("At"), o.get("Bt")
    assert np.abs(At - At.conj().T).max() < 1e-13 * np.abs(At).max()
    assert np.abs(Bt - Bt.conj().T).max() < 1e-13 * np.abs(Bt).max()
    assert np.linalg.eigvalsh(0.5 * (Bt + Bt.conj().T)).min() > 0.1
    o.run()
    r = o.result()
    assert r["flag"] == 1 and r["count"] == inside.sum()
    assert _match(r["lam"], p.lam[inside]) < 1e-12
    assert np.abs(r["lam"].imag).max() < 1e-12
    o.close()
    # the oblique projection of the same pencil: B~ = U2^H B U1 = R2
    g = oracle.Feast(p.A, p.B, p.Y, eps=1e-10, projection=0, **KW)
    R2 = g.get("R2")          # line 2's factor, projected with in the first pass
    g.iterate()
    Bt = g.get("Bt")
    assert np.abs(np.tril(Bt, -1)).max() < 1e-13 * np.abs(Bt).max()
    np.testing.assert_allclose(Bt, R2, atol=1e-13 * np.abs(Bt).max())
    g.close()


def test_rayleigh_ritz_fails_on_example_3_1():
    A, B, eig, inside = load_example_3_1()
    Y = inputs.complex_normal(np.random.default_rng(0), (4, 2))
    kw = dict(contour_kind=0, rule=1, q=16, center=0j, a=1.0, eps=1e-13, max_iter=6)
    o = oracle.Feast(A, B, Y, projection=1, **kw)
    sizes = []
    while True:
        it = o.iterate()
        sizes.append(max(np.abs(o.get("At")).max(), np.abs(o.get("Bt")).max()))
        assert it["count"] == 0
        if it["flag"] != 2:
            break
    r = o.result()
    assert r["flag"] == -1 and r["count"] == 0
    # the projected pair is the filter's leak only, shrinking every pass
    assert sizes[0] < 1e-5 and all(b < 1e-4 * a for a, b in zip(sizes, sizes[1:]))
    o.close()
    g = oracle.Feast(A, B, Y, projection=0, **kw)
    g.run()
    r = g.result()
    assert r["flag"] == 1 and r["count"] == 2
    assert _match(r["lam"], [v for v, _ in inside]) < 1e-13
    g.close()


def test_rayleigh_ritz_general_pencil():
    p = inputs.gapped_pencil(100, 40, 20, seed=4)
    inside = np.abs(p.lam) < 1.0
    for proj in (0, 1):
        o = oracle.Feast(p.A, p.B, p.Y, eps=1e-11, projection=proj, **KW)
        o.run()
        r = o.result()
        assert r["flag"] == 1 and r["count"] == 20
        assert _match(r["lam"], p.lam[inside]) < 1e-11
        o.close()


def test_projection_argument_checked():
    p = inputs.hermitian_pencil(20, 6, seed=2)
    with pytest.raises(ValueError):
        oracle.Feast(p.A, p.B, p.Y, projection=2, **KW)
