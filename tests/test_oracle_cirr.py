"""Pins of the oracle's Block CIRR (Section 2.1, Algorithm Block_CIRR), the
comparison method, and of its one-sided Jacobi SVD:

* the SVD against numpy (singular values, orthonormal U spanning range(a)),
  including an exactly rank-deficient block (zero singular values, zero
  columns);
* steps 1-2 against the closed form of the moment block for the
  prescribed-spectrum pencil A = P diag(lam) Q, B = P Q: (zB - A)^{-1} =
  Q^{-1} diag(1/(z - lam)) P^{-1}, so the quadrature moment block is
  Q^{-1} diag(sum_j w_j zeta_j^i / (z_j - lam)) P^{-1} Y -- its singular
  values must be the oracle's (a dropped power, a stray B or a wrong weight
  changes them);
* the whole method: with enough nodes the selected eigenvalues are the
  prescribed inside ones (Theorem 2.2 of the CIRR section: the projected
  pencil's regular part is the inside Jordan block);
* Example 3.1: the Rayleigh-Ritz pencil of the moment space is zero, so
  Block CIRR accepts nothing -- as the Rayleigh-Ritz FEAST.
"""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs
from test_oracle_pins import load_example_3_1


def test_svd_jacobi_matches_numpy():
    rng = np.random.default_rng(0)
    a = inputs.complex_normal(rng, (30, 12)) @ np.diag(np.logspace(0, -6, 12))
    u, s = oracle.svd_jacobi(a)
    ref = np.linalg.svd(a, compute_uv=False)
    assert np.abs(s - ref).max() < 1e-14 * ref[0]
    assert np.abs(u.conj().T @ u - np.eye(12)).max() < 1e-13
    assert np.abs(u @ (u.conj().T @ a) - a).max() < 1e-14 * ref[0]
    # u_i = a v_i / sigma_i: (u^H a)(u^H a)^H = diag(sigma^2)
    g = (u.conj().T @ a) @ (u.conj().T @ a).conj().T
    assert np.abs(g - np.diag(s ** 2)).max() < 1e-13 * ref[0] ** 2


def test_svd_jacobi_rank_deficient():
    rng = np.random.default_rng(1)
    a = inputs.complex_normal(rng, (20, 3)) @ inputs.complex_normal(rng, (3, 7))
    a[:, 5] = 0.0
    u, s = oracle.svd_jacobi(a)
    ref = np.linalg.svd(a, compute_uv=False)
    assert np.abs(s[:3] - ref[:3]).max() < 1e-13 * ref[0]
    assert np.all(s[3:] < 1e-13 * ref[0])
    assert np.abs(u[:, :3].conj().T @ u[:, :3] - np.eye(3)).max() < 1e-12
    assert np.all(np.linalg.norm(u[:, 6:], axis=0) <= 1.0 + 1e-12)


@pytest.mark.parametrize("q,rule", [(32, 0), (32, 1), (64, 1)])
def test_moment_block_closed_form(q, rule):
    p = inputs.gapped_pencil(120, 24, 12, seed=6, r_out=2.0, lam_radius=3.0)
    Y = inputs.complex_normal(np.random.default_rng(5), (120, 4))
    o = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=rule, q=q, center=0j, a=1.0)
    r = o.cirr(Y, 4)
    z, w = o.get("z"), o.get("w")
    PY = np.linalg.solve(p.P, Y)
    Qi = np.linalg.inv(p.Q)
    blocks = []
    for i in range(4):
        f = np.array([np.sum(w * z ** i / (z - l)) for l in p.lam])
        blocks.append(Qi @ (f[:, None] * PY))
    sc = np.linalg.svd(np.hstack(blocks), compute_uv=False)
    assert np.abs(r["sigma"] - sc).max() < 1e-13 * sc[0]
    o.close()


def test_block_cirr_finds_the_inside_eigenvalues():
    p = inputs.gapped_pencil(120, 24, 12, seed=6, r_out=2.0, lam_radius=3.0)
    inside = np.abs(p.lam) < 1.0
    Y = inputs.complex_normal(np.random.default_rng(5), (120, 4))
    o = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=1, q=64, center=0j, a=1.0)
    r = o.cirr(Y, 4)
    assert r["count"] == inside.sum() == 12
    worst = max(min(abs(l - p.lam[inside])) for l in r["lam"])
    assert worst < 1e-12
    for i in range(r["count"]):
        x = r["X"][:, i]
        res = np.linalg.norm(p.A @ x - r["lam"][i] * (p.B @ x))
        assert res / (np.linalg.norm(p.A @ x) + np.linalg.norm(p.B @ x)) < 1e-11
    o.close()


def test_block_cirr_fails_on_example_3_1():
    A, B, eig, inside = load_example_3_1()
    o = oracle.Feast(A, B, inputs.complex_normal(np.random.default_rng(0), (4, 2)), contour_kind=0,
                     rule=1, q=16, center=0j, a=1.0)
    for h, g in ((2, 1), (1, 2)):
        r = o.cirr(inputs.complex_normal(np.random.default_rng(1), (4, h)), g)
        assert r["count"] == 0
        # the moment block itself has rank 2 (it spans the inside eigenvectors)
        assert r["sigma"][1] > 1e-2 * r["sigma"][0]
    o.close()
