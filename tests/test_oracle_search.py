"""Pins of the oracle's SEARCH (Section 4.1, Algorithm SEARCH) and of its
column-pivoted QR, against numpy (an independent QR / SVD) and the closed
form of the prescribed-spectrum pencil (the spectral projector onto the
inside eigenvectors is Q^{-1} diag(1_inside) Q)."""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs


def test_qrcp_full_rank_matches_numpy():
    rng = np.random.default_rng(0)
    a = inputs.complex_normal(rng, (40, 15)) @ np.diag(np.logspace(0, -3, 15))
    r, jp, rd, q = oracle.qrcp(a, 1e-8)
    assert r == 15
    # Q orthonormal, A[:, jp] = Q R with R = Q^H A[:, jp] upper triangular
    assert np.abs(q.conj().T @ q - np.eye(15)).max() < 1e-13
    R = q.conj().T @ a[:, jp]
    assert np.abs(np.tril(R, -1)).max() < 1e-12
    assert np.abs(q @ R - a[:, jp]).max() < 1e-12
    np.testing.assert_allclose(np.abs(np.diag(R)), rd, rtol=1e-12)
    # greedy pivoting: |R_jj| non-increasing, and the first pivot is the
    # column of largest norm
    assert np.all(np.diff(rd) <= 1e-12 * rd[0])
    assert jp[0] == int(np.argmax(np.linalg.norm(a, axis=0)))
    # the pivoted R has the singular values of A: |det| and the largest
    s = np.linalg.svd(a, compute_uv=False)
    assert abs(np.prod(rd) / np.prod(s) - 1) < 1e-10


def test_qrcp_rank_of_low_rank_plus_noise():
    rng = np.random.default_rng(1)
    for rank in (1, 7, 12):
        a = inputs.complex_normal(rng, (50, rank)) @ inputs.complex_normal(rng, (rank, 20))
        a = a + 1e-13 * inputs.complex_normal(rng, (50, 20))
        r, _, rd, q = oracle.qrcp(a, 1e-8)
        assert r == rank, (r, rank)
        # the rank-r basis spans range(a): projecting a onto it leaves noise
        assert np.abs(a - q @ (q.conj().T @ a)).max() < 1e-10 * np.abs(a).max()


def _exact_projector(p, inside):
    Qi = np.linalg.inv(p.Q)
    return Qi[:, inside] @ p.Q[inside, :]


def test_trace_estimate_is_the_inside_count_in_mean():
    """Line 2: with the exact spectral projector, E[trace(Y^H Q Y)]/p = s and
    the variance of one column's y^H Q y is ||Q||_F^2 (complex Gaussian y)."""
    p = inputs.gapped_pencil(120, 8, 23, seed=3)
    inside = np.abs(p.lam) < 1.0
    Qp = _exact_projector(p, inside)
    s = int(inside.sum())
    rng = np.random.default_rng(4)
    P = 400
    Y = inputs.complex_normal(rng, (120, P))
    est = np.real(np.trace(Y.conj().T @ Qp @ Y)) / P
    sd = np.linalg.norm(Qp) / np.sqrt(P)
    assert abs(est - s) < 5 * sd


@pytest.mark.parametrize("p_start", [6, 30])
def test_search_finds_the_inside_count_across_a_gap(p_start):
    """23 eigenvalues inside |z| < 0.7, the rest beyond 1.5: the filtered
    block (16 trapezoid nodes on |z| = 1) has singular values ~1 for the
    inside directions and < 1e-2 relative for the rest, so with rank_tol 1e-1
    SEARCH must stop at t = 23 -- whether it starts below (p = 6: it grows by
    alpha) or above (p = 30: the first rank-revealing QR shows the
    deficiency) -- and U1 must span the inside eigenvectors (closed form
    Q^{-1} e_i)."""
    n, cap = 120, 48
    p = inputs.gapped_pencil(n, cap, 23, seed=5)
    inside = np.abs(p.lam) < 1.0
    o = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=16, center=0j, a=1.0)
    pool = inputs.complex_normal(np.random.default_rng(9), (n, 200))
    r = o.search(pool, 1.5, p_start, 1e-1)
    assert r["t"] == inside.sum() == 23
    U1 = r["U1"]
    assert np.abs(U1.conj().T @ U1 - np.eye(23)).max() < 1e-12
    X = np.linalg.inv(p.Q)[:, inside]
    Xn = X / np.linalg.norm(X, axis=0)
    resid = np.linalg.norm(Xn - U1 @ (U1.conj().T @ Xn), axis=0)
    # what remains is the filter's leak of the outside part: |rho| <= 1.5e-3
    # beyond |z| = 1.5 with 16 nodes, times the eigenvector basis' spread
    assert resid.max() < 2e-2
    # the estimate of line 2 is an estimate: within a few standard deviations
    assert abs(r["s0"] - 23) <= 3 * np.sqrt(23.0) + 1
    o.close()


def test_search_matches_brute_force_rank():
    """Brute force on a small case: SEARCH's t equals the number of singular
    values of the filtered pool block above rank_tol times the largest
    (numpy SVD), when that count is below the width the search reaches."""
    n, cap = 80, 40
    p = inputs.gapped_pencil(n, cap, 11, seed=7, r_in=0.8, r_out=1.3)
    o = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=16, center=0j, a=1.0)
    pool = inputs.complex_normal(np.random.default_rng(2), (n, 120))
    tol = 1e-1
    r = o.search(pool, 1.5, 20, tol)
    # the whole filtered first-20 block decides when t < 20
    U = o.filter(np.hstack([pool[:, :20], np.zeros((n, cap - 20))]))[:, :20]
    s = np.linalg.svd(U, compute_uv=False)
    brute = int(np.sum(s > tol * s[0]))
    assert r["t"] < 20
    # the pivoted QR's |R_jj| and the singular values agree on a clean gap
    assert r["t"] == brute
    o.close()


def test_line10_reading_scale():
    """Algorithm SEARCH, line 10, prints U = U1 after a full-rank step: the
    orthonormal basis (unit columns) then meets fresh filtered columns whose
    norms are ~sqrt(s) (the filter keeps the inside part of a random column
    whole), and line 9's rank test is relative to the largest |R_jj|.  With a
    coarse threshold (rank_tol 0.1) and a start below the inside count, the
    literal reading discards directions of U1 and stops at t = 25 for s = 41;
    keeping the block as filtered columns (the span of U1 on the scale of
    the columns that join it) finds all 41.  At the threshold the SEARCH
    workload uses (1e-4, 32 nodes) both readings give t = s."""
    n, cap, n_in = 300, 96, 41
    p = inputs.gapped_pencil(n, cap, n_in, seed=11)
    assert int(np.sum(np.abs(p.lam) < 1.0)) == n_in
    pool = inputs.complex_normal(np.random.default_rng(12), (n, 400))

    def t_of(literal, tol, p0):
        o = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=32, center=0j, a=1.0)
        o.set_search_literal(literal)
        r = o.search(pool, 1.5, p0, tol)
        o.close()
        return r["t"]

    assert t_of(False, 0.1, 8) == n_in
    assert t_of(True, 0.1, 8) == 25
    assert t_of(False, 1e-4, 8) == t_of(True, 1e-4, 8) == n_in
    # the scale mismatch itself: unit columns against filtered ones
    o = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=0, q=32, center=0j, a=1.0)
    F = o.filter(np.hstack([pool[:, :20], np.zeros((n, cap - 20))]))[:, :20]
    o.close()
    norms = np.linalg.norm(F, axis=0)
    assert np.median(norms) > 3.0 * np.sqrt(1.0) and np.median(norms) < 3.0 * np.sqrt(n_in)
