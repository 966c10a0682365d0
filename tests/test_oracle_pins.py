"""Pins of the FP64 oracle against values fixed by the paper and by
mathematics: the worked Example 3.1, closed forms of the quadrature filter,
textbook special cases, library routines on small inputs, brute force, and
the exactness theorem (Theorem 3.2).  No expected value here comes from the
GPU path."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1404_1768_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_example_3_1():
    A, B, eig, inside = [], [], [], []
    with open(os.path.join(GOLDEN, "example_3_1.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, *vals = line.split()
            if tag == "A":
                A.append([float(v) for v in vals])
            elif tag == "B":
                B.append([float(v) for v in vals])
            elif tag == "EIG":
                eig = [float(v) for v in vals]
            elif tag == "INSIDE":
                inside.append((float(vals[0]), int(vals[1])))
    return (np.asfortranarray(np.array(A, complex)), np.asfortranarray(np.array(B, complex)),
            eig, inside)


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("q", [1, 2, 3, 8, 16, 32])
def test_gauss_legendre_matches_library_and_is_exact(q):
    t, w = oracle.gauss_legendre(q)
    tl, wl = np.polynomial.legendre.leggauss(q)
    np.testing.assert_allclose(t, tl, atol=1e-14)
    np.testing.assert_allclose(w, wl, atol=1e-14)
    for k in range(2 * q):  # exact for polynomials of degree <= 2q - 1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * t**k) - exact) < 1e-13


@pytest.mark.parametrize("q", [8, 16, 32])
def test_trapezoid_filter_closed_form(q):
    """For offset trapezoid nodes the scalar filter sum_j w_j / (z_j - lam)
    is exactly 1 / (1 + ((lam - gamma)/rho)^q) (the q nodes are the q-th
    roots of -1 on the circle)."""
    gamma, rho = 0.3 - 0.2j, 1.7
    z, w = oracle.contour(0, 0, q, gamma, rho)
    rng = np.random.default_rng(1)
    lam = gamma + rho * 2.0 * (rng.random(50) - 0.5 + 1j * (rng.random(50) - 0.5))
    f = np.array([np.sum(w / (z - l)) for l in lam])
    mu = (lam - gamma) / rho
    np.testing.assert_allclose(f, 1.0 / (1.0 + mu**q), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("rule", [0, 1])
def test_contour_moments(rule):
    """(1/2 pi i) closed-integral of dz = 0 and of dz/(z - gamma) = 1; the
    residue of 1/(z - a) is 1 for a inside and 0 for a outside."""
    gamma, rho, q = 1.0 + 1.0j, 0.5, 32
    z, w = oracle.contour(0, rule, q, gamma, rho)
    assert abs(np.sum(w)) < 1e-14
    assert abs(np.sum(w / (z - gamma)) - 1.0) < 1e-14
    assert abs(np.sum(w / (z - (gamma + 0.1))) - 1.0) < 1e-6
    assert abs(np.sum(w / (z - (gamma + 2.0)))) < 1e-6


def test_gauss_legendre_circle_is_eq_4_1():
    """Eq. 4.1: theta_j = (1 + t_j) pi, z_j = gamma + rho e^{i theta_j},
    w_j = omega_j (z_j - gamma) / 2."""
    gamma, rho, q = -0.5 + 0.25j, 2.0, 16
    t, om = np.polynomial.legendre.leggauss(q)
    theta = (1.0 + t) * np.pi
    zz = gamma + rho * np.exp(1j * theta)
    z, w = oracle.contour(0, 1, q, gamma, rho)
    np.testing.assert_allclose(z, zz, atol=1e-14)
    np.testing.assert_allclose(w, 0.5 * om * (zz - gamma), atol=1e-14)


def test_ellipse_reduces_to_circle_and_integrates():
    gamma, q = 2.0 - 1.0j, 16
    zc, wc = oracle.contour(0, 1, q, gamma, 1.5)
    ze, we = oracle.contour(1, 1, q, gamma, 1.5, 1.5)
    np.testing.assert_allclose(ze, zc, atol=1e-14)
    np.testing.assert_allclose(we, wc, atol=1e-14)
    z, w = oracle.contour(1, 1, 64, gamma, 3.0, 0.75)
    assert abs(np.sum(w / (z - (gamma + 1.0))) - 1.0) < 1e-4   # inside (thin ellipse: slower GL convergence)
    assert abs(np.sum(w / (z - (gamma + 6.0)))) < 1e-4         # outside
    assert abs(np.sum(w)) < 1e-13


def test_inside_is_strict():
    assert oracle.inside(0, 0j, 1.0, 1.0, 0.999 + 0j)
    assert not oracle.inside(0, 0j, 1.0, 1.0, 1.0 + 0j)
    assert oracle.inside(1, 1.0 + 0j, 2.0, 0.5, 2.9 + 0j)
    assert not oracle.inside(1, 1.0 + 0j, 2.0, 0.5, 1.0 + 0.6j)


# ---------------------------------------------------------------- LU / solve
@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
def test_lu_matches_scipy_and_reconstructs(n):
    rng = np.random.default_rng(n)
    A = inputs.complex_normal(rng, (n, n))
    f, piv, info = oracle.lu(A)
    assert info == 0
    # partial pivoting by modulus: every multiplier has modulus <= 1
    assert np.all(np.abs(np.tril(f, -1)) <= 1.0 + 1e-15)
    L = np.tril(f, -1) + np.eye(n)
    U = np.triu(f)
    PA = A.copy()
    for k in range(n):
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    np.testing.assert_allclose(L @ U, PA, atol=1e-12 * n)


def test_solve_triangular_special_case_is_exact():
    """An upper-triangular matrix with power-of-two entries and integer
    right-hand side: no pivoting, and the substitution is exact."""
    n = 12
    U = np.triu(np.full((n, n), 0.5 + 0.25j), 1) + np.diag(np.full(n, 2.0 + 0j))
    x = np.arange(1, n + 1, dtype=complex) * (1 - 1j)
    b = U @ x
    f, piv, info = oracle.lu(U)
    assert info == 0 and np.all(piv == np.arange(n))
    y = oracle.lu_solve(f, piv, b)[:, 0]
    np.testing.assert_array_equal(y, x)


def test_solve_backward_error():
    n, m = 80, 5
    rng = np.random.default_rng(5)
    A = inputs.complex_normal(rng, (n, n))
    b = inputs.complex_normal(rng, (n, m))
    f, piv, _ = oracle.lu(A)
    x = oracle.lu_solve(f, piv, b)
    be = np.linalg.norm(A @ x - b) / (np.linalg.norm(A) * np.linalg.norm(x))
    assert be < 10 * n * 2.2e-16
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_singular_pivot_reported():
    A = np.zeros((3, 3), complex)
    A[0, 0] = 1
    A[1, 2] = 1
    _, _, info = oracle.lu(A)
    assert info == 2


@pytest.mark.parametrize("n,kl,ku", [(1, 0, 0), (9, 1, 2), (30, 4, 3), (64, 8, 8)])
def test_band_lu_solves_like_dense(n, kl, ku):
    rng = np.random.default_rng(n + kl)
    A = np.zeros((n, n), complex)
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            A[i, j] = complex(rng.standard_normal(), rng.standard_normal())
    ab = np.zeros((kl + ku + 1, n), complex, order="F")
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[ku + i - j, j] = A[i, j]
    b = inputs.complex_normal(rng, (n, 3))
    f, piv, info = oracle.band_lu(ab, n, kl, ku)
    assert info == 0
    x = oracle.band_solve(f, piv, n, kl, ku, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-11)
    x2 = sla.solve_banded((kl, ku), ab, b)
    np.testing.assert_allclose(x, x2, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(oracle.band_matmul(ab, n, kl, ku, b), A @ b, atol=1e-12)


# ---------------------------------------------------------------- QR, GEMM
@pytest.mark.parametrize("m,k", [(1, 1), (5, 3), (64, 64), (200, 17)])
def test_qr_orthonormal_and_unique(m, k):
    rng = np.random.default_rng(m * k)
    A = inputs.complex_normal(rng, (m, k))
    Q, R = oracle.qr(A)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0)
    d = np.diag(R)
    assert np.all(np.abs(d.imag) < 1e-14) and np.all(d.real >= 0)
    Ql, Rl = np.linalg.qr(A)
    ph = np.diag(Rl) / np.abs(np.diag(Rl))
    np.testing.assert_allclose(Q, Ql * ph[None, :], atol=1e-12)


def test_gemm_matches_library():
    rng = np.random.default_rng(3)
    a = inputs.complex_normal(rng, (17, 9))
    b = inputs.complex_normal(rng, (17, 5))
    np.testing.assert_allclose(oracle.gemm(a, b, conj_a=True), a.conj().T @ b, atol=1e-13)
    c = inputs.complex_normal(rng, (9, 5))
    np.testing.assert_allclose(oracle.gemm(a, c), a @ c, atol=1e-13)


# ---------------------------------------------------------------- QZ
def _match(a, b):
    """max |a_i - b_pi(i)| over a greedy matching of two multisets."""
    b = list(b)
    worst = 0.0
    for x in sorted(a, key=lambda v: (v.real, v.imag)):
        j = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[j]))
        b.pop(j)
    return worst


def test_qz_example_3_1_projected_pencil():
    """Example 3.1: with U1 = [e1, e2] and the test basis U2 = B U1 = [e4, e3],
    the oblique projection gives A~ = diag(0.2, 0.5), B~ = I, whose
    eigenvalues are the wanted 0.2 and 0.5; the Rayleigh-Ritz pair
    (U1^H A U1, U1^H B U1) is zero."""
    A, B, eig, inside = load_example_3_1()
    U1 = np.eye(4, dtype=complex)[:, :2]
    U2 = B @ U1
    At = oracle.gemm(U2, oracle.gemm(A, U1), conj_a=True)
    Bt = oracle.gemm(U2, oracle.gemm(B, U1), conj_a=True)
    np.testing.assert_allclose(At, np.diag([0.2, 0.5]), atol=0)
    np.testing.assert_allclose(Bt, np.eye(2), atol=0)
    assert np.all(U1.conj().T @ A @ U1 == 0) and np.all(U1.conj().T @ B @ U1 == 0)
    al, be, V = oracle.ggev(At, Bt)
    assert _match(al / be, [v for v, _ in inside]) < 1e-15
    al, be, V = oracle.ggev(A, B)
    assert _match(al / be, eig) < 1e-14


@pytest.mark.parametrize("m", [1, 2, 5, 16, 40, 64])
def test_qz_brute_force_vs_library(m):
    rng = np.random.default_rng(100 + m)
    A = inputs.complex_normal(rng, (m, m))
    B = inputs.complex_normal(rng, (m, m))
    al, be, V = oracle.ggev(A, B)
    lam = al / be
    ref = sla.eigvals(A, B)
    assert _match(lam, ref) < 1e-9 * max(1.0, np.max(np.abs(ref)))
    for i in range(m):  # beta A v = alpha B v, unit v
        r = be[i] * A @ V[:, i] - al[i] * B @ V[:, i]
        assert np.linalg.norm(r) < 1e-12 * (abs(be[i]) * np.linalg.norm(A) + abs(al[i]) * np.linalg.norm(B))
        assert abs(np.linalg.norm(V[:, i]) - 1.0) < 1e-13


def test_qz_triangular_pencil_diagonal_ratios():
    m = 10
    rng = np.random.default_rng(7)
    A = np.triu(inputs.complex_normal(rng, (m, m)))
    B = np.triu(inputs.complex_normal(rng, (m, m))) + 2 * np.eye(m)
    al, be, _ = oracle.ggev(A, B)
    assert _match(al / be, np.diag(A) / np.diag(B)) < 1e-12


def test_qz_prescribed_spectrum_full_pencil():
    """Brute force on the full P diag(lam) Q pencil at n = 64: QZ returns
    exactly the prescribed eigenvalues."""
    p = inputs.prescribed_pencil(64, 8, seed=11)
    al, be, V = oracle.ggev(p.A, p.B)
    assert _match(al / be, p.lam) < 1e-11


# ---------------------------------------------------------------- filter
def test_filter_equals_closed_form_on_prescribed_pencil():
    """For A = P diag(lam) Q, B = P Q:  (z B - A)^{-1} B = Q^{-1} (z - lam)^{-1} Q,
    so the trapezoid quadrature gives U = Q^{-1} diag(f(lam)) Q Y with
    f(lam) = 1 / (1 + ((lam - gamma)/rho)^q)."""
    n, m0, q = 48, 6, 16
    rng = np.random.default_rng(4)
    gp = inputs.complex_normal(rng, (n, n)); gq = inputs.complex_normal(rng, (n, n))
    P = np.eye(n) + 0.1 * gp / math.sqrt(n); Qm = np.eye(n) + 0.1 * gq / math.sqrt(n)
    lam = 2.0 * np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
    A = np.asfortranarray((P * lam) @ Qm); B = np.asfortranarray(P @ Qm)
    Y = inputs.complex_normal(rng, (n, m0))
    gamma, rho = 0.1 + 0.05j, 1.0
    fe = oracle.Feast(A, B, Y, contour_kind=0, rule=0, q=q, center=gamma, a=rho)
    V = inputs.complex_normal(rng, (n, m0))
    U = fe.filter(V)
    f = 1.0 / (1.0 + ((lam - gamma) / rho) ** q)
    Uref = np.linalg.solve(Qm, f[:, None] * (Qm @ V))
    np.testing.assert_allclose(U, Uref, atol=1e-12 * np.abs(Uref).max())
    # the trace of the filter: Y^H U has expectation m0 * sum f (eq. 4.1 of Section 4.1)
    fe.close()


# ---------------------------------------------------------------- Theorem 3.2
def test_exact_subspace_gives_exact_eigenvalues():
    """Theorem 3.2(a): if span(U1) is the exact invariant subspace K of the
    eigenvalues inside, the projected pencil (U2^H A U1, U2^H B U1) with
    U2 = orth(B U1) has exactly those eigenvalues; with t > s extra columns
    the wanted ones are still among the Ritz values with tiny residual."""
    n, m0 = 60, 20
    p = inputs.prescribed_pencil(n, m0, seed=3, radius=1.0)
    ins = np.abs(p.lam) < 1.0
    s = int(ins.sum())
    rng = np.random.default_rng(9)
    # eigenvectors x_i = Q^{-1} e_i; B x_i = P e_i.  Recover Q^{-1} from the
    # pencil: B^{-1} A = Q^{-1} diag(lam) Q.
    w, X = np.linalg.eig(np.linalg.solve(p.B, p.A))
    Xin = X[:, np.abs(w) < 1.0]
    assert Xin.shape[1] == s
    extra = inputs.complex_normal(rng, (n, m0 - s))
    U1 = np.linalg.qr(np.hstack([Xin, extra]))[0]
    fe = oracle.Feast(p.A, p.B, p.Y, q=16, center=0j, a=1.0)
    fe.set_U1(U1)
    fe.iterate()
    lam_r = fe.get("lam")
    res, sel = fe.ritz_info()
    good = lam_r[res < 1e-10]
    assert _match(p.lam[ins], good[np.abs(good) < 1.0]) < 1e-11
    assert int(np.sum(sel)) == s
    fe.close()


# ---------------------------------------------------------------- GFEAST
def test_gfeast_example_3_1():
    """The oblique-projection FEAST recovers 0.2 and 0.5 on Example 3.1."""
    A, B, eig, inside = load_example_3_1()
    rng = np.random.default_rng(0)
    Y = inputs.complex_normal(rng, (4, 2))
    fe = oracle.Feast(A, B, Y, contour_kind=0, rule=1, q=16, center=0j, a=1.0, eps=1e-13)
    fe.run()
    r = fe.result()
    assert r["flag"] == 1 and r["count"] == 2
    assert _match(r["lam"], [v for v, _ in inside]) < 1e-13
    for i in range(2):  # eigenvectors are e1 / e2 up to scale
        x = r["X"][:, i]
        j = int(np.argmax(np.abs(x)))
        assert np.linalg.norm(np.delete(x, j)) < 1e-12 * abs(x[j])
    fe.close()


def test_gfeast_prescribed_pencil_n200():
    """The dense n = 200 workload: all eigenvalues inside |z| < 1 are found,
    the count is exact, eigenvalues match the prescribed ones to 1e-10
    relative and each residual of eq. 5.1 is below 1e-12."""
    cfg = inputs.WORKLOADS["dense_n200_m64_q16"]
    p = inputs.prescribed_pencil(cfg["n"], cfg["m0"], seed=cfg["seed"])
    fe = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=cfg["rule"], q=cfg["q"],
                      center=cfg["center"], a=cfg["radius"], eps=1e-12, eta=1e-3, max_iter=50)
    hist = fe.run()
    r = fe.result()
    assert r["flag"] == 1
    assert r["count"] == p.inside_count()
    ref = p.lam[np.abs(p.lam) < 1.0]
    assert _match(r["lam"], ref) < 1e-10
    assert r["err"] < 1e-12
    # Err decreases over the first iterations (Experiment 5.3)
    errs = [h["err"] for h in hist if h["count"] == r["count"]]
    assert errs[0] > errs[-1]
    fe.close()


def test_gfeast_empty_contour_ends_at_max_iter():
    """No eigenvalue inside: the count never becomes non-zero, so neither
    line 13 nor 14 fires and line 15 ends the run with an empty result."""
    p = inputs.prescribed_pencil(40, 6, seed=2)
    fe = oracle.Feast(p.A, p.B, p.Y, q=16, center=10.0 + 0j, a=0.5, max_iter=3)
    h = fe.run()
    r = fe.result()
    assert len(h) == 3 and r["flag"] == -1 and r["count"] == 0 and r["k"] == 3
    fe.close()


def test_gfeast_max_iter_and_rebound_flags():
    p = inputs.prescribed_pencil(60, 24, seed=5)
    fe = oracle.Feast(p.A, p.B, p.Y, q=8, center=0j, a=1.0, eps=1e-30, max_iter=1)
    fe.run()
    assert fe.result()["flag"] == -1 and fe.result()["k"] == 1
    fe.close()
    # with an unreachable eps the iteration either stagnates (line 14 returns
    # the previous iterate, flag 0) or reaches max_iter (flag -1)
    fe = oracle.Feast(p.A, p.B, p.Y, q=8, center=0j, a=1.0, eps=1e-30, max_iter=40)
    h = fe.run()
    r = fe.result()
    assert r["flag"] in (0, -1)
    if r["flag"] == 0:
        assert r["k"] == len(h) - 1 and h[-1]["err"] > h[-2]["err"]
        assert r["err"] == h[-2]["err"]
    fe.close()


def test_gfeast_line14_returns_the_previous_iterate():
    """Line 14 of Algorithm GFEAST: once the count is fixed, a pass whose
    largest residual e(k) exceeds e(k-1) stops with flag 0 and returns the
    previous iterate.  With an unreachable eps this n = 60 pencil (seed 5,
    8 nodes) reaches the rounding floor and rebounds at pass 25.  A second
    run ended by line 15 one pass earlier (max_iter = 24, flag -1) returns
    that previous iterate as its own result, so the two outputs must be
    identical -- eigenvalues, residuals, vectors, count and e(k)."""
    p = inputs.prescribed_pencil(60, 24, seed=5)
    kw = dict(q=8, center=0j, a=1.0, eps=1e-30)
    fe = oracle.Feast(p.A, p.B, p.Y, max_iter=40, **kw)
    h = fe.run()
    r = fe.result()
    fe.close()
    k = len(h)                        # the pass at which line 14 fired
    assert r["flag"] == 0 and k == 25
    assert h[-1]["count"] == h[-2]["count"] > 0 and h[-1]["err"] > h[-2]["err"]
    assert r["k"] == k - 1 and r["err"] == h[-2]["err"] and r["count"] == h[-2]["count"]
    fe2 = oracle.Feast(p.A, p.B, p.Y, max_iter=k - 1, **kw)
    h2 = fe2.run()
    r2 = fe2.result()
    fe2.close()
    assert len(h2) == k - 1 and r2["flag"] == -1 and r2["k"] == k - 1
    assert r2["count"] == r["count"] and r2["err"] == r["err"]
    assert np.array_equal(r["lam"], r2["lam"]) and np.array_equal(r["res"], r2["res"])
    assert np.array_equal(r["X"], r2["X"])


def test_gfeast_banded_convection_diffusion_closed_form():
    """Banded pencil, B = I: the eigenvalues found inside an ellipse match the
    closed-form spectrum of the 5-point convection-diffusion operator
    lam_{k,l} = (2/h^2) [2 - sqrt(1-(b1 h/2)^2) cos(k pi h) - sqrt(1-(b2 h/2)^2) cos(l pi h)]."""
    nx = 12
    bp = inputs.convection_diffusion(nx, 12, seed=1, beta=(20.0, 10.0))
    h = bp.h
    c1 = math.sqrt(1 - (20.0 * h / 2) ** 2); c2 = math.sqrt(1 - (10.0 * h / 2) ** 2)
    ks = np.arange(1, nx + 1)
    lam = np.sort(((2 / h**2) * (2 - c1 * np.cos(ks[:, None] * np.pi * h) - c2 * np.cos(ks[None, :] * np.pi * h))).ravel())
    # dense QZ of the full operator reproduces the closed form
    al, be, _ = oracle.ggev(bp.dense(), np.eye(bp.n, dtype=complex))
    assert _match(al / be, lam) < 1e-9 * lam.max()
    # ellipse around the lowest 5 eigenvalues (gap to the 6th)
    lo, hi = lam[0] * 0.5, 0.5 * (lam[4] + lam[5])
    cen = 0.5 * (lo + hi); a = 0.5 * (hi - lo)
    fe = oracle.Feast(bp.A_band, None, bp.Y, kind=1, kl=bp.kl, ku=bp.ku, b_identity=True,
                      contour_kind=1, rule=1, q=16, center=complex(cen), a=a, b=a / 4, eps=1e-11)
    fe.run()
    r = fe.result()
    assert r["flag"] == 1 and r["count"] == 5
    assert _match(r["lam"], lam[:5]) < 1e-9 * lam[4]
    fe.close()


def test_count_fixed_only_once_nonzero_reading():
    """Lines 13-14 of GFEAST compare c(k) with c(k-1), and the paper sets
    c(0) = 0.  Read literally, a first pass with no pair below eta would end
    the run at k = 1 with flag 1 and no pairs (c(1) = c(0) = 0 and
    e(1) = 0 < eps).  On the n = 200 workload the first pass selects nothing
    although 44 eigenvalues lie inside the circle -- why the count is taken as
    fixed only once it is non-zero; with that reading the run finds all 44."""
    cfg = inputs.WORKLOADS["dense_n200_m64_q16"]
    p = inputs.prescribed_pencil(cfg["n"], cfg["m0"], seed=cfg["seed"])
    fe = oracle.Feast(p.A, p.B, p.Y, contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"],
                      a=cfg["radius"], eps=cfg["eps"])
    it = fe.iterate()
    assert it["k"] == 1 and it["count"] == 0 and it["err"] == 0.0 and it["flag"] == 2
    fe.run()
    r = fe.result()
    fe.close()
    assert p.inside_count() == 44 and r["flag"] == 1 and r["count"] == 44


def test_stored_n4096_oracle_run_matches_the_prescribed_spectrum():
    """The stored converged oracle run of the n = 4096 workload
    (tests/golden/dense_n4096_m1280_q32_oracle.txt, written by the script
    beside it) against what the construction fixes: its eigenvalues are the
    prescribed ones inside |z| < 1 (count exact, 1e-10 relative), every
    residual of eq. 5.1 is below eps, and line 13 ended the run."""
    g = {"lam": [], "res": []}
    for line in open(os.path.join(GOLDEN, "dense_n4096_m1280_q32_oracle.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, _, rest = line.strip().partition(" ")
        if key == "eig":
            a, b, r = rest.split()
            g["lam"].append(complex(float(a), float(b)))
            g["res"].append(float(r))
        elif key in ("flag", "k", "count", "exact_count"):
            g[key] = int(rest)
    cfg = inputs.WORKLOADS["dense_n4096_m1280_q32"]
    p = inputs.prescribed_pencil(cfg["n"], cfg["m0"], seed=cfg["seed"])
    ref = p.lam[np.abs(p.lam - cfg["center"]) < cfg["radius"]]
    assert g["flag"] == 1 and g["count"] == g["exact_count"] == len(ref) == len(g["lam"])
    pool = list(ref)
    worst = 0.0
    for x in g["lam"]:
        d = np.abs(np.asarray(pool) - x)
        j = int(np.argmin(d))
        worst = max(worst, d[j] / abs(pool[j]))
        pool.pop(j)
    assert worst < 1e-10
    assert max(g["res"]) < cfg["eps"]
