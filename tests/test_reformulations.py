"""The identities behind the GPU path's reformulations of GFEAST steps,
checked in plain numpy on small pencils (no GPU, no oracle internals):

* line 16 in defect form: sum_j w_j M_j^{-1} B X = X rho(Lambda)
  + sum_j w_j M_j^{-1} (R D_j), R = A X - B X Lambda, for ANY X and Lambda
  (so the precision form computes the paper's quadrature sum exactly, up to
  rounding);
* line 16 on the Ritz vectors X = U1 Y spans the same subspace as on U1;
* the second Cholesky-QR pass by the perturbation series: R = I + S with
  S = phi(E - phi(E)^H phi(E)) satisfies R^H R = I + E and
  (I + S)(I - S + S^2) = I up to O(|E|^3).
"""
import numpy as np

from paper_1404_1768_gb300 import inputs


def _contour(q):
    th = 2 * np.pi * (np.arange(q) + 0.5) / q
    z = np.exp(1j * th)
    return z, z / q   # trapezoid on |z| = 1: w_j = (z_j - 0) / q


def _filter(A, B, V, z, w):
    BV = B @ V
    return sum(wj * np.linalg.solve(zj * B - A, BV) for zj, wj in zip(z, w))


def test_defect_form_is_the_quadrature_sum():
    p = inputs.prescribed_pencil(40, 12, seed=2)
    z, w = _contour(8)
    rng = np.random.default_rng(0)
    # arbitrary (not converged) "Ritz" block and values
    X = inputs.complex_normal(rng, (40, 12))
    lam = 0.4 * inputs.complex_normal(rng, (12,))
    direct = _filter(p.A, p.B, X, z, w)
    R = p.A @ X - (p.B @ X) * lam[None, :]
    rho = np.array([np.sum(w / (z - l)) for l in lam])
    defect = X * rho[None, :]
    for zj, wj in zip(z, w):
        d = 1.0 / (zj - lam)
        defect = defect + wj * np.linalg.solve(zj * p.B - p.A, R * d[None, :])
    np.testing.assert_allclose(defect, direct, rtol=0, atol=1e-11 * np.abs(direct).max())


def test_defect_form_error_scales_with_the_residual():
    """A relative error delta on the solves lands on the R term only: with
    Ritz pairs of residual ~r the filtered block's error is ~delta * r, while
    the plain form's is ~delta."""
    p = inputs.prescribed_pencil(60, 10, seed=4)
    z, w = _contour(16)
    # near-exact eigenpairs of (A, B): A Q^-1 = B Q^-1 diag(lam)
    Qi = np.linalg.inv(p.Q)
    idx = np.argsort(np.abs(p.lam))[:10]
    rng = np.random.default_rng(1)
    X = Qi[:, idx] + 1e-6 * inputs.complex_normal(rng, (60, 10))
    lam = p.lam[idx]
    exact = _filter(p.A, p.B, X, z, w)
    delta = 1e-5

    def solve_noisy(M, rhs, k):
        x = np.linalg.solve(M, rhs)
        g = np.random.default_rng(100 + k)
        return x * (1 + delta * g.standard_normal(x.shape))

    BX = p.B @ X
    plain = sum(wj * solve_noisy(zj * p.B - p.A, BX, j) for j, (zj, wj) in enumerate(zip(z, w)))
    R = p.A @ X - BX * lam[None, :]
    rho = np.array([np.sum(w / (z - l)) for l in lam])
    defect = X * rho[None, :]
    for j, (zj, wj) in enumerate(zip(z, w)):
        d = 1.0 / (zj - lam)
        defect = defect + wj * solve_noisy(zj * p.B - p.A, R * d[None, :], j)
    e_plain = np.abs(plain - exact).max() / np.abs(exact).max()
    e_defect = np.abs(defect - exact).max() / np.abs(exact).max()
    assert e_plain > 1e-7
    assert e_defect < 1e-3 * e_plain


def test_filtering_ritz_vectors_keeps_the_subspace():
    p = inputs.prescribed_pencil(50, 14, seed=6)
    z, w = _contour(16)
    U1, _ = np.linalg.qr(_filter(p.A, p.B, p.Y, z, w))
    U2, R2 = np.linalg.qr(p.B @ U1)
    C = np.linalg.solve(R2, U2.conj().T @ p.A @ U1)
    _, Y = np.linalg.eig(C)
    X = U1 @ Y
    Ua, _ = np.linalg.qr(_filter(p.A, p.B, U1, z, w))
    Ub, _ = np.linalg.qr(_filter(p.A, p.B, X, z, w))
    # principal angles between the two subspaces are zero
    s = np.linalg.svd(Ua.conj().T @ Ub, compute_uv=False)
    assert np.all(s > 1 - 1e-9)


def _phi(M):
    S = np.triu(M, 1)
    S[np.diag_indices_from(S)] = 0.5 * np.real(np.diag(M))
    return S


def test_second_cholesky_qr_pass_series():
    rng = np.random.default_rng(3)
    m = 30
    for size in (1e-4, 1e-7):
        G = inputs.complex_normal(rng, (m, m)) * size
        E = 0.5 * (G + G.conj().T)
        S0 = _phi(E)
        S = _phi(E - S0.conj().T @ S0)
        R = np.eye(m) + S
        assert np.allclose(np.tril(R, -1), 0) and np.all(np.isreal(np.diag(R)))
        err = np.abs(R.conj().T @ R - (np.eye(m) + E)).max()
        inv_err = np.abs(R @ (np.eye(m) - S + S @ S) - np.eye(m)).max()
        assert err < 50 * size ** 3 + 1e-15
        assert inv_err < 50 * size ** 3 + 1e-15
        # it is the Cholesky factor (unique with a real positive diagonal)
        Lc = np.linalg.cholesky(np.eye(m) + E)
        assert np.abs(Lc.conj().T - R).max() < 50 * size ** 3 + 1e-15
