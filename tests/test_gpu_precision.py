"""Precision form (complex64 factors and solves on the tensor cores) against
the FP64 oracle.

Tolerances: a complex64 LU agrees with the FP64 one to ~n * 2^-24 relative.
The standalone subspace build (feast_filter) refines each shifted solve with
a residual whose products are FP64-accurate tensor-core GEMMs, to the
refinement target (relative residual 1e-14 -> forward error ~kappa *
1e-14).  Inside the iteration line 16 takes the defect form on the Ritz
pairs (the solves see only the residual block), and the whole method must
reach FP64-level results: exact count, eigenvalues within 1e-10 relative of
the oracle, residuals of eq. 5.1 below 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu

CFG1 = inputs.WORKLOADS["dense_n200_m64_q16"]


def _fg():
    import paper_1404_1768_gb300 as fg
    return fg


def _match(a, b):
    b = list(b)
    worst = 0.0
    for x in sorted(a, key=lambda v: (v.real, v.imag)):
        j = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[j]) / max(abs(b[j]), 1e-300))
        b.pop(j)
    return worst


@pytest.mark.parametrize("n,m0,q", [(200, 64, 16), (77, 13, 8)])
def test_refined_filter_matches_oracle(n, m0, q):
    """U = sum_j w_j (z_j B - A)^{-1} B V with complex64 solves refined to a
    relative residual of 1e-14: agrees with the FP64 oracle to ~1e-11."""
    fg = _fg()
    p = inputs.prescribed_pencil(n, m0, seed=n)
    kw = dict(contour_kind=0, rule=0, q=q, center=0j, a=1.0)
    g = fg.Feast(p.A, p.B, p.Y, prec=fg.FEAST_C64_REFINE, refine_tol=1e-14, max_refine=6, **kw)
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    V = inputs.complex_normal(np.random.default_rng(7), (n, m0))
    Ug, Uo = g.filter(V), o.filter(V)
    err = np.abs(Ug - Uo).max() / np.abs(Uo).max()
    assert err < 1e-11, err
    g.close(); o.close()


def test_unrefined_filter_is_single_precision():
    """Without refinement sweeps the same filter is only complex64-accurate:
    the refinement is what wins the accuracy back."""
    fg = _fg()
    p = inputs.prescribed_pencil(200, 64, seed=200)
    kw = dict(contour_kind=0, rule=0, q=16, center=0j, a=1.0)
    g = fg.Feast(p.A, p.B, p.Y, prec=fg.FEAST_C64_REFINE, refine_tol=1e-14, max_refine=0, **kw)
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    V = inputs.complex_normal(np.random.default_rng(7), (200, 64))
    err = np.abs(g.filter(V) - o.filter(V)).max() / np.abs(o.filter(V)).max()
    assert 1e-9 < err < 1e-3, err
    g.close(); o.close()


def test_gfeast_precision_form_n200():
    """Whole GFEAST in the precision form on the n = 200 workload: exact
    count, eigenvalues within 1e-10 relative of the oracle's and of the
    prescribed spectrum, every residual of eq. 5.1 below 1e-12 -- FP64-level
    accuracy with complex64 solves and no refinement sweep inside the
    iteration (line 16 takes the defect form on the Ritz pairs)."""
    fg = _fg()
    p = inputs.prescribed_pencil(CFG1["n"], CFG1["m0"], seed=CFG1["seed"])
    kw = dict(contour_kind=0, rule=CFG1["rule"], q=CFG1["q"], center=CFG1["center"],
              a=CFG1["radius"], eps=1e-12, eta=1e-3, max_iter=50)
    g = fg.Feast(p.A, p.B, p.Y, prec=fg.FEAST_C64_REFINE, refine_tol=1e-14, max_refine=5, **kw)
    hist = g.run()
    rg = g.eigs()
    o = oracle.Feast(p.A, p.B, p.Y, **kw)
    o.run()
    ro = o.result()
    assert rg["flag"] == 1
    assert rg["count"] == ro["count"] == p.inside_count()
    ref = p.lam[np.abs(p.lam - CFG1["center"]) < CFG1["radius"]]
    assert _match(rg["lam"], ro["lam"]) < 1e-10
    assert _match(rg["lam"], ref) < 1e-10
    assert np.all(rg["res"] < 1e-12)
    for i in range(rg["count"]):
        x = rg["X"][:, i]
        r = p.A @ x - rg["lam"][i] * (p.B @ x)
        assert np.linalg.norm(r) / (np.linalg.norm(p.A @ x) + np.linalg.norm(p.B @ x)) < 1e-12
    assert all(h["refine_sweeps_max"] == 0 for h in hist)
    g.close(); o.close()


@pytest.mark.parametrize("n,m0,cond", [(200, 64, 1e2), (700, 230, 1e4), (700, 230, 1e9), (1000, 300, 3.0),
                                        (1000, 300, 1e2), (1000, 300, 1e5), (1000, 300, 1e9)])
def test_cholesky_qr_of_b_u1(n, m0, cond):
    """U2 R2 = B U1 in the precision form (Cholesky QR twice on tensor-core
    Gram matrices; BCGS2 when the block is too ill-conditioned for it -- the
    cond = 1e9 cases): U2 orthonormal, R2 upper triangular with a real
    positive diagonal, U2 R2 = B U1, and both equal to the unique Householder
    factors with that sign convention (numpy's QR, signs fixed).  From
    m0 = 256 the first factorisation is tried in FP32 on the unit-diagonal
    Gram matrix; the m0 = 300 cases reach its series pass, a second FP64
    Cholesky, its FP64 restart or BCGS2 as their conditioning requires."""
    fg = _fg()
    p = inputs.prescribed_pencil(n, m0, seed=n + 1)
    g = fg.Feast(p.A, p.B, p.Y, prec=fg.FEAST_C64_REFINE, q=8, center=0j, a=1.0)
    rng = np.random.default_rng(11)
    # U1 with the chosen condition number (U1 itself need not be orthonormal
    # for this entry point; B U1 inherits the conditioning)
    Qa, _ = np.linalg.qr(inputs.complex_normal(rng, (n, m0)))
    Qb, _ = np.linalg.qr(inputs.complex_normal(rng, (m0, m0)))
    U1 = (Qa * np.logspace(0, -np.log10(cond), m0)[None, :]) @ Qb
    g.set_subspace(U1)
    U2, R2 = g.get("U2"), g.get("R2")
    BU1 = p.B @ U1
    assert np.abs(U2.conj().T @ U2 - np.eye(m0)).max() < 1e-12
    assert np.allclose(np.tril(R2, -1), 0) and np.all(np.diag(R2).real > 0)
    assert np.abs(np.diag(R2).imag).max() <= 1e-14 * np.abs(R2).max()
    assert np.abs(U2 @ R2 - BU1).max() <= 1e-12 * np.abs(BU1).max()
    Qn, Rn = np.linalg.qr(BU1)
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    Qn, Rn = Qn * ph[None, :], ph.conj()[:, None] * Rn
    if cond <= 1e4:
        np.testing.assert_allclose(U2, Qn, rtol=0, atol=1e-9)
    g.close()
