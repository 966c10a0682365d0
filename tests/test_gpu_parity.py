"""GPU parity: every step of the CUDA path against the FP64 oracle on the
same seeded inputs, through the C ABI.  Tolerances follow from FP64
arithmetic: the kernels sum in a different order than the oracle, so
elementwise agreement is bounded by a small multiple of n * eps times the
condition of the step (stated per test)."""
import math

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
    for x in sorted(a, key=lambda v: (v.real, v.imag)):
        j = int(np.argmin([abs(x - y) for y in b]))
        worst = max(worst, abs(x - b[j]))
        b.pop(j)
    return worst


# ------------------------------------------------------------------ LU
@pytest.mark.parametrize("n", [1, 7, 32, 33, 64, 100])
def test_lu_factors_match_oracle(n):
    """Same partial pivoting rule (largest modulus, first on ties) -> the
    pivots agree exactly and the factors to ~n eps."""
    fg = _fg()
    rng = np.random.default_rng(10 + n)
    Ms = [inputs.complex_normal(rng, (n, n)) for _ in range(3)]
    facs, piv, info = fg.zgetrf_batched(Ms)
    assert info == 0
    for b, M in enumerate(Ms):
        f, p, inf = oracle.lu(M)
        np.testing.assert_array_equal(piv[b], p)
        np.testing.assert_allclose(facs[b], f, rtol=0, atol=1e-12 * max(1, n) * np.abs(f).max())


@pytest.mark.parametrize("n,nrhs", [(1, 1), (33, 5), (100, 70)])
def test_lu_solve_matches_oracle(n, nrhs):
    fg = _fg()
    rng = np.random.default_rng(20 + n)
    Ms = [inputs.complex_normal(rng, (n, n)) for _ in range(2)]
    Rs = [inputs.complex_normal(rng, (n, nrhs)) for _ in range(2)]
    facs, piv, _ = fg.zgetrf_batched(Ms)
    Xs = fg.zgetrs_batched(facs, piv, Rs)
    for b in range(2):
        f, p, _ = oracle.lu(Ms[b])
        xo = oracle.lu_solve(f, p, Rs[b])
        np.testing.assert_allclose(Xs[b], xo, rtol=0, atol=1e-10 * np.abs(xo).max())


def test_singular_matrix_reports_info():
    fg = _fg()
    M = np.zeros((5, 5), complex)
    M[0, 0] = 1.0
    M[1, 2] = 2.0
    _, _, info = fg.zgetrf_batched([np.eye(5, dtype=complex), M])
    assert info == 2   # 1 + block index


# ------------------------------------------------------------------ QZ
@pytest.mark.parametrize("m", [1, 2, 5, 16, 32, 40, 64, 65, 100, 164, 165, 300, 400])
def test_qz_matches_oracle(m):
    """Eigenvalues as multisets (the order of a QZ run is not unique) and the
    generalized eigen-residual of every returned vector.  m <= 64: one-CTA QZ;
    65..164: Hessenberg reduction, then one CTA with the matrix in shared
    memory (single-shift double-single QR, logged rotations applied to the
    Schur vectors afterwards); 165 and up: the cooperative grid QR (single
    shift below 192 active rows, multishift with early deflation above)."""
    fg = _fg()
    rng = np.random.default_rng(30 + m)
    As = [inputs.complex_normal(rng, (m, m)) for _ in range(2)]
    if m <= 64:   # QZ proper: any upper-triangular B, here with a wide condition range
        Bs = [np.triu(inputs.complex_normal(rng, (m, m))) + 2.0 * np.eye(m) for _ in range(2)]
    else:         # standard-form path: B = R2-like, well conditioned as in FEAST
        Bs = [np.eye(m) + 0.1 * np.triu(inputs.complex_normal(rng, (m, m))) / np.sqrt(m)
              for _ in range(2)]
    al, be, Vs, fail = fg.zqz_batched(As, Bs)
    assert fail == 0
    for b in range(2):
        ao, bo, _ = oracle.ggev(As[b], Bs[b])
        lam_g, lam_o = al[b] / be[b], ao / bo
        assert _match(lam_g, lam_o) < 1e-10 * max(1.0, np.abs(lam_o).max())
        for i in range(m):
            v = Vs[b][:, i]
            r = be[b][i] * As[b] @ v - al[b][i] * Bs[b] @ v
            scale = abs(be[b][i]) * np.linalg.norm(As[b]) + abs(al[b][i]) * np.linalg.norm(Bs[b])
            assert np.linalg.norm(r) < 1e-12 * scale
            assert abs(np.linalg.norm(v) - 1.0) < 1e-12


def test_qz_example_3_1():
    """The projected pencil of Example 3.1: A~ = diag(0.2, 0.5), B~ = I."""
    fg = _fg()
    al, be, Vs, fail = fg.zqz_batched([np.diag([0.2, 0.5]).astype(complex)], [np.eye(2, dtype=complex)])
    assert fail == 0
    assert _match(al[0] / be[0], [0.2, 0.5]) < 1e-15


# ------------------------------------------------------------------ pipeline
def _pair(p, cfg, **kw):
    fg = _fg()
    args = dict(contour_kind=0, rule=cfg["rule"], q=cfg["q"], center=cfg["center"],
                a=cfg["radius"], eps=1e-12, eta=1e-3, max_iter=50)
    args.update(kw)
    g = fg.Feast(p.A, p.B, p.Y, **args)
    o = oracle.Feast(p.A, p.B, p.Y, **args)
    return g, o


CFG1 = inputs.WORKLOADS["dense_n200_m64_q16"]


@pytest.mark.parametrize("rule,ck", [(0, 0), (1, 0), (1, 1)])
def test_contour_nodes_match_oracle(rule, ck):
    fg = _fg()
    p = inputs.prescribed_pencil(24, 4, seed=1)
    b = 0.4 if ck == 1 else 0.0
    g = fg.Feast(p.A, p.B, p.Y, contour_kind=ck, rule=rule, q=16, center=0.1 + 0.2j, a=0.9, b=b)
    z, w = oracle.contour(ck, rule, 16, 0.1 + 0.2j, 0.9, b)
    np.testing.assert_allclose(g.get("z"), z, atol=1e-14)
    np.testing.assert_allclose(g.get("w"), w, atol=1e-14)
    g.close()


@pytest.mark.parametrize("n,m0,q", [(200, 64, 16), (77, 13, 8), (130, 70, 5)])
def test_filter_matches_oracle(n, m0, q):
    """U = sum_j w_j (z_j B - A)^{-1} B V (eq. 4.1-4.2): the node-batched LU,
    the blocked solves and the node sum against the oracle, elementwise.
    n = 77, 130 leave ragged tails against the 32-wide panels and 64-wide
    GEMM tiles."""
    p = inputs.prescribed_pencil(n, m0, seed=n)
    cfg = dict(CFG1, q=q)
    g, o = _pair(p, cfg)
    rng = np.random.default_rng(5)
    V = inputs.complex_normal(rng, (n, m0))
    Ug, Uo = g.filter(V), o.filter(V)
    np.testing.assert_allclose(Ug, Uo, rtol=0, atol=1e-11 * np.abs(Uo).max())
    # closed form (independent of both): U = Q^{-1} diag(f(lam)) Q V
    f = 1.0 / (1.0 + ((p.lam - cfg["center"]) / cfg["radius"]) ** q)
    Uc = np.linalg.solve(p.Q, f[:, None] * (p.Q @ V))
    np.testing.assert_allclose(Ug, Uc, rtol=0, atol=1e-10 * np.abs(Uc).max())
    g.close(); o.close()


def test_setup_subspaces_match_oracle():
    """U1 = orth(Q Y), U2 = orth(B U1): both QR factorisations have a real
    positive diagonal in R, so U1 and U2 are unique."""
    p = inputs.prescribed_pencil(CFG1["n"], CFG1["m0"], seed=CFG1["seed"])
    g, o = _pair(p, CFG1)
    for name in ("U1", "U2", "BU1"):
        a, b = g.get(name), o.get(name)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-9 * np.abs(b).max(), err_msg=name)
    U1 = g.get("U1")
    np.testing.assert_allclose(U1.conj().T @ U1, np.eye(CFG1["m0"]), atol=1e-13)
    R2 = g.get("R2")
    assert np.allclose(np.tril(R2, -1), 0) and np.all(np.diag(R2).real > 0)
    g.close(); o.close()


def test_first_passes_match_oracle():
    """Projection, QZ, Ritz residuals and the stopping test of passes 1-3:
    the same count c(k), the same selected eigenvalues, e(k) close."""
    p = inputs.prescribed_pencil(CFG1["n"], CFG1["m0"], seed=CFG1["seed"])
    g, o = _pair(p, CFG1)
    for k in range(3):
        ig, io = g.iterate(), o.iterate()
        assert ig["k"] == io["k"] == k + 1
        assert ig["count"] == io["count"]
        assert ig["flag"] == io["flag"] == 2
        if io["count"]:
            assert abs(ig["err"] - io["err"]) <= 1e-6 * io["err"] + 1e-14
        At_g, At_o = g.get("At"), o.get("At")
        np.testing.assert_allclose(At_g, At_o, rtol=0, atol=1e-9 * np.abs(At_o).max())
        sel_g, sel_o = g.get("sel"), o.ritz_info()[1]
        lam_g, lam_o = g.get("lam"), o.get("lam")
        assert _match(lam_g[sel_g], lam_o[sel_o]) < 1e-9
    g.close(); o.close()


def test_gfeast_end_to_end_n200():
    """The dense n = 200, m0 = 64, 16-node workload to convergence: flag 1,
    the exact count, eigenvalues equal to the prescribed ones to 1e-10
    relative and to the oracle's, residuals below eps."""
    p = inputs.prescribed_pencil(CFG1["n"], CFG1["m0"], seed=CFG1["seed"])
    g, o = _pair(p, CFG1)
    hg, ho = g.run(), o.run()
    rg, ro = g.eigs(), o.result()
    assert rg["flag"] == ro["flag"] == 1
    assert rg["count"] == ro["count"] == p.inside_count()
    assert abs(len(hg) - len(ho)) <= 1
    ref = p.lam[np.abs(p.lam - CFG1["center"]) < CFG1["radius"]]
    assert _match(rg["lam"], ref) < 1e-10
    assert _match(rg["lam"], ro["lam"]) < 1e-10
    assert rg["err"] < 1e-12 and np.all(rg["res"] < 1e-12)
    # returned eigenvectors: A x = lambda B x
    for i in range(rg["count"]):
        x = rg["X"][:, i]
        r = p.A @ x - rg["lam"][i] * (p.B @ x)
        assert np.linalg.norm(r) / (np.linalg.norm(p.A @ x) + np.linalg.norm(p.B @ x)) < 1e-11
    g.close(); o.close()


def test_gfeast_example_3_1_gpu():
    """Example 3.1 through the whole GPU path recovers 0.2 and 0.5."""
    from test_oracle_pins import load_example_3_1
    fg = _fg()
    A, B, eig, inside = load_example_3_1()
    Y = inputs.complex_normal(np.random.default_rng(0), (4, 2))
    g = fg.Feast(A, B, Y, contour_kind=0, rule=1, q=16, center=0j, a=1.0, eps=1e-13)
    g.run()
    r = g.eigs()
    assert r["flag"] == 1 and r["count"] == 2
    assert _match(r["lam"], [v for v, _ in inside]) < 1e-13
    g.close()


def test_gfeast_large_subspace_path():
    """m0 = 96 > 64 takes the whole-GPU projected eigensolver (standard form,
    Hessenberg reduction, chunked QR); end to end it must agree with the
    oracle's QZ-based run.  This pencil has eigenvalues 0.998 and 1.0016
    on either side of the circle, so the filter contracts only ~0.64 per
    pass: both runs end by line 15 (max_iter) with the same count and
    matching eigenvalues."""
    p = inputs.prescribed_pencil(320, 96, seed=12)
    cfg = dict(CFG1, q=16)
    g, o = _pair(p, cfg, max_iter=40)
    hg, ho = g.run(), o.run()
    rg, ro = g.eigs(), o.result()
    assert rg["flag"] == ro["flag"]
    assert len(hg) == len(ho)
    assert rg["count"] == ro["count"] == p.inside_count()
    assert _match(rg["lam"], ro["lam"]) < 1e-8
    ref = p.lam[np.abs(p.lam) < 1.0]
    assert _match(rg["lam"], ref) < 1e-8
    g.close(); o.close()


def test_full_subspace_m0_equals_n():
    """Degenerate width m0 = n: the search space is the whole space."""
    fg = _fg()
    p = inputs.prescribed_pencil(40, 40, seed=4)
    g = fg.Feast(p.A, p.B, p.Y, q=16, center=0j, a=1.0, eps=1e-11)
    g.run()
    r = g.eigs()
    ref = p.lam[np.abs(p.lam) < 1.0]
    assert r["count"] == len(ref) and _match(r["lam"], ref) < 1e-10
    g.close()


def test_non_regular_pencil_reports_singular():
    """det(zB - A) == 0 for all z (a shared zero row): every shifted matrix
    has an exact zero pivot -> FEAST_ESINGULAR, reported at set-up."""
    fg = _fg()
    A = np.diag([1.0, 0.0, 2.0]).astype(complex)
    B = np.diag([1.0, 0.0, 1.0]).astype(complex)
    Y = np.ones((3, 1), complex)
    with pytest.raises(fg.FeastError) as ei:
        fg.Feast(A, B, Y, q=4, center=0j, a=0.5)
    assert ei.value.status == -4


def test_iterate_after_stop_is_refused():
    fg = _fg()
    p = inputs.prescribed_pencil(40, 12, seed=6)
    g = fg.Feast(p.A, p.B, p.Y, q=16, center=0j, a=1.0, eps=1e-10, max_iter=2)
    g.run()
    with pytest.raises(fg.FeastError) as ei:
        g.iterate()
    assert ei.value.status == -8
    g.close()


def test_rebound_flag_returns_previous_iterate():
    """eps unreachable: this pencil (the oracle pin's: n = 60, seed 5, 8
    nodes) reaches the rounding floor and line 14 of GFEAST ends the run with
    flag 0 on both sides; what the GPU returns is the previous pass's
    selection -- the pairs that pass selected (line 10), its count and e(k)."""
    p = inputs.prescribed_pencil(60, 24, seed=5)
    cfg = dict(CFG1, q=8)
    g, o = _pair(p, cfg, eps=1e-30, max_iter=40)
    prev = None
    while True:
        it = g.iterate()
        if it["flag"] != 2:
            break
        lam, res, sel = g.get("lam"), g.get("res"), g.get("sel")
        prev = (lam[sel], res[sel], it)
    o.run()
    rg, ro = g.eigs(), o.result()
    assert rg["flag"] == ro["flag"] == 0
    assert rg["count"] == ro["count"] == prev[2]["count"] == len(prev[0])
    assert rg["err"] == prev[2]["err"]
    np.testing.assert_array_equal(np.sort_complex(rg["lam"]), np.sort_complex(prev[0]))
    np.testing.assert_array_equal(np.sort(rg["res"]), np.sort(prev[1]))
    g.close(); o.close()
