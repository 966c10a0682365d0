"""Sparse pencils on the GPU: feast_csr_to_band writes exactly P M P^T in
band storage, and GFEAST through SparseFeast (reverse Cuthill-McKee, then the
banded path) agrees with the oracle's dense run on the shuffled pencil: the
same count and stop, eigenvalues, and eigenvectors of the original ordering."""
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
        worst = max(worst, abs(x - b[j]) / abs(b[j]))
        b.pop(j)
    return worst


def test_csr_to_band_is_the_permuted_matrix():
    fg = _fg()
    sp = inputs.sparse_pencil(10, 4, seed=2)
    n = sp.n
    perm, kl, ku = fg.csr_rcm(n, sp.A, sp.B)
    for M in (sp.A, sp.B):
        band = fg.csr_to_band(n, M, perm, kl, ku).cpu().numpy().reshape(n, kl + ku + 1).T
        D = inputs.SparsePencil.dense(M, n)[np.ix_(perm, perm)]
        R = np.zeros_like(D)
        for j in range(n):
            for i in range(max(0, j - ku), min(n, j + kl + 1)):
                R[i, j] = band[ku + i - j, j]
        assert np.array_equal(R, D)
    # a band too narrow for the matrix is refused
    with pytest.raises(fg.FeastError) as ei:
        fg.csr_to_band(n, sp.A, perm, kl - 1, ku)
    assert ei.value.status == -1


@pytest.mark.parametrize("prec", [0, 1])
def test_sparse_gfeast_matches_dense_oracle(prec):
    fg = _fg()
    sp = inputs.sparse_pencil(12, 16, seed=1)
    n = sp.n
    A = inputs.SparsePencil.dense(sp.A, n)
    B = inputs.SparsePencil.dense(sp.B, n)
    # circle around the 7 eigenvalues nearest 200 (the next ones are 11 %
    # and 58 % beyond its radius)
    kw = dict(contour_kind=0, rule=1, q=16, center=200.0 + 0j, a=34.0, eps=1e-10)
    g = fg.SparseFeast(n, sp.A, sp.B, sp.Y, prec=prec, **kw)
    assert g.perm.shape == (n,)
    hg = g.run()
    rg = g.eigs()
    o = oracle.Feast(A, B, sp.Y, **kw)
    ho = o.run()
    ro = o.result()
    assert rg["flag"] == ro["flag"] == 1
    assert rg["count"] == ro["count"] == 7
    assert abs(len(hg) - len(ho)) <= 1
    assert _match(rg["lam"], ro["lam"]) < 1e-10
    for i in range(rg["count"]):
        x = rg["X"][:, i]
        r = A @ x - rg["lam"][i] * (B @ x)
        assert np.linalg.norm(r) / (np.linalg.norm(A @ x) + np.linalg.norm(B @ x)) < 1e-10
    g.close(); o.close()
