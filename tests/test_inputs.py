"""The seeded generators state what they build; these checks tie each to
its stated structure (so that the closed forms the tests and the benchmark
use apply): the sparse pencil is the banded operator under a permutation,
the Hermitian pencil has the prescribed real spectrum, the gapped pencil its
gap."""
import numpy as np

from paper_1404_1768_gb300 import inputs


def test_sparse_pencil_is_the_shuffled_band_operator():
    nx = 9
    sp = inputs.sparse_pencil(nx, 3, seed=4, mass=0.0)
    bp = inputs.convection_diffusion(nx, 3, seed=4)
    n = sp.n
    A = inputs.SparsePencil.dense(sp.A, n)
    B = inputs.SparsePencil.dense(sp.B, n)
    # stored index k is grid node shuffle[k]: A[k, l] = A_grid[shuffle[k], shuffle[l]]
    Ag = bp.dense()
    s = sp.shuffle
    assert np.array_equal(np.sort(s), np.arange(n))
    assert np.array_equal(A, Ag[np.ix_(s, s)])
    assert np.array_equal(B, np.eye(n))
    # CSR rows have sorted columns
    for i in range(n):
        cols = sp.A[1][sp.A[0][i]:sp.A[0][i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_sparse_pencil_mass_matrix():
    sp = inputs.sparse_pencil(8, 2, seed=1, mass=0.1)
    B = inputs.SparsePencil.dense(sp.B, sp.n)
    assert np.array_equal(B, B.T)
    ev = np.linalg.eigvalsh(B.real)
    assert ev.min() > 0.9 - 1e-12 and ev.max() < 1.1 + 1e-12


def test_hermitian_pencil_spectrum():
    p = inputs.hermitian_pencil(60, 10, seed=3)
    lam = np.sort(np.linalg.eigvals(np.linalg.solve(p.B, p.A)).real)
    np.testing.assert_allclose(lam, np.sort(p.lam.real), atol=1e-12 * np.abs(p.lam).max())
    assert np.all(np.abs(np.abs(p.lam.real) - 1.0) >= 1e-3)


def test_gapped_pencil_gap():
    p = inputs.gapped_pencil(80, 10, 12, seed=2)
    r = np.abs(p.lam)
    assert np.sum(r < 0.7) == 12 and np.all((r < 0.7) | (r > 1.5))
    lam = np.linalg.eigvals(np.linalg.solve(p.B, p.A))
    assert max(np.min(np.abs(lam - x)) for x in p.lam) < 1e-10
