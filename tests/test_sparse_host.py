"""Host logic of the sparse-pencil path: the reverse Cuthill-McKee ordering
of feast_csr_rcm (a valid permutation; the bandwidths it reports are the
brute-force bandwidths of the permuted matrices; on a shuffled 2D grid it
recovers the grid's bandwidth nx, as scipy's own RCM does) and its argument
checks.  No GPU: the ordering is host code in the library."""
import numpy as np
import pytest

import paper_1404_1768_gb300 as fg
from paper_1404_1768_gb300 import inputs


def _bandwidth(M, n, perm):
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    indptr, indices, _ = M
    rows = np.repeat(np.arange(n), np.diff(indptr))
    d = iperm[rows] - iperm[indices]
    return int(max(d.max(), 0)), int(max((-d).max(), 0))


@pytest.mark.parametrize("nx,seed", [(6, 0), (12, 1), (20, 2)])
def test_rcm_permutation_and_bandwidth(nx, seed):
    sp = inputs.sparse_pencil(nx, 4, seed=seed)
    n = sp.n
    perm, kl, ku = fg.csr_rcm(n, sp.A, sp.B)
    assert np.array_equal(np.sort(perm), np.arange(n))
    bla, bua = _bandwidth(sp.A, n, perm)
    blb, bub = _bandwidth(sp.B, n, perm)
    assert (kl, ku) == (max(bla, blb), max(bua, bub))
    # the shuffled order has bandwidth ~n; the grid's own order has nx
    assert _bandwidth(sp.A, n, np.arange(n))[0] > 2 * nx
    assert kl <= nx + 1 and ku <= nx + 1


def test_rcm_matches_scipy_bandwidth():
    ss = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")
    sp = inputs.sparse_pencil(16, 4, seed=3)
    n = sp.n
    perm, kl, ku = fg.csr_rcm(n, sp.A, sp.B)
    M = ss.csr_matrix((np.ones(len(sp.A[1])), sp.A[1], sp.A[0]), shape=(n, n))
    pr = cg.reverse_cuthill_mckee(M, symmetric_mode=True)
    ref = _bandwidth(sp.A, n, np.asarray(pr, np.int64))[0]
    assert kl <= ref + 2


def test_rcm_disconnected_and_identity_b():
    # two independent grids side by side (block diagonal), B = I
    a = inputs.sparse_pencil(5, 2, seed=4)
    b = inputs.sparse_pencil(7, 2, seed=5)
    n = a.n + b.n
    indptr = np.concatenate([a.A[0], a.A[0][-1] + b.A[0][1:]])
    indices = np.concatenate([a.A[1], b.A[1] + a.n])
    data = np.concatenate([a.A[2], b.A[2]])
    perm, kl, ku = fg.csr_rcm(n, (indptr, indices, data), None)
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert (kl, ku) == _bandwidth((indptr, indices, data), n, perm)
    assert kl <= 8


def test_rcm_rejects_malformed_csr():
    sp = inputs.sparse_pencil(4, 2, seed=0)
    n = sp.n
    bad = (sp.A[0], sp.A[1].copy(), sp.A[2])
    bad[1][3] = n            # column out of range
    with pytest.raises(fg.FeastError) as ei:
        fg.csr_rcm(n, bad, None)
    assert ei.value.status == -1
    ptr = sp.A[0].copy()
    ptr[5], ptr[6] = ptr[6], ptr[5]   # decreasing row pointer
    with pytest.raises(fg.FeastError):
        fg.csr_rcm(n, (ptr, sp.A[1], sp.A[2]), None)
