"""The FP64-accurate complex GEMM on the bf16 tensor cores (exact base-64
digit slicing, FP32 class sums in tensor memory, FP64 combination) against
complex128 products.  Its error bound is per entry: ~2^-47 * k * max_k|A'_ik|
* max_k|B'_kj| (A', B' the real forms), so the checks scale the error by the
row maximum of A and the column maximum of B."""
import numpy as np
import pytest

from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu


def _check(A, B, C0, alpha, beta, out, bits=45):
    ref = beta * C0 + alpha * (A @ B)
    ra = np.max(np.maximum(np.abs(A.real), np.abs(A.imag)), axis=1)
    cb = np.max(np.maximum(np.abs(B.real), np.abs(B.imag)), axis=0)
    k = A.shape[1]
    bound = 2.0 ** -bits * k * abs(alpha) * np.outer(ra, cb) + 1e-15 * np.abs(beta * C0)
    err = np.abs(out - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("m,n,k", [(64, 64, 64), (200, 70, 33), (130, 129, 1100), (1, 1, 1),
                                   (300, 257, 2100)])
def test_zgemm_oz_matches_complex128(m, n, k):
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = inputs.complex_normal(rng, (m, k))
    B = inputs.complex_normal(rng, (k, n))
    C0 = inputs.complex_normal(rng, (m, n))
    alpha, beta = 0.75 - 0.5j, 1.0 + 0.25j
    out = fg.zgemm_oz(A, B, C0, alpha=alpha, beta=beta)
    _check(A, B, C0, alpha, beta, out)


def test_zgemm_oz_row_and_column_scaling():
    """Rows of A and columns of B spanning 1e-12 .. 1e12 keep their own
    relative accuracy (the digit planes are scaled per row / column)."""
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(5)
    m, n, k = 96, 80, 512
    A = inputs.complex_normal(rng, (m, k)) * np.logspace(-12, 12, m)[:, None]
    B = inputs.complex_normal(rng, (k, n)) * np.logspace(8, -8, n)[None, :]
    out = fg.zgemm_oz(A, B)
    _check(A, B, np.zeros((m, n)), 1.0, 0.0, out)


def test_zgemm_oz_exact_on_small_integers():
    """Integer operands with |entries| < 64 are one digit deep: the product
    is exact."""
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(9)
    A = rng.integers(-40, 40, (70, 300)) + 1j * rng.integers(-40, 40, (70, 300))
    B = rng.integers(-40, 40, (300, 90)) + 1j * rng.integers(-40, 40, (300, 90))
    out = fg.zgemm_oz(A, B)
    np.testing.assert_array_equal(out, A @ B)
