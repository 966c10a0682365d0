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


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-2.5, 1.0), (0.5, 0.0), (1.0, -1.0)])
def test_zgemm_oz_real_alpha_unit_beta(alpha, beta):
    """The epilogue's short forms (a real alpha, a unit beta) give the same
    products as the complex-scalar form."""
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(17)
    A = inputs.complex_normal(rng, (150, 700))
    B = inputs.complex_normal(rng, (700, 90))
    C0 = inputs.complex_normal(rng, (150, 90))
    out = fg.zgemm_oz(A, B, C0, alpha=alpha, beta=beta)
    _check(A, B, C0, alpha, beta, out)


def test_zgemm_oz_subnormal_rows():
    """A row whose entries are all subnormal (|a| ~ 1e-310) is sliced from
    its own bits: the row keeps its relative accuracy."""
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(21)
    A = inputs.complex_normal(rng, (40, 200))
    A[7] *= 1e-310
    A[8] *= 5e-322
    B = inputs.complex_normal(rng, (200, 30))
    out = fg.zgemm_oz(A, B)
    assert np.all(np.isfinite(out))
    ref = A @ B
    for i in (7, 8):
        ra = np.max(np.maximum(np.abs(A[i].real), np.abs(A[i].imag)))
        cb = np.max(np.maximum(np.abs(B.real), np.abs(B.imag)), axis=0)
        # subnormal entries carry fewer bits than the digits: the bound is
        # the larger of the method's and the entries' own spacing
        bound = 2.0 ** -45 * 200 * ra * cb + 200 * 5e-324 * cb
        assert np.all(np.abs(out[i] - ref[i]) <= bound)
    _check(np.delete(A, [7, 8], 0), B, np.zeros((38, 30)), 1.0, 0.0, np.delete(out, [7, 8], 0))


def test_zgemm_oz_non_finite_rows_and_columns_are_nan():
    """An Inf or NaN in row i of A or column j of B makes row i / column j of
    the product non-finite (NaN), as in complex128; every other entry is
    unaffected."""
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(23)
    A = inputs.complex_normal(rng, (60, 120))
    B = inputs.complex_normal(rng, (120, 50))
    A[3, 10] = np.nan
    A[11, 0] = complex(np.inf, 0.0)
    B[5, 7] = complex(0.0, -np.inf)
    out = fg.zgemm_oz(A, B)
    bad_r, bad_c = [3, 11], [7]
    assert np.all(np.isnan(out[bad_r, :]))
    assert np.all(np.isnan(out[:, bad_c]))
    keep_r = [i for i in range(60) if i not in bad_r]
    keep_c = [j for j in range(50) if j not in bad_c]
    _check(A[keep_r], B[:, keep_c], np.zeros((58, 49)), 1.0, 0.0, out[np.ix_(keep_r, keep_c)])
