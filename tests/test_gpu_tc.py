"""The tcgen05 complex64 GEMM (TF32 inputs, head/tail split, FP32
accumulation in tensor memory) against a complex128 product.  The split
makes the product ~FP32-accurate: the bound is a few units of 2^-22 times
sqrt(k) relative to |A| |X|."""
import numpy as np
import pytest

from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,batch", [(64, 128, 32, 1), (200, 70, 32, 3), (1000, 300, 96, 2),
                                         (33, 5, 7, 1),
                                         # more 256 x 256 tiles than clusters: every cluster takes
                                         # several tiles, both tensor-memory accumulators in turn
                                         (2048, 1280, 256, 2), (1536, 1000, 256, 3),
                                         # ragged rows and columns in the last tiles, K not a
                                         # multiple of 16
                                         (700, 600, 250, 4)])
def test_tc_cgemm_matches_reference(m, n, k, batch):
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(m + n + k)
    A = [inputs.complex_normal(rng, (m, k)).astype(np.complex64) for _ in range(batch)]
    X = [inputs.complex_normal(rng, (k, n)).astype(np.complex64) for _ in range(batch)]
    C0 = [inputs.complex_normal(rng, (m, n)).astype(np.complex64) for _ in range(batch)]
    out = fg.cgemm_tc(A, X, C0, alpha=-1.0, beta=1.0)
    for b in range(batch):
        ref = C0[b].astype(np.complex128) - A[b].astype(np.complex128) @ X[b].astype(np.complex128)
        scale = np.abs(A[b]).astype(np.float64) @ np.abs(X[b]).astype(np.float64) + np.abs(C0[b])
        err = np.max(np.abs(out[b] - ref) / scale)
        assert err < 2e-6 * max(1.0, np.sqrt(k) / 4), err
