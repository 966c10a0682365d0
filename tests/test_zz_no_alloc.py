"""The eigensolve entry point that allocates no device memory.

Some callers cannot call cudaMalloc -- for instance code running while a
CUDA graph is being captured, or a process whose device memory is owned by
another allocator -- so feast_zqz_batched_noalloc takes its scratch from a
fixed array inside the library instead of from the caller.  This test
checks, through the C ABI, that it returns the same eigenpairs as
feast_zqz_batched (the entry point that takes caller scratch) on two calls
in a row (the second call reuses the shared array left over from the
first), and that requests beyond its fixed capacity are refused.  The file
is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_1404_1768_gb300 import inputs

pytestmark = pytest.mark.gpu


def _pencils(rng, m, batch):
    As = [inputs.complex_normal(rng, (m, m)) for _ in range(batch)]
    Bs = [np.triu(inputs.complex_normal(rng, (m, m))) + 2.0 * np.eye(m) for _ in range(batch)]
    return As, Bs


def test_noalloc_matches_allocating_entry_point_twice():
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(2024)
    for m, batch in ((48, 3), (64, 5)):
        As, Bs = _pencils(rng, m, batch)
        al, be, Vs, fail = fg.zqz_batched(As, Bs)
        assert fail == 0
        for call in range(2):
            al2, be2, Vs2, fail2 = fg.zqz_batched_noalloc(As, Bs)
            assert fail2 == 0
            for b in range(batch):
                lam, lam2 = al[b] / be[b], al2[b] / be2[b]
                scale = max(1.0, np.abs(lam).max())
                # same kernel, same inputs: the same eigenvalues in the same order
                np.testing.assert_allclose(lam2, lam, rtol=0, atol=1e-12 * scale)
                for i in range(m):
                    v, v2 = Vs[b][:, i], Vs2[b][:, i]
                    # unit vectors, equal up to a phase
                    ph = np.vdot(v2, v)
                    assert abs(abs(ph) - 1.0) < 1e-10, (m, b, i, call)


def test_noalloc_rejects_requests_beyond_its_capacity():
    import paper_1404_1768_gb300 as fg
    rng = np.random.default_rng(7)
    As, Bs = _pencils(rng, 65, 1)             # m > 64
    with pytest.raises(fg.FeastError) as ei:
        fg.zqz_batched_noalloc(As, Bs)
    assert ei.value.status == -1
    As, Bs = _pencils(rng, 64, 65)            # 65 * 64 * 64 > 262144 elements
    with pytest.raises(fg.FeastError) as ei:
        fg.zqz_batched_noalloc(As, Bs)
    assert ei.value.status == -1
