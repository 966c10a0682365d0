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


# A fresh process that holds no torch state: it reaches the GPU through the
# CUDA driver API alone (ctypes) and calls the library's C ABI, so the CUDA
# context that is current can be changed between calls.
_CTX_SCRIPT = r'''
import ctypes as C, sys
import numpy as np

cu = C.CDLL("libcuda.so.1")
lib = C.CDLL(sys.argv[1])
P = C.c_void_p
lib.feast_zqz_batched.argtypes = [C.c_int, C.c_int, P, P, P, P, P, P, P, P]
lib.feast_zqz_batched_noalloc.argtypes = [C.c_int, C.c_int, P, P, P, P, P, P, P]
lib.feast_zqz_work_bytes.argtypes = [C.c_int, C.c_int]
lib.feast_zqz_work_bytes.restype = C.c_size_t


def chk(r, what):
    if r != 0:
        raise SystemExit(f"{what}: status {r}")


chk(cu.cuInit(0), "cuInit")
dev = C.c_int()
chk(cu.cuDeviceGet(C.byref(dev), 0), "cuDeviceGet")
m, batch = 48, 3
rng = np.random.default_rng(99)
A = (rng.standard_normal((batch, m, m)) + 1j * rng.standard_normal((batch, m, m))) / np.sqrt(2)
B = np.triu((rng.standard_normal((batch, m, m)) + 1j * rng.standard_normal((batch, m, m))) / np.sqrt(2))
B = B + 2.0 * np.eye(m)
# pencil b as a column-major m x m block
Ah = np.ascontiguousarray(np.transpose(A, (0, 2, 1)))
Bh = np.ascontiguousarray(np.transpose(B, (0, 2, 1)))


def run(noalloc):
    held = []

    def alloc(nbytes):
        p = C.c_uint64()
        chk(cu.cuMemAlloc_v2(C.byref(p), C.c_size_t(max(int(nbytes), 16))), "cuMemAlloc")
        held.append(p.value)
        return p.value

    dA, dB = alloc(Ah.nbytes), alloc(Bh.nbytes)
    dal, dbe, dV, dst = alloc(16 * m * batch), alloc(16 * m * batch), alloc(16 * m * m * batch), alloc(8)
    chk(cu.cuMemcpyHtoD_v2(C.c_uint64(dA), Ah.ctypes.data_as(P), C.c_size_t(Ah.nbytes)), "HtoD")
    chk(cu.cuMemcpyHtoD_v2(C.c_uint64(dB), Bh.ctypes.data_as(P), C.c_size_t(Bh.nbytes)), "HtoD")
    if noalloc:
        st = lib.feast_zqz_batched_noalloc(m, batch, dA, dB, dal, dbe, dV, dst, None)
    else:
        work = alloc(lib.feast_zqz_work_bytes(m, batch))
        st = lib.feast_zqz_batched(m, batch, dA, dB, dal, dbe, dV, work, dst, None)
    chk(st, "feast call")
    chk(cu.cuCtxSynchronize(), "cuCtxSynchronize")
    al = np.zeros(m * batch, np.complex128)
    be = np.zeros(m * batch, np.complex128)
    status = np.zeros(2, np.int32)
    chk(cu.cuMemcpyDtoH_v2(al.ctypes.data_as(P), C.c_uint64(dal), C.c_size_t(al.nbytes)), "DtoH")
    chk(cu.cuMemcpyDtoH_v2(be.ctypes.data_as(P), C.c_uint64(dbe), C.c_size_t(be.nbytes)), "DtoH")
    chk(cu.cuMemcpyDtoH_v2(status.ctypes.data_as(P), C.c_uint64(dst), C.c_size_t(8)), "DtoH")
    for p in held:
        chk(cu.cuMemFree_v2(C.c_uint64(p)), "cuMemFree")
    if status[0] != 0 or status[1] != 0:
        raise SystemExit(f"kernel status {status.tolist()}")
    return al / be


pctx = P()
chk(cu.cuDevicePrimaryCtxRetain(C.byref(pctx), dev), "cuDevicePrimaryCtxRetain")
chk(cu.cuCtxSetCurrent(pctx), "cuCtxSetCurrent")
ref = run(False)                      # the allocating entry point, primary context
lams = [run(True)]                    # primary context: first lookup
for _ in range(2):                    # two contexts made and destroyed in turn
    ctx = P()
    chk(cu.cuCtxCreate_v2(C.byref(ctx), 0, dev), "cuCtxCreate")
    lams.append(run(True))
    lams.append(run(True))
    chk(cu.cuCtxDestroy_v2(ctx), "cuCtxDestroy")
chk(cu.cuCtxSetCurrent(pctx), "cuCtxSetCurrent")
lams.append(run(True))                # back in the primary context
chk(cu.cuDevicePrimaryCtxRelease_v2(dev), "cuDevicePrimaryCtxRelease")
scale = max(1.0, float(np.abs(ref).max()))
worst = max(float(np.abs(l - ref).max()) for l in lams)
print("worst", worst, "scale", scale)
raise SystemExit(0 if worst <= 1e-12 * scale else 3)
'''


def test_noalloc_follows_the_current_context():
    """The scratch array has one device address per CUDA context.  Calls made
    in the primary context, then in two contexts created and destroyed in
    turn (the second may reuse the first one's handle), then in the primary
    context again must each use the address of the context that is current:
    every call returns the allocating entry point's eigenvalues."""
    import subprocess
    import sys

    import paper_1404_1768_gb300 as fg
    fg.load()
    r = subprocess.run([sys.executable, "-c", _CTX_SCRIPT, fg.lib_path()], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
