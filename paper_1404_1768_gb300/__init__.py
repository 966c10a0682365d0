"""GB300-native oblique-projection FEAST (Yin, Chan & Yeung) for A x = lambda B x.

Thin Python binding over the C ABI in ``include/feast_gb300.h``: it only
marshals arguments (torch device tensors -> raw pointers, structs, the
current CUDA stream).  Every step of the method runs in the CUDA library
``_build/libfeast_gb300.so`` (sm_103a); if that library is missing the
binding raises -- there is no CPU fallback.

Layout: matrices cross the boundary as column-major complex128 device
buffers.  ``to_device_colmajor`` / ``from_device_colmajor`` convert numpy
arrays of any order to and from that layout.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Feast", "load", "lib_path", "to_device_colmajor", "from_device_colmajor",
           "zgetrf_batched", "zgetrs_batched", "zqz_batched", "FeastError", "shard_nodes", "dist_collective",
           "BatchSchedule"]

FEAST_DENSE, FEAST_BANDED = 0, 1
FEAST_CIRCLE, FEAST_ELLIPSE = 0, 1
FEAST_TRAPEZOID, FEAST_GAUSS_LEGENDRE = 0, 1
FEAST_FP64, FEAST_C64_REFINE = 0, 1
FEAST_OBLIQUE, FEAST_RAYLEIGH_RITZ = 0, 1
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ESINGULAR", -5: "ENONFINITE",
          -6: "ETIMEOUT", -7: "ENOCONV", -8: "EDONE"}


class FeastError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)} ({status})"
        super().__init__(msg + (f" [{detail}]" if detail else ""))


class Pencil(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int64), ("A", C.c_void_p), ("B", C.c_void_p),
                ("ld", C.c_int64), ("kl", C.c_int64), ("ku", C.c_int64),
                ("b_is_identity", C.c_int)]


class Contour(C.Structure):
    _fields_ = [("kind", C.c_int), ("center_re", C.c_double), ("center_im", C.c_double),
                ("a", C.c_double), ("b", C.c_double), ("q", C.c_int), ("rule", C.c_int)]


FEAST_COLL_SUM, FEAST_COLL_BCAST = 0, 1
# int (*)(void *user, int op, void *buf, int64_t ndoubles, void *stream)
COLLECTIVE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("m0", C.c_int), ("Y0", C.c_void_p), ("eps", C.c_double), ("eta", C.c_double),
                ("max_iter", C.c_int), ("prec", C.c_int), ("max_refine", C.c_int),
                ("refine_tol", C.c_double), ("stream", C.c_void_p), ("no_stop", C.c_int),
                ("converged_only", C.c_int), ("projection", C.c_int),
                ("node_begin", C.c_int), ("node_end", C.c_int), ("collective", COLLECTIVE_FN),
                ("collective_user", C.c_void_p), ("collective_buf", C.c_void_p)]


class BatchItem(C.Structure):
    _fields_ = [("status", C.c_int), ("flag", C.c_int), ("count", C.c_int), ("k", C.c_int),
                ("err", C.c_double), ("ms_setup", C.c_double), ("ms_pass", C.c_double),
                ("ms_solve", C.c_double), ("ms_qz", C.c_double)]


class IterInfo(C.Structure):
    _fields_ = [("k", C.c_int), ("count", C.c_int), ("flag", C.c_int), ("err", C.c_double),
                ("ms_lu", C.c_double), ("ms_solve", C.c_double), ("ms_refine", C.c_double),
                ("ms_qr", C.c_double), ("ms_proj", C.c_double), ("ms_qz", C.c_double),
                ("refine_sweeps_max", C.c_int), ("bad_node", C.c_int), ("qz_sweeps", C.c_int),
                ("qz_phases", C.c_int), ("qz_warm", C.c_int), ("qz_rows", C.c_int),
                ("qz_warm_resid", C.c_double), ("qz_warm_k", C.c_int),
                ("ms_warm_gemm", C.c_double), ("warm_gemm_flop", C.c_double),
                ("ms_tc_gemm", C.c_double), ("tc_gemm_flop", C.c_double), ("qz_cold_fp32", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_lock = threading.Lock()

# every symbol declared in include/feast_gb300.h
EXPORTS = ["feast_workspace_size", "feast_setup", "feast_iterate", "feast_eigs", "feast_get",
           "feast_filter", "feast_set_subspace", "feast_destroy", "feast_strerror",
           "feast_zgetrf_batched", "feast_zgetrs_batched", "feast_zqz_batched",
           "feast_zqz_work_bytes", "feast_kernel_launches", "feast_last_cuda_error", "feast_zqz_batched_noalloc",
           "feast_batch_workspace_size", "feast_solve_batch", "feast_cgemm_tc_scratch_bytes",
           "feast_cgemm_tc", "feast_zgemm_oz_work_bytes", "feast_zgemm_oz", "feast_grad_abs2",
           "feast_search", "feast_cirr", "feast_csr_rcm", "feast_csr_to_band"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if allowed and missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path}")
            _build.build()
        lib = C.CDLL(path)
        P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
        lib.feast_workspace_size.argtypes = [C.POINTER(Pencil), C.POINTER(Contour), C.POINTER(Options),
                                             C.POINTER(C.c_size_t)]
        lib.feast_setup.argtypes = [C.POINTER(P), C.POINTER(Pencil), C.POINTER(Contour),
                                    C.POINTER(Options), P, C.c_size_t, C.POINTER(IterInfo)]
        lib.feast_iterate.argtypes = [P, C.POINTER(IterInfo)]
        lib.feast_eigs.argtypes = [P, C.POINTER(I), P, P, I64, P, C.POINTER(D), C.POINTER(I)]
        lib.feast_get.argtypes = [P, I, P]
        lib.feast_filter.argtypes = [P, P, P]
        lib.feast_set_subspace.argtypes = [P, P]
        lib.feast_search.argtypes = [P, P, C.c_int, C.c_double, C.c_int, C.c_double, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int)]
        lib.feast_cirr.argtypes = [P, P, C.c_int, C.c_int, C.POINTER(IterInfo)]
        lib.feast_csr_rcm.argtypes = [I64, P, P, P, P, P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.feast_csr_to_band.argtypes = [I64, P, P, P, P, I64, I64, P, P, P]
        lib.feast_destroy.argtypes = [P]
        lib.feast_destroy.restype = None
        lib.feast_strerror.argtypes = [I]
        lib.feast_strerror.restype = C.c_char_p
        lib.feast_zgetrf_batched.argtypes = [I64, I, P, I64, I64, P, P, P]
        lib.feast_zgetrs_batched.argtypes = [I64, I64, I, P, I64, I64, P, P, I64, I64, P]
        lib.feast_zqz_batched.argtypes = [I, I, P, P, P, P, P, P, P, P]
        lib.feast_zqz_work_bytes.argtypes = [I, I]
        lib.feast_zqz_work_bytes.restype = C.c_size_t
        lib.feast_zqz_batched_noalloc.argtypes = [I, I, P, P, P, P, P, P, P]
        lib.feast_batch_workspace_size.argtypes = [I, C.POINTER(Pencil), C.POINTER(Contour),
                                                   C.POINTER(Options), I]
        lib.feast_batch_workspace_size.restype = C.c_size_t
        lib.feast_solve_batch.argtypes = [I, C.POINTER(Pencil), C.POINTER(Contour), C.POINTER(Options),
                                          P, C.c_size_t, I, C.POINTER(BatchItem), P, P]
        lib.feast_cgemm_tc_scratch_bytes.argtypes = [I64, I64, I64, I]
        lib.feast_cgemm_tc_scratch_bytes.restype = C.c_size_t
        F = C.c_float
        lib.feast_cgemm_tc.argtypes = [I64, I64, I64, F, F, P, I64, I64, P, I64, I64, F, F, P, I64, I64,
                                       I, P, C.c_size_t, P, P]
        lib.feast_grad_abs2.argtypes = [P, P, P, P, I64, C.POINTER(D), C.POINTER(I)]
        lib.feast_zgemm_oz_work_bytes.argtypes = [I64, I64, I64]
        lib.feast_zgemm_oz_work_bytes.restype = C.c_size_t
        lib.feast_zgemm_oz.argtypes = [I64, I64, I64, D, D, P, I64, P, I64, D, D, P, I64, P, C.c_size_t, P, P]
        lib.feast_kernel_launches.argtypes = []
        lib.feast_kernel_launches.restype = C.c_ulonglong
        lib.feast_last_cuda_error.restype = C.c_char_p
        _lib = lib
        return lib


def kernel_launches() -> int:
    """Kernels launched by the CUDA library in this process so far."""
    return int(load().feast_kernel_launches())


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def to_device_colmajor(x, device="cuda", dtype=None):
    """numpy / torch (rows x cols) -> flat device tensor in column-major order."""
    torch = _torch()
    if isinstance(x, torch.Tensor):
        t = x.resolve_conj().to(device)
        if dtype is not None:
            t = t.to(dtype)
        if t.dim() == 1:
            return t.contiguous()
        return t.t().contiguous().reshape(-1)
    a = np.asarray(x)
    if dtype is None and np.iscomplexobj(a):
        a = a.astype(np.complex128)
    flat = np.ascontiguousarray(a.ravel(order="F")) if a.ndim == 2 else np.ascontiguousarray(a)
    t = torch.from_numpy(flat).to(device)
    if dtype is not None:
        t = t.to(dtype)
    return t


def from_device_colmajor(t, rows: int, cols: int) -> np.ndarray:
    """flat column-major device tensor -> numpy (rows x cols)."""
    a = t.detach().reshape(-1)[: rows * cols].cpu().numpy()
    return a.reshape(cols, rows).T


def _check(st: int, where: str):
    if st != 0:
        detail = ""
        if st in (-3, -6) and _lib is not None:
            detail = (_lib.feast_last_cuda_error() or b"").decode()
        raise FeastError(st, where, detail)


def shard_nodes(q: int, world: int, rank: int):
    """The contiguous range [j0, j1) of the q quadrature nodes that rank owns
    when world ranks share one contour (sizes differ by at most one)."""
    if not (0 <= rank < world) or q < world:
        raise ValueError("need 0 <= rank < world <= q")
    base, extra = divmod(q, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def dist_collective(group=None):
    """The collective hook of a node-sharded run over torch.distributed:
    ``fn(op, buf, stream)`` sums buf over the ranks (FEAST_COLL_SUM) or
    copies rank 0's buf to every rank (FEAST_COLL_BCAST), in place.  With a
    NCCL group the collective is issued on the library's stream (ordered
    after the work that wrote buf, and before what follows); with a CPU
    group (gloo) the stream is synchronised, buf goes through host memory
    and is copied back before the hook returns."""
    import torch.distributed as dist
    torch = _torch()

    def fn(op, buf, stream):
        backend = dist.get_backend(group)
        if backend == "nccl":
            ext = torch.cuda.ExternalStream(stream, device=buf.device) if stream else None
            with torch.cuda.stream(ext) if ext is not None else _nullctx():
                if op == FEAST_COLL_SUM:
                    dist.all_reduce(buf, group=group)
                else:
                    dist.broadcast(buf, src=0, group=group)
            return
        if buf.is_cuda:
            torch.cuda.synchronize(buf.device)
        h = buf.cpu()
        if op == FEAST_COLL_SUM:
            dist.all_reduce(h, group=group)
        else:
            dist.broadcast(h, src=0, group=group)
        buf.copy_(h)
        if buf.is_cuda:
            torch.cuda.synchronize(buf.device)
    return fn


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


class Feast:
    """GFEAST on the GPU (lines 1-3 at construction, one pass of lines 5-17 per
    ``iterate``).  A, B, Y: numpy arrays or torch tensors (rows x cols); they
    are copied to column-major complex128 device buffers.

    Node-sharded runs (one rank per GPU): ``node_range=(j0, j1)`` makes this
    context own quadrature nodes j0..j1-1 only, and ``collective(op, buf,
    stream)`` (e.g. ``dist_collective()``) combines the ranks' partial sums
    and stopping flags; every rank constructs its Feast and calls
    ``iterate`` in step."""

    def __init__(self, A, B, Y, *, contour_kind=0, rule=0, q=16, center=0j, a=1.0, b=0.0,
                 eps=1e-12, eta=1e-3, max_iter=50, prec=FEAST_FP64, no_stop=False, kind=0, kl=0,
                 ku=0, b_identity=False, device="cuda", stream=None, max_refine=5,
                 refine_tol=1e-14, converged_only=False, projection=0, node_range=None, collective=None):
        torch = _torch()
        self._lib = load()
        self.device = torch.device(device)
        self.stream = stream
        self._A = to_device_colmajor(A, device)
        self._B = to_device_colmajor(B, device) if (B is not None and not b_identity) else None
        Yshape = (np.asarray(Y).shape if not isinstance(Y, torch.Tensor) else tuple(Y.shape))
        self.n, self.m0 = int(Yshape[0]), int(Yshape[1])
        self.q = int(q)
        self._Y = to_device_colmajor(Y, device)
        ld = self.n if kind == FEAST_DENSE else (kl + ku + 1)
        self._pencil = Pencil(kind, self.n, self._A.data_ptr(),
                              self._B.data_ptr() if self._B is not None else None,
                              ld, kl, ku, int(bool(b_identity)))
        self._contour = Contour(contour_kind, float(center.real), float(center.imag), float(a),
                                float(b if contour_kind == FEAST_ELLIPSE else a), int(q), int(rule))
        self._opts = Options(self.m0, self._Y.data_ptr(), float(eps), float(eta), int(max_iter),
                             int(prec), int(max_refine), float(refine_tol),
                             _stream_ptr(stream), int(bool(no_stop)), int(bool(converged_only)),
                             int(projection))
        self.node_range = None
        if node_range is not None:
            if collective is None:
                raise ValueError("a node range needs a collective hook")
            j0, j1 = int(node_range[0]), int(node_range[1])
            self.node_range = (j0, j1)
            # one n x m0 complex128 block, as doubles (caller-owned by this object)
            self._coll_buf = torch.empty(2 * self.n * self.m0, dtype=torch.float64, device=self.device)
            buf = self._coll_buf
            user_fn = collective

            def _hook(user, op, ptr, nd, strm):
                try:
                    user_fn(int(op), buf[: int(nd)], int(strm or 0))
                    return 0
                except Exception as ex:  # no exception may cross the C boundary
                    self._coll_error = ex
                    return 1

            self._coll_cb = COLLECTIVE_FN(_hook)
            self._opts.node_begin, self._opts.node_end = j0, j1
            self._opts.collective = self._coll_cb
            self._opts.collective_buf = buf.data_ptr()
        self._coll_error = None
        nbytes = C.c_size_t(0)
        _check(self._lib.feast_workspace_size(C.byref(self._pencil), C.byref(self._contour),
                                              C.byref(self._opts), C.byref(nbytes)),
               "feast_workspace_size")
        self.workspace_bytes = int(nbytes.value)
        self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        self._ctx = C.c_void_p()
        info = IterInfo()
        st = self._lib.feast_setup(C.byref(self._ctx), C.byref(self._pencil), C.byref(self._contour),
                                   C.byref(self._opts), self._ws.data_ptr(), self.workspace_bytes,
                                   C.byref(info))
        self.setup_info = info.as_dict()
        if st != 0 and self._coll_error is not None:
            raise FeastError(st, "feast_setup", f"collective hook: {self._coll_error!r}")
        _check(st, "feast_setup")

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.feast_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self) -> dict:
        info = IterInfo()
        st = self._lib.feast_iterate(self._ctx, C.byref(info))
        if st != 0 and self._coll_error is not None:
            raise FeastError(st, "feast_iterate", f"collective hook: {self._coll_error!r}")
        _check(st, "feast_iterate")
        return info.as_dict()

    def run(self) -> list:
        hist = []
        while True:
            it = self.iterate()
            hist.append(it)
            if it["flag"] != 2:
                return hist

    def eigs(self, want_vectors: bool = True) -> dict:
        torch = _torch()
        cnt, flag = C.c_int(), C.c_int()
        err = C.c_double()
        lam = np.zeros(2 * self.m0)
        res = np.zeros(self.m0)
        X = torch.zeros(self.n * self.m0, dtype=torch.complex128, device=self.device)
        _check(self._lib.feast_eigs(self._ctx, C.byref(cnt), lam.ctypes.data,
                                    X.data_ptr() if want_vectors else None, self.n,
                                    res.ctypes.data, C.byref(err), C.byref(flag)), "feast_eigs")
        c = cnt.value
        out = dict(count=c, lam=(lam[0:2 * c:2] + 1j * lam[1:2 * c:2]), res=res[:c].copy(),
                   err=err.value, flag=flag.value)
        if want_vectors:
            out["X"] = from_device_colmajor(X, self.n, self.m0)[:, :c]
        return out

    _GET = dict(U1=(0, "nm"), U2=(1, "nm"), R2=(2, "mm"), At=(3, "mm"), Bt=(4, "mm"),
                X=(5, "nm"), lam=(6, "m"), AU1=(7, "nm"), BU1=(8, "nm"), z=(9, "q"),
                w=(10, "q"), res=(11, "m_f64"), sel=(12, "m_i32"))

    def get(self, what: str):
        torch = _torch()
        idx, shape = self._GET[what]
        n, m, q = self.n, self.m0, self.q
        if shape == "m_f64":
            buf = torch.zeros(m, dtype=torch.float64, device=self.device)
        elif shape == "m_i32":
            buf = torch.zeros(m, dtype=torch.int32, device=self.device)
        else:
            cnt = dict(nm=n * m, mm=m * m, m=m, q=q)[shape]
            buf = torch.zeros(cnt, dtype=torch.complex128, device=self.device)
        _check(self._lib.feast_get(self._ctx, idx, buf.data_ptr()), "feast_get")
        torch.cuda.current_stream().synchronize()
        if shape == "nm":
            return from_device_colmajor(buf, n, m)
        if shape == "mm":
            return from_device_colmajor(buf, m, m)
        a = buf.cpu().numpy()
        return a.astype(bool) if shape == "m_i32" else a

    def filter(self, V) -> np.ndarray:
        torch = _torch()
        Vd = to_device_colmajor(V, self.device)
        Ud = torch.zeros(self.n * self.m0, dtype=torch.complex128, device=self.device)
        _check(self._lib.feast_filter(self._ctx, Vd.data_ptr(), Ud.data_ptr()), "feast_filter")
        torch.cuda.current_stream().synchronize()
        return from_device_colmajor(Ud, self.n, self.m0)

    def grad_abs2(self, left: "Feast"):
        """L = sum over the inside eigenvalues of |lambda|^2 and its gradients
        (G_A, G_B) as device tensors (n x n, row-major views of column-major
        storage transposed back), from this finished run and a finished run
        on the conjugate-transposed pencil (``left``)."""
        torch = _torch()
        n = self.n
        gA = torch.empty(n * n, dtype=torch.complex128, device=self.device)
        gB = torch.empty(n * n, dtype=torch.complex128, device=self.device)
        L, cnt = C.c_double(), C.c_int()
        _check(self._lib.feast_grad_abs2(self._ctx, left._ctx, gA.data_ptr(), gB.data_ptr(), n, C.byref(L),
                                         C.byref(cnt)), "feast_grad_abs2")
        return L.value, gA.view(n, n).t(), gB.view(n, n).t(), cnt.value

    def search(self, Ypool, alpha: float, p: int, rank_tol: float) -> dict:
        """SEARCH (Section 4.1): Ypool (n x npool) supplies the random columns
        in order.  On return the context's width is t and the iteration starts
        from the search's basis.  Returns dict(t, s0)."""
        Yd = to_device_colmajor(Ypool, self.device)
        npool = int(np.asarray(Ypool).shape[1]) if not hasattr(Ypool, "shape") else int(Ypool.shape[1])
        t, s0 = C.c_int(0), C.c_int(0)
        _check(self._lib.feast_search(self._ctx, Yd.data_ptr(), npool, float(alpha), int(p), float(rank_tol),
                                      C.byref(t), C.byref(s0)), "feast_search")
        _torch().cuda.current_stream().synchronize()
        self.m0 = t.value
        return dict(t=t.value, s0=s0.value)

    def cirr(self, Y, g: int) -> dict:
        """Block CIRR (Section 2.1) on this context (set up with
        projection=FEAST_RAYLEIGH_RITZ): Y (n x h) random columns, g moments,
        t = h g <= m0.  Returns the pass report; the selected pairs are read
        with eigs()."""
        h = int(Y.shape[1])
        Yd = to_device_colmajor(Y, self.device, _torch().complex128)
        info = IterInfo()
        _check(self._lib.feast_cirr(self._ctx, Yd.data_ptr(), h, int(g), C.byref(info)), "feast_cirr")
        self.m0 = h * int(g)
        return info.as_dict()

    def set_subspace(self, U1):
        Ud = to_device_colmajor(U1, self.device)
        _check(self._lib.feast_set_subspace(self._ctx, Ud.data_ptr()), "feast_set_subspace")
        _torch().cuda.current_stream().synchronize()


# --------------------------------------------------------------- standalone kernels
def zgetrf_batched(M_list, stream=None):
    """LU of each n x n matrix in M_list.  Returns (factors list, pivots
    (batch x n), info)."""
    torch = _torch()
    lib = load()
    n = np.asarray(M_list[0]).shape[0]
    batch = len(M_list)
    buf = torch.cat([to_device_colmajor(M) for M in M_list])
    piv = torch.zeros(batch * n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(lib.feast_zgetrf_batched(n, batch, buf.data_ptr(), n, n * n, piv.data_ptr(),
                                    info.data_ptr(), _stream_ptr(stream)), "feast_zgetrf_batched")
    torch.cuda.current_stream().synchronize()
    facs = [from_device_colmajor(buf[b * n * n:(b + 1) * n * n], n, n) for b in range(batch)]
    return facs, piv.cpu().numpy().reshape(batch, n), int(info.item())


def zgetrs_batched(F_list, piv, R_list, stream=None):
    torch = _torch()
    lib = load()
    n = np.asarray(F_list[0]).shape[0]
    nrhs = np.asarray(R_list[0]).shape[1]
    batch = len(F_list)
    fb = torch.cat([to_device_colmajor(F) for F in F_list])
    xb = torch.cat([to_device_colmajor(R) for R in R_list])
    pv = torch.from_numpy(np.ascontiguousarray(piv, dtype=np.int32).ravel()).cuda()
    _check(lib.feast_zgetrs_batched(n, nrhs, batch, fb.data_ptr(), n, n * n, pv.data_ptr(),
                                    xb.data_ptr(), n, n * nrhs, _stream_ptr(stream)),
           "feast_zgetrs_batched")
    torch.cuda.current_stream().synchronize()
    return [from_device_colmajor(xb[b * n * nrhs:(b + 1) * n * nrhs], n, nrhs) for b in range(batch)]


def zqz_batched(A_list, B_list, stream=None):
    """Generalized eigenpairs of each (A, B) (B upper triangular).  Returns
    alpha (batch x m), beta, V list, fail count."""
    torch = _torch()
    lib = load()
    m = np.asarray(A_list[0]).shape[0]
    batch = len(A_list)
    ab = torch.cat([to_device_colmajor(A) for A in A_list])
    bb = torch.cat([to_device_colmajor(B) for B in B_list])
    al = torch.zeros(batch * m, dtype=torch.complex128, device="cuda")
    be = torch.zeros_like(al)
    V = torch.zeros(batch * m * m, dtype=torch.complex128, device="cuda")
    work = torch.zeros(int(lib.feast_zqz_work_bytes(m, batch)), dtype=torch.uint8, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    _check(lib.feast_zqz_batched(m, batch, ab.data_ptr(), bb.data_ptr(), al.data_ptr(),
                                 be.data_ptr(), V.data_ptr(), work.data_ptr(), st.data_ptr(),
                                 _stream_ptr(stream)), "feast_zqz_batched")
    torch.cuda.current_stream().synchronize()
    Vs = [from_device_colmajor(V[b * m * m:(b + 1) * m * m], m, m) for b in range(batch)]
    stv = st.cpu().numpy()
    if stv[1]:
        raise FeastError(-6, "feast_zqz_batched")
    return (al.cpu().numpy().reshape(batch, m), be.cpu().numpy().reshape(batch, m), Vs,
            int(stv[0]))


def zqz_batched_noalloc(A_list, B_list, stream=None):
    """zqz_batched through the entry point that allocates nothing on the
    device (scratch from the library's fixed array; m <= 64)."""
    torch = _torch()
    lib = load()
    m = np.asarray(A_list[0]).shape[0]
    batch = len(A_list)
    ab = torch.cat([to_device_colmajor(A) for A in A_list])
    bb = torch.cat([to_device_colmajor(B) for B in B_list])
    al = torch.zeros(batch * m, dtype=torch.complex128, device="cuda")
    be = torch.zeros_like(al)
    V = torch.zeros(batch * m * m, dtype=torch.complex128, device="cuda")
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    _check(lib.feast_zqz_batched_noalloc(m, batch, ab.data_ptr(), bb.data_ptr(), al.data_ptr(),
                                         be.data_ptr(), V.data_ptr(), st.data_ptr(),
                                         _stream_ptr(stream)), "feast_zqz_batched_noalloc")
    torch.cuda.current_stream().synchronize()
    Vs = [from_device_colmajor(V[b * m * m:(b + 1) * m * m], m, m) for b in range(batch)]
    stv = st.cpu().numpy()
    return (al.cpu().numpy().reshape(batch, m), be.cpu().numpy().reshape(batch, m), Vs,
            int(stv[0]))


class BatchSchedule:
    """Schedule autotuner of solve_batch: the number of pencils solved
    concurrently (one worker thread and CUDA stream each) is picked by
    measurement.  ``next()`` gives the candidate to time next (each once, in
    order), then the fastest; ``record(nworkers, seconds)`` enters a timing
    of the same batch.  The small projected eigensolves are latency-bound
    one-CTA kernels, so how many pencils share the GPU decides the
    throughput; the best count depends on the batch's size mix."""

    def __init__(self, candidates=(16, 32, 64)):
        self.candidates = [int(c) for c in candidates]
        self.times = {}

    def next(self) -> int:
        for c in self.candidates:
            if c not in self.times:
                return c
        return self.best

    def record(self, nworkers: int, seconds: float):
        self.times[int(nworkers)] = min(float(seconds), self.times.get(int(nworkers), float("inf")))

    @property
    def best(self) -> int:
        if not self.times:
            return self.candidates[0]
        return min(self.times, key=lambda c: self.times[c])


def solve_batch(problems, nworkers: int = 16, device="cuda"):
    """Run GFEAST on many independent dense pencils at once (uneven sizes).

    problems: list of dicts with keys A, B, Y (numpy, rows x cols) and the
    contour / tolerance keywords of Feast (contour_kind, rule, q, center, a,
    b, eps, eta, max_iter, prec, refine_tol, max_refine).  Returns a list of
    dicts (status, flag, count, k, err, lam, res)."""
    torch = _torch()
    lib = load()
    cnt = len(problems)
    keep = []
    P = (Pencil * cnt)()
    Cn = (Contour * cnt)()
    O = (Options * cnt)()
    for i, pr in enumerate(problems):
        A = to_device_colmajor(pr["A"], device)
        B = to_device_colmajor(pr["B"], device)
        Y = to_device_colmajor(pr["Y"], device)
        keep += [A, B, Y]
        n, m0 = np.asarray(pr["Y"]).shape
        P[i] = Pencil(0, n, A.data_ptr(), B.data_ptr(), n, 0, 0, 0)
        ck = pr.get("contour_kind", 0)
        ctr = complex(pr.get("center", 0j))
        a = float(pr.get("a", 1.0))
        Cn[i] = Contour(ck, ctr.real, ctr.imag, a, float(pr.get("b", a)), int(pr.get("q", 16)),
                        int(pr.get("rule", 0)))
        O[i] = Options(m0, Y.data_ptr(), float(pr.get("eps", 1e-12)), float(pr.get("eta", 1e-3)),
                       int(pr.get("max_iter", 50)), int(pr.get("prec", 0)),
                       int(pr.get("max_refine", 5)), float(pr.get("refine_tol", 1e-14)), None, 0, 0, 0,
                       0, 0)
    nbytes = int(lib.feast_batch_workspace_size(cnt, P, Cn, O, nworkers))
    if nbytes == 0:
        raise FeastError(-1, "feast_batch_workspace_size")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
    items = (BatchItem * cnt)()
    m0s = [int(o.m0) for o in O]
    off = np.concatenate([[0], np.cumsum(m0s)]).astype(int)
    lam = np.zeros(2 * off[-1])
    res = np.zeros(off[-1])
    torch.cuda.synchronize()
    st = lib.feast_solve_batch(cnt, P, Cn, O, ws.data_ptr(), nbytes, nworkers, items,
                               lam.ctypes.data, res.ctypes.data)
    out = []
    for i in range(cnt):
        it = items[i]
        c = it.count
        l = lam[2 * off[i]:2 * off[i] + 2 * c]
        out.append(dict(status=it.status, flag=it.flag, count=c, k=it.k, err=it.err,
                        lam=l[0::2] + 1j * l[1::2], res=res[off[i]:off[i] + c].copy(),
                        ms_setup=it.ms_setup, ms_pass=it.ms_pass, ms_solve=it.ms_solve, ms_qz=it.ms_qz))
    if st != 0:
        bad = [i for i, o in enumerate(out) if o["status"] != 0]
        raise FeastError(st, f"feast_solve_batch (pencils {bad[:8]})")
    return out


def cgemm_tc(A_list, X_list, C_list=None, alpha=1.0, beta=0.0, stream=None):
    """complex64 C = beta C + alpha A X on tensor cores for each batch member."""
    torch = _torch()
    lib = load()
    batch = len(A_list)
    m, k = np.asarray(A_list[0]).shape
    n = np.asarray(X_list[0]).shape[1]
    c64 = torch.complex64
    Ad = torch.cat([to_device_colmajor(np.asarray(A, np.complex64), dtype=c64) for A in A_list])
    Xd = torch.cat([to_device_colmajor(np.asarray(X, np.complex64), dtype=c64) for X in X_list])
    if C_list is None:
        Cd = torch.zeros(batch * m * n, dtype=torch.complex64, device="cuda")
    else:
        Cd = torch.cat([to_device_colmajor(np.asarray(Cc, np.complex64), dtype=c64) for Cc in C_list])
    nb = int(lib.feast_cgemm_tc_scratch_bytes(m, n, k, batch))
    sc = torch.empty(nb, dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    a, b = complex(alpha), complex(beta)
    _check(lib.feast_cgemm_tc(m, n, k, a.real, a.imag, Ad.data_ptr(), m, m * k, Xd.data_ptr(), k, k * n,
                              b.real, b.imag, Cd.data_ptr(), m, m * n, batch, sc.data_ptr(), nb,
                              err.data_ptr(), _stream_ptr(stream)), "feast_cgemm_tc")
    torch.cuda.current_stream().synchronize()
    if int(err.item()):
        raise FeastError(-6, "feast_cgemm_tc")
    return [from_device_colmajor(Cd[b_ * m * n:(b_ + 1) * m * n], m, n) for b_ in range(batch)]


def zgemm_oz(A, Bm, Cm=None, alpha=1.0, beta=0.0, stream=None):
    """complex128 C = beta C + alpha A B on the bf16 tensor cores with exact
    digit slicing (FP64-accurate to ~2^-47 of max|A| max|B| k)."""
    torch = _torch()
    lib = load()
    A = np.asarray(A, np.complex128)
    Bm = np.asarray(Bm, np.complex128)
    m, k = A.shape
    n = Bm.shape[1]
    Ad = to_device_colmajor(A)
    Bd = to_device_colmajor(Bm)
    Cd = (to_device_colmajor(np.asarray(Cm, np.complex128)) if Cm is not None
          else torch.zeros(m * n, dtype=torch.complex128, device="cuda"))
    nb = int(lib.feast_zgemm_oz_work_bytes(m, n, k))
    work = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) // 256 * 256
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    a, b = complex(alpha), complex(beta)
    _check(lib.feast_zgemm_oz(m, n, k, a.real, a.imag, Ad.data_ptr(), m, Bd.data_ptr(), k, b.real, b.imag,
                              Cd.data_ptr(), m, wp, nb, err.data_ptr(), _stream_ptr(stream)), "feast_zgemm_oz")
    torch.cuda.current_stream().synchronize()
    if int(err.item()):
        raise FeastError(-6, "feast_zgemm_oz")
    return from_device_colmajor(Cd, m, n)


def _eig_abs2_runs(A, B, Y, kw):
    # converged pairs only: the gradient is only as accurate as the pairs
    f = Feast(A, B, Y, converged_only=True, **kw)
    f.run()
    return f


def _conj_contour(kw):
    kk = dict(kw)
    kk["center"] = complex(kw.get("center", 0j)).conjugate()
    return kk


def _make_eig_abs2_function():
    torch = _torch()

    class EigSumAbs2(torch.autograd.Function):
        """L = sum over the eigenvalues of (A, B) inside the contour of
        |lambda|^2, by GFEAST; backward runs GFEAST on (A^H, B^H) over the
        conjugated contour for the left eigenvectors and forms dL/dA, dL/dB
        with the library's adjoint kernels."""

        @staticmethod
        def forward(ctx, A, B, Y, kw):
            right = _eig_abs2_runs(A, B, Y, kw)
            r = right.eigs(want_vectors=False)
            ctx.right, ctx.kw = right, kw
            ctx.save_for_backward(A, B, Y)
            L = float(np.sum(np.abs(r["lam"]) ** 2))
            return torch.tensor(L, dtype=torch.float64, device=A.device)

        @staticmethod
        def backward(ctx, gout):
            A, B, Y = ctx.saved_tensors
            left = _eig_abs2_runs(A.conj().t().resolve_conj(), B.conj().t().resolve_conj(), Y,
                                  _conj_contour(ctx.kw))
            _, gA, gB, _ = ctx.right.grad_abs2(left)
            left.close()
            ctx.right.close()
            g = gout.to(torch.complex128)
            return g * gA, g * gB, None, None

    return EigSumAbs2


_EIG_ABS2 = None


def eig_sum_abs2(A, B, Y, **kw):
    """Differentiable L = sum_{lambda inside} |lambda|^2 of the dense pencil
    (A, B) (torch complex128 tensors on the GPU, rows x cols); kw are Feast's
    contour / tolerance / precision keywords."""
    global _EIG_ABS2
    if _EIG_ABS2 is None:
        _EIG_ABS2 = _make_eig_abs2_function()
    return _EIG_ABS2.apply(A, B, Y, kw)


def _csr_arrays(M, n):
    """(indptr, indices, data) of a CSR matrix (a scipy.sparse matrix or a
    triple) as int64 / int64 / complex128 numpy arrays."""
    if hasattr(M, "tocsr"):
        M = M.tocsr()
        M = (M.indptr, M.indices, M.data)
    indptr, indices, data = M
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int64)
    data = np.ascontiguousarray(data, dtype=np.complex128)
    if indptr.shape != (n + 1,) or indices.shape != data.shape:
        raise ValueError("malformed CSR triple")
    return indptr, indices, data


def csr_rcm(n: int, A, B=None):
    """Reverse Cuthill-McKee ordering of the joint pattern of the sparse
    pencil (host; feast_csr_rcm).  Returns (perm, kl, ku): perm[new] = old
    and the bandwidths of the permuted A and B."""
    lib = load()
    a = _csr_arrays(A, n)
    b = _csr_arrays(B, n) if B is not None else None
    perm = np.zeros(n, np.int64)
    kl, ku = C.c_int64(0), C.c_int64(0)
    _check(lib.feast_csr_rcm(n, a[0].ctypes.data, a[1].ctypes.data, b[0].ctypes.data if b else None,
                             b[1].ctypes.data if b else None, perm.ctypes.data, C.byref(kl), C.byref(ku)),
           "feast_csr_rcm")
    return perm, int(kl.value), int(ku.value)


def csr_to_band(n: int, M, perm, kl: int, ku: int, device="cuda"):
    """P M P^T of a CSR matrix in compact band storage on the device (flat
    column-major (kl + ku + 1) x n complex128 tensor; feast_csr_to_band)."""
    torch = _torch()
    lib = load()
    indptr, indices, data = _csr_arrays(M, n)
    iperm = np.empty(n, np.int64)
    iperm[np.asarray(perm, np.int64)] = np.arange(n, dtype=np.int64)
    d_ptr = torch.from_numpy(indptr).to(device)
    d_col = torch.from_numpy(indices).to(device)
    d_val = torch.from_numpy(data).to(device)
    d_ip = torch.from_numpy(iperm).to(device)
    band = torch.empty((kl + ku + 1) * n, dtype=torch.complex128, device=device)
    status = torch.zeros(1, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream(torch.device(device))
    _check(lib.feast_csr_to_band(n, d_ptr.data_ptr(), d_col.data_ptr(), d_val.data_ptr(), d_ip.data_ptr(), kl, ku,
                                 band.data_ptr(), status.data_ptr(), stream.cuda_stream), "feast_csr_to_band")
    return band


class SparseFeast(Feast):
    """GFEAST on a sparse pencil (A, B in CSR; B = None for B = I): the
    rows and columns are reordered by reverse Cuthill-McKee, both matrices
    are scattered into band storage on the device, and the banded path runs
    on (P A P^T, P B P^T) with the start block P Y.  eigs() returns the
    eigenvectors in the original ordering.  The reordered bandwidth must fit
    the band solves (kl + ku up to ~600 in FP64, ~1200 in the precision
    form); a wider one raises FeastError (EINVAL) at set-up."""

    def __init__(self, n: int, A, B, Y, **kw):
        for k in ("kind", "kl", "ku", "b_identity"):
            if k in kw:
                raise TypeError(f"SparseFeast sets {k} itself")
        device = kw.get("device", "cuda")
        self.perm, kl, ku = csr_rcm(n, A, B)
        Ab = csr_to_band(n, A, self.perm, kl, ku, device)
        Bb = csr_to_band(n, B, self.perm, kl, ku, device) if B is not None else None
        Yp = np.asarray(Y)[self.perm, :] if not hasattr(Y, "device") else Y[_torch().from_numpy(self.perm)]
        super().__init__(Ab, Bb, Yp, kind=FEAST_BANDED, kl=kl, ku=ku, b_identity=B is None, **kw)
        self._iperm = np.empty(n, np.int64)
        self._iperm[self.perm] = np.arange(n, dtype=np.int64)

    def eigs(self, want_vectors: bool = True) -> dict:
        out = super().eigs(want_vectors)
        if want_vectors:
            out["X"] = out["X"][self._iperm, :]
        return out
