"""Plain FP64 CPU oracle for oblique-projection FEAST (Yin, Chan & Yeung).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
never links, loads or calls it, and this package never imports the GPU
package: the two share no code.  The C source (``feast_oracle.c``) restates
the method from the paper:

* contour nodes / weights -- Section 4.3, eq. 4.1 (Gauss-Legendre on a circle);
  trapezoid and ellipse variants derived the same way from z'(theta);
* LU with partial pivoting + substitution for the shifted systems, eq. 4.2;
* banded LU (LAPACK band layout) for the same systems with banded pencils;
* Householder QR (GFEAST lines 2, 17);
* oblique projection A~ = U2^H A U1, B~ = U2^H B U1 (eq. 3.10, GFEAST line 5);
* complex QZ for the projected pencil (GFEAST line 6);
* residual of eq. 5.1, selection, and the three stopping tests (lines 7-15);
* the Rayleigh-Ritz projection of Algorithm FEAST (Section 3) as an option
  of the same driver (test space = search space), for comparison;
* Block CIRR (Section 2.1, Algorithm Block_CIRR), the comparison method:
  quadrature moments F_i Y, a one-sided Jacobi SVD of the moment block, the
  Rayleigh-Ritz pencil and its eigenpairs, selected like GFEAST's;
* SEARCH (Section 4.1): trace estimate of the inside count and the
  numerical rank of the filtered block by Householder QR with column
  pivoting (lines 1-10 of the algorithm);
* the derivative of sum_{lambda inside} |lambda|^2 with respect to A and B
  from first-order perturbation of simple eigenvalues (left / right
  eigenvectors of the whole pencil by the own QZ) -- for the
  differentiation form built on top of the method.

Every entry point takes numpy complex128 arrays in Fortran (column-major)
order.  Parity of each routine is pinned in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "feast_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfeast_oracle.so")
_lib = None
_lock = threading.Lock()

OR_OK, OR_EINVAL, OR_ENOMEM, OR_ESINGULAR, OR_ENOCONV = 0, -1, -2, -4, -7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over nodes/columns)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, I, D = C.c_void_p, C.c_int, C.c_double
            lib.or_gauss_legendre.argtypes = [I, P, P]
            lib.or_contour.argtypes = [I, I, I, D, D, D, D, P, P]
            lib.or_inside.argtypes = [I, D, D, D, D, D, D]
            lib.or_zgetrf.argtypes = [I, P, I, P]
            lib.or_zgetrs.argtypes = [I, I, P, I, P, P, I]
            lib.or_zgetrs_cols.argtypes = [I, I, P, I, P, P, I]
            lib.or_zgbtrf.argtypes = [I, I, I, P, I, P]
            lib.or_zgbtrs.argtypes = [I, I, I, I, P, I, P, P, I]
            lib.or_zgemm.argtypes = [I, I, I, I, P, I, P, I, P, I]
            lib.or_band_matmul.argtypes = [I, I, I, P, I, I, P, I, P, I]
            lib.or_zqr.argtypes = [I, I, P, I, P, I, P, I]
            lib.or_zggev.argtypes = [I, P, I, P, I, P, P, P, I]
            lib.or_setup.argtypes = [I, I, P, P, I, I, I, I, I, I, I, D, D, D, D, I, P, D, D, I,
                                     C.POINTER(C.c_int)]
            lib.or_setup.restype = P
            lib.or_iterate.argtypes = [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(D)]
            lib.or_filter.argtypes = [P, P, P]
            lib.or_get.argtypes = [P, I, P]
            lib.or_get_ritz_info.argtypes = [P, P, P]
            lib.or_set_U1.argtypes = [P, P]
            lib.or_result.argtypes = [P, C.POINTER(I), P, P, P, C.POINTER(D), C.POINTER(I),
                                      C.POINTER(I)]
            lib.or_free.argtypes = [P]
            lib.or_zqrcp.argtypes = [I, I, P, I, D, P, P, C.POINTER(I), P, I]
            lib.or_set_projection.argtypes = [P, I]
            lib.or_set_search_literal.argtypes = [P, I]
            lib.or_zsvd_jacobi.argtypes = [I, I, P, I, P, I, P]
            lib.or_cirr.argtypes = [P, P, I, I, C.POINTER(I), P, P, P, P]
            lib.or_search.argtypes = [P, P, I, D, I, D, P, C.POINTER(I), C.POINTER(I)]
            lib.or_num_threads.restype = I
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _zf(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.complex128))


def num_threads() -> int:
    return _load().or_num_threads()


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------
def gauss_legendre(q: int):
    t = np.zeros(q); w = np.zeros(q)
    _load().or_gauss_legendre(q, _p(t), _p(w))
    return t, w


def contour(ckind: int, rule: int, q: int, center: complex, a: float, b: float = 0.0):
    """Nodes z_j and weights w_j (complex128, length q).  ckind 0 circle /
    1 ellipse; rule 0 trapezoid / 1 Gauss-Legendre."""
    z = np.zeros(q, np.complex128); w = np.zeros(q, np.complex128)
    st = _load().or_contour(ckind, rule, q, center.real, center.imag, a, b, _p(z), _p(w))
    if st:
        raise ValueError(f"or_contour status {st}")
    return z, w


def inside(ckind: int, center: complex, a: float, b: float, lam: complex) -> bool:
    return bool(_load().or_inside(ckind, center.real, center.imag, a, b, lam.real, lam.imag))


def lu(a):
    """P A = L U (partial pivoting). Returns (lu, piv, info)."""
    f = _zf(a).copy(order="F")
    n = f.shape[0]
    piv = np.zeros(n, np.int32)
    info = _load().or_zgetrf(n, _p(f), n, _p(piv))
    return f, piv, info


def lu_solve(f, piv, b):
    x = _zf(b).copy(order="F")
    if x.ndim == 1:
        x = x.reshape(-1, 1, order="F")
    n = f.shape[0]
    _load().or_zgetrs(n, x.shape[1], _p(f), n, _p(piv), _p(x), n)
    return x


def lu_solve_cols(f, piv, b):
    """lu_solve with the columns solved in parallel (OpenMP)."""
    x = _zf(b).copy(order="F")
    n = f.shape[0]
    _load().or_zgetrs_cols(n, x.shape[1], _p(f), n, _p(piv), _p(x), n)
    return x


def band_lu(ab_compact, n: int, kl: int, ku: int):
    """Band LU.  ab_compact: (kl+ku+1) x n compact band storage (entry (i,j)
    at row ku+i-j).  Returns factor storage (2kl+ku+1) x n and pivots."""
    ldab = 2 * kl + ku + 1
    f = np.zeros((ldab, n), np.complex128, order="F")
    f[kl:, :] = _zf(ab_compact)
    piv = np.zeros(n, np.int32)
    info = _load().or_zgbtrf(n, kl, ku, _p(f), ldab, _p(piv))
    return f, piv, info


def band_solve(f, piv, n: int, kl: int, ku: int, b):
    x = _zf(b).copy(order="F")
    if x.ndim == 1:
        x = x.reshape(-1, 1, order="F")
    _load().or_zgbtrs(n, kl, ku, x.shape[1], _p(f), f.shape[0], _p(piv), _p(x), n)
    return x


def band_matmul(ab_compact, n: int, kl: int, ku: int, x):
    x = _zf(x)
    if x.ndim == 1:
        x = x.reshape(-1, 1, order="F")
    ab = _zf(ab_compact)
    y = np.zeros((n, x.shape[1]), np.complex128, order="F")
    _load().or_band_matmul(n, kl, ku, _p(ab), ab.shape[0], x.shape[1], _p(x), n, _p(y), n)
    return y


def gemm(a, b, conj_a: bool = False):
    a = _zf(a); b = _zf(b)
    m = a.shape[1] if conj_a else a.shape[0]
    k = a.shape[0] if conj_a else a.shape[1]
    n = b.shape[1]
    c = np.zeros((m, n), np.complex128, order="F")
    _load().or_zgemm(int(conj_a), m, n, k, _p(a), a.shape[0], _p(b), b.shape[0], _p(c), m)
    return c


def qr(a):
    a = _zf(a)
    m, k = a.shape
    q = np.zeros((m, k), np.complex128, order="F"); r = np.zeros((k, k), np.complex128, order="F")
    st = _load().or_zqr(m, k, _p(a), m, _p(q), m, _p(r), k)
    if st:
        raise ValueError(f"or_zqr status {st}")
    return q, r


def ggev(a, b):
    """Generalized eigenpairs of (a, b): returns alpha, beta, V (unit columns)."""
    a = _zf(a); b = _zf(b)
    m = a.shape[0]
    al = np.zeros(m, np.complex128); be = np.zeros(m, np.complex128)
    v = np.zeros((m, m), np.complex128, order="F")
    st = _load().or_zggev(m, _p(a), m, _p(b), m, _p(al), _p(be), _p(v), m)
    if st:
        raise RuntimeError(f"or_zggev status {st}")
    return al, be, v


# --------------------------------------------------------------------------
# Derivative of L = sum over the eigenvalues inside the contour of |lambda|^2
# --------------------------------------------------------------------------
def eig_grad_abs2(A, B, ckind: int, center: complex, a: float, b: float = 0.0):
    """L and its gradients with respect to A and B for a real loss of complex
    inputs (dL = Re sum conj(G_A) * dA + Re sum conj(G_B) * dB).

    A simple eigenvalue with right vector x (A x = lam B x) and left vector
    v (v^H A = lam v^H B) moves by d lam = v^H (dA - lam dB) x / (v^H B x);
    with dL = sum 2 Re(conj(lam) d lam) this gives
        G_A = sum_i 2 lam_i v_i x_i^H / conj(c_i),
        G_B = -sum_i 2 |lam_i|^2 v_i x_i^H / conj(c_i),   c_i = v_i^H B x_i.
    Right vectors come from the QZ of (A, B), left vectors from the QZ of
    (A^H, B^H) (its eigenvalues are the conjugates), both over the whole
    pencil.  Returns (L, G_A, G_B, inside eigenvalues)."""
    A = _zf(A); B = _zf(B)
    n = A.shape[0]
    al, be, X = ggev(A, B)
    lam = al / be
    alL, beL, V = ggev(np.conj(A.T), np.conj(B.T))
    mu = np.conj(alL / beL)
    ins = [i for i in range(n) if inside(ckind, center, a, b, complex(lam[i]))]
    free = list(range(n))
    gA = np.zeros((n, n), np.complex128)
    gB = np.zeros((n, n), np.complex128)
    L = 0.0
    for i in ins:
        k = min(free, key=lambda j: abs(mu[j] - lam[i]))
        free.remove(k)
        x = X[:, i]
        v = V[:, k]
        c = np.vdot(v, B @ x)
        outer = np.outer(v, np.conj(x)) / np.conj(c)
        gA += 2.0 * lam[i] * outer
        gB -= 2.0 * abs(lam[i]) ** 2 * outer
        L += abs(lam[i]) ** 2
    return L, gA, gB, lam[ins]


# --------------------------------------------------------------------------
# GFEAST driver
# --------------------------------------------------------------------------
def qrcp(a, tol: float):
    """Householder QR with column pivoting (largest remaining norm first).
    Returns (rank, jpvt, |R_jj|, Q[:, :rank]); rank counts |R_jj| > tol |R_00|."""
    a = _zf(a)
    m, k = a.shape
    jp = np.zeros(k, np.int32)
    rd = np.zeros(k)
    q = np.zeros((m, k), np.complex128, order="F")
    r = C.c_int(0)
    st = _load().or_zqrcp(m, k, _p(a), m, float(tol), _p(jp), _p(rd), C.byref(r), _p(q), m)
    if st:
        raise RuntimeError(f"or_zqrcp status {st}")
    return r.value, jp, rd, q[:, :r.value].copy()


def svd_jacobi(a):
    """One-sided Jacobi SVD of the m x k matrix a (m >= k): returns (U, sigma),
    the left singular vectors (m x k) and singular values, decreasing."""
    a = _zf(a)
    m, k = a.shape
    u = np.zeros((m, k), np.complex128, order="F")
    sg = np.zeros(k)
    st = _load().or_zsvd_jacobi(m, k, _p(a), m, _p(u), m, _p(sg))
    if st:
        raise RuntimeError(f"or_zsvd_jacobi status {st}")
    return u, sg


class Feast:
    """Lines 1-17 of GFEAST with the start block Y in place of SEARCH.

    kind 0: dense A, B (n x n).  kind 1: compact band storage ((kl+ku+1) x n).
    """

    def __init__(self, A, B, Y, *, contour_kind=0, rule=0, q=16, center=0j, a=1.0, b=0.0,
                 eps=1e-12, eta=1e-3, max_iter=50, kind=0, kl=0, ku=0, b_identity=False, projection=0):
        lib = _load()
        self.A = _zf(A)
        self.B = _zf(B) if B is not None else np.zeros_like(self.A)
        self.Y = _zf(Y)
        self.n = self.Y.shape[0] if kind == 0 else self.A.shape[1]
        self.m0 = self.Y.shape[1]
        self.q = q
        ld = self.A.shape[0]
        st = C.c_int(0)
        self._c = lib.or_setup(kind, self.n, _p(self.A), _p(self.B), ld, kl, ku, int(b_identity),
                               contour_kind, rule, q, center.real, center.imag, a, b,
                               self.m0, _p(self.Y), eps, eta, max_iter, C.byref(st))
        if not self._c:
            raise RuntimeError(f"or_setup status {st.value}")
        if lib.or_set_projection(self._c, int(projection)):
            raise ValueError("projection must be 0 (oblique) or 1 (Rayleigh-Ritz)")

    def close(self):
        if getattr(self, "_c", None):
            _load().or_free(self._c)
            self._c = None

    def __del__(self):
        self.close()

    def iterate(self):
        k, cnt, flag = C.c_int(), C.c_int(), C.c_int()
        err = C.c_double()
        st = _load().or_iterate(self._c, C.byref(k), C.byref(cnt), C.byref(flag), C.byref(err))
        if st < 0:
            raise RuntimeError(f"or_iterate status {st}")
        return dict(k=k.value, count=cnt.value, flag=flag.value, err=err.value, done=(st == 1))

    def run(self):
        hist = []
        while True:
            it = self.iterate()
            hist.append(it)
            if it["flag"] != 2:
                return hist

    def filter(self, V):
        V = _zf(V)
        U = np.zeros((self.n, self.m0), np.complex128, order="F")
        _load().or_filter(self._c, _p(V), _p(U))
        return U

    def get(self, what: str):
        idx = dict(U1=0, U2=1, R2=2, At=3, Bt=4, X=5, lam=6, AU1=7, BU1=8, z=9, w=10)[what]
        if what in ("U1", "U2", "X", "AU1", "BU1"):
            out = np.zeros((self.n, self.m0), np.complex128, order="F")
        elif what in ("R2", "At", "Bt"):
            out = np.zeros((self.m0, self.m0), np.complex128, order="F")
        elif what == "lam":
            out = np.zeros(self.m0, np.complex128)
        else:
            out = np.zeros(self.q, np.complex128)
        _load().or_get(self._c, idx, _p(out))
        return out

    def ritz_info(self):
        res = np.zeros(self.m0); sel = np.zeros(self.m0, np.int32)
        _load().or_get_ritz_info(self._c, _p(res), _p(sel))
        return res, sel.astype(bool)

    def set_search_literal(self, literal: bool):
        """Read SEARCH's line 10 literally (U = U1 after a full-rank step)
        instead of keeping the block as filtered columns."""
        _load().or_set_search_literal(self._c, int(bool(literal)))

    def search(self, Ypool, alpha: float, p: int, rank_tol: float):
        """Algorithm SEARCH (Section 4.1) with the random columns supplied by
        Ypool (n x npool, used in order); the working width is bounded by
        this context's m0.  Returns dict(t, s0, U1 (n x t))."""
        Ypool = _zf(Ypool)
        U1 = np.zeros((self.n, self.m0), np.complex128, order="F")
        t, s0 = C.c_int(0), C.c_int(0)
        st = _load().or_search(self._c, _p(Ypool), Ypool.shape[1], float(alpha), int(p), float(rank_tol),
                               _p(U1), C.byref(t), C.byref(s0))
        if st:
            raise RuntimeError(f"or_search status {st}")
        return dict(t=t.value, s0=s0.value, U1=U1[:, :t.value].copy())

    def cirr(self, Y, g: int):
        """Algorithm Block_CIRR (Section 2.1) on this context's pencil and
        quadrature: Y (n x h) random columns, g moments, t = h g.  Returns
        dict(count, lam, X, res) of the selected pairs and sigma, the
        singular values of the moment block."""
        Y = _zf(Y)
        h = Y.shape[1]
        t = h * g
        lam = np.zeros(t, np.complex128)
        X = np.zeros((self.n, t), np.complex128, order="F")
        res = np.zeros(t)
        sg = np.zeros(t)
        cnt = C.c_int(0)
        st = _load().or_cirr(self._c, _p(Y), h, int(g), C.byref(cnt), _p(lam), _p(X), _p(res), _p(sg))
        if st:
            raise RuntimeError(f"or_cirr status {st}")
        c = cnt.value
        return dict(count=c, lam=lam[:c].copy(), X=X[:, :c].copy(), res=res[:c].copy(), sigma=sg)

    def set_U1(self, U1):
        U1 = _zf(U1)
        st = _load().or_set_U1(self._c, _p(U1))
        if st:
            raise RuntimeError(f"or_set_U1 status {st}")

    def result(self):
        cnt, flag, k = C.c_int(), C.c_int(), C.c_int()
        err = C.c_double()
        lam = np.zeros(self.m0, np.complex128)
        X = np.zeros((self.n, self.m0), np.complex128, order="F")
        res = np.zeros(self.m0)
        st = _load().or_result(self._c, C.byref(cnt), _p(lam), _p(X), _p(res), C.byref(err),
                               C.byref(flag), C.byref(k))
        if st:
            raise RuntimeError("GFEAST has not stopped yet")
        c = cnt.value
        return dict(count=c, lam=lam[:c].copy(), X=X[:, :c].copy(), res=res[:c].copy(),
                    err=err.value, flag=flag.value, k=k.value)
