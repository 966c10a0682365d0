"""Seeded synthetic pencils -- the only module shared by the GPU path's tests
and the oracle.  It holds input construction only: no quadrature, no
factorisation, no projection.

The paper's experiments use Matrix Market pencils that are not available
here; these generators stand in for them with the same kind of structure:

* ``prescribed_pencil``: dense complex A = P diag(lam) Q, B = P Q with
  P, Q = I + 0.1 G / sqrt(n) (G complex Gaussian).  Then A x = lam B x has
  exactly the eigenvalues ``lam`` (eigenvectors Q^{-1} e_i), which is the
  canonical form of Theorem 2.1 with T = P^{-1}, S = Q^{-1}.
* ``convection_diffusion``: -Lap u + (b1, b2) . grad u on the unit square,
  Dirichlet, 5-point central differences on an nx x nx grid (B = I), in
  compact band storage; its spectrum has a closed form.
* ``ragged_batch``: many prescribed-spectrum pencils of uneven size.
* ``hermitian_pencil``: A Hermitian, B Hermitian positive definite, real
  prescribed spectrum (the Rayleigh-Ritz comparison case).
* ``sparse_pencil``: the convection-diffusion operator with a non-identity
  sparse B, rows and columns in a random order, in CSR (the structure of
  the paper's sparse test pencils without a banded ordering).

Random draws use ``numpy.random.default_rng(seed)`` (PCG64) in a fixed
order: lam (u then v, then any re-draws), G_P, G_Q, Y.  With seed 0 and
n = 200 this order puts 44 eigenvalues inside |z| < 1 (the dense n = 200
workload is specified as having about 50 inside).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    """(N(0,1) + i N(0,1)) / sqrt(2), Fortran order."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return np.asfortranarray((re + 1j * im) / math.sqrt(2.0))


@dataclass
class DensePencil:
    A: np.ndarray          # n x n complex128, column-major
    B: np.ndarray
    Y: np.ndarray          # n x m0 start block
    lam: np.ndarray        # prescribed eigenvalues (length n)
    center: complex
    radius: float
    P: np.ndarray = None   # A = P diag(lam) Q, B = P Q
    Q: np.ndarray = None

    @property
    def n(self) -> int:
        return self.A.shape[0]

    def inside_count(self) -> int:
        return int(np.sum(np.abs(self.lam - self.center) < self.radius))


def draw_spectrum(rng: np.random.Generator, n: int, lam_radius: float, center: complex,
                  radius: float, guard: float = 1e-3) -> np.ndarray:
    """lam = lam_radius * sqrt(u) * exp(2 pi i v) (uniform in the disk), with
    any eigenvalue within a relative distance ``guard`` of the contour
    re-drawn so that the inside count is well posed."""
    u = rng.random(n)
    v = rng.random(n)
    lam = lam_radius * np.sqrt(u) * np.exp(2j * np.pi * v)
    for _ in range(1000):
        bad = np.abs(np.abs(lam - center) / radius - 1.0) < guard
        if not bad.any():
            break
        k = int(bad.sum())
        u2 = rng.random(k)
        v2 = rng.random(k)
        lam[bad] = lam_radius * np.sqrt(u2) * np.exp(2j * np.pi * v2)
    return lam


def prescribed_pencil(n: int, m0: int, seed: int = 0, center: complex = 0j, radius: float = 1.0,
                      lam_radius: float = 2.0, lam_center: complex = 0j) -> DensePencil:
    rng = np.random.default_rng(seed)
    lam = lam_center + draw_spectrum(rng, n, lam_radius, center - lam_center, radius)
    gp = complex_normal(rng, (n, n))
    gq = complex_normal(rng, (n, n))
    Y = complex_normal(rng, (n, m0))
    eye = np.eye(n, dtype=np.complex128)
    P = eye + 0.1 * gp / math.sqrt(n)
    Q = eye + 0.1 * gq / math.sqrt(n)
    B = np.asfortranarray(P @ Q)
    A = np.asfortranarray((P * lam[None, :]) @ Q)
    return DensePencil(A=A, B=B, Y=Y, lam=lam, center=center, radius=radius, P=P, Q=Q)


def gapped_pencil(n: int, m0: int, n_in: int, seed: int = 0, r_in: float = 0.7, r_out: float = 1.5,
                  lam_radius: float = 2.0) -> DensePencil:
    """A = P diag(lam) Q, B = P Q (as prescribed_pencil) with n_in eigenvalues
    uniform in |z| < r_in and the rest uniform in the annulus r_out < |z| <
    lam_radius: a clean gap around the unit circle, so that the filtered
    block has a well-defined numerical rank (SEARCH).  Draw order: inside
    radii/angles, outside radii/angles, G_P, G_Q, Y."""
    rng = np.random.default_rng(seed)
    u, v = rng.random(n_in), rng.random(n_in)
    lam_in = r_in * np.sqrt(u) * np.exp(2j * np.pi * v)
    k = n - n_in
    u2, v2 = rng.random(k), rng.random(k)
    rad = np.sqrt(r_out ** 2 + (lam_radius ** 2 - r_out ** 2) * u2)
    lam = np.concatenate([lam_in, rad * np.exp(2j * np.pi * v2)])
    gp = complex_normal(rng, (n, n))
    gq = complex_normal(rng, (n, n))
    Y = complex_normal(rng, (n, m0))
    eye = np.eye(n, dtype=np.complex128)
    P = eye + 0.1 * gp / math.sqrt(n)
    Q = eye + 0.1 * gq / math.sqrt(n)
    B = np.asfortranarray(P @ Q)
    A = np.asfortranarray((P * lam[None, :]) @ Q)
    return DensePencil(A=A, B=B, Y=Y, lam=lam, center=0j, radius=1.0, P=P, Q=Q)


def hermitian_pencil(n: int, m0: int, seed: int = 0, lam_radius: float = 2.0,
                     guard: float = 1e-3) -> DensePencil:
    """A Hermitian / B Hermitian positive definite: A = Q^H diag(lam) Q,
    B = Q^H Q with Q = I + 0.1 G / sqrt(n) and lam real, uniform in
    (-lam_radius, lam_radius) (values within ``guard`` of +-1 re-drawn).  It is
    the prescribed pencil with P = Q^H, so the eigenvalues are ``lam`` and the
    eigenvectors Q^{-1} e_i -- the class of pencils Algorithm FEAST's
    Rayleigh-Ritz projection is made for.  Draw order: lam (then re-draws),
    G_Q, Y."""
    rng = np.random.default_rng(seed)
    lam = lam_radius * (2.0 * rng.random(n) - 1.0)
    for _ in range(1000):
        bad = np.abs(np.abs(lam) - 1.0) < guard
        if not bad.any():
            break
        lam[bad] = lam_radius * (2.0 * rng.random(int(bad.sum())) - 1.0)
    gq = complex_normal(rng, (n, n))
    Y = complex_normal(rng, (n, m0))
    Q = np.eye(n, dtype=np.complex128) + 0.1 * gq / math.sqrt(n)
    P = np.ascontiguousarray(Q.conj().T)
    B = np.asfortranarray(P @ Q)
    A = np.asfortranarray((P * lam[None, :]) @ Q)
    A = np.asfortranarray(0.5 * (A + A.conj().T))   # exactly Hermitian in floating point
    B = np.asfortranarray(0.5 * (B + B.conj().T))
    return DensePencil(A=A, B=B, Y=Y, lam=lam.astype(np.complex128), center=0j, radius=1.0, P=P, Q=Q)


@dataclass
class BandPencil:
    A_band: np.ndarray     # (kl + ku + 1) x n compact band storage, row ku + i - j
    n: int
    kl: int
    ku: int
    Y: np.ndarray
    nx: int
    h: float
    beta: tuple

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n), np.complex128, order="F")
        for j in range(self.n):
            for i in range(max(0, j - self.ku), min(self.n, j + self.kl + 1)):
                A[i, j] = self.A_band[self.ku + i - j, j]
        return A


def convection_diffusion(nx: int, m0: int, seed: int = 0, beta=(20.0, 10.0)) -> BandPencil:
    """A = (1/h^2) [tridiag(-1 - b1 h/2, 4, -1 + b1 h/2) in x  (+)  the same
    in y with b2], lexicographic order with x fastest, h = 1/(nx + 1).
    Half-bandwidth nx; B = I."""
    n = nx * nx
    h = 1.0 / (nx + 1)
    kl = ku = nx
    ab = np.zeros((kl + ku + 1, n), np.complex128, order="F")
    b1, b2 = beta
    inv = 1.0 / (h * h)
    for gy in range(nx):
        for gx in range(nx):
            i = gx + gy * nx
            ab[ku, i] = 4.0 * inv
            if gx > 0:       # (i, i-1): x-lower
                ab[ku + 1, i - 1] = (-1.0 - b1 * h / 2) * inv
            if gx < nx - 1:  # (i, i+1): x-upper
                ab[ku - 1, i + 1] = (-1.0 + b1 * h / 2) * inv
            if gy > 0:       # (i, i-nx): y-lower
                ab[ku + nx, i - nx] = (-1.0 - b2 * h / 2) * inv
            if gy < nx - 1:  # (i, i+nx): y-upper
                ab[ku - nx, i + nx] = (-1.0 + b2 * h / 2) * inv
    rng = np.random.default_rng(seed)
    Y = complex_normal(rng, (n, m0))
    return BandPencil(A_band=ab, n=n, kl=kl, ku=ku, Y=Y, nx=nx, h=h, beta=tuple(beta))


@dataclass
class SparsePencil:
    n: int
    nx: int
    A: tuple               # CSR (indptr int64, indices int64, data complex128)
    B: tuple
    Y: np.ndarray          # n x m0 start block (stored ordering)
    shuffle: np.ndarray    # stored index k is grid node shuffle[k]

    @staticmethod
    def dense(M, n: int) -> np.ndarray:
        indptr, indices, data = M
        D = np.zeros((n, n), np.complex128, order="F")
        for i in range(n):
            for p in range(indptr[i], indptr[i + 1]):
                D[i, indices[p]] += data[p]
        return D


def sparse_pencil(nx: int, m0: int, seed: int = 0, beta=(20.0, 10.0), mass: float = 0.1) -> SparsePencil:
    """A sparse pencil with the structure of a discretised PDE and no useful
    ordering: A = the convection-diffusion operator of convection_diffusion,
    B = I + mass * (sum of the 4 grid neighbours) / 4 (symmetric, eigenvalues
    in (1 - mass, 1 + mass)), both with rows and columns in a random order
    (rng.permutation, drawn first; then Y), in CSR with sorted columns."""
    n = nx * nx
    h = 1.0 / (nx + 1)
    b1, b2 = beta
    inv = 1.0 / (h * h)
    rng = np.random.default_rng(seed)
    shuffle = rng.permutation(n).astype(np.int64)
    pos = np.empty(n, np.int64)
    pos[shuffle] = np.arange(n, dtype=np.int64)       # grid node -> stored index
    ra, ca, va, rb, cb, vb = [], [], [], [], [], []
    for gy in range(nx):
        for gx in range(nx):
            i = gx + gy * nx
            ra.append(i); ca.append(i); va.append(4.0 * inv)
            rb.append(i); cb.append(i); vb.append(1.0)
            for (ok, j, coef) in ((gx > 0, i - 1, -1.0 - b1 * h / 2), (gx < nx - 1, i + 1, -1.0 + b1 * h / 2),
                                  (gy > 0, i - nx, -1.0 - b2 * h / 2), (gy < nx - 1, i + nx, -1.0 + b2 * h / 2)):
                if ok:
                    ra.append(i); ca.append(j); va.append(coef * inv)
                    rb.append(i); cb.append(j); vb.append(mass / 4.0)

    def csr(r, c, v):
        r = pos[np.asarray(r)]
        c = pos[np.asarray(c)]
        v = np.asarray(v, np.complex128)
        order = np.lexsort((c, r))
        r, c, v = r[order], c[order], v[order]
        indptr = np.zeros(n + 1, np.int64)
        np.add.at(indptr, r + 1, 1)
        return np.cumsum(indptr).astype(np.int64), c.astype(np.int64), v

    Y = complex_normal(rng, (n, m0))
    return SparsePencil(n=n, nx=nx, A=csr(ra, ca, va), B=csr(rb, cb, vb), Y=Y, shuffle=shuffle)


@dataclass
class RaggedBatch:
    pencils: list          # list of DensePencil
    m0: list               # per-pencil start-block width


def ragged_batch(count: int, n_lo: int, n_hi: int, seed: int = 0, lam_radius: float = 2.0) -> RaggedBatch:
    """count pencils, n ~ U[n_lo, n_hi], circle centre uniform in |z| <= 1,
    radius U[0.5, 1]; m0 = max(8, ceil(1.5 s / 8) * 8) capped at n, where s is
    the exact inside count."""
    rng = np.random.default_rng(seed)
    out, m0s = [], []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        cr = math.sqrt(rng.random())
        ca = 2 * math.pi * rng.random()
        center = complex(cr * math.cos(ca), cr * math.sin(ca))
        radius = 0.5 + 0.5 * rng.random()
        sub_seed = int(rng.integers(0, 2**31 - 1))
        # the start block width depends on the spectrum (drawn first)
        lam = draw_spectrum(np.random.default_rng(sub_seed), n, lam_radius, center, radius)
        s = int(np.sum(np.abs(lam - center) < radius))
        m0 = min(n, max(8, int(math.ceil(1.5 * s / 8.0)) * 8))
        p = prescribed_pencil(n, m0, seed=sub_seed, center=center, radius=radius,
                              lam_radius=lam_radius)
        out.append(p)
        m0s.append(m0)
    return RaggedBatch(pencils=out, m0=m0s)


# The workloads of the benchmark and the tests, by name.
WORKLOADS = {
    # plain method, FP64 dense, n = 200, circle |z| < 1, 16 trapezoid nodes,
    # m0 = 64, stopping tolerance 1e-12
    "dense_n200_m64_q16": dict(n=200, m0=64, q=16, rule=0, center=0j, radius=1.0, seed=0,
                               eps=1e-12),
    # precision form, dense n = 4096, m0 = 1280, 32 trapezoid nodes; compared
    # at residual <= 1e-10
    "dense_n4096_m1280_q32": dict(n=4096, m0=1280, q=32, rule=0, center=0j, radius=1.0, seed=0,
                                  eps=1e-10),
    # mid-size dense case for kernel profiles (same generator)
    "dense_n1024_m256_q8": dict(n=1024, m0=256, q=8, rule=0, center=0j, radius=1.0, seed=0,
                                eps=1e-10),
    # profiling size whose operands exceed the 129 MB L2 with ~3 GB on the device
    "dense_n2048_m512_q8": dict(n=2048, m0=512, q=8, rule=0, center=0j, radius=1.0, seed=0,
                                eps=1e-10),
    # banded convection-diffusion, 128 x 128 grid (n = 16384, kl = ku = 128),
    # B = I, ellipse around the lowest 41 eigenvalues, 16 Gauss-Legendre nodes
    "band_n16384_m64_q16": dict(nx=128, m0=64, q=16, rule=1, center=422.0 + 0j, a=322.0,
                                b=80.5, seed=0, eps=1e-10, beta=(20.0, 10.0)),
    # ragged batch: 256 dense pencils, n ~ U[64, 1024], own circles, 16 nodes
    "batch_256_n64_1024_q16": dict(batch=256, n_lo=64, n_hi=1024, q=16, seed=0, eps=1e-10),
    # differentiation form: dense n = 2048, circle |z| < 1, 24 trapezoid nodes,
    # m0 = 640; gradient of the sum of |lambda|^2 over the inside eigenvalues
    "grad_n2048_m640_q24": dict(n=2048, m0=640, q=24, rule=0, center=0j, radius=1.0, seed=0, eps=1e-10,
                                grad=True),
    # SEARCH then GFEAST (the complete algorithm): dense gapped pencil
    # n = 2048 with 400 eigenvalues inside |z| < 0.7 and the rest beyond 1.5,
    # 32 trapezoid nodes on |z| = 1 (the filter leaves < 3e-6 of the outside
    # part), a workspace of width 640, first sample p = 64, growth alpha =
    # 1.5, rank threshold 1e-4
    "search_n2048_s400_q32": dict(n=2048, m0=640, n_in=400, q=32, rule=0, center=0j, radius=1.0, seed=0,
                                  eps=1e-10, search=dict(p=64, alpha=1.5, rank_tol=1e-4, pool=1024)),
    # the banded workload's operator stored as a sparse matrix in a random
    # order (CSR), B = I stored explicitly: reverse Cuthill-McKee must
    # recover the band before the banded path runs; closed-form spectrum
    "sparse_n16384_m64_q16": dict(nx=128, m0=64, q=16, rule=1, center=422.0 + 0j, a=322.0, b=80.5, seed=0,
                                  eps=1e-10, beta=(20.0, 10.0), sparse=dict(mass=0.0)),
    # the comparison of Section 5 on a gapped pencil: GFEAST (oblique), the
    # Rayleigh-Ritz FEAST of Section 3 and Block CIRR of Section 2.1 (h = 80
    # random columns, g = 4 moments), all at width 320 for 200 inside
    "compare_n2048_s200_q32": dict(n=2048, m0=320, n_in=200, q=32, rule=0, center=0j, radius=1.0, seed=0,
                                   eps=1e-10, compare=dict(h=80, g=4)),
}


def convection_diffusion_spectrum(nx: int, beta=(20.0, 10.0)) -> np.ndarray:
    """Closed-form eigenvalues of the operator built by convection_diffusion
    (ascending): lam_{k,l} = (2/h^2) [2 - sqrt(1-(b1 h/2)^2) cos(k pi h)
    - sqrt(1-(b2 h/2)^2) cos(l pi h)], k, l = 1..nx.  Used by tests as a pin;
    the method's code never calls it."""
    h = 1.0 / (nx + 1)
    c1 = math.sqrt(1 - (beta[0] * h / 2) ** 2)
    c2 = math.sqrt(1 - (beta[1] * h / 2) ** 2)
    k = np.arange(1, nx + 1)
    lam = (2 / h**2) * (2 - c1 * np.cos(k[:, None] * np.pi * h) - c2 * np.cos(k[None, :] * np.pi * h))
    return np.sort(lam.ravel())
