// Batched complex QZ for the projected pencil (A~, B~) of GFEAST line 6, in
// FP64, one CTA per pencil.
//
// B~ = U2^H B U1 is upper triangular by construction (U2 R2 = B U1, so
// B~ = R2 up to rounding), so the usual initial QR of B is skipped and its
// strictly lower part is treated as zero.  Then: Hessenberg-triangular
// reduction by Givens rotations, single-shift complex QZ sweeps with
// deflation (Moler-Stewart), and right eigenvectors by back-substitution on
// the generalized Schur form (beta S - alpha P) y = 0 mapped back by Z.
//
// The sweep is a chain of dependent 2x2 rotations, each applied to a row or
// column pair; the CTA's four warps share each rotation's updates of H, T
// and Z (one merged index range, so every SM partition's FP64 units work)
// and meet at a barrier between rotations.  The three m x m arrays live in
// shared memory (m <= 64).  Larger projected problems go to k_zeig.cu.
#include "common.cuh"

namespace feast {

namespace {

__device__ __forceinline__ zd zsqrt_d(zd z)
{
    double r = hypot(z.x, z.y);
    if (r == 0.0) return zmake(0.0, 0.0);
    if (z.x >= 0.0) {
        double t = sqrt(0.5 * (r + z.x));
        return zmake(t, z.y / (2.0 * t));
    }
    double t = sqrt(0.5 * (r - z.x));
    return zmake(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

// Left rotation G = [c s; -conj(s) c], G [x; y] = [r; 0].
__device__ __forceinline__ void giv_left(zd x, zd y, double &c, zd &s)
{
    double ax = zabs(x), ay = zabs(y);
    if (ay == 0.0) { c = 1.0; s = zmake(0.0, 0.0); return; }
    if (ax == 0.0) { c = 0.0; s = zmake(1.0, 0.0); return; }
    double r = hypot(ax, ay);
    c = ax / r;
    s = zscale(zmul(zscale(x, 1.0 / ax), zconj(y)), 1.0 / r);
}
// Right rotation R = [c -conj(s); s c] on a column pair, [t0 t1] R = [0 r].
__device__ __forceinline__ void giv_right(zd t0, zd t1, double &c, zd &s)
{
    double a0 = zabs(t0), a1 = zabs(t1);
    if (a0 == 0.0) { c = 1.0; s = zmake(0.0, 0.0); return; }
    if (a1 == 0.0) { c = 0.0; s = zmake(1.0, 0.0); return; }
    double r = hypot(a0, a1);
    c = a1 / r;
    zd t = zscale(zmul(t0, zconj(t1)), -1.0 / (a1 * r));
    s = t;
}

struct Mat {
    zd *p;
    int ld;
    __device__ __forceinline__ zd &operator()(int i, int j) const { return p[i + (int64_t)j * ld]; }
};

template <int NT>
struct Team {
    __device__ __forceinline__ static void bar()
    {
        if (NT == 32) __syncwarp(); else __syncthreads();
    }
};

// rows (i, j) of M over columns [c0, c1]; optionally force M(j, zc) = 0
template <int NT>
__device__ __forceinline__ void rot_rows(Mat M, int i, int j, int c0, int c1, double c, zd s,
                                         int zc)
{
    for (int col = c0 + (int)threadIdx.x; col <= c1; col += NT) {
        zd a = M(i, col), b = M(j, col);
        zd ni = zadd(zscale(a, c), zmul(s, b));
        zd nj = zadd(zscale(zmul(zconj(s), a), -1.0), zscale(b, c));
        M(i, col) = ni;
        M(j, col) = (col == zc) ? zmake(0.0, 0.0) : nj;
    }
}
// columns (i, j) of M over rows [r0, r1]; optionally force M(zr, i) = 0
template <int NT>
__device__ __forceinline__ void rot_cols(Mat M, int i, int j, int r0, int r1, double c, zd s,
                                         int zr)
{
    for (int row = r0 + (int)threadIdx.x; row <= r1; row += NT) {
        zd a = M(row, i), b = M(row, j);
        zd ni = zadd(zscale(a, c), zmul(b, s));
        zd nj = zadd(zscale(zmul(a, zconj(s)), -1.0), zscale(b, c));
        M(row, i) = (row == zr) ? zmake(0.0, 0.0) : ni;
        M(row, j) = nj;
    }
}

// Left rotation on rows (i, j) of two matrices at once: M1 over columns
// [a0, a1] (optionally zeroing M1(j, z1)), M2 over [b0, b1]; the threads
// share the concatenated index range so all warps stay busy.
template <int NT>
__device__ __forceinline__ void rot_rows2(Mat M1, int a0, int a1, int z1, Mat M2, int b0, int b1,
                                          int i, int j, double c, zd s)
{
    const int na = a1 - a0 + 1, nb = b1 - b0 + 1;
    for (int t = (int)threadIdx.x; t < na + nb; t += NT) {
        Mat M = (t < na) ? M1 : M2;
        const int col = (t < na) ? a0 + t : b0 + (t - na);
        zd a = M(i, col), b = M(j, col);
        zd ni = zadd(zscale(a, c), zmul(s, b));
        zd nj = zadd(zscale(zmul(zconj(s), a), -1.0), zscale(b, c));
        M(i, col) = ni;
        M(j, col) = (t < na && col == z1) ? zmake(0.0, 0.0) : nj;
    }
}
// Right rotation on columns (i, j) of three matrices at once: M1 rows
// [0, r1], M2 rows [0, r2] (optionally zeroing M2(z2, i)), M3 rows [0, r3].
template <int NT>
__device__ __forceinline__ void rot_cols3(Mat M1, int r1, Mat M2, int r2, int z2, Mat M3, int r3,
                                          int i, int j, double c, zd s)
{
    const int n1 = r1 + 1, n2 = r2 + 1, n3 = r3 + 1;
    for (int t = (int)threadIdx.x; t < n1 + n2 + n3; t += NT) {
        Mat M;
        int row;
        bool zero_ok = false;
        if (t < n1) { M = M1; row = t; }
        else if (t < n1 + n2) { M = M2; row = t - n1; zero_ok = true; }
        else { M = M3; row = t - n1 - n2; }
        zd a = M(row, i), b = M(row, j);
        zd ni = zadd(zscale(a, c), zmul(b, s));
        zd nj = zadd(zscale(zmul(a, zconj(s)), -1.0), zscale(b, c));
        M(row, i) = (zero_ok && row == z2) ? zmake(0.0, 0.0) : ni;
        M(row, j) = nj;
    }
}

template <int NT>
__device__ double block_max(double v, double *red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (NT == 32) return v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < NT / 32; ++w) r = fmax(r, red[w]);
    __syncthreads();
    return r;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_qz(int m, zd *A, int64_t lda, int64_t sA, zd *B,
                                           int64_t ldb, int64_t sB, zd *alpha, zd *beta, zd *V,
                                           int64_t ldv, int64_t sV, zd *work, int use_smem,
                                           int *fail)
{
    extern __shared__ zd smem[];
    __shared__ double red[32];
    const int b = blockIdx.x;
    A += (int64_t)b * sA;
    B += (int64_t)b * sB;
    V += (int64_t)b * sV;
    alpha += (int64_t)b * m;
    beta += (int64_t)b * m;
    zd *Wk = work + (int64_t)b * m * m;
    const int tid = threadIdx.x;
    const double eps = 2.220446049250313e-16;

    Mat H, T, Z, Yh;
    if (use_smem) {
        H = Mat{smem, m};
        T = Mat{smem + m * m, m};
        Z = Mat{smem + 2 * m * m, m};
    } else {
        H = Mat{A, (int)lda};
        T = Mat{B, (int)ldb};
        Z = Mat{Wk, m};
    }
    Yh = Mat{use_smem ? Wk : V, use_smem ? m : (int)ldv};
    // load / initialise
    for (int e = tid; e < m * m; e += NT) {
        int r = e % m, c = e / m;
        if (use_smem) {
            H(r, c) = A[r + c * lda];
            T(r, c) = (r <= c) ? B[r + c * ldb] : zmake(0.0, 0.0);
        } else if (r > c) {
            T(r, c) = zmake(0.0, 0.0);
        }
        Z(r, c) = zmake(r == c ? 1.0 : 0.0, 0.0);
    }
    Team<NT>::bar();
    double c;
    zd s;
    // Hessenberg-triangular reduction
    for (int j = 0; j + 2 < m; ++j)
        for (int i = m - 1; i >= j + 2; --i) {
            giv_left(H(i - 1, j), H(i, j), c, s);
            Team<NT>::bar();
            rot_rows2<NT>(H, j, m - 1, j, T, i - 1, m - 1, i - 1, i, c, s);
            Team<NT>::bar();
            giv_right(T(i, i - 1), T(i, i), c, s);
            Team<NT>::bar();
            rot_cols3<NT>(H, m - 1, T, i, i, Z, m - 1, i - 1, i, c, s);
            Team<NT>::bar();
        }
    // norms for the deflation tests
    double hn = 0.0, tn = 0.0;
    for (int e = tid; e < m * m; e += NT) {
        hn = fmax(hn, zabs(H(e % m, e / m)));
        tn = fmax(tn, zabs(T(e % m, e / m)));
    }
    hn = block_max<NT>(hn, red);
    tn = block_max<NT>(tn, red);
    const double htol = eps * fmax(hn, 1e-300);
    // QZ sweeps
    int ihi = m - 1, iter = 0, total = 0, failed = 0;
    while (ihi > 0) {
        int l = ihi;
        bool found = false;
        while (l > 0) {
            double sub = zabs(H(l, l - 1));
            double loc = zabs(H(l - 1, l - 1)) + zabs(H(l, l));
            if (sub <= eps * loc || sub <= htol) { found = true; break; }
            --l;
        }
        Team<NT>::bar();
        if (found) {
            if (tid == 0) H(l, l - 1) = zmake(0.0, 0.0);
            Team<NT>::bar();
        }
        if (l == ihi) { --ihi; iter = 0; continue; }
        if (++total > 60 * m) { failed = 1; break; }
        ++iter;
        zd sigma;
        zd h00 = H(ihi - 1, ihi - 1), h01 = H(ihi - 1, ihi), h10 = H(ihi, ihi - 1), h11 = H(ihi, ihi);
        zd t00 = T(ihi - 1, ihi - 1), t01 = T(ihi - 1, ihi), t11 = T(ihi, ihi);
        if (iter % 11 == 10) {
            zd den = (t11.x != 0.0 || t11.y != 0.0) ? t11 : zmake(1.0, 0.0);
            double a = zabs(h10);
            sigma = zadd(zdiv(h11, den), zmake(a, 0.5 * a));
        } else if (zabs(t00) > eps * tn && zabs(t11) > eps * tn) {
            zd qa = zmul(t00, t11);
            zd qb = zscale(zsub(zadd(zmul(h00, t11), zmul(h11, t00)), zmul(t01, h10)), -1.0);
            zd qc = zsub(zmul(h00, h11), zmul(h01, h10));
            zd disc = zsqrt_d(zsub(zmul(qb, qb), zscale(zmul(qa, qc), 4.0)));
            zd twoa = zscale(qa, 2.0);
            zd r1 = zdiv(zadd(zscale(qb, -1.0), disc), twoa);
            zd r2 = zdiv(zsub(zscale(qb, -1.0), disc), twoa);
            zd ref = zdiv(h11, t11);
            sigma = (zabs(zsub(r1, ref)) < zabs(zsub(r2, ref))) ? r1 : r2;
        } else {
            sigma = zmake(0.0, 0.0);
        }
        for (int k = l; k < ihi; ++k) {
            zd x, y;
            if (k == l) { x = zsub(H(l, l), zmul(sigma, T(l, l))); y = H(l + 1, l); }
            else        { x = H(k, k - 1); y = H(k + 1, k - 1); }
            giv_left(x, y, c, s);
            Team<NT>::bar();
            rot_rows2<NT>(H, (k > l) ? k - 1 : l, m - 1, (k > l) ? k - 1 : -1, T, k, m - 1, k, k + 1, c, s);
            Team<NT>::bar();
            giv_right(T(k + 1, k), T(k + 1, k + 1), c, s);
            Team<NT>::bar();
            int rl = (k + 2 < ihi) ? k + 2 : ihi;
            rot_cols3<NT>(H, rl, T, k + 1, k + 1, Z, m - 1, k, k + 1, c, s);
            Team<NT>::bar();
        }
    }
    if (failed && tid == 0 && fail) atomicAdd(fail, 1);
    // eigenvalues
    for (int k = tid; k < m; k += NT) { alpha[k] = H(k, k); beta[k] = T(k, k); }
    // y_hat_k by back-substitution, one thread per eigenvector
    const double small = eps * (hn + tn);
    for (int k = tid; k < m; k += NT) {
        const zd al = H(k, k), be = T(k, k);
        const double g = small * (zabs(al) + zabs(be));
        for (int i = k + 1; i < m; ++i) Yh(i, k) = zmake(0.0, 0.0);
        Yh(k, k) = zmake(1.0, 0.0);
        for (int i = k - 1; i >= 0; --i) {
            zd sum = zmake(0.0, 0.0);
            for (int p = i + 1; p <= k; ++p)
                zfma(sum, zsub(zmul(be, H(i, p)), zmul(al, T(i, p))), Yh(p, k));
            zd d = zsub(zmul(be, H(i, i)), zmul(al, T(i, i)));
            if (zabs(d) < g) d = zmake(g, 0.0);
            if (d.x == 0.0 && d.y == 0.0) d = zmake(1e-300, 0.0);
            zd q = zdiv(sum, d);
            Yh(i, k) = zmake(-q.x, -q.y);
        }
    }
    Team<NT>::bar();
    // V = Z * Y_hat with unit columns.  The product column k needs Y_hat(:, k)
    // only, and is written to a buffer that holds neither Z nor Y_hat: V
    // itself in the shared-memory layout (Y_hat is in work), H's storage in
    // the global layout (Y_hat is in V; H is no longer needed).
    Mat P = use_smem ? Mat{V, (int)ldv} : H;
    for (int k = tid; k < m; k += NT) {
        double nrm = 0.0;
        for (int r = 0; r < m; ++r) {
            zd acc = zmake(0.0, 0.0);
            for (int p = 0; p <= k; ++p) zfma(acc, Z(r, p), Yh(p, k));
            P(r, k) = acc;
            nrm += zabs2(acc);
        }
        nrm = sqrt(nrm);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 1.0;
        for (int r = 0; r < m; ++r) P(r, k) = zscale(P(r, k), inv);
    }
    Team<NT>::bar();
    if (use_smem) {
        for (int e = tid; e < m * m; e += NT) {
            int r = e % m, cc = e / m;
            A[r + cc * lda] = H(r, cc);
            B[r + cc * ldb] = T(r, cc);
        }
    } else {
        for (int e = tid; e < m * m; e += NT) {
            int r = e % m, cc = e / m;
            V[r + cc * ldv] = H(r, cc);
        }
    }
}
}  // namespace

size_t zqz_work_bytes(int m)
{
    size_t small = (size_t)m * m * sizeof(zd);
    if (m <= 64) return small;
    size_t big = zeig_large_work_bytes(m);
    return (big + 255) & ~(size_t)255;
}

int zqz_batched(cudaStream_t s, int m, int batch, zd *A, int64_t lda, int64_t sA, zd *B,
                int64_t ldb, int64_t sB, zd *alpha, zd *beta, zd *V, int64_t ldv, int64_t sV,
                void *work, int *fail, int *timeout, int *stats, double defl)
{
    if (m <= 0 || batch <= 0) return FEAST_OK;
    if (m <= 64) {
        size_t sm = 3 * (size_t)m * m * sizeof(zd);
        FEAST_CUDA_TRY(ensure_dyn_smem(k_qz<128>, sm));
        k_qz<128><<<batch, 128, sm, s>>>(m, A, lda, sA, B, ldb, sB, alpha, beta, V, ldv, sV, (zd *)work, 1, fail);
        FEAST_LAUNCH_CHECK();
        return FEAST_OK;
    }
    if (lda != m || ldb != m || ldv != m) return FEAST_EINVAL;
    const size_t wb = zqz_work_bytes(m);
    for (int b = 0; b < batch; ++b) {
        int e = zeig_large(s, m, A + (int64_t)b * sA, B + (int64_t)b * sB, alpha + (int64_t)b * m,
                           beta + (int64_t)b * m, V + (int64_t)b * sV, (char *)work + b * wb, fail,
                           timeout, stats, defl);
        if (e) return e;
    }
    return FEAST_OK;
}

}  // namespace feast
