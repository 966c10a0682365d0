// Projected eigenproblem for large subspaces (m0 > 64), FP64, GFEAST line 6.
//
// B~ = U2^H B U1 equals R2 of the QR B U1 = U2 R2 (upper triangular; its
// condition number is that of B on the search space), so the projected
// pencil is reduced to the standard problem C = B~^{-1} A~, whose
// eigenpairs are those of (A~, B~).  Then:
//   1. Hessenberg reduction C = Q H Q^H by Householder reflectors, one
//      column per step, each step a handful of grid-wide kernels;
//   2. single-shift complex QR sweeps on H with deflation, accumulating the
//      Schur vectors into Q.  A sweep's rotations form a dependent chain,
//      so they are generated in chunks of CH rotations by one warp on a small
//      diagonal block held in shared memory, and the rest of each rotation
//      (the long row / column / Schur-vector segments, which no later
//      rotation of the chunk reads) is applied by the whole grid in one
//      parallel pass.  The grid is a cooperative launch; its barriers spin
//      with an iteration limit and report a timeout instead of hanging;
//   3. right eigenvectors of the triangular Schur form by back-substitution
//      (one warp per eigenvector), mapped back by Q (a GEMM), unit norm.
// The small-pencil path (m0 <= 64, one warp, shared memory) is the QZ
// kernel in k_zqz.cu.
#include <cooperative_groups.h>

#include "common.cuh"

namespace feast {

namespace {

constexpr int CH = 32;           // rotations per chunk
constexpr int BLK = CH + 3;      // local block edge
constexpr int QT = 256;          // threads per CTA of the QR kernel
constexpr long long SPIN_LIMIT = 1ll << 24;

// ------------------------------------------------------------- Householder
// v = x - beta e1 with beta = -(x0/|x0|) ||x||, tau = 2 / ||v||^2, for
// x = C[j+1:m, j]; column j becomes (beta, 0, ..., 0).  One CTA.
__global__ void k_house(int m, int j, zd *C, int ld, zd *v, double *tau)
{
    __shared__ double red[32];
    __shared__ double s_norm;
    const int len = m - j - 1;
    zd *x = C + (j + 1) + (int64_t)j * ld;
    double part = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) part += zabs2(x[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        s_norm = sqrt(s);
    }
    __syncthreads();
    const double nrm = s_norm;
    const zd x0 = x[0];
    const double a0 = zabs(x0);
    const zd ph = a0 > 0.0 ? zscale(x0, 1.0 / a0) : zmake(1.0, 0.0);
    const zd beta = zscale(ph, -nrm);
    // v = x - beta e1 ;  ||v||^2 = 2 nrm (nrm + |x0|)
    const double vv = 2.0 * nrm * (nrm + a0);
    for (int i = threadIdx.x; i < len; i += blockDim.x) v[i] = (i == 0) ? zsub(x0, beta) : x[i];
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) x[i] = (i == 0) ? beta : zmake(0.0, 0.0);
    if (threadIdx.x == 0) *tau = vv > 0.0 ? 2.0 / vv : 0.0;
}

// w[c] = sum_i conj(v[i]) M[r0 + i, c0 + c]   (one warp per column)
__global__ void k_vh_times(int rows, int cols, const zd *M, int ld, const zd *v, zd *w)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= cols) return;
    const zd *col = M + (int64_t)warp * ld;
    zd acc = zmake(0.0, 0.0);
    for (int i = lane; i < rows; i += 32) zfma_conj(acc, v[i], col[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) w[warp] = acc;
}

// M[i, c] -= tau v[i] w[c]
__global__ void k_rank1_left(int rows, int cols, zd *M, int ld, const zd *v, const zd *w,
                             const double *tau)
{
    const double t = *tau;
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % rows), c = (int)(e / rows);
        zd a = M[i + (int64_t)c * ld];
        zfma(a, zscale(v[i], -t), w[c]);
        M[i + (int64_t)c * ld] = a;
    }
}

// u[r] = sum_c M[r, c0 + c] v[c]  for the rows of two matrices stacked
// (C and Q, each m rows); one thread per row
__global__ void k_times_v2(int m, int cols, const zd *C, const zd *Q, int ld, const zd *v, zd *u)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 2 * m) return;
    const zd *M = (r < m) ? C : Q;
    const int rr = (r < m) ? r : r - m;
    zd acc = zmake(0.0, 0.0);
    for (int c = 0; c < cols; ++c) zfma(acc, M[rr + (int64_t)c * ld], v[c]);
    u[r] = acc;
}

// M[r, c] -= tau u[r] conj(v[c]) for both stacked matrices
__global__ void k_rank1_right2(int m, int cols, zd *C, zd *Q, int ld, const zd *u, const zd *v,
                               const double *tau)
{
    const double t = *tau;
    const int64_t total = (int64_t)2 * m * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % (2 * m)), c = (int)(e / (2 * m));
        zd *M = (r < m) ? C : Q;
        int rr = (r < m) ? r : r - m;
        zd a = M[rr + (int64_t)c * ld];
        zfma(a, zscale(u[r], -t), zconj(v[c]));
        M[rr + (int64_t)c * ld] = a;
    }
}

__global__ void k_eye(int m, zd *Q, int ld)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % m), c = (int)(e / m);
        Q[r + (int64_t)c * ld] = zmake(r == c ? 1.0 : 0.0, 0.0);
    }
}

// ------------------------------------------------------------- QR sweeps
struct GridSync {
    unsigned *count;
    unsigned *gen;
    int *err;
};

// Sense-counting grid barrier for a cooperative launch, with a bounded spin:
// on timeout it raises *err and returns (every caller then bails out).
__device__ bool grid_barrier(const GridSync &g)
{
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = g.gen;
        const unsigned my = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(g.count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            *g.count = 0;
            __threadfence();
            atomicAdd(g.gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == my) {
                if (++it > SPIN_LIMIT || *(volatile int *)g.err) { ok = 0; atomicExch(g.err, 1); break; }
                __nanosleep(20);
            }
        }
        __threadfence();
        s_ok = ok && !*(volatile int *)g.err;
    }
    __syncthreads();
    return s_ok != 0;
}

struct Rot {
    double c;
    zd s;
};

__device__ __forceinline__ Rot make_rot(zd x, zd y)
{
    double ax = zabs(x), ay = zabs(y);
    Rot r;
    if (ay == 0.0) { r.c = 1.0; r.s = zmake(0.0, 0.0); return r; }
    if (ax == 0.0) { r.c = 0.0; r.s = zmake(1.0, 0.0); return r; }
    double h = hypot(ax, ay);
    r.c = ax / h;
    r.s = zscale(zmul(zscale(x, 1.0 / ax), zconj(y)), 1.0 / h);
    return r;
}
// left: [a; b] <- [c a + s b; -conj(s) a + c b]
__device__ __forceinline__ void rot_left(const Rot &g, zd &a, zd &b)
{
    zd na = zadd(zscale(a, g.c), zmul(g.s, b));
    zd nb = zsub(zscale(b, g.c), zmul(zconj(g.s), a));
    a = na;
    b = nb;
}
// right by G^H: [a b] <- [a c + b conj(s), -a s + b c]
__device__ __forceinline__ void rot_right(const Rot &g, zd &a, zd &b)
{
    zd na = zadd(zscale(a, g.c), zmul(b, zconj(g.s)));
    zd nb = zsub(zscale(b, g.c), zmul(a, g.s));
    a = na;
    b = nb;
}

__device__ __forceinline__ zd zsqrt_e(zd z)
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

// Whole QR phase: all CTAs run the same control flow (every decision is a
// function of values read after a grid barrier), CTA 0 generates each chunk
// of rotations, everybody applies the far parts.
__global__ void __launch_bounds__(QT) k_hqr(int m, zd *H, zd *Z, int ld, Rot *rots, GridSync g,
                                            int *fail, double hnorm)
{
    __shared__ zd blk[BLK][BLK + 1];
    __shared__ Rot srot[CH];
    const double eps = 2.220446049250313e-16;
    const double htol = eps * fmax(hnorm, 1e-300);
    const int gtid = blockIdx.x * QT + threadIdx.x, gthreads = gridDim.x * QT;
    int ihi = m - 1, iter = 0, total = 0;
    while (ihi > 0) {
        // deflation scan (identical in every CTA)
        int l = ihi;
        while (l > 0) {
            double sub = zabs(__ldcg(H + l + (int64_t)(l - 1) * ld));
            double loc = zabs(__ldcg(H + (l - 1) + (int64_t)(l - 1) * ld)) + zabs(__ldcg(H + l + (int64_t)l * ld));
            if (sub <= eps * loc || sub <= htol) break;
            --l;
        }
        if (l == ihi) { --ihi; iter = 0; continue; }
        if (++total > 40 * m) { if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(fail, 1); return; }
        ++iter;
        // Wilkinson shift from the trailing 2 x 2 block (exceptional shift
        // every 11th sweep without deflation)
        zd sigma;
        {
            zd h00 = __ldcg(H + (ihi - 1) + (int64_t)(ihi - 1) * ld), h01 = __ldcg(H + (ihi - 1) + (int64_t)ihi * ld);
            zd h10 = __ldcg(H + ihi + (int64_t)(ihi - 1) * ld), h11 = __ldcg(H + ihi + (int64_t)ihi * ld);
            if (iter % 11 == 10) {
                double a = zabs(h10);
                sigma = zadd(h11, zmake(a, 0.5 * a));
            } else {
                zd tr = zadd(h00, h11), det = zsub(zmul(h00, h11), zmul(h01, h10));
                zd disc = zsqrt_e(zsub(zscale(zmul(tr, tr), 0.25), det));
                zd half = zscale(tr, 0.5);
                zd r1 = zadd(half, disc), r2 = zsub(half, disc);
                sigma = (zabs(zsub(r1, h11)) < zabs(zsub(r2, h11))) ? r1 : r2;
            }
        }
        // every CTA has read what it needs for l, ihi and sigma before CTA 0
        // starts rewriting the leading block of the sweep
        if (!grid_barrier(g)) return;
        for (int k0 = l; k0 < ihi; k0 += CH) {
            const int k1 = (k0 + CH < ihi) ? k0 + CH : ihi;   // rotations k0 .. k1-1
            const int b0 = (k0 - 1 > 0) ? k0 - 1 : 0;
            const int b1 = (k1 + 1 < m - 1) ? k1 + 1 : m - 1;
            const int nb = b1 - b0 + 1;
            if (blockIdx.x == 0) {
                for (int e = threadIdx.x; e < nb * nb; e += QT) {
                    int r = e % nb, c = e / nb;
                    blk[r][c] = __ldcg(H + (b0 + r) + (int64_t)(b0 + c) * ld);
                }
                __syncthreads();
                if (threadIdx.x < 32) {
                    const int lane = threadIdx.x;
                    for (int k = k0; k < k1; ++k) {
                        const int kr = k - b0;
                        zd x, y;
                        if (k == l) {
                            x = zsub(blk[kr][kr], sigma);
                            y = blk[kr + 1][kr];
                        } else {
                            x = blk[kr][kr - 1];
                            y = blk[kr + 1][kr - 1];
                        }
                        Rot gr = make_rot(x, y);
                        __syncwarp();
                        const int cs = (k == l) ? kr : kr - 1;
                        for (int c = cs + lane; c < nb; c += 32) rot_left(gr, blk[kr][c], blk[kr + 1][c]);
                        __syncwarp();
                        if (k > l && lane == 0) blk[kr + 1][kr - 1] = zmake(0.0, 0.0);
                        const int rl = ((k + 2 < ihi) ? k + 2 : ihi) - b0;
                        for (int r = lane; r <= rl && r < nb; r += 32) rot_right(gr, blk[r][kr], blk[r][kr + 1]);
                        __syncwarp();
                        if (lane == 0) srot[k - k0] = gr;
                    }
                }
                __syncthreads();
                for (int e = threadIdx.x; e < nb * nb; e += QT) {
                    int r = e % nb, c = e / nb;
                    __stcg(H + (b0 + r) + (int64_t)(b0 + c) * ld, blk[r][c]);
                }
                for (int e = threadIdx.x; e < k1 - k0; e += QT) {
                    __stcg(&rots[e].c, srot[e].c);
                    __stcg(&rots[e].s, srot[e].s);
                }
            }
            if (!grid_barrier(g)) return;
            // far parts: left rotations on rows k0..k1 for columns > b1,
            // right rotations on columns k0..k1 for rows < b0 of H and all
            // rows of Z
            const int nrot = k1 - k0;
            const int ncol = m - 1 - b1, nrowH = b0;
            const int lines = ncol + nrowH + m;
            if (blockIdx.x != 0) {
                for (int e = threadIdx.x; e < nrot; e += QT) {
                    srot[e].c = __ldcg(&rots[e].c);
                    srot[e].s = __ldcg(&rots[e].s);
                }
            }
            __syncthreads();
            for (int t = gtid; t < lines; t += gthreads) {
                zd seg[CH + 1];
                if (t < ncol) {
                    zd *col = H + (int64_t)(b1 + 1 + t) * ld + k0;
#pragma unroll
                    for (int i = 0; i <= CH; ++i)
                        if (i <= nrot) seg[i] = __ldcg(col + i);
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        if (i < nrot) rot_left(srot[i], seg[i], seg[i + 1]);
#pragma unroll
                    for (int i = 0; i <= CH; ++i)
                        if (i <= nrot) __stcg(col + i, seg[i]);
                } else {
                    const int r = (t < ncol + nrowH) ? t - ncol : t - ncol - nrowH;
                    zd *row = ((t < ncol + nrowH) ? H : Z) + r + (int64_t)k0 * ld;
#pragma unroll
                    for (int i = 0; i <= CH; ++i)
                        if (i <= nrot) seg[i] = __ldcg(row + (int64_t)i * ld);
#pragma unroll
                    for (int i = 0; i < CH; ++i)
                        if (i < nrot) rot_right(srot[i], seg[i], seg[i + 1]);
#pragma unroll
                    for (int i = 0; i <= CH; ++i)
                        if (i <= nrot) __stcg(row + (int64_t)i * ld, seg[i]);
                }
            }
            if (!grid_barrier(g)) return;
        }
    }
}

// Eigenvector k of the upper-triangular Schur form S: (S - S_kk I) y = 0,
// y_k = 1, back-substitution; one warp per eigenvector.  Y is m x m
// (upper triangular on output).
__global__ void k_schur_vectors(int m, const zd *S, int ld, zd *Y, double snorm)
{
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= m) return;
    const double eps = 2.220446049250313e-16;
    const double small = eps * fmax(snorm, 1e-300);
    zd *y = Y + (int64_t)k * ld;
    const zd lam = S[k + (int64_t)k * ld];
    for (int i = k + 1 + lane; i < m; i += 32) y[i] = zmake(0.0, 0.0);
    if (lane == 0) y[k] = zmake(1.0, 0.0);
    __syncwarp();
    for (int i = k - 1; i >= 0; --i) {
        zd acc = zmake(0.0, 0.0);
        for (int p = i + 1 + lane; p <= k; p += 32) zfma(acc, S[i + (int64_t)p * ld], y[p]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) {
            zd d = zsub(S[i + (int64_t)i * ld], lam);
            if (zabs(d) < small) d = zmake(small, 0.0);
            zd q = zdiv(acc, d);
            y[i] = zmake(-q.x, -q.y);
        }
        __syncwarp();
    }
}

__global__ void k_normalise_cols(int m, zd *V, int ld)
{
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= m) return;
    zd *v = V + (int64_t)k * ld;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += zabs2(v[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    for (int i = lane; i < m; i += 32) v[i] = zscale(v[i], inv);
}

__global__ void k_diag_out(int m, const zd *S, int ld, zd *alpha, zd *beta)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    alpha[k] = S[k + (int64_t)k * ld];
    beta[k] = zmake(1.0, 0.0);
}

__global__ void k_absmax(int64_t count, const zd *x, double *out)
{
    __shared__ double red[32];
    double v = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        v = fmax(v, zabs(x[e]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = fmax(r, red[w]);
        // non-negative doubles order like their bit patterns
        atomicMax((unsigned long long *)out, (unsigned long long)__double_as_longlong(r));
    }
}

}  // namespace

size_t zeig_large_work_bytes(int m)
{
    // Q (m*m) + v (m) + w (m) + u (2m) complex, tau, absmax, rotations,
    // barrier words
    return sizeof(zd) * ((size_t)m * m + 4 * (size_t)m) + 64 + sizeof(Rot) * CH + 64;
}

// A (m x m, overwritten), Bt (m x m upper triangular, overwritten by the
// solve), alpha/beta (beta = 1), V (m x m unit eigenvectors).
int zeig_large(cudaStream_t s, int m, zd *A, zd *Bt, zd *alpha, zd *beta, zd *V, void *work,
               int *fail, int *timeout)
{
    if (m <= 0) return FEAST_OK;
    char *w = (char *)work;
    zd *Q = (zd *)w;
    zd *v = Q + (size_t)m * m;
    zd *wv = v + m;
    zd *u = wv + m;
    double *tau = (double *)(u + 2 * m);
    double *hmax = tau + 1;
    Rot *rots = (Rot *)(hmax + 7);
    unsigned *bar = (unsigned *)(rots + CH);
    int e;
    // C = B~^{-1} A~  (upper-triangular solve with m right-hand sides)
    if ((e = trsm_upper_batched<zd>(s, m, m, 1, Bt, m, 0, A, m, 0))) return e;
    zd *C = A;
    k_eye<<<cdiv((size_t)m * m, 256) > 2048 ? 2048 : cdiv((size_t)m * m, 256), 256, 0, s>>>(m, Q, m);
    FEAST_LAUNCH_CHECK();
    // Hessenberg reduction C <- Q^H C Q
    for (int j = 0; j + 2 < m; ++j) {
        const int len = m - j - 1;
        k_house<<<1, 256, 0, s>>>(m, j, C, m, v, tau);
        FEAST_LAUNCH_CHECK();
        zd *blkC = C + (j + 1) + (int64_t)(j + 1) * m;
        k_vh_times<<<cdiv((size_t)len * 32, 256), 256, 0, s>>>(len, len, blkC, m, v, wv);
        FEAST_LAUNCH_CHECK();
        unsigned g1 = cdiv((size_t)len * len, 256);
        k_rank1_left<<<g1 > 4096 ? 4096 : g1, 256, 0, s>>>(len, len, blkC, m, v, wv, tau);
        FEAST_LAUNCH_CHECK();
        k_times_v2<<<cdiv((size_t)2 * m, 128), 128, 0, s>>>(m, len, C + (int64_t)(j + 1) * m,
                                                           Q + (int64_t)(j + 1) * m, m, v, u);
        FEAST_LAUNCH_CHECK();
        unsigned g2 = cdiv((size_t)2 * m * len, 256);
        k_rank1_right2<<<g2 > 4096 ? 4096 : g2, 256, 0, s>>>(m, len, C + (int64_t)(j + 1) * m,
                                                             Q + (int64_t)(j + 1) * m, m, u, v, tau);
        FEAST_LAUNCH_CHECK();
    }
    // norm for the deflation test
    FEAST_CUDA_TRY(cudaMemsetAsync(hmax, 0, sizeof(double), s));
    k_absmax<<<64, 256, 0, s>>>((int64_t)m * m, C, hmax);
    FEAST_LAUNCH_CHECK();
    double hn = 0.0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&hn, hmax, sizeof(double), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaMemsetAsync(bar, 0, 16, s));
    FEAST_CUDA_TRY(cudaMemsetAsync(timeout, 0, sizeof(int), s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    // QR sweeps: cooperative grid, one CTA per SM at most
    int dev = 0, sms = 0, per = 0;
    FEAST_CUDA_TRY(cudaGetDevice(&dev));
    FEAST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hqr, QT, 0));
    if (per < 1) return FEAST_ECUDA;
    // one CTA per SM (the far-part pass has ~3 m independent lines, each a
    // chain of up to CH rotations on the FP64 pipe, so every SM's FP64 units
    // are worth having even when there are fewer lines than threads)
    int grid = sms * (per < 1 ? 1 : 1);
    GridSync gs{bar, bar + 1, timeout};
    double hnorm = hn;
    int mm = m, ldh = m;
    void *args[] = {&mm, &C, &Q, &ldh, &rots, &gs, &fail, &hnorm};
    FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_hqr, dim3(grid), dim3(QT), args, 0, s));
    FEAST_LAUNCH_CHECK();
    // eigenvalues and eigenvectors
    k_diag_out<<<cdiv(m, 128), 128, 0, s>>>(m, C, m, alpha, beta);
    FEAST_LAUNCH_CHECK();
    zd *Yh = Bt;  // B~ is no longer needed
    k_schur_vectors<<<cdiv((size_t)m * 32, 256), 256, 0, s>>>(m, C, m, Yh, hn);
    FEAST_LAUNCH_CHECK();
    if ((e = zgemm_batched(s, 0, m, m, m, zmake(1.0, 0.0), Q, m, 0, Yh, m, 0, zmake(0.0, 0.0), V, m, 0, 1)))
        return e;
    k_normalise_cols<<<cdiv((size_t)m * 32, 256), 256, 0, s>>>(m, V, m);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
