// FP64 complex dense kernels of the plain GPU path: batched GEMM, formation
// of the shifted matrices z_j B - A (eq. 4.2), blocked right-looking LU with
// partial pivoting, blocked triangular solves with many right-hand sides,
// and the quadrature node-sum U = sum_j w_j X_j (eq. 4.1).
//
// GB300 runs FP64 at ~2 DFMA per clock per SM (1.05 TFLOP/s measured for
// the whole GPU), so these kernels are bound by the FP64 pipe, not by
// memory: a modest register tile (4 x 4 complex per thread) already keeps
// the pipe busy, and the work is spread over all 152 SMs through the batch
// (node) dimension and the tile grid.
#include "common.cuh"

namespace feast {

// ------------------------------------------------------------------ GEMM
namespace {
constexpr int GB_M = 64, GB_N = 64, GB_K = 8, GB_T = 256;

__global__ void __launch_bounds__(GB_T) k_zgemm(int conj_a, int64_t m, int64_t n, int64_t k,
                                                zd alpha, const zd *__restrict__ A, int64_t lda,
                                                int64_t sA, const zd *__restrict__ B,
                                                int64_t ldb, int64_t sB, zd beta,
                                                zd *__restrict__ C, int64_t ldc, int64_t sC)
{
    __shared__ zd As[GB_K][GB_M + 1];
    __shared__ zd Bs[GB_K][GB_N + 1];
    const int b = blockIdx.z;
    A += (int64_t)b * sA;
    B += (int64_t)b * sB;
    C += (int64_t)b * sC;
    const int64_t i0 = (int64_t)blockIdx.x * GB_M, j0 = (int64_t)blockIdx.y * GB_N;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    zd acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = zmake(0.0, 0.0);

    for (int64_t k0 = 0; k0 < k; k0 += GB_K) {
        // A tile: op(A)(i0 + r, k0 + kk)
        for (int e = threadIdx.x; e < GB_M * GB_K; e += GB_T) {
            int r, kk;
            if (!conj_a) { r = e % GB_M; kk = e / GB_M; }
            else         { kk = e % GB_K; r = e / GB_K; }
            int64_t gi = i0 + r, gk = k0 + kk;
            zd v = zmake(0.0, 0.0);
            if (gi < m && gk < k) v = conj_a ? zconj(A[gk + gi * lda]) : A[gi + gk * lda];
            As[kk][r] = v;
        }
        for (int e = threadIdx.x; e < GB_N * GB_K; e += GB_T) {
            int kk = e % GB_K, c = e / GB_K;
            int64_t gj = j0 + c, gk = k0 + kk;
            Bs[kk][c] = (gj < n && gk < k) ? B[gk + gj * ldb] : zmake(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            zd av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) zfma(acc[a][c], av[a], bv[c]);
        }
        __syncthreads();
    }
    const bool beta0 = (beta.x == 0.0 && beta.y == 0.0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * c;
            if (gi < m && gj < n) {
                zd v = zmul(alpha, acc[a][c]);
                if (!beta0) v = zadd(v, zmul(beta, C[gi + gj * ldc]));
                C[gi + gj * ldc] = v;
            }
        }
}
}  // namespace

int zgemm_batched(cudaStream_t s, int conj_a, int64_t m, int64_t n, int64_t k, zd alpha,
                  const zd *A, int64_t lda, int64_t sA, const zd *B, int64_t ldb, int64_t sB,
                  zd beta, zd *C, int64_t ldc, int64_t sC, int batch)
{
    if (m <= 0 || n <= 0 || batch <= 0) return FEAST_OK;
    if (batch > 65535) return FEAST_EINVAL;
    dim3 grid(cdiv(m, GB_M), cdiv(n, GB_N), batch);
    if (grid.y > 65535) return FEAST_EINVAL;
    k_zgemm<<<grid, GB_T, 0, s>>>(conj_a, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// ------------------------------------------------------------------ z_j B - A
namespace {
__global__ void k_form_shifted(int64_t n, const zd *__restrict__ A, const zd *__restrict__ B,
                               int64_t ld, const zd *__restrict__ z, zd *__restrict__ F,
                               int64_t ldf, int64_t sF)
{
    const int j = blockIdx.y;
    const zd zj = z[j];
    const int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        zd bij = B ? B[r + c * ld] : zmake(r == c ? 1.0 : 0.0, 0.0);
        F[(int64_t)j * sF + r + c * ldf] = zsub(zmul(zj, bij), A[r + c * ld]);
    }
}
}  // namespace

int zform_shifted(cudaStream_t s, int64_t n, int q, const zd *A, const zd *B, int64_t ld,
                  const zd *z, zd *F, int64_t ldf, int64_t sF)
{
    unsigned gx = cdiv(n * n, 256);
    if (gx > 1024) gx = 1024;
    k_form_shifted<<<dim3(gx, q), 256, 0, s>>>(n, A, B, ld, z, F, ldf, sF);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// ------------------------------------------------------------------ LU
namespace {
constexpr int LU_NB = 32;     // panel width
constexpr int LU_PT = 512;    // panel threads

// Factor the panel [k0, k0 + nb) x [k0, n) of every batch member: pivot by
// largest modulus (ties -> smallest row), swap within the panel columns,
// scale, rank-1 update of the remaining panel columns.
__global__ void __launch_bounds__(LU_PT) k_lu_panel(int64_t n, int64_t k0, int nb, zd *F,
                                                   int64_t ldf, int64_t sF, int *piv,
                                                   int *info, int *row)
{
    const int b = blockIdx.x;
    zd *Am = F + (int64_t)b * sF;
    __shared__ double s_val[LU_PT / 32];
    __shared__ int64_t s_idx[LU_PT / 32];
    __shared__ int64_t s_p;
    __shared__ zd s_row[LU_NB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < nb; ++j) {
        const int64_t col = k0 + j;
        double best = -1.0;
        int64_t bi = col;
        for (int64_t i = col + threadIdx.x; i < n; i += LU_PT) {
            double v = zabs2(Am[i + col * ldf]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double ov = __shfl_down_sync(0xffffffffu, best, off);
            int64_t oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double bv = s_val[0];
            int64_t bx = s_idx[0];
            for (int w = 1; w < LU_PT / 32; ++w)
                if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bx)) { bv = s_val[w]; bx = s_idx[w]; }
            s_p = bx;
            piv[(int64_t)b * n + col] = (int)bx;
            if (bv == 0.0 && info) {
                // record the first failing block (1-based) and column
                if (atomicCAS(info, 0, b + 1) == 0 && row) *row = (int)col + 1;
            }
        }
        __syncthreads();
        const int64_t p = s_p;
        if (p != col && threadIdx.x < nb) {
            int64_t c = k0 + threadIdx.x;
            zd t = Am[col + c * ldf];
            Am[col + c * ldf] = Am[p + c * ldf];
            Am[p + c * ldf] = t;
        }
        __syncthreads();
        if (threadIdx.x < nb) s_row[threadIdx.x] = Am[col + (k0 + threadIdx.x) * ldf];
        __syncthreads();
        const zd d = s_row[j];
        if (d.x != 0.0 || d.y != 0.0) {
            for (int64_t i = col + 1 + threadIdx.x; i < n; i += LU_PT) {
                zd l = zdiv(Am[i + col * ldf], d);
                Am[i + col * ldf] = l;
                for (int c = j + 1; c < nb; ++c) {
                    zd &a = Am[i + (k0 + c) * ldf];
                    zd v = a;
                    zfma(v, zmake(-l.x, -l.y), s_row[c]);
                    a = v;
                }
            }
        }
        __syncthreads();
    }
}

// Apply the panel's row interchanges to the columns outside the panel.
__global__ void k_laswp_outside(int64_t n, int64_t k0, int nb, zd *F, int64_t ldf, int64_t sF,
                                const int *piv)
{
    const int b = blockIdx.y;
    zd *Am = F + (int64_t)b * sF;
    const int *pv = piv + (int64_t)b * n;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= k0 && c < k0 + nb) continue;
        for (int j = 0; j < nb; ++j) {
            int64_t r = k0 + j, p = pv[r];
            if (p != r) {
                zd t = Am[r + c * ldf];
                Am[r + c * ldf] = Am[p + c * ldf];
                Am[p + c * ldf] = t;
            }
        }
    }
}

// U12 = L11^{-1} A12 for the nb rows of the panel (L11 unit lower), one
// thread per column to the right of the panel.
__global__ void k_trsm_u12(int64_t n, int64_t k0, int nb, zd *F, int64_t ldf, int64_t sF)
{
    const int b = blockIdx.y;
    zd *Am = F + (int64_t)b * sF;
    __shared__ zd L[LU_NB][LU_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e % nb, c = e / nb;
        L[r][c] = Am[(k0 + r) + (k0 + c) * ldf];
    }
    __syncthreads();
    const int64_t c = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    zd x[LU_NB];
#pragma unroll
    for (int r = 0; r < LU_NB; ++r)
        if (r < nb) x[r] = Am[(k0 + r) + c * ldf];
#pragma unroll
    for (int i = 0; i < LU_NB; ++i) {
        if (i >= nb) break;
#pragma unroll
        for (int r = i + 1; r < LU_NB; ++r)
            if (r < nb) zfma(x[r], zmake(-L[r][i].x, -L[r][i].y), x[i]);
    }
#pragma unroll
    for (int r = 0; r < LU_NB; ++r)
        if (r < nb) Am[(k0 + r) + c * ldf] = x[r];
}
}  // namespace

int zgetrf_batched(cudaStream_t s, int64_t n, int batch, zd *F, int64_t ldf, int64_t sF,
                   int *piv, int *info, int *row)
{
    if (n <= 0 || batch <= 0) return FEAST_OK;
    for (int64_t k0 = 0; k0 < n; k0 += LU_NB) {
        int nb = (int)((n - k0) < LU_NB ? (n - k0) : LU_NB);
        k_lu_panel<<<batch, LU_PT, 0, s>>>(n, k0, nb, F, ldf, sF, piv, info, row);
        FEAST_LAUNCH_CHECK();
        unsigned gx = cdiv(n, 128);
        k_laswp_outside<<<dim3(gx, batch), 128, 0, s>>>(n, k0, nb, F, ldf, sF, piv);
        FEAST_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest > 0) {
            k_trsm_u12<<<dim3(cdiv(rest, 128), batch), 128, 0, s>>>(n, k0, nb, F, ldf, sF);
            FEAST_LAUNCH_CHECK();
            int e = zgemm_batched(s, 0, rest, rest, nb, zmake(-1.0, 0.0), F + k0 + nb + k0 * ldf,
                                  ldf, sF, F + k0 + (k0 + nb) * ldf, ldf, sF, zmake(1.0, 0.0),
                                  F + (k0 + nb) + (k0 + nb) * ldf, ldf, sF, batch);
            if (e) return e;
        }
    }
    return FEAST_OK;
}

// ------------------------------------------------------------------ solves
namespace {
constexpr int SV_NB = 32;

// X rows [k0, k0+nb) <- T^{-1} X rows [k0, k0+nb) for the diagonal block T of
// the factor (lower = unit lower L, else upper U).  One thread per column.
__global__ void k_trsv_diag(int64_t n, int64_t nrhs, int64_t k0, int nb, int lower,
                            const zd *F, int64_t ldf, int64_t sF, zd *X, int64_t ldx, int64_t sX)
{
    const int b = blockIdx.y;
    const zd *Am = F + (int64_t)b * sF;
    zd *Xb = X + (int64_t)b * sX;
    __shared__ zd T[SV_NB][SV_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e % nb, c = e / nb;
        T[r][c] = Am[(k0 + r) + (k0 + c) * ldf];
    }
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    zd x[SV_NB];
#pragma unroll
    for (int r = 0; r < SV_NB; ++r)
        if (r < nb) x[r] = Xb[(k0 + r) + c * ldx];
    if (lower) {
#pragma unroll
        for (int i = 0; i < SV_NB; ++i) {
            if (i >= nb) break;
#pragma unroll
            for (int r = i + 1; r < SV_NB; ++r)
                if (r < nb) zfma(x[r], zmake(-T[r][i].x, -T[r][i].y), x[i]);
        }
    } else {
#pragma unroll
        for (int i = SV_NB - 1; i >= 0; --i) {
            if (i >= nb) continue;
            x[i] = zdiv(x[i], T[i][i]);
#pragma unroll
            for (int r = 0; r < SV_NB; ++r)
                if (r < i) zfma(x[r], zmake(-T[r][i].x, -T[r][i].y), x[i]);
        }
    }
#pragma unroll
    for (int r = 0; r < SV_NB; ++r)
        if (r < nb) Xb[(k0 + r) + c * ldx] = x[r];
}

// Apply the interchanges piv[0..n) to each column of X in sequence.
__global__ void k_laswp_rhs(int64_t n, int64_t nrhs, const int *piv, zd *X, int64_t ldx,
                            int64_t sX)
{
    const int b = blockIdx.y;
    zd *Xb = X + (int64_t)b * sX;
    const int *pv = piv + (int64_t)b * n;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = pv[k];
        if (p != k) {
            zd t = Xb[k + c * ldx];
            Xb[k + c * ldx] = Xb[p + c * ldx];
            Xb[p + c * ldx] = t;
        }
    }
}

// Composition of the interchanges: perm[i] = original row that ends at i.
__global__ void k_piv_to_perm(int64_t n, const int *piv, int *perm)
{
    const int b = blockIdx.x;
    const int *pv = piv + (int64_t)b * n;
    int *pm = perm + (int64_t)b * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) pm[i] = (int)i;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int64_t k = 0; k < n; ++k) {
            int64_t p = pv[k];
            if (p != k) { int t = pm[k]; pm[k] = pm[p]; pm[p] = t; }
        }
}

__global__ void k_gather_rows(int64_t n, int64_t nrhs, const int *perm, const zd *R, int64_t ldr,
                              zd *X, int64_t ldx, int64_t sX)
{
    const int b = blockIdx.y;
    const int *pm = perm + (int64_t)b * n;
    zd *Xb = X + (int64_t)b * sX;
    const int64_t total = n * nrhs;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        Xb[r + c * ldx] = R[pm[r] + c * ldr];
    }
}
}  // namespace

int zpiv_to_perm(cudaStream_t s, int64_t n, int batch, const int *piv, int *perm)
{
    k_piv_to_perm<<<batch, 256, 0, s>>>(n, piv, perm);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int zgather_rows(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const int *perm,
                 const zd *R, int64_t ldr, zd *X, int64_t ldx, int64_t sX)
{
    unsigned gx = cdiv(n * nrhs, 256);
    if (gx > 2048) gx = 2048;
    k_gather_rows<<<dim3(gx, batch), 256, 0, s>>>(n, nrhs, perm, R, ldr, X, ldx, sX);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// L U solve of already-permuted right-hand sides.
int ztrsm_lu_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const zd *F,
                     int64_t ldf, int64_t sF, zd *X, int64_t ldx, int64_t sX)
{
    if (n <= 0 || nrhs <= 0 || batch <= 0) return FEAST_OK;
    dim3 g(cdiv(nrhs, 64), batch);
    // forward: L (unit lower)
    for (int64_t k0 = 0; k0 < n; k0 += SV_NB) {
        int nb = (int)((n - k0) < SV_NB ? (n - k0) : SV_NB);
        k_trsv_diag<<<g, 64, 0, s>>>(n, nrhs, k0, nb, 1, F, ldf, sF, X, ldx, sX);
        FEAST_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest > 0) {
            int e = zgemm_batched(s, 0, rest, nrhs, nb, zmake(-1.0, 0.0), F + (k0 + nb) + k0 * ldf,
                                  ldf, sF, X + k0, ldx, sX, zmake(1.0, 0.0), X + k0 + nb, ldx, sX,
                                  batch);
            if (e) return e;
        }
    }
    // backward: U
    int64_t last = ((n - 1) / SV_NB) * SV_NB;
    for (int64_t k0 = last; k0 >= 0; k0 -= SV_NB) {
        int nb = (int)((n - k0) < SV_NB ? (n - k0) : SV_NB);
        k_trsv_diag<<<g, 64, 0, s>>>(n, nrhs, k0, nb, 0, F, ldf, sF, X, ldx, sX);
        FEAST_LAUNCH_CHECK();
        if (k0 > 0) {
            int e = zgemm_batched(s, 0, k0, nrhs, nb, zmake(-1.0, 0.0), F + k0 * ldf, ldf, sF,
                                  X + k0, ldx, sX, zmake(1.0, 0.0), X, ldx, sX, batch);
            if (e) return e;
        }
    }
    return FEAST_OK;
}

int zgetrs_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const zd *F,
                   int64_t ldf, int64_t sF, const int *piv, zd *X, int64_t ldx, int64_t sX)
{
    if (n <= 0 || nrhs <= 0 || batch <= 0) return FEAST_OK;
    k_laswp_rhs<<<dim3(cdiv(nrhs, 64), batch), 64, 0, s>>>(n, nrhs, piv, X, ldx, sX);
    FEAST_LAUNCH_CHECK();
    return ztrsm_lu_batched(s, n, nrhs, batch, F, ldf, sF, X, ldx, sX);
}

// ------------------------------------------------------------------ node sum
namespace {
__global__ void k_node_sum(int64_t n, int64_t m, int q, const zd *__restrict__ w,
                           const zd *__restrict__ X, int64_t ldx, int64_t sX, zd *__restrict__ U,
                           int64_t ldu)
{
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        zd acc = zmake(0.0, 0.0);
        for (int j = 0; j < q; ++j) zfma(acc, w[j], X[(int64_t)j * sX + r + c * ldx]);
        U[r + c * ldu] = acc;
    }
}
}  // namespace

int znode_sum(cudaStream_t s, int64_t n, int64_t m, int q, const zd *w, const zd *X,
              int64_t ldx, int64_t sX, zd *U, int64_t ldu)
{
    unsigned gx = cdiv(n * m, 256);
    if (gx > 152 * 16) gx = 152 * 16;
    k_node_sum<<<gx, 256, 0, s>>>(n, m, q, w, X, ldx, sX, U, ldu);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
