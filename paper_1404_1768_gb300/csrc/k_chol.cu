// QR of a tall block by Cholesky QR, twice (precision form; GFEAST lines 2
// and 17):
//
//     G = V^H V = R_a^H R_a,  Q_1 = V R_a^{-1};   Q_1^H Q_1 = R_b^H R_b,
//     Q = Q_1 R_b^{-1},  R = R_b R_a.
//
// The Gram matrices and the products V R^{-1} are FP64-accurate GEMMs on the
// tensor cores (k_oz.cu); the Cholesky factorisations and the triangular
// inverses are FP64.  The first pass leaves Q_1 orthonormal to ~eps
// cond(V)^2, the second to ~eps, while cond(V) stays below ~1e6.  Every
// pivot is checked against its column's original norm: a pivot below
// 1e-12 of it (cond(V) out of reach) reports failure and the caller runs
// the column-by-column BCGS2 instead.  R has a real positive diagonal, like
// the Householder QR with that sign convention, so Q and R are the same
// unique factors.
#include "common.cuh"

namespace feast {
namespace {

constexpr int CB = 32;  // Cholesky block

__global__ void k_diag_copy(int m, const zd *__restrict__ G, double *__restrict__ d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) d[i] = G[i + (int64_t)i * m].x;
}

// Unblocked Cholesky of the diagonal block G[k0:k0+nb, k0:k0+nb] (upper
// triangle in, R's upper triangle out).  Thread (i, k) of 32 x 32 owns
// entry (i, k); three barriers per column.
__global__ void __launch_bounds__(CB * CB) k_chol_diag(int m, zd *__restrict__ G, int k0, int nb,
                                                       const double *__restrict__ d0, int *__restrict__ fail)
{
    __shared__ zd T[CB][CB + 1];
    __shared__ double rinv;
    const int i = threadIdx.x % CB, k = threadIdx.x / CB;
    const bool live = (i < nb && k < nb);
    if (live) T[i][k] = G[(k0 + i) + (int64_t)(k0 + k) * m];
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double d = T[j][j].x;
            const double ref = d0[k0 + j];
            double r;
            if (!(d > 1e-12 * ref) || !(ref > 0.0)) {
                *fail = 1;
                r = 1.0;
            } else {
                r = sqrt(d);
            }
            T[j][j] = zmake(r, 0.0);
            rinv = 1.0 / r;
        }
        __syncthreads();
        if (live && i == j && k > j) T[j][k] = zscale(T[j][k], rinv);
        __syncthreads();
        if (live && i > j && k >= i) {
            const zd rji = T[j][i], rjk = T[j][k];
            // T[i][k] -= conj(r_ji) r_jk
            T[i][k] = zsub(T[i][k], zmake(rji.x * rjk.x + rji.y * rjk.y, rji.x * rjk.y - rji.y * rjk.x));
        }
        __syncthreads();
    }
    if (live && k >= i) G[(k0 + i) + (int64_t)(k0 + k) * m] = T[i][k];
}

// Row block of R right of the diagonal block: R[k0:k0+nb, c] solves
// R_kk^H x = G[k0:k0+nb, c] (forward substitution), thread per column c.
__global__ void k_chol_row(int m, zd *__restrict__ G, int k0, int nb)
{
    __shared__ zd T[CB][CB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        T[r][c] = G[(k0 + r) + (int64_t)(k0 + c) * m];
    }
    __syncthreads();
    const int c = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    zd x[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i)
        if (i < nb) x[i] = G[(k0 + i) + (int64_t)c * m];
#pragma unroll
    for (int i = 0; i < CB; ++i) {
        if (i >= nb) break;
        zd acc = x[i];
#pragma unroll
        for (int p = 0; p < CB; ++p) {
            if (p >= i) break;
            const zd t = T[p][i];  // R_pi; (R^H)_ip = conj(R_pi)
            acc = zsub(acc, zmake(t.x * x[p].x + t.y * x[p].y, t.x * x[p].y - t.y * x[p].x));
        }
        x[i] = zscale(acc, 1.0 / T[i][i].x);
    }
#pragma unroll
    for (int i = 0; i < CB; ++i)
        if (i < nb) G[(k0 + i) + (int64_t)c * m] = x[i];
}

// Zero the strictly lower triangle (m x m, leading dim ld).
__global__ void k_zero_lower(int m, zd *__restrict__ R, int64_t ld)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        if (i > j) R[i + (int64_t)j * ld] = zmake(0.0, 0.0);
    }
}

// Inverse of each CB x CB diagonal block of the upper triangular R (ld
// ldr) into Ri (ld m): block b by CTA b, thread k builds column k of the
// block's inverse by back-substitution.
__global__ void __launch_bounds__(CB) k_trinv_diag(int m, const zd *__restrict__ R, int64_t ldr, zd *__restrict__ Ri)
{
    __shared__ zd T[CB][CB + 1];
    const int b0 = blockIdx.x * CB;
    const int nb = (m - b0) < CB ? (m - b0) : CB;
    const int k = threadIdx.x;
    for (int i = 0; i < nb; ++i)
        if (k < nb) T[i][k] = R[(b0 + i) + (int64_t)(b0 + k) * ldr];
    __syncthreads();
    if (k >= nb) return;
    zd x[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) x[i] = zmake(0.0, 0.0);
    x[k] = zdiv(zmake(1.0, 0.0), T[k][k]);
#pragma unroll
    for (int i = CB - 1; i >= 0; --i) {
        if (i >= k) continue;
        zd acc = zmake(0.0, 0.0);
#pragma unroll
        for (int p = 0; p < CB; ++p)
            if (p > i && p <= k) zfma(acc, T[i][p], x[p]);
        x[i] = zdiv(zmake(-acc.x, -acc.y), T[i][i]);
    }
#pragma unroll
    for (int i = 0; i < CB; ++i)
        if (i < nb) Ri[(b0 + i) + (int64_t)(b0 + k) * m] = x[i];
}

unsigned grid_for(size_t count)
{
    const unsigned g = cdiv(count, 256);
    return g > 4096 ? 4096 : g;
}

// G (m x m, Hermitian positive definite) -> R upper triangular in place,
// G = R^H R.  Right-looking, CB-wide blocks; FP64.
int cholesky(cudaStream_t s, int m, zd *G, double *d0, int *fail)
{
    k_diag_copy<<<cdiv(m, 128), 128, 0, s>>>(m, G, d0);
    FEAST_LAUNCH_CHECK();
    const zd mone = zmake(-1.0, 0.0), one = zmake(1.0, 0.0);
    for (int k0 = 0; k0 < m; k0 += CB) {
        const int nb = (m - k0) < CB ? (m - k0) : CB;
        k_chol_diag<<<1, CB * CB, 0, s>>>(m, G, k0, nb, d0, fail);
        FEAST_LAUNCH_CHECK();
        const int k1 = k0 + nb;
        if (k1 >= m) break;
        k_chol_row<<<cdiv(m - k1, 32), 32, 0, s>>>(m, G, k0, nb);
        FEAST_LAUNCH_CHECK();
        // only the upper triangle of the trailing block is ever read
        int e = zgemm_batched(s, 1, m - k1, m - k1, nb, mone, G + k0 + (int64_t)k1 * m, m, 0,
                              G + k0 + (int64_t)k1 * m, m, 0, one, G + k1 + (int64_t)k1 * m, m, 0, 1, 3);
        if (e) return e;
    }
    return FEAST_OK;
}

}  // namespace

// Ri (m x m, ld m) = R^{-1} for upper triangular R (ld ldr): inverses of
// the 32 x 32 diagonal blocks, then, level by level, adjacent inverted
// blocks [A^{-1} X; 0 C^{-1}] get X = -A^{-1} B C^{-1} (B the block of R
// between them) -- batched GEMMs over the equal pairs of a level, one more
// pair for a shorter last block.  T: scratch of m * m / 2 + 32 * m entries.
int tri_inverse(cudaStream_t s, int m, const zd *R, int64_t ldr, zd *Ri, zd *T)
{
    if (m <= 0) return FEAST_OK;
    FEAST_CUDA_TRY(cudaMemsetAsync(Ri, 0, sizeof(zd) * (size_t)m * m, s));
    k_trinv_diag<<<cdiv(m, CB), CB, 0, s>>>(m, R, ldr, Ri);
    FEAST_LAUNCH_CHECK();
    const zd one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0), zero = zmake(0.0, 0.0);
    int e;
    for (int64_t L = CB; L < m; L *= 2) {
        const int64_t full = m / (2 * L);  // pairs with two L-blocks
        const int64_t sR = 2 * L * (ldr + 1), sI = 2 * L * ((int64_t)m + 1);
        if (full > 0) {
            // T_p = A_p^{-1} B_p, then X_p = -T_p C_p^{-1}
            if ((e = zgemm_batched(s, 0, L, L, L, one, Ri, m, sI, R + L * ldr, ldr, sR, zero, T, L, L * L, (int)full,
                                   1)))
                return e;
            if ((e = zgemm_batched(s, 0, L, L, L, mone, T, L, L * L, Ri + L + L * (int64_t)m, m, sI, zero,
                                   Ri + L * (int64_t)m, m, sI, (int)full, 2)))
                return e;
        }
        const int64_t a0 = full * 2 * L, b0 = a0 + L;  // a leftover pair with a shorter second block
        if (b0 < m) {
            const int64_t w = m - b0;
            if ((e = zgemm_batched(s, 0, L, w, L, one, Ri + a0 + a0 * (int64_t)m, m, 0, R + a0 + b0 * ldr, ldr, 0,
                                   zero, T, L, 0, 1, 1)))
                return e;
            if ((e = zgemm_batched(s, 0, L, w, w, mone, T, L, 0, Ri + b0 + b0 * (int64_t)m, m, 0, zero,
                                   Ri + a0 + b0 * (int64_t)m, m, 0, 1, 2)))
                return e;
        }
    }
    return FEAST_OK;
}

size_t tri_inverse_scratch_elems(int m)
{
    return (size_t)m * m / 2 + (size_t)CB * m + 64;
}

size_t zorth_chol_work_bytes(int64_t m)
{
    return sizeof(zd) * (3 * (size_t)m * m + tri_inverse_scratch_elems((int)m)) + sizeof(double) * (size_t)m + 64;
}

int zorth_chol(cudaStream_t s, int64_t n, int64_t m, zd *V, int64_t ldv, zd *R, int64_t ldr, void *work,
               const OzScratch &oz, int *ok)
{
    *ok = 0;
    if (m <= 0) {
        *ok = 1;
        return FEAST_OK;
    }
    if (m > n) return FEAST_EINVAL;
    const size_t mm = (size_t)m * m;
    zd *F0 = (zd *)work;
    zd *F1 = F0 + mm;
    zd *Ti = F1 + mm;
    zd *Ts = Ti + mm;
    double *d0 = (double *)(Ts + tri_inverse_scratch_elems((int)m));
    int *fail = (int *)(d0 + m);
    const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
    int e;
    FEAST_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), s));
    for (int pass = 0; pass < 2; ++pass) {
        zd *F = pass == 0 ? F0 : F1;
        // G = V^H V
        if ((e = oz_prepare_rows(s, m, n, V, ldv, oz.rows, 1))) return e;
        if ((e = oz_prepare_cols(s, n, m, V, ldv, oz.cols))) return e;
        if ((e = oz_gemm(s, m, m, n, oz.rows, oz.cols, one, nullptr, 0, zero, F, m, oz.err))) return e;
        if ((e = cholesky(s, (int)m, F, d0, fail))) return e;
        if (pass == 0) {
            int hf = 0;
            FEAST_CUDA_TRY(cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
            FEAST_CUDA_TRY(cudaStreamSynchronize(s));
            if (hf) return FEAST_OK;  // V too ill-conditioned: caller falls back
        }
        k_zero_lower<<<grid_for(mm), 256, 0, s>>>((int)m, F, m);
        FEAST_LAUNCH_CHECK();
        // V <- V F^{-1} (the digit planes of V are taken before V is overwritten)
        if ((e = tri_inverse(s, (int)m, F, m, Ti, Ts))) return e;
        if ((e = oz_prepare_rows(s, n, m, V, ldv, oz.rows))) return e;
        if ((e = oz_prepare_cols(s, m, m, Ti, m, oz.cols))) return e;
        if ((e = oz_gemm(s, n, m, m, oz.rows, oz.cols, one, nullptr, 0, zero, V, ldv, oz.err))) return e;
    }
    // R = R_b R_a
    if (R) {
        if ((e = oz_prepare_rows(s, m, m, F1, m, oz.rows))) return e;
        if ((e = oz_prepare_cols(s, m, m, F0, m, oz.cols))) return e;
        if ((e = oz_gemm(s, m, m, m, oz.rows, oz.cols, one, nullptr, 0, zero, R, ldr, oz.err))) return e;
        k_zero_lower<<<grid_for(mm), 256, 0, s>>>((int)m, R, ldr);
        FEAST_LAUNCH_CHECK();
    }
    *ok = 1;
    return FEAST_OK;
}

}  // namespace feast
