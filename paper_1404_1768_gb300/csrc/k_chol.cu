// QR of a tall block by Cholesky QR, twice (precision form; GFEAST lines 2
// and 17):
//
//     G = V^H V = R_a^H R_a,  Q_1 = V R_a^{-1};   Q_1^H Q_1 = R_b^H R_b,
//     Q = Q_1 R_b^{-1},  R = R_b R_a.
//
// The Gram matrices and the products V R^{-1} are FP64-accurate GEMMs on the
// tensor cores (k_oz.cu); the triangular inverses are FP64 (recursive
// doubling), the Cholesky factorisations one cooperative launch each: FP64,
// or -- the first one, on the digit-sliced path from m = 256 -- FP32 on the
// unit-diagonal Gram matrix, since the second pass corrects whatever the
// first leaves.  The first pass leaves Q_1 orthonormal to ~eps cond(V)^2
// (FP64) or ~2^-24 cond of the scaled Gram matrix (FP32), the second to
// ~eps, while cond(V) stays below ~1e6.  Every FP64 pivot is checked
// against its column's original norm: a pivot below 1e-12 of it (cond(V)
// out of reach) reports failure and the caller runs the column-by-column
// BCGS2 instead.  R has a real positive diagonal, like the Householder QR
// with that sign convention, so Q and R are the same unique factors.
#include "common.cuh"

namespace feast {
namespace {

constexpr int CB = 32;  // Cholesky block
constexpr int kChol32MinM = 256;      // the FP32 first factorisation from this block width up
constexpr double kChol32Tol = 1e-4;   // its pivots against the unit diagonal
constexpr double kSeriesMax = 1e-2;   // largest Gram defect repeated series rounds take on (no R)

__global__ void k_diag_copy(int m, const zd *__restrict__ G, double *__restrict__ d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) d[i] = G[i + (int64_t)i * m].x;
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

// The whole right-looking Cholesky in one cooperative launch (one CTA per
// SM): per 32-column step, CTA 0 factors and inverts the diagonal block;
// after a grid barrier every warp takes columns of the row panel
// R12 = R11^{-H} G12; after another, the CTAs share the 32 x 32 tiles of the
// trailing block's upper triangle (G22 -= R12^H R12).  The launch sequence
// of the blocked form (three launches per step, each too small to fill the
// GPU) becomes grid barriers.  T = double2 (FP64) or float2 (FP32: the
// first factorisation of Cholesky QR, on a unit-diagonal Gram matrix).  A
// pivot at or below tol times its reference (d0, or 1 without one) sets
// *fail.
constexpr int PT = 256;
template <typename T>
__global__ void __launch_bounds__(PT, 1) k_chol_grid(int m, T *__restrict__ G, const double *__restrict__ d0,
                                                     double tol, int *__restrict__ fail, T *__restrict__ rinv,
                                                     GridSync gs)
{
    using R = typename CxReal<T>::type;
    __shared__ T Tb[CB][CB + 1];
    __shared__ T P2[CB][CB + 1];
    __shared__ R rsh;
    const int tid = threadIdx.x, lane = tid & 31;
    const int gwarp = blockIdx.x * (PT / 32) + (tid >> 5), nwarp = gridDim.x * (PT / 32);
    for (int k0 = 0; k0 < m; k0 += CB) {
        const int nb = (m - k0) < CB ? (m - k0) : CB;
        const int k1 = k0 + nb;
        if (blockIdx.x == 0) {
            for (int e = tid; e < CB * CB; e += PT) {
                const int i = e % CB, k = e / CB;
                Tb[i][k] = (i < nb && k < nb) ? G[(k0 + i) + (int64_t)(k0 + k) * m] : cx<T>(0, 0);
            }
            __syncthreads();
            for (int j = 0; j < nb; ++j) {
                if (tid == 0) {
                    const double d = (double)Tb[j][j].x, ref = d0 ? d0[k0 + j] : 1.0;
                    R r;
                    if (!(d > tol * ref) || !(ref > 0.0)) {
                        *fail = 1;
                        r = (R)1;
                    } else {
                        r = sqrt((R)d);
                    }
                    Tb[j][j] = cx<T>(r, 0);
                    rsh = (R)1 / r;
                }
                __syncthreads();
                for (int k = j + 1 + tid; k < nb; k += PT) Tb[j][k] = cx<T>(Tb[j][k].x * rsh, Tb[j][k].y * rsh);
                __syncthreads();
                for (int e = tid; e < CB * CB; e += PT) {
                    const int i = e % CB, k = e / CB;
                    if (i > j && k >= i && k < nb) {
                        const T rji = Tb[j][i], rjk = Tb[j][k];
                        Tb[i][k] = cx<T>(Tb[i][k].x - (rji.x * rjk.x + rji.y * rjk.y),
                                         Tb[i][k].y - (rji.x * rjk.y - rji.y * rjk.x));
                    }
                }
                __syncthreads();
            }
            for (int e = tid; e < CB * CB; e += PT) {
                const int i = e % CB, k = e / CB;
                if (i < nb && k < nb && k >= i) G[(k0 + i) + (int64_t)(k0 + k) * m] = Tb[i][k];
            }
            // R11^{-1} (upper), column k by thread k: back-substitution
            if (tid < nb) {
                const int k = tid;
                T x[CB];
#pragma unroll
                for (int i = 0; i < CB; ++i) x[i] = cx<T>(0, 0);
                x[k] = cx<T>((R)1 / Tb[k][k].x, 0);
#pragma unroll
                for (int i = CB - 1; i >= 0; --i) {
                    if (i >= k) continue;
                    T acc = cx<T>(0, 0);
#pragma unroll
                    for (int p = 0; p < CB; ++p)
                        if (p > i && p <= k) cfma(acc, Tb[i][p], x[p]);
                    const R di = (R)1 / Tb[i][i].x;
                    x[i] = cx<T>(-acc.x * di, -acc.y * di);
                }
#pragma unroll
                for (int i = 0; i < CB; ++i) rinv[i + k * CB] = x[i];
            }
        }
        if (!grid_barrier(gs)) return;
        if (k1 >= m) break;
        // row panel: column c by one warp, lane i -> entry i
        for (int e = tid; e < CB * CB; e += PT) {
            const int i = e % CB, k = e / CB;
            Tb[i][k] = (i < nb && k < nb) ? rinv[i + k * CB] : cx<T>(0, 0);
        }
        __syncthreads();
        for (int c = k1 + gwarp; c < m; c += nwarp) {
            const T g = (lane < nb) ? G[(k0 + lane) + (int64_t)c * m] : cx<T>(0, 0);
            T acc = cx<T>(0, 0);
            for (int p = 0; p < nb; ++p) {
                T gp;
                gp.x = __shfl_sync(0xffffffffu, g.x, p);
                gp.y = __shfl_sync(0xffffffffu, g.y, p);
                if (p <= lane) {
                    const T rp = Tb[p][lane];  // (R11^{-H})_{lane, p} = conj(rinv_{p, lane})
                    acc = cadd(acc, cx<T>(rp.x * gp.x + rp.y * gp.y, rp.x * gp.y - rp.y * gp.x));
                }
            }
            if (lane < nb) G[(k0 + lane) + (int64_t)c * m] = acc;
        }
        if (!grid_barrier(gs)) return;
        // trailing update, upper-triangle tiles (ti <= tj) of G[k1:, k1:]
        const int nt = (m - k1 + CB - 1) / CB;
        const int ntiles = nt * (nt + 1) / 2;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int tj = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
            while ((tj + 1) * (tj + 2) / 2 <= t) ++tj;
            while (tj * (tj + 1) / 2 > t) --tj;
            const int ti = t - tj * (tj + 1) / 2;
            const int r0 = k1 + ti * CB, c0 = k1 + tj * CB;
            __syncthreads();
            for (int e = tid; e < CB * CB; e += PT) {
                const int p = e % CB, a = e / CB;
                const bool okp = p < nb;
                Tb[p][a] = (okp && r0 + a < m) ? G[(k0 + p) + (int64_t)(r0 + a) * m] : cx<T>(0, 0);
                P2[p][a] = (okp && c0 + a < m) ? G[(k0 + p) + (int64_t)(c0 + a) * m] : cx<T>(0, 0);
            }
            __syncthreads();
            for (int e = tid; e < CB * CB; e += PT) {
                const int a = e % CB, b = e / CB;
                const int gi = r0 + a, gj = c0 + b;
                if (gi >= m || gj >= m) continue;
                R ax = 0, ay = 0;
#pragma unroll 8
                for (int p = 0; p < CB; ++p) {
                    const T x = Tb[p][a], y = P2[p][b];  // conj(x) y
                    ax += x.x * y.x + x.y * y.y;
                    ay += x.x * y.y - x.y * y.x;
                }
                T &gv = G[gi + (int64_t)gj * m];
                gv = cx<T>(gv.x - ax, gv.y - ay);
            }
        }
        if (!grid_barrier(gs)) return;
    }
}

// Unit-diagonal scaling for the FP32 factorisation: dsq_j = sqrt(G_jj) and
// its reciprocal (dsq[m + j]), then S = (D^-1 G D^-1) in complex64 (m x m).
__global__ void k_chol_dsq(int m, const zd *__restrict__ G, double *__restrict__ dsq)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double d = sqrt(G[j + (int64_t)j * m].x);
    dsq[j] = d;
    dsq[m + j] = 1.0 / d;
}

__global__ void k_chol_scale(int m, const zd *__restrict__ G, const double *__restrict__ dsq, cf *__restrict__ S)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        const double f = dsq[m + i] * dsq[m + j];
        S[e] = cmakef((float)(G[e].x * f), (float)(G[e].y * f));
    }
}

// R = R32 D in FP64 (upper triangle; zeros below): the factor of G = D S D.
__global__ void k_chol_unscale(int m, const cf *__restrict__ R32, const double *__restrict__ dsq,
                               zd *__restrict__ R)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        R[e] = (i <= j) ? zmake((double)R32[e].x * dsq[j], (double)R32[e].y * dsq[j]) : zmake(0.0, 0.0);
    }
}

// S = phi(G - I - P) (P may be null): strictly upper part plus half the
// (real) diagonal; zero below.
__global__ void k_phi(int m, const zd *__restrict__ G, const zd *__restrict__ P, zd *__restrict__ S)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        zd v = zmake(0.0, 0.0);
        if (i <= j) {
            v = G[e];
            if (P) v = zsub(v, P[e]);
            if (i == j) v = zmake(0.5 * (v.x - 1.0), 0.0);
        }
        S[e] = v;
    }
}

// *out = max |G_ij - delta_ij| (non-negative doubles order like their bits)
__global__ void k_offident_max(int m, const zd *__restrict__ G, unsigned long long *__restrict__ out)
{
    const int64_t total = (int64_t)m * m;
    double mx = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        zd v = G[e];
        if (i == j) v.x -= 1.0;
        const double a = zabs(v);
        mx = (a > mx || !(a == a)) ? a : mx;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (!(mx == mx)) mx = 1e300;
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

unsigned grid_for(size_t count)
{
    const unsigned g = cdiv(count, 256);
    return g > 4096 ? 4096 : g;
}

// C = alpha op(A) B + beta C on the digit-sliced tensor-core GEMM (op(A) =
// A^H when conj_a; C may alias A or B: their digit planes are taken first).
int oz_mm(cudaStream_t s, const OzScratch &oz, int conj_a, int64_t M, int64_t N, int64_t K, zd alpha, const zd *A,
          int64_t lda, const zd *B, int64_t ldb, zd beta, zd *C, int64_t ldc)
{
    // (without digit-plane scratch: the FP64 GEMM; C must not overlap A, B)
    if (!oz.rows) return zgemm_batched(s, conj_a, M, N, K, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, 1);
    int e;
    if ((e = oz_prepare_rows(s, M, K, A, lda, oz.rows, conj_a))) return e;
    if ((e = oz_prepare_cols(s, K, N, B, ldb, oz.cols))) return e;
    return oz_gemm(s, M, N, K, oz.rows, oz.cols, alpha, nullptr, 0, beta, C, ldc, oz.err);
}

// G (m x m, Hermitian positive definite) -> R upper triangular in place,
// G = R^H R (upper triangle; the lower one is left as it was).  One
// cooperative launch (k_chol_grid<T>); pivots checked against tol d0 (d0
// null: against tol).  work: 2 barrier words + a 32 x 32 scratch.
template <typename T>
int chol_launch(cudaStream_t s, int m, T *G, const double *d0, double tol, int *fail, unsigned *bar, T *rinv,
                int *timeout)
{
    int dev = 0, sms = 0, per = 0;
    FEAST_CUDA_TRY(cudaGetDevice(&dev));
    FEAST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_grid<T>, PT, 0));
    if (per < 1) return FEAST_ECUDA;
    FEAST_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    GridSync gs{bar, bar + 1, timeout, TO_CHOL};
    void *args[] = {&m, &G, &d0, &tol, &fail, &rinv, &gs};
    // as many CTAs as the first trailing update has ~4 tiles for (at least
    // 8, at most one per SM): a small factorisation leaves the rest of the
    // GPU to other work (the pencils of a batch)
    const int nt = (m + CB - 1) / CB;
    int grid = nt * (nt + 1) / 8;
    if (grid < 8) grid = 8;
    if (grid > sms) grid = sms;
    FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_chol_grid<T>, dim3(grid), dim3(PT), args, 0, s));
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// The FP64 factorisation, pivots against 1e-12 of the original diagonal.
int cholesky(cudaStream_t s, int m, zd *G, double *d0, int *fail, unsigned *bar, zd *rinv, int *timeout)
{
    k_diag_copy<<<cdiv(m, 128), 128, 0, s>>>(m, G, d0);
    FEAST_LAUNCH_CHECK();
    return chol_launch<zd>(s, m, G, d0, 1e-12, fail, bar, rinv, timeout);
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
    return sizeof(zd) * (4 * (size_t)m * m + tri_inverse_scratch_elems((int)m) + CB * CB) +
           sizeof(double) * (size_t)m + 64;
}

// V <- V X (beta = 0) or V <- V + V X (beta = 1), X m x m: on the digit
// slices in place, or in FP64 through tmp (n x m, a copy of V).
static int mul_right(cudaStream_t s, const OzScratch &oz, int64_t n, int64_t m, zd *V, int64_t ldv, const zd *X,
                     zd beta, zd *tmp)
{
    const zd one = zmake(1.0, 0.0);
    int e;
    if (oz.rows) {
        if ((e = oz_prepare_rows(s, n, m, V, ldv, oz.rows))) return e;
        if ((e = oz_prepare_cols(s, m, m, X, m, oz.cols))) return e;
        return oz_gemm(s, n, m, m, oz.rows, oz.cols, one, nullptr, 0, beta, V, ldv, oz.err);
    }
    FEAST_CUDA_TRY(cudaMemcpy2DAsync(tmp, sizeof(zd) * n, V, sizeof(zd) * ldv, sizeof(zd) * n, m,
                                     cudaMemcpyDeviceToDevice, s));
    return zgemm_batched(s, 0, n, m, m, one, tmp, n, 0, X, m, 0, beta, V, ldv, 0, 1);
}

// G = V^H V (m x m) and max |G - I| (read back).
static int gram_defect(cudaStream_t s, const OzScratch &oz, int64_t n, int64_t m, const zd *V, int64_t ldv, zd *G,
                       unsigned long long *emax, double *hemax)
{
    const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
    int e;
    if ((e = oz_mm(s, oz, 1, m, m, n, one, V, ldv, V, ldv, zero, G, m))) return e;
    FEAST_CUDA_TRY(cudaMemsetAsync(emax, 0, sizeof(unsigned long long), s));
    k_offident_max<<<grid_for((size_t)m * m), 256, 0, s>>>((int)m, G, emax);
    FEAST_LAUNCH_CHECK();
    unsigned long long hb = 0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&hb, emax, sizeof(hb), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    memcpy(hemax, &hb, sizeof(double));
    return FEAST_OK;
}

int zorth_chol(cudaStream_t s, int64_t n, int64_t m, zd *V, int64_t ldv, zd *R, int64_t ldr, void *work,
               const OzScratch &oz, int *ok, zd *tmp)
{
    if (!oz.rows && !tmp) return FEAST_EINVAL;
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
    zd *rinv = Ts + tri_inverse_scratch_elems((int)m);
    zd *rinv_big = rinv + CB * CB;  // m x m
    double *d0 = (double *)(rinv_big + mm);
    int *fail = (int *)(d0 + m);
    unsigned *bar = (unsigned *)(fail + 2);
    unsigned long long *emax = (unsigned long long *)(bar + 2);
    const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
    int e;
    // The first factorisation only has to bring V R_a^{-1} close to
    // orthonormal (the second pass corrects it; R stays exact because V is
    // multiplied by the FP64 inverse of the R_a used): on the digit-sliced
    // path it runs in FP32 on the unit-diagonal Gram matrix D^-1 G D^-1,
    // with V kept in tmp.  A pivot at or below 1e-4 there, or a second-pass
    // defect max|E| above 1/2, starts again from V in FP64.
    const bool try32 = oz.rows != nullptr && tmp != nullptr && m >= kChol32MinM;
    bool dirty = false;   // V holds the product of a discarded FP32 first pass
    for (int attempt = try32 ? 0 : 1; attempt < 2; ++attempt) {
        const bool use32 = attempt == 0;
        if (use32)
            FEAST_CUDA_TRY(cudaMemcpy2DAsync(tmp, sizeof(zd) * n, V, sizeof(zd) * ldv, sizeof(zd) * n, m,
                                             cudaMemcpyDeviceToDevice, s));
        else if (dirty)
            FEAST_CUDA_TRY(cudaMemcpy2DAsync(V, sizeof(zd) * ldv, tmp, sizeof(zd) * n, sizeof(zd) * n, m,
                                             cudaMemcpyDeviceToDevice, s));
        FEAST_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), s));
        // pass 1: G = V^H V = R_a^H R_a, V <- V R_a^{-1}
        if ((e = oz_mm(s, oz, 1, m, m, n, one, V, ldv, V, ldv, zero, F0, m))) return e;
        int hf = 0;
        if (use32) {
            cf *S32 = (cf *)F1;          // (F1 is free until pass 2)
            double *dsq = (double *)Ti;  // 2m: (Ti is written after the unscaling)
            k_chol_dsq<<<cdiv(m, 128), 128, 0, s>>>((int)m, F0, dsq);
            FEAST_LAUNCH_CHECK();
            k_chol_scale<<<grid_for(mm), 256, 0, s>>>((int)m, F0, dsq, S32);
            FEAST_LAUNCH_CHECK();
            if ((e = chol_launch<cf>(s, (int)m, S32, nullptr, kChol32Tol, fail, bar, (cf *)rinv, oz.err))) return e;
            FEAST_CUDA_TRY(cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
            FEAST_CUDA_TRY(cudaStreamSynchronize(s));
            if (hf) continue;            // beyond FP32: the FP64 factorisation
            k_chol_unscale<<<grid_for(mm), 256, 0, s>>>((int)m, S32, dsq, F0);
            FEAST_LAUNCH_CHECK();
        } else {
            if ((e = cholesky(s, (int)m, F0, d0, fail, bar, rinv, oz.err))) return e;
            FEAST_CUDA_TRY(cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
            FEAST_CUDA_TRY(cudaStreamSynchronize(s));
            if (hf) return FEAST_OK;     // V too ill-conditioned: caller falls back
            k_zero_lower<<<grid_for(mm), 256, 0, s>>>((int)m, F0, m);
            FEAST_LAUNCH_CHECK();
        }
        if ((e = tri_inverse(s, (int)m, F0, m, Ti, Ts))) return e;
        if ((e = mul_right(s, oz, n, m, V, ldv, Ti, zero, tmp))) return e;
        dirty = use32;
        // pass 2: G = V^H V = I + E with E ~ eps cond(V)^2 (FP64 first
        // pass; ~2^-24 cond(D^-1 G D^-1) after the FP32 one).  R_b = I + S
        // with S + S^H = E - S^H S; S_0 = phi(E), S = phi(E - S_0^H S_0)
        // (error O(|E|^3), phi = strict upper part + half the diagonal),
        // R_b^{-1} = I - S + S^2 (error O(|E|^3)): V <- V + V (S^2 - S).
        double hemax = 0.0;
        if ((e = gram_defect(s, oz, n, m, V, ldv, F1, emax, &hemax))) return e;
        if (use32 && !(hemax <= 0.5)) continue;
        // Series rounds, each taking a defect E to O(|E|^3): one when max|E|
        // <= 1e-4 (R = (I + S) R_a then holds to O(|E|^3) as well).  Without
        // R (only Q's span and orthonormality wanted, and every round is an
        // upper triangular map with a positive diagonal, so Q is still the
        // unique factor) up to three from max|E| <= kSeriesMax, the Gram
        // matrix and its defect measured again after each round that started
        // above 1e-4.  A defect out of their reach gets a second Cholesky and
        // inverse instead.
        const double series_max = R ? 1e-4 : kSeriesMax;
        bool finished = false;
        int rounds = 0;
        while (hemax <= series_max && rounds < 3) {
            // S_0 = phi(G - I) into Ti; S = phi(G - I - S_0^H S_0) into Ti
            // (the products of these small corrections on the tensor cores:
            // the digit planes scale per row and column, so their error is
            // relative to the corrections themselves)
            zd *S = Ti, *D = rinv_big;
            k_phi<<<grid_for(mm), 256, 0, s>>>((int)m, F1, nullptr, S);
            FEAST_LAUNCH_CHECK();
            if ((e = oz_mm(s, oz, 1, m, m, m, one, S, m, S, m, zero, D, m))) return e;   // S_0^H S_0
            k_phi<<<grid_for(mm), 256, 0, s>>>((int)m, F1, D, S);
            FEAST_LAUNCH_CHECK();
            // D = S^2 - S, then V <- V + V D
            FEAST_CUDA_TRY(cudaMemcpyAsync(D, S, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, s));
            if ((e = oz_mm(s, oz, 0, m, m, m, one, S, m, S, m, zmake(-1.0, 0.0), D, m))) return e;
            if ((e = mul_right(s, oz, n, m, V, ldv, D, one, tmp))) return e;
            // R = (I + S) R_a (R: a single round)
            if (R) {
                FEAST_CUDA_TRY(cudaMemcpy2DAsync(R, sizeof(zd) * ldr, F0, sizeof(zd) * m, sizeof(zd) * m, m,
                                                 cudaMemcpyDeviceToDevice, s));
                if ((e = oz_mm(s, oz, 0, m, m, m, one, S, m, F0, m, one, R, ldr))) return e;
            }
            ++rounds;
            if (hemax <= 1e-4) {
                finished = true;
                break;
            }
            if ((e = gram_defect(s, oz, n, m, V, ldv, F1, emax, &hemax))) return e;
        }
        if (!finished) {
            if ((e = cholesky(s, (int)m, F1, d0, fail, bar, rinv, oz.err))) return e;
            k_zero_lower<<<grid_for(mm), 256, 0, s>>>((int)m, F1, m);
            FEAST_LAUNCH_CHECK();
            if ((e = tri_inverse(s, (int)m, F1, m, Ti, Ts))) return e;
            if ((e = mul_right(s, oz, n, m, V, ldv, Ti, zero, tmp))) return e;
            // R = R_b R_a (with R no series round has run)
            if (R && (e = oz_mm(s, oz, 0, m, m, m, one, F1, m, F0, m, zero, R, ldr))) return e;
        }
        if (R) {
            k_zero_lower<<<grid_for(mm), 256, 0, s>>>((int)m, R, ldr);
            FEAST_LAUNCH_CHECK();
        }
        *ok = 1;
        return FEAST_OK;
    }
    return FEAST_OK;
}

}  // namespace feast
