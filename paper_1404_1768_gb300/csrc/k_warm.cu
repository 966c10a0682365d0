// Warm-started solve of the projected eigenproblem (GFEAST line 6).
//
// When the filter of line 16 is applied to the Ritz vectors of the previous
// pass, ordered by their expected residual after filtering (r_i /
// |rho(lambda_i)|, rho the filter function of eq. 4.1, so the most
// converged pairs come first), the QR factorisation of line 17
// keeps the order, and every leading group of converged Ritz vectors spans
// an (almost) invariant subspace.  The projected matrix C = B~^{-1} A~ is
// then block upper triangular up to a small remainder:
//
//     C = [ T11 + E11   C12 ]      T11 upper triangular (k x k),
//         [ E21         C22 ]      E11 strictly lower, E11 and E21 small.
//
// The solve below takes k from the column norms of C's strictly lower
// part, computes the Schur form of the trailing block only (C22 = Z T22
// Z^H, the double-single multishift QR of k_zeig.cu on m - k instead of m
// rows), and treats what is left as a perturbation: with Zh = diag(I, Z)
// and C' = Zh^H C Zh = T^ + D (T^ upper triangular, D small), one Newton
// step for the eigen-decomposition of C' starting from the eigenvectors V^
// of T^ gives
//
//     F = V^{-1} C' V^,   lambda_i = F_ii,   G_ij = F_ij / (lambda_j - lambda_i),
//     Y' = V^ (I + G),    Y = Zh Y'          (error O(|D|^2 / gap)).
//
// The products that define C and C' (B~^{-1} A~, the similarity with Z)
// are FP64 GEMMs; the triangular solves are products with explicit
// triangular inverses.  The Newton step itself runs in defect form: with
// T^ V^ = V^ Lh (Lh = diag T^), W' = C' V^ - V^ Lh = D V^ is small, F =
// Lh + V^{-1} W', and the residual C' Y' - Y' L = V^ S1 + W' (I + G) with
// S1 small too.  Every one of these products has a small operand, so they
// run on the digit-sliced tensor-core GEMM (48-bit fixed point per row and
// column of its operands) at FP64 accuracy; computed as plain products of
// O(1) matrices on it, the step's residual stalled near 3e-12 at m0 = 1280
// instead of 1e-13.  (Without the digit-sliced scratch every product is an
// FP64 GEMM.)  The eigenpairs are accepted only if each
// ||C' y'_i - lambda_i y'_i|| / ((max|C_ij| + |lambda_i|) ||y'_i||) is at
// most accept_tol; otherwise the caller runs the cold solve (Hessenberg
// reduction and QR of the whole matrix).  The subspace of every pass is the
// paper's (span of the filtered Ritz vectors = span of the filtered U1);
// only the way the projected problem is solved changes.
#include "common.cuh"

namespace feast {
namespace {

// Per column j: ||C[j+1:m, j]||_2 and max_i |C_ij|.  Warp per column.
__global__ void k_col_stats(int m, const zd *__restrict__ C, double *__restrict__ lower, double *__restrict__ cmax)
{
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= m) return;
    const zd *c = C + (int64_t)j * m;
    double s = 0.0, mx = 0.0;
    for (int i = lane; i < m; i += 32) {
        const double a2 = zabs2(c[i]);
        if (i > j) s += a2;
        mx = fmax(mx, a2);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) {
        lower[j] = sqrt(s);
        cmax[j] = sqrt(mx);
    }
}

__global__ void k_diag_lambda(int m, const zd *__restrict__ F, zd *__restrict__ alpha, zd *__restrict__ beta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    alpha[i] = F[i + (int64_t)i * m];
    beta[i] = zmake(1.0, 0.0);
}

// G_ij = F_ij / (lambda_j - lambda_i) off the diagonal, G_ii = 0 (in place).
// A correction entry above 1/4 means the first-order step is not valid for
// this pair: *bad is set and the solve is not accepted.
__global__ void k_newton_g(int m, zd *__restrict__ F, const zd *__restrict__ lam, int *__restrict__ bad)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        if (i == j) {
            F[e] = zmake(0.0, 0.0);
            continue;
        }
        const zd d = zsub(lam[j], lam[i]);
        const zd f = F[e];
        const double d2 = zabs2(d), f2 = zabs2(f);
        if (!(f2 <= 0.0625 * d2)) {
            if (f2 > 0.0) *bad = 1;
            F[e] = zmake(0.0, 0.0);
            continue;
        }
        F[e] = zdiv(f, d);
    }
}

// max_i ||W_i - lambda_i Y_i|| / ((cnorm + |lambda_i|) ||Y_i||) into *out
// (non-negative doubles order like their bit patterns); is_resid: W holds
// the residual block itself.  Warp per column.
__global__ void k_eig_resid(int m, const zd *__restrict__ W, const zd *__restrict__ Y, const zd *__restrict__ lam,
                            double cnorm, unsigned long long *__restrict__ out, int is_resid = 0)
{
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= m) return;
    const zd l = lam[i];
    const zd *w = W + (int64_t)i * m;
    const zd *y = Y + (int64_t)i * m;
    double r = 0.0, yy = 0.0;
    for (int p = lane; p < m; p += 32) {
        const zd yv = y[p];
        const zd d = is_resid ? w[p] : zsub(w[p], zmul(l, yv));
        r += zabs2(d);
        yy += zabs2(yv);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        r += __shfl_xor_sync(0xffffffffu, r, off);
        yy += __shfl_xor_sync(0xffffffffu, yy, off);
    }
    if (lane == 0) {
        double rel = (yy > 0.0) ? sqrt(r / yy) / (cnorm + zabs(l)) : 1e300;
        if (!(rel == rel)) rel = 1e300;
        atomicMax(out, (unsigned long long)__double_as_longlong(rel));
    }
}

// D = C' - T^ (m x m; T^ upper triangular) and lamh = diag(T^).
__global__ void k_defect_split(int m, const zd *__restrict__ Cq, const zd *__restrict__ Th, zd *__restrict__ D,
                               zd *__restrict__ lamh)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        const zd t = Th[e];
        D[e] = (i <= j) ? zsub(Cq[e], t) : Cq[e];
        if (i == j) lamh[i] = t;
    }
}

// F_ii += lamh_i, then lambda_i = F_ii (alpha), beta_i = 1.
__global__ void k_add_diag_lambda(int m, zd *__restrict__ F, const zd *__restrict__ lamh, zd *__restrict__ alpha,
                                  zd *__restrict__ beta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const zd f = zadd(F[i + (int64_t)i * m], lamh[i]);
    F[i + (int64_t)i * m] = f;
    alpha[i] = f;
    beta[i] = zmake(1.0, 0.0);
}

// S1 = (Lh - L) + Lh G - G L (Lh = diag(lamh), L = diag(lam)):
// S1_ij = G_ij (lamh_i - lam_j) off the diagonal, lamh_i - lam_i on it
// (G_ii = 0).
__global__ void k_newton_s1(int m, const zd *__restrict__ G, const zd *__restrict__ lamh, const zd *__restrict__ lam,
                            zd *__restrict__ S1)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        S1[e] = (i == j) ? zsub(lamh[i], lam[i]) : zmul(G[e], zsub(lamh[i], lam[j]));
    }
}

// E <- (E - I) / 2 in place (m x m): the first-order term of (I + E)^{-1/2}.
__global__ void k_sub_identity_half(int m, zd *__restrict__ E)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        zd v = E[e];
        if (i == j) v.x -= 1.0;
        E[e] = zmake(0.5 * v.x, 0.5 * v.y);
    }
}

// Column gather: Vout[:, i] = Vin[:, perm[i]] (rows x m, leading dim rows).
__global__ void k_permute_cols(int64_t rows, int m, const int *__restrict__ perm, const zd *__restrict__ Vin,
                               zd *__restrict__ Vout)
{
    const int64_t total = rows * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows;
        const int j = (int)(e / rows);
        Vout[e] = Vin[i + (int64_t)perm[j] * rows];
    }
}

struct WarmCarve {
    zd *Cp, *W, *Yp, *S, *Z, *Ts;
    double *lower, *cmax;
    unsigned long long *res;
    int *bad;
};

WarmCarve warm_carve(void *work, int m)
{
    WarmCarve w;
    const size_t mm = (size_t)m * m;
    zd *p = (zd *)work;
    w.Cp = p;
    w.W = p + mm;
    w.Yp = p + 2 * mm;
    w.S = p + 3 * mm;
    w.Z = p + 4 * mm;
    w.Ts = p + 5 * mm;
    w.lower = (double *)(w.Ts + tri_inverse_scratch_elems(m));
    w.cmax = w.lower + m;
    w.res = (unsigned long long *)(w.cmax + m);
    w.bad = (int *)(w.res + 1);
    return w;
}

unsigned grid_for(size_t count)
{
    const unsigned g = cdiv(count, 256);
    return g > 4096 ? 4096 : g;
}

}  // namespace

size_t zeig_warm_work_bytes(int m)
{
    return sizeof(zd) * (5 * (size_t)m * m + tri_inverse_scratch_elems(m)) + sizeof(double) * 2 * (size_t)m + 64;
}

int permute_cols(cudaStream_t s, int64_t rows, int m, const int *perm, const zd *Vin, zd *Vout)
{
    k_permute_cols<<<grid_for((size_t)rows * m), 256, 0, s>>>(rows, m, perm, Vin, Vout);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int zeig_warm(cudaStream_t s, int m, zd *A, zd *Bt, zd *alpha, zd *beta, zd *V, void *warm_work, void *qz_work,
              const WarmParams &prm, WarmResult *res, int *fail, int *timeout, int *stats, GemmTimer *gt,
              const OzScratch *oz)
{
    *res = WarmResult{};
    if (m < prm.min_m) return FEAST_OK;
    const WarmCarve w = warm_carve(warm_work, m);
    const size_t mm = (size_t)m * m;
    const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
    const double m3 = (double)m * m * m, tri_inv = 8.0 * m3 / 6.0;   // m^3/6 MACs
    // segment marks: begin, then end with the segment's algorithmic flops
    auto mark = [&](double flops) -> int {
        if (!gt || gt->used >= GemmTimer::kMax) return FEAST_OK;
        FEAST_CUDA_TRY(cudaEventRecord(gt->ev[gt->used++], s));
        gt->flops += flops;
        return FEAST_OK;
    };
    int e;
    // C = beta C + alpha op(A) B: the FP64 GEMM (tri: the triangular zeros it
    // may skip), or -- with oz, for a pass whose pairs are needed only well
    // above FP64 rounding -- the FP64-accurate digit-sliced tensor-core GEMM
    auto mul = [&](int conj_a, int64_t M, int64_t N, int64_t K, zd alpha, const zd *Am, int64_t lda, const zd *Bm,
                   int64_t ldb, zd beta, zd *Cm, int64_t ldc, int tri) -> int {
        if (!oz) return zgemm_batched(s, conj_a, M, N, K, alpha, Am, lda, 0, Bm, ldb, 0, beta, Cm, ldc, 0, 1, tri);
        int r;
        if ((r = oz_prepare_rows(s, M, K, Am, lda, oz->rows, conj_a))) return r;
        if ((r = oz_prepare_cols(s, K, N, Bm, ldb, oz->cols))) return r;
        return oz_gemm(s, M, N, K, oz->rows, oz->cols, alpha, nullptr, 0, beta, Cm, ldc, oz->err);
    };
    // the products that define C and C' themselves: FP64 unless the pass's
    // pairs are needed only well above the digit-sliced GEMM's resolution
    auto mulc = [&](int conj_a, int64_t M, int64_t N, int64_t K, zd alpha, const zd *Am, int64_t lda, const zd *Bm,
                    int64_t ldb, zd beta, zd *Cm, int64_t ldc, int tri) -> int {
        if (!prm.cold_fp32) return zgemm_batched(s, conj_a, M, N, K, alpha, Am, lda, 0, Bm, ldb, 0, beta, Cm, ldc, 0, 1, tri);
        return mul(conj_a, M, N, K, alpha, Am, lda, Bm, ldb, beta, Cm, ldc, tri);
    };
    // C = B~^{-1} A~ (B~ = R2 is upper triangular), into Cp
    if ((e = mark(0.0))) return e;
    if ((e = tri_inverse(s, m, Bt, m, w.W, w.Ts))) return e;
    if ((e = mulc(0, m, m, m, one, w.W, m, A, m, zero, w.Cp, m, 1))) return e;
    if ((e = mark(tri_inv + 4.0 * m3))) return e;
    const zd *C = w.Cp;
    k_col_stats<<<cdiv((size_t)m * 32, 256), 256, 0, s>>>(m, C, w.lower, w.cmax);
    FEAST_LAUNCH_CHECK();
    double *h = (double *)malloc(sizeof(double) * 2 * (size_t)m);
    if (!h) return FEAST_EINVAL;
    if (cudaMemcpyAsync(h, w.lower, sizeof(double) * 2 * (size_t)m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        free(h);
        return FEAST_ECUDA;
    }
    double hn = 0.0;
    for (int j = 0; j < m; ++j) hn = fmax(hn, h[m + j]);
    int k = 0;
    if (!prm.cold_fp32)
        while (k < m && h[k] <= prm.tau * hn) ++k;
    free(h);
    res->k = k;
    if (prm.cold_fp32) {
        k = 0;           // the whole matrix is the "tail"
    } else if (k < m - prm.min_tail) {
        if (k < m / 4) return FEAST_OK;  // too little has converged: cold solve
    } else {
        k = m - prm.min_tail;
    }
    const int mb = m - k;
    // Schur form of the trailing block: C22 = Z T22 Z^H
    FEAST_CUDA_TRY(cudaMemcpy2DAsync(w.S, sizeof(zd) * mb, C + k + (int64_t)k * m, sizeof(zd) * m, sizeof(zd) * mb,
                                     mb, cudaMemcpyDeviceToDevice, s));
    if (prm.cold_fp32) {
        // FP32 QR, then Z made unitary to FP64 rounding (BCGS2 in FP64;
        // Z moves by its FP32 error, ~1e-6), so that Zh^H C Zh below is a
        // similarity of C and its lower part is that small
        FEAST_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), s));
        if ((e = schur_large_fp32(s, mb, w.S, w.Z, qz_work, fail, timeout, stats, nullptr, 0.0))) return e;
        // Z^H Z = I + E with |E| ~ 1e-6: Z (I - E / 2) is unitary to O(|E|^2)
        // (one step of the series of (I + E)^{-1/2}), i.e. to ~1e-12
        if ((e = mark(0.0))) return e;
        if ((e = mul(1, mb, mb, mb, one, w.Z, mb, w.Z, mb, zero, w.Yp, mb, 0))) return e;
        k_sub_identity_half<<<grid_for((size_t)mb * mb), 256, 0, s>>>(mb, w.Yp);
        FEAST_LAUNCH_CHECK();
        FEAST_CUDA_TRY(cudaMemcpyAsync(w.W, w.Z, sizeof(zd) * (size_t)mb * mb, cudaMemcpyDeviceToDevice, s));
        if ((e = mul(0, mb, mb, mb, zmake(-1.0, 0.0), w.W, mb, w.Yp, mb, one, w.Z, mb, 0))) return e;
        if ((e = mark(16.0 * (double)mb * mb * mb))) return e;
    } else if ((e = schur_large(s, mb, w.S, w.Z, qz_work, fail, timeout, stats, nullptr, prm.tail_defl))) {
        return e;
    }
    // C' = Zh^H C Zh, Zh = diag(I_k, Z), into A (Bt as the row-block scratch)
    zd *Cq = A;
    FEAST_CUDA_TRY(cudaMemcpyAsync(Cq, C, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, s));
    if ((e = mark(0.0))) return e;
    if ((e = mulc(0, m, mb, mb, one, C + (int64_t)k * m, m, w.Z, mb, zero, Cq + (int64_t)k * m, m, 0))) return e;
    if ((e = mulc(1, mb, m, mb, one, w.Z, mb, Cq + k, m, zero, Bt + k, m, 0))) return e;
    if ((e = mark(16.0 * (double)m * mb * mb))) return e;
    FEAST_CUDA_TRY(cudaMemcpy2DAsync(Cq + k, sizeof(zd) * m, Bt + k, sizeof(zd) * m, sizeof(zd) * mb, m,
                                     cudaMemcpyDeviceToDevice, s));
    // T^: C' with T22 from the QR in its trailing block (upper triangles are
    // all that the eigenvector recurrence reads), into Cp -- or C' itself
    // after the FP32 QR, whose T22 is only FP32-accurate
    FEAST_CUDA_TRY(cudaMemcpyAsync(w.Cp, Cq, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, s));
    if (!prm.cold_fp32)
        FEAST_CUDA_TRY(cudaMemcpy2DAsync(w.Cp + k + (int64_t)k * m, sizeof(zd) * m, w.S, sizeof(zd) * mb,
                                         sizeof(zd) * mb, mb, cudaMemcpyDeviceToDevice, s));
    zd *Vh = Bt;  // V^, unit upper triangular
    if ((e = schur_vectors(s, m, w.Cp, Vh, hn, w.W))) return e;
    zd *F = V;
    if (!oz) {
        // F = V^{-1} (C' V^)
        if ((e = mark(0.0))) return e;
        if ((e = mul(0, m, m, m, one, Cq, m, Vh, m, zero, w.W, m, 2))) return e;
        if ((e = tri_inverse(s, m, Vh, m, w.Cp, w.Ts))) return e;
        if ((e = mul(0, m, m, m, one, w.Cp, m, w.W, m, zero, F, m, 1))) return e;
        if ((e = mark(8.0 * m3 + tri_inv))) return e;
        k_diag_lambda<<<cdiv(m, 128), 128, 0, s>>>(m, F, alpha, beta);
        FEAST_LAUNCH_CHECK();
        FEAST_CUDA_TRY(cudaMemsetAsync(w.res, 0, 16, s));
        k_newton_g<<<grid_for(mm), 256, 0, s>>>(m, F, alpha, w.bad);
        FEAST_LAUNCH_CHECK();
        // Y' = V^ + V^ G, and its residual against C'
        FEAST_CUDA_TRY(cudaMemcpyAsync(w.Yp, Vh, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, s));
        if ((e = mark(0.0))) return e;
        if ((e = mul(0, m, m, m, one, Vh, m, F, m, one, w.Yp, m, 1))) return e;
        if ((e = mul(0, m, m, m, one, Cq, m, w.Yp, m, zero, w.W, m, 0))) return e;
        if ((e = mark(12.0 * m3))) return e;
        k_eig_resid<<<cdiv((size_t)m * 32, 256), 256, 0, s>>>(m, w.W, w.Yp, alpha, hn, w.res);
        FEAST_LAUNCH_CHECK();
    } else {
        // The same step in defect form, every product on the digit-sliced
        // GEMM with one small operand (its error is relative to the
        // operands' row / column maxima): with C' = T^ + D and T^ V^ = V^ Lh,
        //   W' = C' V^ - V^ Lh = D V^,   F = Lh + V^{-1} W',
        //   Y' = V^ + V^ G,   C' Y' - Y' L = V^ S1 + W' + W' G,
        //   S1 = (Lh - L) + Lh G - G L   (L = diag(F), G as above).
        zd *lamh = (zd *)w.lower;   // diag(T^) (the column statistics are spent)
        k_defect_split<<<grid_for(mm), 256, 0, s>>>(m, Cq, w.Cp, w.W, lamh);
        FEAST_LAUNCH_CHECK();
        if ((e = mark(0.0))) return e;
        if ((e = mul(0, m, m, m, one, w.W, m, Vh, m, zero, w.S, m, 2))) return e;       // W'
        if ((e = tri_inverse(s, m, Vh, m, w.Cp, w.Ts))) return e;
        if ((e = mul(0, m, m, m, one, w.Cp, m, w.S, m, zero, F, m, 1))) return e;       // V^{-1} W'
        if ((e = mark(8.0 * m3 + tri_inv))) return e;   // (algorithmic: V^ triangular)
        k_add_diag_lambda<<<cdiv(m, 128), 128, 0, s>>>(m, F, lamh, alpha, beta);
        FEAST_LAUNCH_CHECK();
        FEAST_CUDA_TRY(cudaMemsetAsync(w.res, 0, 16, s));
        k_newton_g<<<grid_for(mm), 256, 0, s>>>(m, F, alpha, w.bad);
        FEAST_LAUNCH_CHECK();
        FEAST_CUDA_TRY(cudaMemcpyAsync(w.Yp, Vh, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, s));
        k_newton_s1<<<grid_for(mm), 256, 0, s>>>(m, F, lamh, alpha, w.W);
        FEAST_LAUNCH_CHECK();
        FEAST_CUDA_TRY(cudaMemcpyAsync(Cq, w.S, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, s));   // R = W'
        if ((e = mark(0.0))) return e;
        if ((e = mul(0, m, m, m, one, Vh, m, F, m, one, w.Yp, m, 1))) return e;       // Y' = V^ + V^ G
        if ((e = mul(0, m, m, m, one, Vh, m, w.W, m, one, Cq, m, 1))) return e;       // R += V^ S1
        if ((e = mul(0, m, m, m, one, w.S, m, F, m, one, Cq, m, 0))) return e;        // R += W' G
        if ((e = mark(16.0 * m3))) return e;
        k_eig_resid<<<cdiv((size_t)m * 32, 256), 256, 0, s>>>(m, Cq, w.Yp, alpha, hn, w.res, 1);
        FEAST_LAUNCH_CHECK();
    }
    struct {
        unsigned long long r;
        int bad;
        int pad;
    } hr{};
    int qfail = 0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&hr, w.res, 16, cudaMemcpyDeviceToHost, s));
    if (prm.cold_fp32) FEAST_CUDA_TRY(cudaMemcpyAsync(&qfail, fail, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    double worst;
    memcpy(&worst, &hr.r, sizeof(double));
    res->resid = worst;
    res->tail = mb;
    if (hr.bad || qfail || !(worst <= prm.accept_tol)) return FEAST_OK;
    // Y = Zh Y', unit columns
    FEAST_CUDA_TRY(cudaMemcpy2DAsync(V, sizeof(zd) * m, w.Yp, sizeof(zd) * m, sizeof(zd) * k, m,
                                     cudaMemcpyDeviceToDevice, s));
    if ((e = mulc(0, mb, m, mb, one, w.Z, mb, w.Yp + k, m, zero, V + k, m, 0))) return e;
    if ((e = normalise_cols(s, m, V))) return e;
    res->accepted = 1;
    return FEAST_OK;
}

}  // namespace feast
