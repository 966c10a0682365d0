// Differentiation form: gradients of L = sum over the eigenvalues inside the
// contour of |lambda|^2 with respect to A and B (real loss of complex
// inputs, dL = Re sum conj(G) * dA).
//
// A simple eigenvalue lambda_i with right vector x_i (A x = lambda B x) and
// left vector v_i (v^H A = lambda v^H B) moves by
//     d lambda_i = v_i^H (dA - lambda_i dB) x_i / c_i,   c_i = v_i^H B x_i,
// so with dL = sum_i 2 Re(conj(lambda_i) d lambda_i)
//     G_A = sum_i alpha_i v_i x_i^H,  alpha_i = 2 lambda_i / conj(c_i),
//     G_B = sum_i beta_i  v_i x_i^H,  beta_i = -2 |lambda_i|^2 / conj(c_i).
// The right pairs come from a FEAST run on (A, B); the left vectors are the
// right Ritz vectors of a FEAST run on (A^H, B^H) over the conjugated
// contour (its eigenvalues are the conjugates).  Two kernels: the pair
// coefficients (one warp per pair) and the fused rank-s products that form
// both gradients from one pass over V and X.
#include "common.cuh"

namespace feast {

namespace {

// alpha_i, beta_i from c_i = v_{k_i}^H (B x)_i; one warp per pair.
__global__ void k_adj_coef(int64_t n, int s, const zd *__restrict__ V, int64_t ldv, const int *__restrict__ kidx,
                           const zd *__restrict__ BX, int64_t ldb, const zd *__restrict__ lam,
                           zd *__restrict__ alpha, zd *__restrict__ beta)
{
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= s) return;
    const zd *v = V + (int64_t)kidx[i] * ldv;
    const zd *bx = BX + (int64_t)i * ldb;
    zd acc = zmake(0.0, 0.0);
    for (int64_t r = lane; r < n; r += 32) zfma_conj(acc, v[r], bx[r]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) {
        const zd li = lam[i];
        const zd cc = zconj(acc);
        const double d = zabs2(cc);
        // 1 / conj(c) = c / |c|^2
        const zd inv = (d > 0.0) ? zscale(acc, 1.0 / d) : zmake(0.0, 0.0);
        alpha[i] = zscale(zmul(li, inv), 2.0);
        beta[i] = zscale(inv, -2.0 * zabs2(li));
    }
}

constexpr int AT = 64;      // output tile edge
constexpr int AK = 16;      // pairs per stage

// G_A[r, l] = sum_i alpha_i V[r, k_i] conj(X[l, i]),  G_B likewise with beta.
// 64 x 64 tiles of both outputs, 256 threads, 4 x 4 entries per thread.
__global__ void __launch_bounds__(256) k_adj_grad(int64_t n, int s, const zd *__restrict__ V, int64_t ldv,
                                                  const int *__restrict__ kidx, const zd *__restrict__ X,
                                                  int64_t ldx, const zd *__restrict__ alpha,
                                                  const zd *__restrict__ beta, zd *__restrict__ GA,
                                                  zd *__restrict__ GB, int64_t ldg)
{
    __shared__ zd sV[AK][AT + 1];
    __shared__ zd sX[AK][AT + 1];
    __shared__ zd sa[AK], sb[AK];
    const int64_t r0 = (int64_t)blockIdx.x * AT, l0 = (int64_t)blockIdx.y * AT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    zd ga[4][4], gb[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { ga[a][b] = zmake(0.0, 0.0); gb[a][b] = zmake(0.0, 0.0); }
    for (int i0 = 0; i0 < s; i0 += AK) {
        for (int e = threadIdx.x; e < AK * AT; e += 256) {
            const int ii = e / AT, rr = e % AT;
            const bool ok = (i0 + ii < s);
            const int64_t gr = r0 + rr, gl = l0 + rr;
            sV[ii][rr] = (ok && gr < n) ? V[gr + (int64_t)kidx[i0 + ii] * ldv] : zmake(0.0, 0.0);
            sX[ii][rr] = (ok && gl < n) ? zconj(X[gl + (int64_t)(i0 + ii) * ldx]) : zmake(0.0, 0.0);
        }
        if (threadIdx.x < AK) {
            const bool ok = (i0 + (int)threadIdx.x < s);
            sa[threadIdx.x] = ok ? alpha[i0 + threadIdx.x] : zmake(0.0, 0.0);
            sb[threadIdx.x] = ok ? beta[i0 + threadIdx.x] : zmake(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int ii = 0; ii < AK; ++ii) {
            zd va[4], vb[4], xr[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const zd v = sV[ii][ty + 16 * a];
                va[a] = zmul(sa[ii], v);
                vb[a] = zmul(sb[ii], v);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) xr[b] = sX[ii][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    zfma(ga[a][b], va[a], xr[b]);
                    zfma(gb[a][b], vb[a], xr[b]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t gr = r0 + ty + 16 * a, gl = l0 + tx + 16 * b;
            if (gr < n && gl < n) {
                GA[gr + gl * ldg] = ga[a][b];
                GB[gr + gl * ldg] = gb[a][b];
            }
        }
}

}  // namespace

int adjoint_coef(cudaStream_t s, int64_t n, int cnt, const zd *V, int64_t ldv, const int *kidx, const zd *BX,
                 int64_t ldb, const zd *lam, zd *alpha, zd *beta)
{
    if (cnt <= 0) return FEAST_OK;
    k_adj_coef<<<cdiv((size_t)cnt * 32, 256), 256, 0, s>>>(n, cnt, V, ldv, kidx, BX, ldb, lam, alpha, beta);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int adjoint_grad(cudaStream_t s, int64_t n, int cnt, const zd *V, int64_t ldv, const int *kidx, const zd *X,
                 int64_t ldx, const zd *alpha, const zd *beta, zd *GA, zd *GB, int64_t ldg)
{
    if (n <= 0) return FEAST_OK;
    dim3 g(cdiv(n, AT), cdiv(n, AT));
    k_adj_grad<<<g, 256, 0, s>>>(n, cnt, V, ldv, kidx, X, ldx, alpha, beta, GA, GB, ldg);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
