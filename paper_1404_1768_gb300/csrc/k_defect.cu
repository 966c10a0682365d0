// Line 16 of GFEAST applied to Ritz pairs, in defect form (precision form).
//
// For a Ritz pair (lambda, x) with residual r = A x - lambda B x, and any
// node z_j != lambda,
//
//     (z_j B - A) x = (z_j - lambda) B x - r
//     =>  (z_j B - A)^{-1} B x = [x + (z_j B - A)^{-1} r] / (z_j - lambda),
//
// so the quadrature sum of eq. 4.1-4.2 over the Ritz block X is, exactly,
//
//     U = sum_j w_j M_j^{-1} B X = X rho(Lambda) + sum_j w_j M_j^{-1} (R D_j),
//     R = A X - B X Lambda,  D_j = diag(1 / (z_j - lambda_i)),
//     rho(lambda) = sum_j w_j / (z_j - lambda).
//
// The first term is exact (FP64); the solves only see R, whose size is the
// residual already reached, so the complex64 factors' relative error
// (~1e-6) lands on a term that shrinks with the residual: the filtered
// block is as accurate as FP64 solves would make it without refinement
// sweeps.  A X and B X are the products of line 9 (FP64-accurate).  A
// column whose Ritz value is non-finite or within dmin of a node takes the
// plain right-hand side B x (and no rho term).
#include "common.cuh"

namespace feast {
namespace {

// Per Ritz value: d_ji = 1 / (z_j - lambda_i) (complex64 table, q x m),
// rho_i, and whether the column is plain.
__global__ void k_defect_coef(int m, int q, const zd *__restrict__ z, const zd *__restrict__ w,
                              const zd *__restrict__ lam, double dmin, cf *__restrict__ d32, zd *__restrict__ rho,
                              int *__restrict__ plain)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const zd l = lam[i];
    bool ok = (l.x == l.x) && (l.y == l.y) && fabs(l.x) < 1e300 && fabs(l.y) < 1e300;
    for (int j = 0; ok && j < q; ++j) ok = zabs(zsub(z[j], l)) >= dmin;
    zd r = zmake(0.0, 0.0);
    for (int j = 0; j < q; ++j) {
        zd d = zmake(1.0, 0.0);
        if (ok) {
            d = zdiv(zmake(1.0, 0.0), zsub(z[j], l));
            r = zadd(r, zmul(w[j], d));
        }
        d32[(int64_t)j * m + i] = make_float2((float)d.x, (float)d.y);
    }
    rho[i] = r;
    plain[i] = ok ? 0 : 1;
}

// S = R = A X - B X Lambda (defect columns) or B X (plain columns), complex64.
__global__ void k_defect_src(int64_t n, int m, const zd *__restrict__ AX, const zd *__restrict__ BX,
                             const zd *__restrict__ lam, const int *__restrict__ plain, cf *__restrict__ S)
{
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const zd bx = BX[e];
        zd v = bx;
        if (!plain[c]) v = zsub(AX[e], zmul(bx, lam[c]));
        S[e] = make_float2((float)v.x, (float)v.y);
    }
}

// Right-hand side of node j: RHS_j[r, c] = S[src, c] d_jc with src =
// perm_j[r] (the LU's row interchanges; identity when perm is null).
__global__ void k_defect_rhs(int64_t n, int m, const int *__restrict__ perm, const cf *__restrict__ S,
                             const cf *__restrict__ d32, cf *__restrict__ X, int64_t sX)
{
    const int j = blockIdx.y;
    const int *pj = perm ? perm + (int64_t)j * n : nullptr;
    const cf *dj = d32 + (int64_t)j * m;
    cf *Xj = X + (int64_t)j * sX;
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % n;
        const int c = (int)(e / n);
        const int64_t src = pj ? pj[r] : r;
        const cf sv = S[src + (int64_t)c * n];
        const cf d = dj[c];
        Xj[e] = make_float2(sv.x * d.x - sv.y * d.y, sv.x * d.y + sv.y * d.x);
    }
}

// U[:, c] = sum_j w_j Y_j[:, c] (complex64 accumulation of the correction)
// + rho_c X[:, c] (FP64).
__global__ void k_defect_sum(int64_t n, int m, int q, const cf *__restrict__ Y, int64_t sY, const zd *__restrict__ w,
                             const zd *__restrict__ X, const zd *__restrict__ rho, zd *__restrict__ U)
{
    __shared__ cf ws[256];
    for (int j = threadIdx.x; j < q && j < 256; j += blockDim.x) ws[j] = make_float2((float)w[j].x, (float)w[j].y);
    __syncthreads();
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        float ar = 0.f, ai = 0.f;
        for (int j = 0; j < q; ++j) {
            const cf y = Y[(int64_t)j * sY + e];
            const cf wj = j < 256 ? ws[j] : make_float2((float)w[j].x, (float)w[j].y);
            ar = fmaf(wj.x, y.x, fmaf(-wj.y, y.y, ar));
            ai = fmaf(wj.x, y.y, fmaf(wj.y, y.x, ai));
        }
        const int c = (int)(e / n);
        const zd t = zmul(rho[c], X[e]);
        U[e] = zmake(t.x + (double)ar, t.y + (double)ai);
    }
}

unsigned grid_for(size_t count)
{
    const unsigned g = cdiv(count, 256);
    return g > 8192 ? 8192 : g;
}

}  // namespace

int defect_prepare(cudaStream_t s, int64_t n, int m, int q, const zd *z, const zd *w, const zd *lam, double dmin,
                   const zd *AX, const zd *BX, DefectScratch &d)
{
    k_defect_coef<<<cdiv(m, 128), 128, 0, s>>>(m, q, z, w, lam, dmin, d.d32, d.rho, d.plain);
    FEAST_LAUNCH_CHECK();
    k_defect_src<<<grid_for((size_t)n * m), 256, 0, s>>>(n, m, AX, BX, lam, d.plain, d.S);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int defect_rhs(cudaStream_t s, int64_t n, int m, int q, const int *perm, const DefectScratch &d, cf *X, int64_t sX)
{
    unsigned gx = grid_for((size_t)n * m);
    if (gx > 2048) gx = 2048;
    k_defect_rhs<<<dim3(gx, q), 256, 0, s>>>(n, m, perm, d.S, d.d32, X, sX);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int defect_sum(cudaStream_t s, int64_t n, int m, int q, const cf *Y, int64_t sY, const zd *w, const zd *X,
               const DefectScratch &d, zd *U)
{
    k_defect_sum<<<grid_for((size_t)n * m), 256, 0, s>>>(n, m, q, Y, sY, w, X, d.rho, U);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
