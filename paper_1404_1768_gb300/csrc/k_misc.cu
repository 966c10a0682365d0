// Small kernels of the FEAST pass: quadrature nodes and weights on the
// device (eq. 4.1 and its trapezoid / ellipse variants), the residuals of
// eq. 5.1 for every Ritz pair, the selection and stopping tests of GFEAST
// lines 7-15, and the compaction of the accepted pairs.
#include "common.cuh"

namespace feast {

namespace {
// One thread per node.  Gauss-Legendre: t_j is found by Newton's method on
// P_q (three-term recurrence), omega_j = 2 / ((1 - t^2) P_q'(t)^2); nodes
// are returned in ascending t.  The weight w_j folds in the 1/(2 pi i)
// factor and z'(theta_j) so that the contour integral is sum_j w_j f(z_j).
__global__ void k_contour(int kind, int rule, int q, double cre, double cim, double a, double b,
                          zd *z, zd *w)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= q) return;
    if (kind == FEAST_CIRCLE) b = a;
    double theta, dth;
    if (rule == FEAST_GAUSS_LEGENDRE) {
        // the (q-1-j)-th largest root -> ascending order
        const int jj = q - 1 - j;
        double x = cos(M_PI * (jj + 0.75) / (q + 0.5));
        double p0 = 1.0, p1 = x, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0;
            p1 = x;
            for (int k = 1; k < q; ++k) {
                double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = q * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-15) break;
        }
        p0 = 1.0;
        p1 = x;
        for (int k = 1; k < q; ++k) {
            double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = q * (x * p1 - p0) / (x * x - 1.0);
        const double om = 2.0 / ((1.0 - x * x) * dp * dp);
        theta = (1.0 + x) * M_PI;
        dth = M_PI * om;
    } else {
        theta = 2.0 * M_PI * (j + 0.5) / q;
        dth = 2.0 * M_PI / q;
    }
    const double ct = cos(theta), stt = sin(theta);
    z[j] = zmake(cre + a * ct, cim + b * stt);
    // w = dth * z'(theta) / (2 pi i),  z'(theta) = -a sin + i b cos
    const double f = dth / (2.0 * M_PI);
    w[j] = zmake(f * b * ct, f * a * stt);
}

// r_i = ||A x_i - lambda_i B x_i|| / (||A x_i|| + ||B x_i||) with A x_i, B x_i
// the columns of AX, BX; lambda_i = alpha_i / beta_i.  One CTA per pair.
__global__ void k_ritz_residual(int64_t n, int m, const zd *AX, const zd *BX, int64_t ld,
                                const zd *alpha, const zd *beta, zd *lam, double *res,
                                DevStatus *st)
{
    const int i = blockIdx.x;
    __shared__ double red[3][32];
    const zd be = beta[i], al = alpha[i];
    const bool finite = (be.x != 0.0 || be.y != 0.0);
    const zd l = finite ? zdiv(al, be) : zmake(INFINITY, 0.0);
    double num = 0.0, na = 0.0, nb = 0.0;
    if (finite)
        for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
            zd ax = AX[r + i * ld], bx = BX[r + i * ld];
            zd d = ax;
            zfma(d, zmake(-l.x, -l.y), bx);
            num += zabs2(d);
            na += zabs2(ax);
            nb += zabs2(bx);
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, off);
        na += __shfl_xor_sync(0xffffffffu, na, off);
        nb += __shfl_xor_sync(0xffffffffu, nb, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = num; red[1][wid] = na; red[2][wid] = nb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { s0 += red[0][w]; s1 += red[1][w]; s2 += red[2][w]; }
        double r = finite ? sqrt(s0) / (sqrt(s1) + sqrt(s2)) : INFINITY;
        lam[i] = l;
        res[i] = r;
        if (finite && !isfinite(r) && st) atomicExch(&st->nonfinite, 1);
    }
}

__device__ __forceinline__ bool inside_contour(int kind, double cre, double cim, double a,
                                               double b, zd l)
{
    if (kind == FEAST_CIRCLE) b = a;
    if (!isfinite(l.x) || !isfinite(l.y)) return false;
    double x = (l.x - cre) / a, y = (l.y - cim) / b;
    return x * x + y * y < 1.0;
}

// Lines 7-15 in one thread: selection (inside and r_i < eta) in Ritz order,
// c(k), e(k) = max r over the selection (0 if empty), and the flag.  The
// count is taken as fixed (lines 13-14) only once it is non-zero.
__global__ void k_stop(int m, feast_contour c, const zd *lam, const double *res, double eta,
                       double eps, int k, int max_iter, int c_prev, double e_prev, int converged_only,
                       int *sel, int *idx, DevStatus *st)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int cnt = 0;
    double e = 0.0;
    for (int i = 0; i < m; ++i) {
        bool s = inside_contour(c.kind, c.center_re, c.center_im, c.a, c.b, lam[i]) && res[i] < eta;
        sel[i] = s ? 1 : 0;
        if (s) {
            idx[cnt++] = i;
            e = fmax(e, res[i]);
        }
    }
    const bool fixed = (cnt == c_prev) && cnt > 0;
    int flag = 2;
    if (fixed && e < eps) flag = 1;
    else if (fixed && e > e_prev && !converged_only) flag = 0;
    else if (k == max_iter) flag = -1;
    st->count = cnt;
    st->err = e;
    st->flag = flag;
}

// Accepted pairs to the front: Xc[:, p] = X[:, idx[p]], p < count.
__global__ void k_compact(int64_t n, int m, const int *idx, const DevStatus *st, const zd *X,
                          int64_t ldx, const zd *lam, const double *res, zd *Xc, zd *lamc,
                          double *resc)
{
    const int cnt = st->count;
    const int64_t total = n * (int64_t)m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n;
        int p = (int)(e / n);
        if (p >= cnt) continue;
        int src = idx[p];
        Xc[r + p * n] = X[r + (int64_t)src * ldx];
        if (r == 0) { lamc[p] = lam[src]; resc[p] = res[src]; }
    }
}
}  // namespace

int contour_nodes(cudaStream_t s, const feast_contour *c, zd *z, zd *w)
{
    k_contour<<<cdiv(c->q, 64), 64, 0, s>>>(c->kind, c->rule, c->q, c->center_re, c->center_im,
                                            c->a, c->b, z, w);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int ritz_residuals(cudaStream_t s, int64_t n, int m, const zd *AX, const zd *BX, int64_t ld,
                   const zd *alpha, const zd *beta, zd *lam, double *res, DevStatus *st)
{
    k_ritz_residual<<<m, 256, 0, s>>>(n, m, AX, BX, ld, alpha, beta, lam, res, st);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int stop_test(cudaStream_t s, int m, const feast_contour *c, const zd *lam, const double *res,
              double eta, double eps, int k, int max_iter, int c_prev, double e_prev, int converged_only,
              int *sel, int *idx, DevStatus *st)
{
    k_stop<<<1, 32, 0, s>>>(m, *c, lam, res, eta, eps, k, max_iter, c_prev, e_prev, converged_only, sel, idx,
                            st);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int compact_pairs(cudaStream_t s, int64_t n, int m, const int *idx, const DevStatus *st,
                  const zd *X, int64_t ldx, const zd *lam, const double *res, zd *Xc, zd *lamc,
                  double *resc)
{
    unsigned gx = cdiv(n * m, 256);
    if (gx > 4096) gx = 4096;
    k_compact<<<gx, 256, 0, s>>>(n, m, idx, st, X, ldx, lam, res, Xc, lamc, resc);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
