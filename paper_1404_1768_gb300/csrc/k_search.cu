// SEARCH (Section 4.1, Algorithm SEARCH) on the GPU: the trace estimate of
// line 2 and the rank-revealing factorisation of line 9.
//
// Line 9's column-pivoted QR U Pi = Q R is taken through the Gram matrix:
// a pivoted Cholesky factorisation Pi^H (U^H U) Pi = R^H R picks, step by
// step, the column with the largest remaining norm -- the same greedy rule
// as Householder QR with column pivoting, with the same R in exact
// arithmetic -- and stops when that norm falls to rank_tol of the first.
// The Gram matrix squares the condition number, so ranks are resolved down
// to ~1e-7 relative (plenty for SEARCH's thresholds).  The factorisation
// is one cooperative launch: per step every CTA proposes the largest
// remaining diagonal entry of its columns, a grid barrier, every CTA takes
// the same winner and computes its share of row k of R (a warp per column,
// lanes over the previous rows), another barrier.
#include "common.cuh"

namespace feast {
namespace {

constexpr int ST = 256;

// out += sum_j Re(y_j^H u_j) over p columns (n rows, leading dims ldy, ldu)
__global__ void k_trace_real(int64_t n, int p, const zd *__restrict__ Y, int64_t ldy, const zd *__restrict__ U,
                             int64_t ldu, double *__restrict__ out)
{
    __shared__ double red[ST / 32];
    double s = 0.0;
    const int64_t total = n * p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        const zd y = Y[i + j * ldy], u = U[i + j * ldu];
        s += y.x * u.x + y.y * u.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < ST / 32; ++w) t += red[w];
        atomicAdd(out, t);
    }
}

// Pivoted Cholesky of the m x m Gram matrix G (leading dim m).  R (m x m,
// leading dim m, columns in the ORIGINAL order: R[k + j m] = row k, column
// j of R Pi^H), piv[k] = original column of step k, d = the remaining
// diagonal, used = 0 / 1 per column, pval / pidx = per-CTA proposals.
// *rank = number of steps with R_kk > rank_tol R_00.
__global__ void __launch_bounds__(ST) k_pchol_grid(int m, const zd *__restrict__ G, zd *__restrict__ R,
                                                   int *__restrict__ piv, double *__restrict__ d,
                                                   int *__restrict__ used, double *__restrict__ pval,
                                                   int *__restrict__ pidx, double rank_tol, int *__restrict__ rank,
                                                   GridSync gs)
{
    __shared__ double sv[ST / 32];
    __shared__ int si[ST / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gwarp = blockIdx.x * (ST / 32) + wid, nwarp = gridDim.x * (ST / 32);
    for (int j = blockIdx.x * ST + tid; j < m; j += gridDim.x * ST) {
        d[j] = G[j + (int64_t)j * m].x;
        used[j] = 0;
    }
    if (!grid_barrier(gs)) return;
    double r00 = 0.0;
    int k = 0;
    for (; k < m; ++k) {
        // proposals: largest remaining d over this CTA's columns (ties: lowest index)
        double bv = -1.0;
        int bi = m;
        for (int j = blockIdx.x * ST + tid; j < m; j += gridDim.x * ST)
            if (!used[j] && (d[j] > bv || (d[j] == bv && j < bi))) { bv = d[j]; bi = j; }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { sv[wid] = bv; si[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < ST / 32; ++w)
                if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
            pval[blockIdx.x] = bv;
            pidx[blockIdx.x] = bi;
        }
        if (!grid_barrier(gs)) return;
        // every CTA reduces all proposals the same way
        double vmax = -1.0;
        int jmax = m;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            const double v = pval[b];
            const int i = pidx[b];
            if (v > vmax || (v == vmax && i < jmax)) { vmax = v; jmax = i; }
        }
        const double rkk = vmax > 0.0 ? sqrt(vmax) : 0.0;
        if (k == 0) r00 = rkk;
        if (jmax >= m || !(rkk > rank_tol * r00) || !(rkk > 0.0)) break;
        if (blockIdx.x == 0 && tid == 0) {
            piv[k] = jmax;
            used[jmax] = 1;
            R[k + (int64_t)jmax * m] = zmake(rkk, 0.0);
        }
        // row k: R[k, j] = (G[jmax, j] - sum_{i<k} conj(R[i, jmax]) R[i, j]) / rkk
        const zd *rp = R + (int64_t)jmax * m;
        for (int j = gwarp; j < m; j += nwarp) {
            if (j == jmax || used[j]) continue;
            const zd *rj = R + (int64_t)j * m;
            double ax = 0.0, ay = 0.0;
            for (int i = lane; i < k; i += 32) {
                const zd a = rp[i], b = rj[i];   // conj(a) b
                ax += a.x * b.x + a.y * b.y;
                ay += a.x * b.y - a.y * b.x;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, off);
                ay += __shfl_xor_sync(0xffffffffu, ay, off);
            }
            if (lane == 0) {
                const zd g = G[jmax + (int64_t)j * m];
                const zd v = zmake((g.x - ax) / rkk, (g.y - ay) / rkk);
                R[k + (int64_t)j * m] = v;
                d[j] -= v.x * v.x + v.y * v.y;
            }
        }
        if (!grid_barrier(gs)) return;
    }
    if (blockIdx.x == 0 && tid == 0) *rank = k;
}

// Up[:, c] = U[:, piv[c]] (n rows) and Rt[i, c] = R[i, piv[c]] (t x t).
__global__ void k_gather_pivoted(int64_t n, int t, const int *__restrict__ piv, const zd *__restrict__ U,
                                 int64_t ldu, zd *__restrict__ Up, const zd *__restrict__ R, int m,
                                 zd *__restrict__ Rt)
{
    const int64_t total = n * t;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n;
        const int c = (int)(e / n);
        const int src = piv[c];
        Up[i + (int64_t)c * n] = U[i + (int64_t)src * ldu];
        if (i < t) Rt[i + (int64_t)c * t] = (i <= c) ? R[i + (int64_t)src * m] : zmake(0.0, 0.0);
    }
}

unsigned grid_for(size_t count)
{
    const unsigned g = cdiv(count, 256);
    return g > 4096 ? 4096 : g;
}

}  // namespace

size_t rrqr_work_bytes(int64_t n, int m)
{
    return sizeof(zd) * (3 * (size_t)m * m + (size_t)n * m + tri_inverse_scratch_elems(m)) +
           sizeof(double) * (size_t)m + sizeof(int) * 2 * (size_t)m + 2048 * (sizeof(double) + sizeof(int)) + 256;
}

int trace_real(cudaStream_t s, int64_t n, int p, const zd *Y, int64_t ldy, const zd *U, int64_t ldu, double *out)
{
    FEAST_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
    k_trace_real<<<grid_for((size_t)n * p), ST, 0, s>>>(n, p, Y, ldy, U, ldu, out);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int rrqr_basis(cudaStream_t s, int64_t n, int m, const zd *U, zd *Q, double rank_tol, void *work, int *timeout,
               int *t_out)
{
    *t_out = 0;
    if (m <= 0) return FEAST_OK;
    const size_t mm = (size_t)m * m;
    zd *G = (zd *)work;
    zd *R = G + mm;
    zd *Rt = R + mm;
    zd *Up = Rt + mm;
    zd *Ts = Up + (size_t)n * m;
    double *d = (double *)(Ts + tri_inverse_scratch_elems(m));
    int *piv = (int *)(d + m);
    int *used = piv + m;
    double *pval = (double *)(used + m);
    int *pidx = (int *)(pval + 1024);
    unsigned *bar = (unsigned *)(pidx + 1024);
    int *rk = (int *)(bar + 2);
    const zd one = zmake(1.0, 0.0), zero = zmake(0.0, 0.0);
    int e;
    // G = U^H U (FP64)
    if ((e = zgemm_batched(s, 1, m, m, n, one, U, n, 0, U, n, 0, zero, G, m, 0, 1))) return e;
    FEAST_CUDA_TRY(cudaMemsetAsync(R, 0, sizeof(zd) * mm, s));
    int dev = 0, sms = 0, per = 0;
    FEAST_CUDA_TRY(cudaGetDevice(&dev));
    FEAST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pchol_grid, ST, 0));
    if (per < 1) return FEAST_ECUDA;
    int grid = (m + ST - 1) / ST * 4;
    if (grid < 4) grid = 4;
    if (grid > sms) grid = sms;
    if (grid > 1024) grid = 1024;
    FEAST_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    GridSync gs{bar, bar + 1, timeout, TO_PCHOL};
    int mm_ = m;
    void *args[] = {&mm_, &G, &R, &piv, &d, &used, &pval, &pidx, &rank_tol, &rk, &gs};
    FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_pchol_grid, dim3(grid), dim3(ST), args, 0, s));
    FEAST_LAUNCH_CHECK();
    int t = 0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&t, rk, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    *t_out = t;
    if (t <= 0) return FEAST_OK;
    // basis: U[:, piv[:t]] R_t^{-1}, into Q[:, :t]
    k_gather_pivoted<<<grid_for((size_t)n * t), 256, 0, s>>>(n, t, piv, U, n, Up, R, m, Rt);
    FEAST_LAUNCH_CHECK();
    if ((e = tri_inverse(s, t, Rt, t, G, Ts))) return e;
    if ((e = zgemm_batched(s, 0, n, t, t, one, Up, n, 0, G, t, 0, zero, Q, n, 0, 1, 2))) return e;
    return FEAST_OK;
}

}  // namespace feast
