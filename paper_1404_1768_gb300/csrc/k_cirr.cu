// Block CIRR (Section 2.1, Algorithm Block_CIRR), step 1: the moment block
// R_i = F_i Y, i = 0..g-1, from the per-node solutions X_j = (z_j B - A)^{-1} Y
// already in HBM:  R_i = sum_j w_j zeta_j^i X_j with zeta_j = (z_j - c) / a
// (the shifted, scaled moments; degree by degree they span what z^i spans).
//
// One thread per (row, column) of the n x h solutions: it reads X_j(r, col)
// once per chunk of MC moments and keeps the chunk's sums in registers, so
// the q n h solutions are read ceil(g / MC) times and the n h g block is
// written once -- an HBM-bound pass.
#include "common.cuh"

namespace feast {
namespace {

constexpr int MC = 8;   // moments per register chunk

__global__ void k_moment_sum(int64_t n, int h, int q, int g, const zd *__restrict__ z, const zd *__restrict__ w,
                             double cre, double cim, double inv_scale, const zd *__restrict__ X, int64_t sX,
                             zd *__restrict__ R, int64_t ldr)
{
    const int64_t total = n * h;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % n;
        const int col = (int)(e / n);
        for (int i0 = 0; i0 < g; i0 += MC) {
            zd acc[MC];
#pragma unroll
            for (int k = 0; k < MC; ++k) acc[k] = zmake(0.0, 0.0);
            for (int j = 0; j < q; ++j) {
                const zd zj = z[j];
                const zd zeta = zmake((zj.x - cre) * inv_scale, (zj.y - cim) * inv_scale);
                zd pw = w[j];
                for (int k = 0; k < i0; ++k) pw = zmul(pw, zeta);   // w_j zeta_j^i0
                const zd x = X[(int64_t)j * sX + r + (int64_t)col * n];
#pragma unroll
                for (int k = 0; k < MC; ++k) {
                    zfma(acc[k], pw, x);
                    pw = zmul(pw, zeta);
                }
            }
#pragma unroll
            for (int k = 0; k < MC; ++k)
                if (i0 + k < g) R[r + (int64_t)((i0 + k) * h + col) * ldr] = acc[k];
        }
    }
}

}  // namespace

int moment_sum(cudaStream_t s, int64_t n, int h, int q, int g, const zd *z, const zd *w, double cre, double cim,
               double scale, const zd *X, int64_t sX, zd *R, int64_t ldr)
{
    if (n <= 0 || h <= 0 || g <= 0) return FEAST_OK;
    if (!(scale > 0.0)) return FEAST_EINVAL;
    unsigned gx = cdiv(n * h, 256);
    if (gx > 152 * 16) gx = 152 * 16;
    k_moment_sum<<<gx, 256, 0, s>>>(n, h, q, g, z, w, cre, cim, 1.0 / scale, X, sX, R, ldr);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
