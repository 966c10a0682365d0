// Kernels of the precision form: complex64 shifted matrices, conversions
// between complex128 solutions and complex64 corrections, and the pieces of
// the refinement residual R_j = B U1 - M_j X_j other than its two products
// (which run on the tensor cores, k_oz.cu): R_j's initial value and the
// per-node squared norms.
#include "common.cuh"

namespace feast {

namespace {

// M32_j = fl32(z_j B - A), complex64 (B = I when B is null).
__global__ void k_form_shifted32(int64_t n, const zd *__restrict__ A, const zd *__restrict__ B, int64_t ld,
                                 const zd *__restrict__ z, cf *__restrict__ M32, int64_t sF)
{
    const int j = blockIdx.y;
    const zd zj = z[j];
    const int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        zd bij = B ? B[r + c * ld] : zmake(r == c ? 1.0 : 0.0, 0.0);
        zd v = zsub(zmul(zj, bij), A[r + c * ld]);
        M32[(int64_t)j * sF + r + c * n] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void k_z2c(int64_t count, const zd *__restrict__ x, cf *__restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        zd v = x[e];
        y[e] = make_float2((float)v.x, (float)v.y);
    }
}

__global__ void k_c2z(int64_t count, const cf *__restrict__ x, zd *__restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        cf v = x[e];
        y[e] = zmake((double)v.x, (double)v.y);
    }
}

__global__ void k_add_c32(int64_t count, zd *__restrict__ x, const cf *__restrict__ c)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        cf v = c[e];
        zd a = x[e];
        x[e] = zmake(a.x + (double)v.x, a.y + (double)v.y);
    }
}

__global__ void k_sumsq(int64_t count, const zd *__restrict__ x, double *__restrict__ out)
{
    __shared__ double red[32];
    double part = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        part += zabs2(x[e]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        atomicAdd(out, s);
    }
}

__global__ void k_resid_init(int64_t n, int64_t m, const zd *__restrict__ BV, const zd *__restrict__ xz,
                             const zd *__restrict__ z, zd *__restrict__ R)
{
    const int j = blockIdx.y;
    const int64_t nm = n * m;
    const zd zj = z[j];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nm; e += (int64_t)gridDim.x * blockDim.x) {
        zd v = BV[e];
        if (xz) {
            zd x = xz[(int64_t)j * nm + e];
            v = zsub(v, zmul(zj, x));
        }
        R[(int64_t)j * nm + e] = v;
    }
}

__global__ void k_sumsq_blocks(int64_t count, const zd *__restrict__ x, double *__restrict__ out)
{
    __shared__ double red[32];
    const int j = blockIdx.y;
    const zd *xj = x + (int64_t)j * count;
    double part = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        part += zabs2(xj[e]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        atomicAdd(out + j, s);
    }
}

unsigned grid_for(int64_t count)
{
    unsigned g = cdiv(count, 256);
    return g > 152 * 32 ? 152 * 32 : (g == 0 ? 1 : g);
}
}  // namespace

int form_shifted32(cudaStream_t s, int64_t n, int q, const zd *A, const zd *B, int64_t ld, const zd *z, cf *M32)
{
    unsigned gx = cdiv(n * n, 256);
    if (gx > 1024) gx = 1024;
    k_form_shifted32<<<dim3(gx, q), 256, 0, s>>>(n, A, B, ld, z, M32, n * n);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int z2c(cudaStream_t s, int64_t count, const zd *x, cf *y)
{
    k_z2c<<<grid_for(count), 256, 0, s>>>(count, x, y);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int c2z(cudaStream_t s, int64_t count, const cf *x, zd *y)
{
    k_c2z<<<grid_for(count), 256, 0, s>>>(count, x, y);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int add_c32(cudaStream_t s, int64_t count, zd *x, const cf *c)
{
    k_add_c32<<<grid_for(count), 256, 0, s>>>(count, x, c);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int sumsq(cudaStream_t s, int64_t count, const zd *x, double *out)
{
    FEAST_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
    k_sumsq<<<grid_for(count), 256, 0, s>>>(count, x, out);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int resid_init(cudaStream_t s, int64_t n, int64_t m, int q, const zd *BV, const zd *xz, const zd *z, zd *R)
{
    unsigned gx = cdiv(n * m, 256);
    if (gx > 256) gx = 256;
    k_resid_init<<<dim3(gx, q), 256, 0, s>>>(n, m, BV, xz, z, R);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int sumsq_blocks(cudaStream_t s, int64_t count, int q, const zd *x, double *out)
{
    FEAST_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * q, s));
    unsigned gx = cdiv(count, 256);
    if (gx > 128) gx = 128;
    k_sumsq_blocks<<<dim3(gx, q), 256, 0, s>>>(count, x, out);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
