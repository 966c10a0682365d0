// Kernels of the precision form: complex64 shifted matrices and their
// factors, conversions, and the refinement residual R_j = B U1 - M_j X_j
// evaluated to ~48-bit accuracy without the FP64 pipe.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the residual uses
// double-single arithmetic on the FP32 pipe: M_j and X_j are held as
// unevaluated sums hi + lo of two floats; each product hi*hi is formed
// exactly (FMA error term), the cross terms hi*lo + lo*hi are added to that
// error, and the running sum is kept as a float pair by an error-free
// two-sum and renormalised.  The result carries ~44-48 significant bits
// (worst case K * 2^-48 relative to the partial sums) at ~15 FP32
// operations per real multiply-add.
#include "common.cuh"

namespace feast {

namespace {

// M32_j = fl32(z_j B - A)  and the double-single split Mhi + Mlo of the
// FP64 value (for the residual).  Any of the outputs may be null.
__global__ void k_form_shifted_split(int64_t n, const zd *__restrict__ A, const zd *__restrict__ B,
                                     int64_t ld, const zd *__restrict__ z, cf *__restrict__ M32,
                                     cf *__restrict__ Mhi, cf *__restrict__ Mlo, int64_t sF)
{
    const int j = blockIdx.y;
    const zd zj = z[j];
    const int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        zd bij = B ? B[r + c * ld] : zmake(r == c ? 1.0 : 0.0, 0.0);
        zd v = zsub(zmul(zj, bij), A[r + c * ld]);
        float hr = (float)v.x, hi = (float)v.y;
        const int64_t o = (int64_t)j * sF + r + c * n;
        if (M32) M32[o] = make_float2(hr, hi);
        if (Mhi) {
            Mhi[o] = make_float2(hr, hi);
            Mlo[o] = make_float2((float)(v.x - (double)hr), (float)(v.y - (double)hi));
        }
    }
}

__global__ void k_split(int64_t count, const zd *__restrict__ x, cf *__restrict__ hi,
                        cf *__restrict__ lo)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        zd v = x[e];
        float hr = (float)v.x, him = (float)v.y;
        hi[e] = make_float2(hr, him);
        lo[e] = make_float2((float)(v.x - (double)hr), (float)(v.y - (double)him));
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

// ---------------------------------------------------------------- residual
constexpr int RT_M = 64, RT_N = 64, RT_K = 16, RT_T = 256;

struct DS {  // double-single accumulator
    float h, l;
};

// acc += a * x for reals given as (hi, lo) pairs
__device__ __forceinline__ void ds_mac(DS &acc, float ah, float al, float xh, float xl)
{
    // explicit round-to-nearest intrinsics: the compiler must not contract
    // these additions into FMAs, or the error terms stop being exact
    float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    float s = __fadd_rn(acc.h, p);                                   // two-sum of the high parts
    float bb = __fsub_rn(s, acc.h);
    float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    float t = __fadd_rn(acc.l, __fadd_rn(err, e));
    float h = __fadd_rn(s, t);                                       // renormalise (fast two-sum)
    acc.l = __fsub_rn(t, __fsub_rn(h, s));
    acc.h = h;
}

// R_j = RHS - M_j X_j for one 64 x 64 tile of node j.  Complex operands as
// (hi, lo) float2 planes: M (q x n x n), X (q x n x m, leading dim n).
// nrm2[j] += ||tile of R_j||_F^2.
__global__ void __launch_bounds__(RT_T) k_ds_residual(int64_t n, int64_t m, const cf *__restrict__ Mhi,
                                                      const cf *__restrict__ Mlo,
                                                      const cf *__restrict__ Xhi,
                                                      const cf *__restrict__ Xlo,
                                                      const zd *__restrict__ RHS, zd *__restrict__ R,
                                                      double *__restrict__ nrm2)
{
    __shared__ cf sAh[RT_K][RT_M + 1], sAl[RT_K][RT_M + 1];
    __shared__ cf sXh[RT_K][RT_N + 1], sXl[RT_K][RT_N + 1];
    __shared__ double red[RT_T / 32];
    const int j = blockIdx.z;
    const cf *Ah = Mhi + (int64_t)j * n * n, *Al = Mlo + (int64_t)j * n * n;
    const cf *Xh = Xhi + (int64_t)j * n * m, *Xl = Xlo + (int64_t)j * n * m;
    zd *Rj = R + (int64_t)j * n * m;
    const int64_t i0 = (int64_t)blockIdx.x * RT_M, c0 = (int64_t)blockIdx.y * RT_N;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    DS re[4][4], im[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { re[a][b] = DS{0.f, 0.f}; im[a][b] = DS{0.f, 0.f}; }
    for (int64_t k0 = 0; k0 < n; k0 += RT_K) {
        for (int e = threadIdx.x; e < RT_M * RT_K; e += RT_T) {
            int r = e % RT_M, kk = e / RT_M;
            int64_t gi = i0 + r, gk = k0 + kk;
            bool ok = gi < n && gk < n;
            sAh[kk][r] = ok ? Ah[gi + gk * n] : make_float2(0.f, 0.f);
            sAl[kk][r] = ok ? Al[gi + gk * n] : make_float2(0.f, 0.f);
        }
        for (int e = threadIdx.x; e < RT_N * RT_K; e += RT_T) {
            int kk = e % RT_K, c = e / RT_K;
            int64_t gk = k0 + kk, gc = c0 + c;
            bool ok = gk < n && gc < m;
            sXh[kk][c] = ok ? Xh[gk + gc * n] : make_float2(0.f, 0.f);
            sXl[kk][c] = ok ? Xl[gk + gc * n] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < RT_K; ++kk) {
            cf ah[4], al[4], xh[4], xl[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) { ah[a] = sAh[kk][ty + 16 * a]; al[a] = sAl[kk][ty + 16 * a]; }
#pragma unroll
            for (int b = 0; b < 4; ++b) { xh[b] = sXh[kk][tx + 16 * b]; xl[b] = sXl[kk][tx + 16 * b]; }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // (ar + i ai)(xr + i xi): re = ar xr - ai xi, im = ar xi + ai xr
                    ds_mac(re[a][b], ah[a].x, al[a].x, xh[b].x, xl[b].x);
                    ds_mac(re[a][b], -ah[a].y, -al[a].y, xh[b].y, xl[b].y);
                    ds_mac(im[a][b], ah[a].x, al[a].x, xh[b].y, xl[b].y);
                    ds_mac(im[a][b], ah[a].y, al[a].y, xh[b].x, xl[b].x);
                }
        }
        __syncthreads();
    }
    double part = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int64_t gi = i0 + ty + 16 * a, gc = c0 + tx + 16 * b;
            if (gi < n && gc < m) {
                zd rhs = RHS[gi + gc * n];
                double pr = (double)re[a][b].h + (double)re[a][b].l;
                double pi = (double)im[a][b].h + (double)im[a][b].l;
                zd v = zmake(rhs.x - pr, rhs.y - pi);
                Rj[gi + gc * n] = v;
                part += zabs2(v);
            }
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < RT_T / 32; ++w) s += red[w];
        atomicAdd(nrm2 + j, s);
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

unsigned grid_for(int64_t count)
{
    unsigned g = cdiv(count, 256);
    return g > 152 * 32 ? 152 * 32 : (g == 0 ? 1 : g);
}
}  // namespace

int form_shifted_split(cudaStream_t s, int64_t n, int q, const zd *A, const zd *B, int64_t ld,
                       const zd *z, cf *M32, cf *Mhi, cf *Mlo)
{
    unsigned gx = cdiv(n * n, 256);
    if (gx > 1024) gx = 1024;
    k_form_shifted_split<<<dim3(gx, q), 256, 0, s>>>(n, A, B, ld, z, M32, Mhi, Mlo, n * n);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int split_hilo(cudaStream_t s, int64_t count, const zd *x, cf *hi, cf *lo)
{
    k_split<<<grid_for(count), 256, 0, s>>>(count, x, hi, lo);
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

int ds_residual(cudaStream_t s, int64_t n, int64_t m, int q, const cf *Mhi, const cf *Mlo,
                const cf *Xhi, const cf *Xlo, const zd *RHS, zd *R, double *nrm2)
{
    FEAST_CUDA_TRY(cudaMemsetAsync(nrm2, 0, sizeof(double) * q, s));
    dim3 g(cdiv(n, RT_M), cdiv(m, RT_N), q);
    k_ds_residual<<<g, RT_T, 0, s>>>(n, m, Mhi, Mlo, Xhi, Xlo, RHS, R, nrm2);
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

}  // namespace feast
