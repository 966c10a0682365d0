// Projected eigenproblem for large subspaces (m0 > 64), FP64, GFEAST line 6.
//
// B~ = U2^H B U1 equals R2 of the QR B U1 = U2 R2 (upper triangular; its
// condition number is that of B on the search space), so the projected
// pencil is reduced to the standard problem C = B~^{-1} A~, whose
// eigenpairs are those of (A~, B~).  Then:
//   1. Hessenberg reduction C = Q H Q^H by Householder reflectors, one
//      column per step, each step a handful of grid-wide kernels;
//   2. QR iteration on H with deflation, accumulating the Schur vectors
//      into Q, in double-single arithmetic (~46 bits) on the FP32 pipe (the
//      FP64 pipe is 64x slower): aggressive early deflation on a trailing
//      window (Schur form of the window by one CTA, deflation by the spike
//      test, reordering, Householder back to Hessenberg), then multishift
//      sweeps whose bulges are chased concurrently, one CTA each, on small
//      diagonal blocks in shared memory, with the long row / column /
//      Schur-vector segments of each chunk of rotations applied by the whole
//      grid.  The grid is a cooperative launch; its barriers spin with an
//      iteration limit and report a timeout instead of hanging;
//   3. right eigenvectors of the triangular Schur form by back-substitution
//      (one warp per eigenvector), mapped back by Q (a GEMM), unit norm.
// The small-pencil path (m0 <= 64, one warp, shared memory) is the QZ
// kernel in k_zqz.cu.
#include <cooperative_groups.h>

#include "common.cuh"

#ifndef FEAST_QR_FP32
#define FEAST_QR_FP32 0
#endif

namespace feast {

namespace {

constexpr int CH = 32;           // rotations per chunk
constexpr int BLK = CH + 3;      // local block edge
constexpr int QT = 256;          // threads per CTA of the QR kernel
constexpr int NSH = 16;          // most shifts (bulges) of a multishift sweep
constexpr int DSEP = 2;          // phases between the entries of consecutive bulges
constexpr int MS_MIN = 192;      // smallest active window that takes multishift sweeps

// ------------------------------------------------------------- Householder
// v = x - beta e1 with beta = -(x0/|x0|) ||x||, tau = 2 / ||v||^2, for
// x = C[j+1:m, j]; column j becomes (beta, 0, ..., 0).  One CTA.
__global__ void k_house(int m, int j, zd *C, int ld, zd *v, double *tau)
{
    __shared__ double red[32];
    __shared__ double s_norm;
    const int len = m - j - 1;
    zd *x = C + (j + 1) + (int64_t)j * ld;
    double part = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) part += zabs2(x[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        s_norm = sqrt(s);
    }
    __syncthreads();
    const double nrm = s_norm;
    const zd x0 = x[0];
    const double a0 = zabs(x0);
    const zd ph = a0 > 0.0 ? zscale(x0, 1.0 / a0) : zmake(1.0, 0.0);
    const zd beta = zscale(ph, -nrm);
    // v = x - beta e1 ;  ||v||^2 = 2 nrm (nrm + |x0|)
    const double vv = 2.0 * nrm * (nrm + a0);
    for (int i = threadIdx.x; i < len; i += blockDim.x) v[i] = (i == 0) ? zsub(x0, beta) : x[i];
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) x[i] = (i == 0) ? beta : zmake(0.0, 0.0);
    if (threadIdx.x == 0) *tau = vv > 0.0 ? 2.0 / vv : 0.0;
}

// w[c] = sum_i conj(v[i]) M[r0 + i, c0 + c]   (one warp per column)
__global__ void k_vh_times(int rows, int cols, const zd *M, int ld, const zd *v, zd *w)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= cols) return;
    const zd *col = M + (int64_t)warp * ld;
    zd acc = zmake(0.0, 0.0);
    for (int i = lane; i < rows; i += 32) zfma_conj(acc, v[i], col[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) w[warp] = acc;
}

// M[i, c] -= tau v[i] w[c]
__global__ void k_rank1_left(int rows, int cols, zd *M, int ld, const zd *v, const zd *w,
                             const double *tau)
{
    const double t = *tau;
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % rows), c = (int)(e / rows);
        zd a = M[i + (int64_t)c * ld];
        zfma(a, zscale(v[i], -t), w[c]);
        M[i + (int64_t)c * ld] = a;
    }
}

// u[r] = sum_c M[r, c0 + c] v[c]  for the rows of two matrices stacked
// (C and Q, each m rows).  A CTA takes TV_R rows; its TV_G thread groups
// split the columns (reads stay coalesced down each column) and the partial
// sums meet in shared memory.
constexpr int TV_R = 16, TV_G = 16;
__global__ void __launch_bounds__(TV_R * TV_G) k_times_v2(int m, int cols, const zd *C, const zd *Q, int ld,
                                                          const zd *v, zd *u)
{
    __shared__ zd part[TV_G][TV_R];
    const int tr = threadIdx.x % TV_R, tg = threadIdx.x / TV_R;
    const int r = blockIdx.x * TV_R + tr;
    zd acc = zmake(0.0, 0.0);
    if (r < 2 * m) {
        const zd *M = (r < m) ? C : Q;
        const int rr = (r < m) ? r : r - m;
        for (int c = tg; c < cols; c += TV_G) zfma(acc, M[rr + (int64_t)c * ld], v[c]);
    }
    part[tg][tr] = acc;
    __syncthreads();
    if (tg == 0 && r < 2 * m) {
        zd s = part[0][tr];
        for (int g = 1; g < TV_G; ++g) s = zadd(s, part[g][tr]);
        u[r] = s;
    }
}

// M[r, c] -= tau u[r] conj(v[c]) for both stacked matrices
__global__ void k_rank1_right2(int m, int cols, zd *C, zd *Q, int ld, const zd *u, const zd *v,
                               const double *tau)
{
    const double t = *tau;
    const int64_t total = (int64_t)2 * m * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % (2 * m)), c = (int)(e / (2 * m));
        zd *M = (r < m) ? C : Q;
        int rr = (r < m) ? r : r - m;
        zd a = M[rr + (int64_t)c * ld];
        zfma(a, zscale(u[r], -t), zconj(v[c]));
        M[rr + (int64_t)c * ld] = a;
    }
}

// The whole Hessenberg reduction C <- Q^H C Q (Q <- Q P_0 P_1 ..., P_j =
// I - tau v v^H from column j) in one cooperative launch, two grid barriers
// per column instead of five launches: every CTA forms the same reflector
// from column j (the same reduction in the same order, so the CTAs agree
// bit for bit) and keeps v in shared memory; the CTAs' warps own columns of
// the trailing block for the left update w = v^H C, C -= tau v w (read,
// then rewrite, the same column); after a barrier the CTAs own 16-row
// slabs of [C; Q] for the right update u = M v, M -= tau u v^H; column j
// becomes (beta, 0, ..., 0).  The same arithmetic as the five-kernel form.
constexpr int HG_T = 256;        // threads per CTA
constexpr int HG_R = 16;         // rows per slab of the right update
constexpr int HG_U = 8;          // loads in flight per thread
template <typename T>
__device__ __forceinline__ T hg_scale(T a, typename CxReal<T>::type s)
{
    return cx<T>(a.x * s, a.y * s);
}
// T = double2 (the double-single QR's input), or float2 in the FP32 build
// (its Schur form is polished in FP64 afterwards, and GB300's FP32 pipe is
// 64x its FP64 one)
template <typename T>
__global__ void __launch_bounds__(HG_T) k_hess_grid(int m, T *C, T *Q, int ld, GridSync g)
{
    typedef typename CxReal<T>::type R;
    extern __shared__ __align__(16) unsigned char hv_raw[];
    T *hv = reinterpret_cast<T *>(hv_raw);       // v (m - 1 entries at most)
    __shared__ R red[HG_T / 32];
    __shared__ T part[HG_T / HG_R][HG_R];
    __shared__ T uslab[HG_R];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * (HG_T / 32) + wid, nwarps = gridDim.x * (HG_T / 32);
    const T zero = cx<T>(0, 0);
    for (int j = 0; j + 2 < m; ++j) {
        const int len = m - j - 1;
        const T *x = C + (j + 1) + (int64_t)j * ld;
        // reflector (every CTA, same order)
        R pn = 0;
        for (int i = threadIdx.x; i < len; i += HG_T) pn += cabs2(__ldcg(x + i));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) pn += __shfl_xor_sync(0xffffffffu, pn, off);
        if (lane == 0) red[wid] = pn;
        __syncthreads();
        R ss = 0;
        for (int w = 0; w < HG_T / 32; ++w) ss += red[w];
        const R nrm = sqrt(ss);
        const T x0 = __ldcg(x);
        const R a0 = sqrt(cabs2(x0));
        const T ph = a0 > 0 ? hg_scale(x0, (R)1 / a0) : cx<T>(1, 0);
        const T beta = hg_scale(ph, -nrm);
        const R vv = (R)2 * nrm * (nrm + a0);
        const R tau = vv > 0 ? (R)2 / vv : (R)0;
        for (int i = threadIdx.x; i < len; i += HG_T) hv[i] = (i == 0) ? cadd(x0, cneg(beta)) : __ldcg(x + i);
        __syncthreads();
        // left update of the trailing block, one warp per column (HG_U
        // loads in flight per lane: the steps are latency-bound otherwise)
        for (int c = gwarp; c < len; c += nwarps) {
            T *col = C + (j + 1) + (int64_t)(j + 1 + c) * ld;
            T acc = zero;
            for (int i0 = lane; i0 < len; i0 += 32 * HG_U) {
                T a[HG_U];
#pragma unroll
                for (int u = 0; u < HG_U; ++u) {
                    const int i = i0 + 32 * u;
                    a[u] = (i < len) ? __ldcg(col + i) : zero;
                }
#pragma unroll
                for (int u = 0; u < HG_U; ++u) {
                    const int i = i0 + 32 * u;
                    if (i < len) cfma(acc, cconj(hv[i]), a[u]);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            const T f = hg_scale(acc, -tau);
            for (int i0 = lane; i0 < len; i0 += 32 * HG_U) {
                T a[HG_U];
#pragma unroll
                for (int u = 0; u < HG_U; ++u) {
                    const int i = i0 + 32 * u;
                    a[u] = (i < len) ? __ldcg(col + i) : zero;
                }
#pragma unroll
                for (int u = 0; u < HG_U; ++u) {
                    const int i = i0 + 32 * u;
                    if (i < len) {
                        cfma(a[u], hv[i], f);
                        __stcg(col + i, a[u]);
                    }
                }
            }
        }
        if (!grid_barrier(g)) return;
        // right update of the stacked [C; Q] over columns j+1 .., 16-row slabs
        const int tr = threadIdx.x % HG_R, tg = threadIdx.x / HG_R;
        for (int slab = blockIdx.x; slab * HG_R < 2 * m; slab += gridDim.x) {
            const int r = slab * HG_R + tr;
            T *M = (r < m) ? C : Q;
            const int rr = (r < m) ? r : r - m;
            constexpr int CG = HG_T / HG_R;          // column groups
            T acc = zero;
            if (r < 2 * m)
                for (int c0 = tg; c0 < len; c0 += CG * HG_U) {
                    T a[HG_U];
#pragma unroll
                    for (int u = 0; u < HG_U; ++u) {
                        const int c = c0 + CG * u;
                        a[u] = (c < len) ? __ldcg(M + rr + (int64_t)(j + 1 + c) * ld) : zero;
                    }
#pragma unroll
                    for (int u = 0; u < HG_U; ++u) {
                        const int c = c0 + CG * u;
                        if (c < len) cfma(acc, a[u], hv[c]);
                    }
                }
            part[tg][tr] = acc;
            __syncthreads();
            if (tg == 0) {
                T sum = part[0][tr];
                for (int q = 1; q < HG_T / HG_R; ++q) sum = cadd(sum, part[q][tr]);
                uslab[tr] = hg_scale(sum, -tau);
            }
            __syncthreads();
            if (r < 2 * m) {
                const T f = uslab[tr];
                for (int c0 = tg; c0 < len; c0 += CG * HG_U) {
                    T a[HG_U];
#pragma unroll
                    for (int u = 0; u < HG_U; ++u) {
                        const int c = c0 + CG * u;
                        a[u] = (c < len) ? __ldcg(M + rr + (int64_t)(j + 1 + c) * ld) : zero;
                    }
#pragma unroll
                    for (int u = 0; u < HG_U; ++u) {
                        const int c = c0 + CG * u;
                        if (c < len) {
                            cfma(a[u], f, cconj(hv[c]));
                            __stcg(M + rr + (int64_t)(j + 1 + c) * ld, a[u]);
                        }
                    }
                }
            }
            __syncthreads();
        }
        // column j: (beta, 0, ..., 0) -- every CTA has read it
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i < len; i += HG_T)
                __stcg(C + (j + 1 + i) + (int64_t)j * ld, (i == 0) ? beta : zero);
        if (!grid_barrier(g)) return;
    }
}

// complex128 <-> complex64 copies of an m x m matrix, and the identity
__global__ void k_z2c(int64_t count, const zd *__restrict__ x, cf *__restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = make_float2((float)x[e].x, (float)x[e].y);
}
__global__ void k_c2z(int64_t count, const cf *__restrict__ x, zd *__restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = zmake((double)x[e].x, (double)x[e].y);
}
__global__ void k_eye_c(int m, cf *Q)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        Q[e] = make_float2((e % m) == (e / m) ? 1.f : 0.f, 0.f);
}

__global__ void k_eye(int m, zd *Q, int ld)
{
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % m), c = (int)(e / m);
        Q[r + (int64_t)c * ld] = zmake(r == c ? 1.0 : 0.0, 0.0);
    }
}

// ------------------------------------------------------------- QR sweeps
// ---------------------------------------------------------- double-single
// The QR sweeps run in double-single arithmetic (a value is an unevaluated
// sum h + l of two floats, ~46 significant bits) on the FP32 pipe: on
// GB300 a warp-wide FP64 instruction issues about 64x slower than an FP32
// one, and the chase is a chain of dependent rotations.  Error-free
// transformations use explicit round-to-nearest intrinsics so that the
// compiler cannot contract them into FMAs.
struct ds {
    float h, l;
};
struct cds {
    ds re, im;
};

#if FEAST_QR_FP32
// Plain FP32 build (k_zeig32.cu): the same algorithm with every value a
// single float (the low word stays zero), for projected problems whose
// Schur form is polished afterwards in FP64 (the Newton step of k_warm.cu).
__device__ __forceinline__ ds ds_make(float h, float l) { ds r; r.h = h + l; r.l = 0.f; return r; }
__device__ __forceinline__ ds ds_qts(float a, float b) { return ds_make(a + b, 0.f); }
__device__ __forceinline__ ds ds_add(ds x, ds y) { return ds_make(x.h + y.h, 0.f); }
__device__ __forceinline__ ds ds_neg(ds x) { return ds_make(-x.h, 0.f); }
__device__ __forceinline__ ds ds_sub(ds x, ds y) { return ds_make(x.h - y.h, 0.f); }
__device__ __forceinline__ ds ds_mul(ds x, ds y) { return ds_make(x.h * y.h, 0.f); }
__device__ __forceinline__ ds ds_from(double d) { return ds_make((float)d, 0.f); }
__device__ __forceinline__ ds ds_rsqrt(ds x) { return ds_make(rsqrtf(x.h), 0.f); }
#else
__device__ __forceinline__ ds ds_make(float h, float l) { ds r; r.h = h; r.l = l; return r; }
__device__ __forceinline__ ds ds_qts(float a, float b)   // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    return ds_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ds ds_add(ds x, ds y)
{
    float s = __fadd_rn(x.h, y.h);
    float bb = __fsub_rn(s, x.h);
    float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bb)), __fsub_rn(y.h, bb));
    e = __fadd_rn(e, __fadd_rn(x.l, y.l));
    return ds_qts(s, e);
}
__device__ __forceinline__ ds ds_neg(ds x) { return ds_make(-x.h, -x.l); }
__device__ __forceinline__ ds ds_sub(ds x, ds y) { return ds_add(x, ds_neg(y)); }
__device__ __forceinline__ ds ds_mul(ds x, ds y)
{
    float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return ds_qts(p, e);
}
__device__ __forceinline__ ds ds_from(double d)
{
    float h = (float)d;
    return ds_make(h, (float)(d - (double)h));
}
// 1/sqrt(x), x > 0: float seed and one Newton step in double-single
__device__ __forceinline__ ds ds_rsqrt(ds x)
{
    float y0 = rsqrtf(x.h);
    ds y = ds_make(y0, 0.f);
    ds t = ds_mul(x, ds_mul(y, y));                 // x y0^2 ~ 1
    ds e = ds_sub(ds_make(1.f, 0.f), t);            // 1 - x y0^2
    ds corr = ds_mul(ds_mul(y, e), ds_make(0.5f, 0.f));
    return ds_add(y, corr);
}
#endif
__device__ __forceinline__ cds cds_add(cds a, cds b) { cds r; r.re = ds_add(a.re, b.re); r.im = ds_add(a.im, b.im); return r; }
__device__ __forceinline__ cds cds_sub(cds a, cds b) { cds r; r.re = ds_sub(a.re, b.re); r.im = ds_sub(a.im, b.im); return r; }
__device__ __forceinline__ cds cds_mul(cds a, cds b)
{
    cds r;
    r.re = ds_sub(ds_mul(a.re, b.re), ds_mul(a.im, b.im));
    r.im = ds_add(ds_mul(a.re, b.im), ds_mul(a.im, b.re));
    return r;
}
__device__ __forceinline__ cds cds_conj(cds a) { cds r; r.re = a.re; r.im = ds_neg(a.im); return r; }
__device__ __forceinline__ cds cds_scale(cds a, ds s) { cds r; r.re = ds_mul(a.re, s); r.im = ds_mul(a.im, s); return r; }
__device__ __forceinline__ ds cds_abs2(cds a) { return ds_add(ds_mul(a.re, a.re), ds_mul(a.im, a.im)); }
__device__ __forceinline__ float cds_absf(cds a) { return hypotf(a.re.h, a.im.h); }
__device__ __forceinline__ cds cds_zero() { cds r; r.re = ds_make(0.f, 0.f); r.im = r.re; return r; }

// storage: float4 (re.h, re.l, im.h, im.l)
__device__ __forceinline__ cds ld_cds(const float4 *p)
{
    float4 v = __ldcg(p);
    cds r;
    r.re = ds_make(v.x, v.y);
    r.im = ds_make(v.z, v.w);
    return r;
}
__device__ __forceinline__ void st_cds(float4 *p, cds v) { __stcg(p, make_float4(v.re.h, v.re.l, v.im.h, v.im.l)); }

struct RotDS {
    ds c;   // real
    cds s;
};
// G = [c s; -conj(s) c] with G [x; y] = [r; 0]
__device__ __forceinline__ cds cds_ldexp(cds a, float f)
{
    // exact scaling by a power of two f
    cds r;
    r.re = ds_make(a.re.h * f, a.re.l * f);
    r.im = ds_make(a.im.h * f, a.im.l * f);
    return r;
}
__device__ __forceinline__ RotDS make_rot_ds(cds x, cds y)
{
    RotDS g;
    // the rotation depends only on the direction of (x, y): bring the
    // larger entry near 1 first, so that |x|^2 and |y|^2 neither underflow
    // nor overflow the float exponent range (a bulge running into an
    // almost deflated stretch carries entries far below 1e-19)
    const float mx = fmaxf(fmaxf(fabsf(x.re.h), fabsf(x.im.h)), fmaxf(fabsf(y.re.h), fabsf(y.im.h)));
    if (mx == 0.f) { g.c = ds_make(1.f, 0.f); g.s = cds_zero(); return g; }
    int ex;
    frexpf(mx, &ex);
    const float f = ldexpf(1.f, -ex);
    x = cds_ldexp(x, f);
    y = cds_ldexp(y, f);
    ds ax2 = cds_abs2(x), ay2 = cds_abs2(y);
    if (ay2.h == 0.f) { g.c = ds_make(1.f, 0.f); g.s = cds_zero(); return g; }
    if (ax2.h == 0.f) { g.c = ds_make(0.f, 0.f); g.s = cds_zero(); g.s.re = ds_make(1.f, 0.f); return g; }
    ds ia = ds_rsqrt(ax2), ir = ds_rsqrt(ds_add(ax2, ay2));
    ds k = ds_mul(ia, ir);
    g.c = ds_mul(ax2, k);                            // |x| / r
    g.s = cds_scale(cds_mul(x, cds_conj(y)), k);     // (x/|x|) conj(y) / r
    return g;
}
__device__ __forceinline__ void rot_left_ds(const RotDS &g, cds &a, cds &b)
{
    cds na = cds_add(cds_scale(a, g.c), cds_mul(g.s, b));
    cds nb = cds_sub(cds_scale(b, g.c), cds_mul(cds_conj(g.s), a));
    a = na;
    b = nb;
}
__device__ __forceinline__ void rot_right_ds(const RotDS &g, cds &a, cds &b)
{
    cds na = cds_add(cds_scale(a, g.c), cds_mul(b, cds_conj(g.s)));
    cds nb = cds_sub(cds_scale(b, g.c), cds_mul(a, g.s));
    a = na;
    b = nb;
}

__global__ void k_to_ds(int64_t count, const zd *x, float4 *y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        zd v = x[e];
        ds r = ds_from(v.x), i = ds_from(v.y);
        y[e] = make_float4(r.h, r.l, i.h, i.l);
    }
}
__global__ void k_from_ds(int64_t count, const float4 *x, zd *y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        float4 v = x[e];
        y[e] = zmake((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}

__device__ __forceinline__ cds csqrt_ds_approx(cds z)
{
    // shift selection only needs a float-accurate square root
    float zr = z.re.h, zi = z.im.h;
    float r = hypotf(zr, zi);
    cds o = cds_zero();
    if (r == 0.f) return o;
    if (zr >= 0.f) {
        float t = sqrtf(0.5f * (r + zr));
        o.re = ds_make(t, 0.f);
        o.im = ds_make(zi / (2.f * t), 0.f);
    } else {
        float t = sqrtf(0.5f * (r - zr));
        o.re = ds_make(fabsf(zi) / (2.f * t), 0.f);
        o.im = ds_make(copysignf(t, zi), 0.f);
    }
    return o;
}

// ------------------------------------------------------------ QR sweeps
// Bulge bookkeeping for the multishift sweep: bulge b enters the active
// window [l, ihi] DSEP phases after bulge b-1 and moves CH rows per phase,
// so the diagonal blocks of concurrent bulges (CH + 3 wide, DSEP * CH
// apart) never overlap.
struct Bulge {
    int k0, nrot, b0, b1;
};
__device__ __forceinline__ Bulge bulge_at(int t, int b, int l, int ihi, int m)
{
    Bulge g{0, 0, 0, 0};
    const int c = t - DSEP * b;
    if (c < 0) return g;
    const int k0 = l + c * CH;
    if (k0 >= ihi) return g;
    const int k1 = (k0 + CH < ihi) ? k0 + CH : ihi;
    g.k0 = k0;
    g.nrot = k1 - k0;
    g.b0 = (k0 - 1 > 0) ? k0 - 1 : 0;
    g.b1 = (k1 + 1 < m - 1) ? k1 + 1 : m - 1;
    return g;
}

// One chunk of a bulge chase (rotations k0 .. k0+nrot-1) on the diagonal
// block [b0, b1] held in shared memory: a dependent chain of rotations, each
// formed by every thread from the same shared values and applied by the
// whole CTA.  A bulge enters at k == l with the first column of H - sigma I.
// The rotations go to rots_g (global) for the far-part pass.
__device__ __forceinline__ void chase_chunk(int m, float4 *H, int ld, int l, int ihi, const Bulge &bg, cds sigma,
                            cds (*blk)[BLK + 1], RotDS *lrot, RotDS *rots_g)
{
    const int b0 = bg.b0, nb = bg.b1 - bg.b0 + 1, k0 = bg.k0, k1 = bg.k0 + bg.nrot;
    for (int e = threadIdx.x; e < nb * nb; e += QT) {
        int r = e % nb, c = e / nb;
        blk[r][c] = ld_cds(H + (b0 + r) + (int64_t)(b0 + c) * ld);
    }
    __syncthreads();
    // every thread forms the rotation (same shared values); the row pair and
    // the column pair it acts on take one element pair per thread
    const int t = threadIdx.x;
    for (int k = k0; k < k1; ++k) {
        const int kr = k - b0;
        cds x, y;
        if (k == l) {
            x = cds_sub(blk[kr][kr], sigma);
            y = blk[kr + 1][kr];
        } else {
            x = blk[kr][kr - 1];
            y = blk[kr + 1][kr - 1];
        }
        const RotDS gr = make_rot_ds(x, y);
        __syncthreads();
        const int cs = (k == l) ? kr : kr - 1;
        if (cs + t < nb) {
            rot_left_ds(gr, blk[kr][cs + t], blk[kr + 1][cs + t]);
            if (t == 0 && k > l) blk[kr + 1][kr - 1] = cds_zero();   // the bulge, annihilated exactly
        }
        __syncthreads();
        const int rl = ((k + 2 < ihi) ? k + 2 : ihi) - b0;
        if (t <= rl && t < nb) rot_right_ds(gr, blk[t][kr], blk[t][kr + 1]);
        if (t == 0) lrot[k - k0] = gr;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += QT) {
        int r = e % nb, c = e / nb;
        st_cds(H + (b0 + r) + (int64_t)(b0 + c) * ld, blk[r][c]);
    }
    for (int e = threadIdx.x; e < bg.nrot * (int)(sizeof(RotDS) / sizeof(float)); e += QT)
        __stcg(((float *)rots_g) + e, ((const float *)lrot)[e]);
}

// Left rotations of one chunk on the column segment col[0 .. nrot]: rotation
// i mixes entries i and i+1, so entry i is final once rotation i is done and
// only one entry is carried forward; loads go out FG entries at a time.
constexpr int FG = 8;
__device__ __forceinline__ void far_left(float4 *col, int nrot, const RotDS *rot)
{
    cds carry = ld_cds(col);
    for (int g0 = 0; g0 < nrot; g0 += FG) {
        cds buf[FG];
#pragma unroll
        for (int j = 0; j < FG; ++j)
            if (g0 + j < nrot) buf[j] = ld_cds(col + g0 + j + 1);
#pragma unroll
        for (int j = 0; j < FG; ++j) {
            if (g0 + j < nrot) {
                rot_left_ds(rot[g0 + j], carry, buf[j]);
                st_cds(col + g0 + j, carry);
                carry = buf[j];
            }
        }
    }
    st_cds(col + nrot, carry);
}
// Right rotations of one chunk on the row segment row[0], row[ld], ...
__device__ __forceinline__ void far_right(float4 *row, int ld, int nrot, const RotDS *rot)
{
    cds carry = ld_cds(row);
    for (int g0 = 0; g0 < nrot; g0 += FG) {
        cds buf[FG];
#pragma unroll
        for (int j = 0; j < FG; ++j)
            if (g0 + j < nrot) buf[j] = ld_cds(row + (int64_t)(g0 + j + 1) * ld);
#pragma unroll
        for (int j = 0; j < FG; ++j) {
            if (g0 + j < nrot) {
                rot_right_ds(rot[g0 + j], carry, buf[j]);
                st_cds(row + (int64_t)(g0 + j) * ld, carry);
                carry = buf[j];
            }
        }
    }
    st_cds(row + (int64_t)nrot * ld, carry);
}

// ------------------------------------------------- aggressive early deflation
// A trailing window of the active block is brought to Schur form by one CTA
// in shared memory; eigenvalues whose "spike" entry (the window's coupling
// column times the first row of its Schur vectors) is negligible deflate
// at once, the others are moved to the top of the window and serve as the
// next sweep's shifts; the rest of the window goes back to Hessenberg form
// by Householder reflections and the whole window transform is applied to
// the rest of H and to Z by the grid.
// largest deflation window (the FP32 build's window is solved by one warp,
// and its rotation chain grows with the window: a smaller one there)
constexpr int NW = FEAST_QR_FP32 ? 32 : 48;
constexpr int NWP = NW + 1;

__device__ __forceinline__ ds ds_sqrt(ds x) { return (x.h > 0.f) ? ds_mul(x, ds_rsqrt(x)) : ds_make(0.f, 0.f); }
__device__ __forceinline__ cds cds_neg(cds a) { cds r; r.re = ds_neg(a.re); r.im = ds_neg(a.im); return r; }
__device__ __forceinline__ cds cds_shfl_xor(cds a, int m)
{
    cds r;
    r.re = ds_make(__shfl_xor_sync(0xffffffffu, a.re.h, m), __shfl_xor_sync(0xffffffffu, a.re.l, m));
    r.im = ds_make(__shfl_xor_sync(0xffffffffu, a.im.h, m), __shfl_xor_sync(0xffffffffu, a.im.l, m));
    return r;
}
__device__ __forceinline__ cds cds_shfl(cds a, int src)
{
    cds r;
    r.re = ds_make(__shfl_sync(0xffffffffu, a.re.h, src), __shfl_sync(0xffffffffu, a.re.l, src));
    r.im = ds_make(__shfl_sync(0xffffffffu, a.im.h, src), __shfl_sync(0xffffffffu, a.im.l, src));
    return r;
}

// Apply a rotation (as the bulge chase does) to the w x w window T and its
// Schur vectors V: rows (k, k+1) of T from column c0, columns (k, k+1) of T
// over rows 0 .. r1, columns (k, k+1) of V.  Whole CTA; ends synchronised.
__device__ __forceinline__ void win_rot(const RotDS &gr, int k, int c0, int r1, int w, cds (*T)[NWP],
                                        cds (*V)[NWP], bool zero_bulge = false)
{
    const int t = threadIdx.x;
    if (c0 + t < w) {
        rot_left_ds(gr, T[k][c0 + t], T[k + 1][c0 + t]);
        if (zero_bulge && t == 0) T[k + 1][c0] = cds_zero();   // the bulge, annihilated exactly
    }
    __syncthreads();
    if (t <= r1) rot_right_ds(gr, T[t][k], T[t][k + 1]);
    if (t >= 64 && t - 64 < w) rot_right_ds(gr, V[t - 64][k], V[t - 64][k + 1]);
    __syncthreads();
}

// Schur form of the w x w upper Hessenberg T (in place) with Schur vectors
// accumulated into V (which starts as I): single-shift QR with full window
// updates.  Whole CTA; false if the iteration budget runs out.
__device__ bool win_schur(int w, cds (*T)[NWP], cds (*V)[NWP], float tol_rel, float tol_abs)
{
    int hi = w - 1, it = 0, tot = 0;
    while (hi > 0) {
        int lo = hi;
        while (lo > 0) {
            const float sub = cds_absf(T[lo][lo - 1]);
            const float loc = cds_absf(T[lo - 1][lo - 1]) + cds_absf(T[lo][lo]);
            if (sub <= tol_rel * loc || sub <= tol_abs) break;
            --lo;
        }
        __syncthreads();
        if (lo > 0 && threadIdx.x == 0) T[lo][lo - 1] = cds_zero();
        if (lo == hi) { --hi; it = 0; __syncthreads(); continue; }
        if (++tot > 40 * w) return false;
        ++it;
        cds sigma;
        {
            const cds h00 = T[hi - 1][hi - 1], h01 = T[hi - 1][hi], h10 = T[hi][hi - 1], h11 = T[hi][hi];
            if (it % 11 == 10) {
                const float a = cds_absf(h10);
                sigma = h11;
                sigma.re = ds_add(sigma.re, ds_make(a, 0.f));
                sigma.im = ds_add(sigma.im, ds_make(0.5f * a, 0.f));
            } else {
                cds half = cds_scale(cds_add(h00, h11), ds_make(0.5f, 0.f));
                cds det = cds_sub(cds_mul(h00, h11), cds_mul(h01, h10));
                cds disc = csqrt_ds_approx(cds_sub(cds_mul(half, half), det));
                cds r1 = cds_add(half, disc), r2 = cds_sub(half, disc);
                sigma = (cds_absf(cds_sub(r1, h11)) < cds_absf(cds_sub(r2, h11))) ? r1 : r2;
            }
        }
        __syncthreads();
        for (int k = lo; k < hi; ++k) {
            cds x, y;
            if (k == lo) { x = cds_sub(T[k][k], sigma); y = T[k + 1][k]; }
            else { x = T[k][k - 1]; y = T[k + 1][k - 1]; }
            const RotDS gr = make_rot_ds(x, y);
            __syncthreads();
            win_rot(gr, k, (k == lo) ? k : k - 1, (k + 2 < hi) ? k + 2 : hi, w, T, V, k > lo);
        }
    }
    __syncthreads();
    return true;
}

#if FEAST_QR_FP32
// FP32 build: the same single-shift QR by one warp.  The window's rows and
// columns (at most NW) take one or two lanes each, and in FP32 a
// rotation is a few operations per lane -- less than the CTA barriers the
// whole-CTA form spends on each one; lanes order their shared-memory
// updates with __syncwarp.  The other warps of the CTA wait at the caller's
// barrier.
__device__ bool win_schur_warp(int w, cds (*T)[NWP], cds (*V)[NWP], float tol_rel, float tol_abs)
{
    const int lane = threadIdx.x & 31;
    int hi = w - 1, it = 0, tot = 0;
    while (hi > 0) {
        // lo: the largest p in [1, hi] with a negligible subdiagonal entry, else 0
        int lo = 0;
        for (int base = hi; base >= 1 && lo == 0; base -= 32) {
            const int p = base - lane;
            bool neg = false;
            if (p >= 1) {
                const float sub = cds_absf(T[p][p - 1]);
                const float loc = cds_absf(T[p - 1][p - 1]) + cds_absf(T[p][p]);
                neg = (sub <= tol_rel * loc || sub <= tol_abs);
            }
            const unsigned b = __ballot_sync(0xffffffffu, neg);
            if (b) lo = base - (__ffs(b) - 1);
        }
        __syncwarp();
        if (lo > 0 && lane == 0) T[lo][lo - 1] = cds_zero();
        __syncwarp();
        if (lo == hi) { --hi; it = 0; continue; }
        if (++tot > 40 * w) return false;
        ++it;
        cds sigma;
        {
            const cds h00 = T[hi - 1][hi - 1], h01 = T[hi - 1][hi], h10 = T[hi][hi - 1], h11 = T[hi][hi];
            if (it % 11 == 10) {
                const float a = cds_absf(h10);
                sigma = h11;
                sigma.re = ds_add(sigma.re, ds_make(a, 0.f));
                sigma.im = ds_add(sigma.im, ds_make(0.5f * a, 0.f));
            } else {
                cds half = cds_scale(cds_add(h00, h11), ds_make(0.5f, 0.f));
                cds det = cds_sub(cds_mul(h00, h11), cds_mul(h01, h10));
                cds disc = csqrt_ds_approx(cds_sub(cds_mul(half, half), det));
                cds r1 = cds_add(half, disc), r2 = cds_sub(half, disc);
                sigma = (cds_absf(cds_sub(r1, h11)) < cds_absf(cds_sub(r2, h11))) ? r1 : r2;
            }
        }
        __syncwarp();
        for (int k = lo; k < hi; ++k) {
            cds x, y;
            if (k == lo) { x = cds_sub(T[k][k], sigma); y = T[k + 1][k]; }
            else { x = T[k][k - 1]; y = T[k + 1][k - 1]; }
            const RotDS gr = make_rot_ds(x, y);
            __syncwarp();
            const int c0 = (k == lo) ? k : k - 1;
            for (int j = c0 + lane; j < w; j += 32) rot_left_ds(gr, T[k][j], T[k + 1][j]);
            if (k > lo && lane == 0) T[k + 1][k - 1] = cds_zero();   // (lane 0 rotated that column)
            __syncwarp();
            const int r1 = (k + 2 < hi) ? k + 2 : hi;
            for (int i = lane; i <= r1; i += 32) rot_right_ds(gr, T[i][k], T[i][k + 1]);
            for (int i = lane; i < w; i += 32) rot_right_ds(gr, V[i][k], V[i][k + 1]);
            __syncwarp();
        }
    }
    return true;
}
#endif

// Swap the adjacent diagonal entries p-1, p of the upper-triangular T (and
// update V): the rotation that maps the eigenvector of T[p][p], (c, b - a),
// onto e1.  Whole CTA.
__device__ __forceinline__ void win_swap(int p, int w, cds (*T)[NWP], cds (*V)[NWP])
{
    const cds a = T[p - 1][p - 1], b = T[p][p], c = T[p - 1][p];
    const RotDS gr = make_rot_ds(c, cds_sub(b, a));
    __syncthreads();
    win_rot(gr, p - 1, p - 1, p, w, T, V);
    if (threadIdx.x == 0) T[p][p - 1] = cds_zero();
    __syncthreads();
}

// Householder reflector I - tau v v^H mapping x (len entries, stride sx
// through shared memory) onto alpha e1; v written to vout, tau to *tau
// (0: identity).  One warp (lanes take entries i = lane, lane + 32).
__device__ void win_house(const cds *x, int sx, int len, cds *vout, ds *tau, cds *alpha_out)
{
    const int lane = threadIdx.x & 31;
    ds s = ds_make(0.f, 0.f);
    for (int i = lane; i < len; i += 32) s = ds_add(s, cds_abs2(x[i * sx]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        s = ds_add(s, ds_make(__shfl_xor_sync(0xffffffffu, s.h, off), __shfl_xor_sync(0xffffffffu, s.l, off)));
    const cds x0 = x[0];
    const ds a02 = cds_abs2(x0);
    const ds nrm = ds_sqrt(s), a0 = ds_sqrt(a02);
    const bool trivial = (s.h == 0.f) || (ds_sub(s, a02).h <= 0.f);   // nothing below the first entry
    for (int i = lane; i < len; i += 32) {
        cds v = x[i * sx];
        if (i == 0 && !trivial) {
            // v0 = x0 + (x0/|x0|) ||x||
            cds ph;
            if (a0.h > 0.f) ph = cds_scale(x0, ds_rsqrt(a02));
            else { ph = cds_zero(); ph.re = ds_make(1.f, 0.f); }
            v = cds_add(x0, cds_scale(ph, nrm));
        }
        vout[i] = v;
    }
    if (lane == 0) {
        if (trivial) {
            *tau = ds_make(0.f, 0.f);
            *alpha_out = x0;
        } else {
            cds ph;
            if (a0.h > 0.f) ph = cds_scale(x0, ds_rsqrt(a02));
            else { ph = cds_zero(); ph.re = ds_make(1.f, 0.f); }
            const ds d = ds_mul(nrm, ds_add(nrm, a0));                 // ||v||^2 / 2
            const ds r = ds_rsqrt(d);
            *tau = ds_mul(r, r);
            *alpha_out = cds_neg(cds_scale(ph, nrm));
        }
    }
}

// M <- H M over rows r0 .. r0+len-1, columns c0 .. c1-1, H = I - tau v v^H.
// Four threads per column.  Whole CTA; ends synchronised.
__device__ __forceinline__ void win_house_left(cds (*M)[NWP], int r0, int len, int c0, int c1, const cds *v, ds tau)
{
    const int col = c0 + (int)(threadIdx.x >> 2), part = threadIdx.x & 3;
    cds acc = cds_zero();
    if (col < c1)
        for (int i = part; i < len; i += 4) acc = cds_add(acc, cds_mul(cds_conj(v[i]), M[r0 + i][col]));
    acc = cds_add(acc, cds_shfl_xor(acc, 1));
    acc = cds_add(acc, cds_shfl_xor(acc, 2));
    __syncthreads();
    if (col < c1) {
        const cds f = cds_scale(acc, tau);
        for (int i = part; i < len; i += 4) M[r0 + i][col] = cds_sub(M[r0 + i][col], cds_mul(v[i], f));
    }
    __syncthreads();
}
// M <- M H over columns c0 .. c0+len-1, rows 0 .. rows-1.  Whole CTA.
__device__ __forceinline__ void win_house_right(cds (*M)[NWP], int rows, int c0, int len, const cds *v, ds tau)
{
    const int row = (int)(threadIdx.x >> 2), part = threadIdx.x & 3;
    cds acc = cds_zero();
    if (row < rows)
        for (int i = part; i < len; i += 4) acc = cds_add(acc, cds_mul(M[row][c0 + i], v[i]));
    acc = cds_add(acc, cds_shfl_xor(acc, 1));
    acc = cds_add(acc, cds_shfl_xor(acc, 2));
    __syncthreads();
    if (row < rows) {
        const cds f = cds_scale(acc, tau);
        for (int i = part; i < len; i += 4) M[row][c0 + i] = cds_sub(M[row][c0 + i], cds_mul(f, cds_conj(v[i])));
    }
    __syncthreads();
}

struct AedShared {
    cds T[NW][NWP];
    cds V[NW][NWP];
    cds hv[NW];          // Householder vector
    cds spk[NW];         // spike
    ds tau;
    cds alpha;
    int nd, ok;
};

// AED on the window [kw, kw + w - 1] (kw = ihi - w + 1) of the active block
// starting at l.  CTA 0 only.  Writes the window's new contents to H, the
// spike column, the total window transform to vg (w x w), shifts of the
// undeflated part (up to ns, the bottom-most) to shifts, and returns nd
// (deflated count) in sh->nd; nd = 0 leaves H untouched.
__device__ void aed_window(int m, float4 *H, int ld, int l, int kw, int w, int ns, float tol_rel, float tol_abs,
                           AedShared *sh, float4 *vg, float2 *shifts)
{
    const int t = threadIdx.x;
    for (int e = t; e < w * w; e += QT) {
        const int r = e % w, c = e / w;
        sh->T[r][c] = (r > c + 1) ? cds_zero() : ld_cds(H + (kw + r) + (int64_t)(kw + c) * ld);
        cds v = cds_zero();
        if (r == c) v.re = ds_make(1.f, 0.f);
        sh->V[r][c] = v;
    }
    if (t == 0) { sh->nd = 0; sh->ok = 1; }
    __syncthreads();
#if FEAST_QR_FP32
    if (t < 32) {
        const bool r = win_schur_warp(w, sh->T, sh->V, tol_rel, tol_abs);
        if (t == 0) sh->ok = r ? 1 : 0;
    }
    __syncthreads();
    const bool ok = sh->ok != 0;
#else
    const bool ok = win_schur(w, sh->T, sh->V, tol_rel, tol_abs);
#endif
    const cds s = (kw > l) ? ld_cds(H + kw + (int64_t)(kw - 1) * ld) : cds_zero();
    const float sabs = cds_absf(s);
    int nd = 0;
    if (ok) {
        // deflation test from the bottom; undeflatable eigenvalues move to the top
        int top = 0, cur = w - 1;
        while (cur >= top) {
            const float spike = sabs * cds_absf(sh->V[0][cur]);
            const float d = cds_absf(sh->T[cur][cur]);
            if (spike <= tol_rel * d || spike <= tol_abs) {
                ++nd;
                --cur;
                continue;
            }
            // moving it up only pays if some candidate above could still
            // deflate (a swap changes spike entries by rotations of
            // neighbours, so a candidate far above the threshold stays above)
            bool any = false;
            for (int j = top; j < cur && !any; ++j)
                any = sabs * cds_absf(sh->V[0][j]) <= 64.f * (tol_rel * cds_absf(sh->T[j][j]) + tol_abs);
            if (!any) break;
            for (int p = cur; p > top; --p) win_swap(p, w, sh->T, sh->V);
            ++top;
        }
    }
    const int u = w - nd;
    // shifts: the bottom-most undeflated eigenvalues (all of them if fewer)
    if (t < ns) {
        const int idx = (u > ns) ? u - ns + t : (u > 0 ? t % u : 0);
        const cds e = (u > 0) ? sh->T[idx][idx] : sh->T[w - 1][w - 1];
        shifts[t] = make_float2(e.re.h + e.re.l, e.im.h + e.im.l);
    }
    if (t == 0) sh->nd = (ok ? nd : 0);
    __syncthreads();
    if (!ok || nd == 0) return;
    // spike of the undeflated part; Hessenberg form back by Householder
    // reflections on the window rows/cols 0 .. u-1 (the spike is column -1)
    for (int j = t; j < u; j += QT) sh->spk[j] = cds_mul(s, cds_conj(sh->V[0][j]));
    __syncthreads();
    if (kw > l && u > 1) {
        // reflector for the spike
        if (t < 32) win_house(sh->spk, 1, u, sh->hv, &sh->tau, &sh->alpha);
        __syncthreads();
        win_house_left(sh->T, 0, u, 0, w, sh->hv, sh->tau);
        win_house_right(sh->T, u, 0, u, sh->hv, sh->tau);
        win_house_right(sh->V, w, 0, u, sh->hv, sh->tau);
        if (t == 0) {
            sh->spk[0] = sh->alpha;
        }
        for (int j = 1 + t; j < u; j += QT) sh->spk[j] = cds_zero();
        __syncthreads();
        // Hessenberg reduction of the leading u x u block
        for (int j = 0; j + 2 < u; ++j) {
            if (t < 32) win_house(&sh->T[j + 1][j], NWP, u - j - 1, sh->hv, &sh->tau, &sh->alpha);
            __syncthreads();
            win_house_left(sh->T, j + 1, u - j - 1, j, w, sh->hv, sh->tau);
            win_house_right(sh->T, u, j + 1, u - j - 1, sh->hv, sh->tau);
            win_house_right(sh->V, w, j + 1, u - j - 1, sh->hv, sh->tau);
            for (int i = j + 2 + t; i < u; i += QT) sh->T[i][j] = cds_zero();
            __syncthreads();
        }
    }
    // window and spike back to H; the window transform to vg
    for (int e = t; e < w * w; e += QT) {
        const int r = e % w, c = e / w;
        st_cds(H + (kw + r) + (int64_t)(kw + c) * ld, (r > c + 1) ? cds_zero() : sh->T[r][c]);
        st_cds(vg + r + (int64_t)c * w, sh->V[r][c]);
    }
    if (kw > l)
        for (int j = t; j < w; j += QT) st_cds(H + (kw + j) + (int64_t)(kw - 1) * ld, (j < u) ? sh->spk[j] : cds_zero());
}

// Apply the window transform W (w x w, in shared memory) to the rest of H
// and to Z: H[0:kw, win] <- H[0:kw, win] W, H[win, c] <- W^H H[win, c] for
// c > kw + w - 1, Z[:, win] <- Z[:, win] W.  One warp per line.
__device__ void aed_apply(int m, float4 *H, float4 *Z, int ld, int kw, int w, const cds (*W)[NWP])
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * QT + threadIdx.x) >> 5, nwarps = (gridDim.x * QT) >> 5;
    const int right = m - (kw + w);
    const int lines = kw + m + right;
    for (int x = gw; x < lines; x += nwarps) {
        float4 *base;
        int64_t stride;
        bool colline;
        if (x < kw) { base = H + x + (int64_t)kw * ld; stride = ld; colline = false; }
        else if (x < kw + m) { base = Z + (x - kw) + (int64_t)kw * ld; stride = ld; colline = false; }
        else { base = H + kw + (int64_t)(kw + w + (x - kw - m)) * ld; stride = 1; colline = true; }
        cds in0 = cds_zero(), in1 = cds_zero();
        if (lane < w) in0 = ld_cds(base + (int64_t)lane * stride);
        if (lane + 32 < w) in1 = ld_cds(base + (int64_t)(lane + 32) * stride);
        cds o0 = cds_zero(), o1 = cds_zero();
        for (int k = 0; k < w; ++k) {
            const cds xk = (k < 32) ? cds_shfl(in0, k) : cds_shfl(in1, k - 32);
            if (colline) {
                // (W^H x)_j = sum_k conj(W[k][j]) x_k
                if (lane < w) o0 = cds_add(o0, cds_mul(cds_conj(W[k][lane]), xk));
                if (lane + 32 < w) o1 = cds_add(o1, cds_mul(cds_conj(W[k][lane + 32]), xk));
            } else {
                // (x W)_j = sum_k x_k W[k][j]
                if (lane < w) o0 = cds_add(o0, cds_mul(xk, W[k][lane]));
                if (lane + 32 < w) o1 = cds_add(o1, cds_mul(xk, W[k][lane + 32]));
            }
        }
        if (lane < w) st_cds(base + (int64_t)lane * stride, o0);
        if (lane + 32 < w) st_cds(base + (int64_t)(lane + 32) * stride, o1);
    }
}

// Largest p in [1, ihi] whose subdiagonal entry H[p][p-1] is negligible
// (|h| <= tol_rel (|H[p-1][p-1]| + |H[p][p]|) or |h| <= tol_abs), else 0.
// The CTA tests QT candidates at a time from the bottom (the first hit of a
// scan from ihi downwards).  Whole CTA, ihi uniform; every CTA finds the
// same p from the same H.
__device__ int scan_deflation(const float4 *H, int ld, int ihi, float tol_rel, float tol_abs)
{
    __shared__ int s_l;
    for (int top = ihi; top >= 1; top -= QT) {
        __syncthreads();
        if (threadIdx.x == 0) s_l = 0;
        __syncthreads();
        const int p = top - (int)threadIdx.x;
        if (p >= 1) {
            const float sub = cds_absf(ld_cds(H + p + (int64_t)(p - 1) * ld));
            const float loc = cds_absf(ld_cds(H + (p - 1) + (int64_t)(p - 1) * ld)) +
                              cds_absf(ld_cds(H + p + (int64_t)p * ld));
            if (sub <= tol_rel * loc || sub <= tol_abs) atomicMax(&s_l, p);
        }
        __syncthreads();
        const int v = s_l;
        if (v > 0) return v;
    }
    return 0;
}

// Whole QR phase in double-single: all CTAs run the same control flow (every
// decision is a function of values read after a grid barrier).  Active
// blocks of at least MS_MIN rows take aggressive early deflation on their
// bottom NW rows (CTA 0), whose undeflated eigenvalues then serve as the ns
// shifts of a multishift sweep: ns bulges through the block, each chased by
// its own CTA on its own diagonal block, and after each phase the whole
// grid applies the chunks' far parts -- first every bulge's left rotations
// (row segments right of its block), then every bulge's right rotations
// (column segments above its block, and Z), so no two writers meet.  Blocks
// of at most NW rows are brought to Schur form at once by the window
// routine; those in between take single-shift sweeps (Wilkinson shift,
// exceptional shift every 11th sweep).  H, Z: m x m double-single (float4),
// leading dim ld; rots: NSH * CH rotations; shifts: NSH entries; vwin: the
// NW x NW window transform; ctl: the window's deflation count.
__global__ void __launch_bounds__(QT, 1) k_hqr(int m, float4 *H, float4 *Z, int ld, RotDS *rots, float2 *shifts,
                                               float4 *vwin, int *ctl, GridSync g, int *fail, float tol_rel,
                                               float tol_abs, int *stats)
{
    extern __shared__ __align__(16) unsigned char hqr_dyn[];
    AedShared *sh = (AedShared *)hqr_dyn;
    __shared__ cds blk[BLK][BLK + 1];
    __shared__ RotDS srot[NSH][CH];
    const int gtid = blockIdx.x * QT + threadIdx.x, gthreads = gridDim.x * QT;
    int ihi = m - 1, iter = 0, total = 0;
    while (ihi > 0) {
        const int l = scan_deflation(H, ld, ihi, tol_rel, tol_abs);
        if (l == ihi) { --ihi; iter = 0; continue; }
        const int L = ihi - l + 1;
        int ns = 1;
        if (L >= MS_MIN) {
            ns = L / (DSEP * CH);
            if (ns > NSH) ns = NSH;
            if (ns > (int)gridDim.x) ns = gridDim.x;
        }
        // budget: 30 shifts per eigenvalue
        total += ns;
        if (total > 30 * m) { if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(fail, 1); return; }
        ++iter;
        if (L <= NW) {
            // the whole active block fits a window: its Schur form at once
            if (blockIdx.x == 0) {
                aed_window(m, H, ld, l, l, L, 1, tol_rel, tol_abs, sh, vwin, shifts);
                if (threadIdx.x == 0) __stcg(ctl, sh->nd);
            }
            if (!grid_barrier(g)) return;
            if (__ldcg(ctl) > 0) {
                for (int e = threadIdx.x; e < L * L; e += QT) sh->T[e % L][e / L] = ld_cds(vwin + e);
                __syncthreads();
                aed_apply(m, H, Z, ld, l, L, sh->T);
                if (!grid_barrier(g)) return;
                if (stats && blockIdx.x == 0 && threadIdx.x == 0) stats[2] += 1;
                continue;
            }
            // (window iteration budget ran out: fall through to a single-shift sweep)
        }
        if (ns > 1) {
            // ------------------------------------------------ multishift sweep
            // aggressive early deflation on the bottom NW rows first; its
            // undeflated eigenvalues are the sweep's shifts
            const int kw = ihi - NW + 1;
            if (blockIdx.x == 0) {
                aed_window(m, H, ld, l, kw, NW, ns, tol_rel, tol_abs, sh, vwin, shifts);
                if (threadIdx.x == 0) __stcg(ctl, sh->nd);
                if (iter % 6 == 5) {
                    // exceptional shifts: perturbed trailing diagonal
                    __syncthreads();
                    const int nd = sh->nd;
                    for (int b = threadIdx.x; b < ns; b += QT) {
                        const int i = ihi - nd - b;
                        float4 d = __ldcg(H + i + (int64_t)i * ld), e = __ldcg(H + i + (int64_t)(i - 1) * ld);
                        const float s = hypotf(e.x, e.z);
                        shifts[b] = make_float2(d.x + 0.75f * s, d.z + 0.4f * s);
                    }
                }
            }
            // every CTA has finished its scan; window, shifts and ctl are out
            if (!grid_barrier(g)) return;
            const int nd = __ldcg(ctl);
            if (nd > 0) {
                for (int e = threadIdx.x; e < NW * NW; e += QT) sh->T[e % NW][e / NW] = ld_cds(vwin + e);
                __syncthreads();
                aed_apply(m, H, Z, ld, kw, NW, sh->T);
                if (!grid_barrier(g)) return;
                if (stats && blockIdx.x == 0 && threadIdx.x == 0) stats[2] += 1;
                iter = 0;
                // many deflations: look again before sweeping
                if (nd * 100 >= NW * 14) continue;
                ihi -= nd;
                if (ihi - l + 1 < MS_MIN) continue;
            }
            const int nphase = (ihi - l + CH - 1) / CH + DSEP * (ns - 1);
            if (stats && blockIdx.x == 0 && threadIdx.x == 0) {
                stats[0] += 1;
                stats[1] += nphase;
            }
            for (int t = 0; t < nphase; ++t) {
                if ((int)blockIdx.x < ns) {
                    const int b = blockIdx.x;
                    const Bulge bg = bulge_at(t, b, l, ihi, m);
                    if (bg.nrot > 0) {
                        const float2 sf = __ldcg(shifts + b);
                        cds sigma = cds_zero();
                        sigma.re = ds_make(sf.x, 0.f);
                        sigma.im = ds_make(sf.y, 0.f);
                        chase_chunk(m, H, ld, l, ihi, bg, sigma, blk, srot[0], rots + (size_t)b * CH);
                    }
                }
                if (!grid_barrier(g)) return;
                for (int e = threadIdx.x; e < ns * CH * (int)(sizeof(RotDS) / sizeof(float)); e += QT)
                    ((float *)srot)[e] = __ldcg(((const float *)rots) + e);
                __syncthreads();
                // left rotations: column segments right of each block
                {
                    int total_l = 0;
                    for (int b = 0; b < ns; ++b) {
                        const Bulge bg = bulge_at(t, b, l, ihi, m);
                        if (bg.nrot > 0) total_l += m - 1 - bg.b1;
                    }
                    for (int x = gtid; x < total_l; x += gthreads) {
                        int rem = x, b = 0;
                        Bulge bg;
                        for (;; ++b) {
                            bg = bulge_at(t, b, l, ihi, m);
                            const int cnt = (bg.nrot > 0) ? m - 1 - bg.b1 : 0;
                            if (rem < cnt) break;
                            rem -= cnt;
                        }
                        far_left(H + (int64_t)(bg.b1 + 1 + rem) * ld + bg.k0, bg.nrot, srot[b]);
                    }
                }
                if (!grid_barrier(g)) return;
                // right rotations: row segments above each block, and Z
                {
                    int total_r = 0;
                    for (int b = 0; b < ns; ++b) {
                        const Bulge bg = bulge_at(t, b, l, ihi, m);
                        if (bg.nrot > 0) total_r += bg.b0 + m;
                    }
                    for (int x = gtid; x < total_r; x += gthreads) {
                        int rem = x, b = 0;
                        Bulge bg;
                        for (;; ++b) {
                            bg = bulge_at(t, b, l, ihi, m);
                            const int cnt = (bg.nrot > 0) ? bg.b0 + m : 0;
                            if (rem < cnt) break;
                            rem -= cnt;
                        }
                        float4 *row = (rem < bg.b0) ? H + rem + (int64_t)bg.k0 * ld
                                                    : Z + (rem - bg.b0) + (int64_t)bg.k0 * ld;
                        far_right(row, ld, bg.nrot, srot[b]);
                    }
                }
                if (!grid_barrier(g)) return;
            }
            continue;
        }
        // ---------------------------------------------------- single-shift sweep
        cds sigma;
        {
            cds h00 = ld_cds(H + (ihi - 1) + (int64_t)(ihi - 1) * ld), h01 = ld_cds(H + (ihi - 1) + (int64_t)ihi * ld);
            cds h10 = ld_cds(H + ihi + (int64_t)(ihi - 1) * ld), h11 = ld_cds(H + ihi + (int64_t)ihi * ld);
            if (iter % 11 == 10) {
                float a = cds_absf(h10);
                sigma = h11;
                sigma.re = ds_add(sigma.re, ds_make(a, 0.f));
                sigma.im = ds_add(sigma.im, ds_make(0.5f * a, 0.f));
            } else {
                // Wilkinson shift: eigenvalue of the trailing 2 x 2 closest to h11
                cds tr = cds_add(h00, h11);
                cds half = cds_scale(tr, ds_make(0.5f, 0.f));
                cds det = cds_sub(cds_mul(h00, h11), cds_mul(h01, h10));
                cds disc = csqrt_ds_approx(cds_sub(cds_mul(half, half), det));
                cds r1 = cds_add(half, disc), r2 = cds_sub(half, disc);
                sigma = (cds_absf(cds_sub(r1, h11)) < cds_absf(cds_sub(r2, h11))) ? r1 : r2;
            }
        }
        if (stats && blockIdx.x == 0 && threadIdx.x == 0) {
            stats[0] += 1;
            stats[1] += (ihi - l + CH - 1) / CH;
        }
        // every CTA has read what it needs for l, ihi and sigma before CTA 0
        // starts rewriting the leading block of the sweep
        if (!grid_barrier(g)) return;
        for (int k0 = l; k0 < ihi; k0 += CH) {
            const int k1 = (k0 + CH < ihi) ? k0 + CH : ihi;   // rotations k0 .. k1-1
            Bulge bg;
            bg.k0 = k0;
            bg.nrot = k1 - k0;
            bg.b0 = (k0 - 1 > 0) ? k0 - 1 : 0;
            bg.b1 = (k1 + 1 < m - 1) ? k1 + 1 : m - 1;
            if (blockIdx.x == 0) chase_chunk(m, H, ld, l, ihi, bg, sigma, blk, srot[0], rots);
            if (!grid_barrier(g)) return;
            if (blockIdx.x != 0) {
                for (int e = threadIdx.x; e < bg.nrot * (int)(sizeof(RotDS) / sizeof(float)); e += QT)
                    ((float *)srot[0])[e] = __ldcg(((const float *)rots) + e);
            }
            __syncthreads();
            // one writer per element: the column segments right of the block
            // and the row segments above it do not meet
            const int ncol = m - 1 - bg.b1, nrowH = bg.b0;
            const int lines = ncol + nrowH + m;
            for (int x = gtid; x < lines; x += gthreads) {
                if (x < ncol) {
                    far_left(H + (int64_t)(bg.b1 + 1 + x) * ld + k0, bg.nrot, srot[0]);
                } else {
                    const int r = (x < ncol + nrowH) ? x - ncol : x - ncol - nrowH;
                    float4 *row = ((x < ncol + nrowH) ? H : Z) + r + (int64_t)k0 * ld;
                    far_right(row, ld, bg.nrot, srot[0]);
                }
            }
            if (!grid_barrier(g)) return;
        }
    }
}

// Eigenvector k of the upper-triangular Schur form S: (S - S_kk I) y = 0,
// y_k = 1, back-substitution; one warp per eigenvector.  St is S
// transposed (St[p + i ld] = S[i, p]), so that a warp's dot product over a
// row of S reads contiguous memory.  Y is m x m (upper triangular on output).
__global__ void k_schur_vectors(int m, const zd *St, int ld, zd *Y, double snorm)
{
    // eigenvector k costs ~k^2 / 2 complex MACs on the FP64 pipe: the warps
    // of a CTA take eigenvectors gridDim.x apart, so that every SM gets a
    // mix of short and long ones (consecutive k put the longest ones of all
    // on one SM)
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x + (int)gridDim.x * (threadIdx.x >> 5);
    if (k >= m) return;
    const double eps = 2.220446049250313e-16;
    const double small = eps * fmax(snorm, 1e-300);
    zd *y = Y + (int64_t)k * ld;
    const zd lam = St[k + (int64_t)k * ld];
    for (int i = k + 1 + lane; i < m; i += 32) y[i] = zmake(0.0, 0.0);
    if (lane == 0) y[k] = zmake(1.0, 0.0);
    __syncwarp();
    for (int i = k - 1; i >= 0; --i) {
        const zd *srow = St + (int64_t)i * ld;   // S[i, :]
        // four independent partial sums: four loads of each operand in
        // flight per lane (the step is bound by their latency)
        zd acc = zmake(0.0, 0.0), a1 = acc, a2 = acc, a3 = acc;
        int p = i + 1 + lane;
        for (; p + 96 <= k; p += 128) {
            zfma(acc, srow[p], y[p]);
            zfma(a1, srow[p + 32], y[p + 32]);
            zfma(a2, srow[p + 64], y[p + 64]);
            zfma(a3, srow[p + 96], y[p + 96]);
        }
        for (; p <= k; p += 32) zfma(acc, srow[p], y[p]);
        acc = zadd(zadd(acc, a1), zadd(a2, a3));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) {
            zd d = zsub(srow[i], lam);
            if (zabs(d) < small) d = zmake(small, 0.0);
            zd q = zdiv(acc, d);
            y[i] = zmake(-q.x, -q.y);
        }
        __syncwarp();
    }
}

__global__ void k_transpose(int m, const zd *__restrict__ A, int ld, zd *__restrict__ At)
{
    __shared__ zd tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int i = bx + tx, j = by + r;
        if (i < m && j < m) tile[r][tx] = A[i + (int64_t)j * ld];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = by + tx, j = bx + r;
        if (i < m && j < m) At[i + (int64_t)j * ld] = tile[tx][r];
    }
}

__global__ void k_normalise_cols(int m, zd *V, int ld)
{
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= m) return;
    zd *v = V + (int64_t)k * ld;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += zabs2(v[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    for (int i = lane; i < m; i += 32) v[i] = zscale(v[i], inv);
}

__global__ void k_diag_out(int m, const zd *S, int ld, zd *alpha, zd *beta)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    alpha[k] = S[k + (int64_t)k * ld];
    beta[k] = zmake(1.0, 0.0);
}

__global__ void k_absmax(int64_t count, const zd *x, double *out)
{
    __shared__ double red[32];
    double v = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        v = fmax(v, zabs(x[e]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = fmax(r, red[w]);
        // non-negative doubles order like their bit patterns
        atomicMax((unsigned long long *)out, (unsigned long long)__double_as_longlong(r));
    }
}

}  // namespace

#if FEAST_QR_FP32
namespace {   // the FP32 build's own copies of the one-CTA kernels
#endif
// ------------------------------------------------- small matrices: one CTA
// Schur form of an m x m upper Hessenberg matrix, m <= SQ_MAX, by one CTA
// with the whole matrix in shared memory: packed by columns (column j keeps
// rows 0 .. j+2, one row below the subdiagonal for the bulge), double-single
// entries.  Single-shift QR sweeps (Wilkinson shift, an exceptional shift
// every 11th sweep at one eigenvalue), the standard deflation test on the
// subdiagonal.  Each rotation G_k (rows k, k+1) is applied to the full rows
// and the columns above and logged; the Schur vectors are the Hessenberg
// reduction's Q times the logged rotations (k_apply_rotlog, one thread per
// row of Q), so the serial chain here touches shared memory only.
constexpr int SQ_MAX = 164;      // largest m: the packed matrix fills ~222 KB
constexpr int SQ_T = 256;        // threads of the one-CTA kernel
constexpr int SQ_LOG = 4;        // rotation log capacity: SQ_LOG * m^2 entries

struct RotLog {
    float ch, cl, srh, srl, sih, sil;  // c (real) and s (complex), double-single
    int k;
    int pad;
};

__host__ __device__ inline int sq_elems(int m)
{
    int e = 0;
    for (int j = 0; j < m; ++j) e += (j + 3 < m) ? j + 3 : m;
    return e;
}
inline size_t sq_smem_bytes(int m) { return sizeof(float4) * (size_t)sq_elems(m) + sizeof(int) * (size_t)(m + 1); }

__device__ __forceinline__ cds sq_ld(const float4 *S, const int *off, int i, int j)
{
    const float4 v = S[off[j] + i];
    cds r;
    r.re = ds_make(v.x, v.y);
    r.im = ds_make(v.z, v.w);
    return r;
}
__device__ __forceinline__ void sq_st(float4 *S, const int *off, int i, int j, cds v)
{
    S[off[j] + i] = make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
}

// status[0]: 0 done, 1 iteration budget spent, 2 rotation log full;
// status[1]: rotations logged; status[2]: sweeps.  T (= H in place) is
// written only when status[0] = 0.
__global__ void __launch_bounds__(SQ_T, 1) k_small_schur(int m, zd *__restrict__ H, RotLog *__restrict__ log,
                                                         int max_log, int *__restrict__ status, float tol_rel,
                                                         float tol_abs)
{
    extern __shared__ float4 S[];
    int *off = (int *)(S + sq_elems(m));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        int o = 0;
        for (int j = 0; j < m; ++j) {
            off[j] = o;
            o += (j + 3 < m) ? j + 3 : m;
        }
        off[m] = o;
    }
    __syncthreads();
    for (int j = warp; j < m; j += SQ_T / 32) {
        const int len = (j + 3 < m) ? j + 3 : m;
        for (int i = lane; i < len; i += 32) {
            cds v = cds_zero();
            if (i <= j + 1) {
                const zd h = H[i + (int64_t)j * m];
                v.re = ds_from(h.x);
                v.im = ds_from(h.y);
            }
            sq_st(S, off, i, j, v);
        }
    }
    __syncthreads();
    __shared__ RotDS g_sh;
    __shared__ int ctl[2];   // lo of the active block, sweep status (0 go, 1 deflated one, 2 stop)
    int hi = m - 1, it = 0, tot = 0, nr = 0, st = 0;
    while (hi > 0) {
        // warp 0: deflation scan, shift and every rotation of the sweep;
        // the CTA applies them
        if (warp == 0) {
            int lo = hi;
            while (lo > 0) {
                const float sub = cds_absf(sq_ld(S, off, lo, lo - 1));
                const float loc = cds_absf(sq_ld(S, off, lo - 1, lo - 1)) + cds_absf(sq_ld(S, off, lo, lo));
                if (sub <= tol_rel * loc || sub <= tol_abs) break;
                --lo;
            }
            if (lane == 0) {
                if (lo > 0) sq_st(S, off, lo, lo - 1, cds_zero());
                ctl[0] = lo;
                ctl[1] = (lo == hi) ? 1 : 0;
            }
        }
        __syncthreads();
        const int lo = ctl[0];
        const int defl = ctl[1];
        __syncthreads();  // everyone has read ctl before warp 0 writes it again
        if (defl == 1) {
            --hi;
            it = 0;
            continue;
        }
        if (++tot > 30 * m) {
            st = 1;
            break;
        }
        if (nr + (hi - lo) > max_log) {
            st = 2;
            break;
        }
        ++it;
        cds sigma = cds_zero();
        if (warp == 0) {
            const cds h00 = sq_ld(S, off, hi - 1, hi - 1), h01 = sq_ld(S, off, hi - 1, hi);
            const cds h10 = sq_ld(S, off, hi, hi - 1), h11 = sq_ld(S, off, hi, hi);
            if (it % 11 == 10) {
                const float a = cds_absf(h10);
                sigma = h11;
                sigma.re = ds_add(sigma.re, ds_make(a, 0.f));
                sigma.im = ds_add(sigma.im, ds_make(0.5f * a, 0.f));
            } else {
                // Wilkinson shift: eigenvalue of the trailing 2 x 2 closest to h11
                cds half = cds_scale(cds_add(h00, h11), ds_make(0.5f, 0.f));
                cds det = cds_sub(cds_mul(h00, h11), cds_mul(h01, h10));
                cds disc = csqrt_ds_approx(cds_sub(cds_mul(half, half), det));
                cds r1 = cds_add(half, disc), r2 = cds_sub(half, disc);
                sigma = (cds_absf(cds_sub(r1, h11)) < cds_absf(cds_sub(r2, h11))) ? r1 : r2;
            }
        }
        for (int k = lo; k < hi; ++k) {
            if (warp == 0) {
                cds x, y;
                if (k == lo) {
                    x = cds_sub(sq_ld(S, off, k, k), sigma);
                    y = sq_ld(S, off, k + 1, k);
                } else {
                    x = sq_ld(S, off, k, k - 1);
                    y = sq_ld(S, off, k + 1, k - 1);
                }
                const RotDS gr = make_rot_ds(x, y);
                if (lane == 0) {
                    g_sh = gr;
                    RotLog L;
                    L.ch = gr.c.h;
                    L.cl = gr.c.l;
                    L.srh = gr.s.re.h;
                    L.srl = gr.s.re.l;
                    L.sih = gr.s.im.h;
                    L.sil = gr.s.im.l;
                    L.k = k;
                    L.pad = 0;
                    log[nr] = L;
                }
            }
            ++nr;
            __syncthreads();
            const RotDS gr = g_sh;
            // rows k, k+1 (columns from the bulge's column to the right edge)
            const int c0 = (k == lo) ? k : k - 1;
            for (int c = c0 + t; c < m; c += SQ_T) {
                cds a = sq_ld(S, off, k, c), b = sq_ld(S, off, k + 1, c);
                rot_left_ds(gr, a, b);
                sq_st(S, off, k, c, a);
                sq_st(S, off, k + 1, c, b);
            }
            __syncthreads();
            // columns k, k+1 (rows from the top to the new bulge)
            const int r1 = (k + 2 < hi) ? k + 2 : hi;
            for (int r = t; r <= r1; r += SQ_T) {
                cds a = sq_ld(S, off, r, k), b = sq_ld(S, off, r, k + 1);
                rot_right_ds(gr, a, b);
                sq_st(S, off, r, k, a);
                sq_st(S, off, r, k + 1, b);
            }
            // the annihilated bulge entry (k+1, k-1) is set to zero exactly
            if (k > lo && t == 0) sq_st(S, off, k + 1, k - 1, cds_zero());
            __syncthreads();
        }
    }
    if (t == 0) {
        status[0] = st;
        status[1] = nr;
        status[2] = tot;
    }
    if (st) return;
    for (int j = warp; j < m; j += SQ_T / 32)
        for (int i = lane; i < m; i += 32) {
            zd v = zmake(0.0, 0.0);
            if (i <= j) {
                const cds c = sq_ld(S, off, i, j);
                v = zmake((double)c.re.h + (double)c.re.l, (double)c.im.h + (double)c.im.l);
            }
            H[i + (int64_t)j * m] = v;
        }
}

__global__ void k_add_stats(int *stats, int sweeps) { stats[0] += sweeps; }

// Q <- Q G_1^H G_2^H ... (the logged rotations, in order): thread per row of
// Q, the row held in shared memory (double-single) and the log streamed
// through shared memory in chunks, the two entries a rotation touches
// carried in registers along a sweep.  AR rows per CTA.
constexpr int AR = 32, ALOG = 256;
__global__ void __launch_bounds__(AR) k_apply_rotlog(int m, zd *__restrict__ Q, const RotLog *__restrict__ log,
                                                    const int *__restrict__ status)
{
    extern __shared__ float4 zrow[];             // AR rows x m entries
    __shared__ RotLog chunk[ALOG];
    const int t = threadIdx.x;
    const int r = blockIdx.x * AR + t;
    const int nr = status[1];
    float4 *zr = zrow + (size_t)t * m;
    if (r < m)
        for (int c = 0; c < m; ++c) {
            const zd v = Q[r + (int64_t)c * m];
            const ds re = ds_from(v.x), im = ds_from(v.y);
            zr[c] = make_float4(re.h, re.l, im.h, im.l);
        }
    int cur = -2;
    cds a = cds_zero(), b = cds_zero();
    for (int e0 = 0; e0 < nr; e0 += ALOG) {
        const int cnt = (nr - e0) < ALOG ? (nr - e0) : ALOG;
        __syncthreads();
        for (int e = t; e < cnt; e += AR) chunk[e] = log[e0 + e];
        __syncthreads();
        if (r >= m) continue;
        for (int e = 0; e < cnt; ++e) {
            const RotLog L = chunk[e];
            const int k = L.k;
            if (k != cur) {
                if (k == cur + 1) {
                    zr[cur] = make_float4(a.re.h, a.re.l, a.im.h, a.im.l);
                    a = b;
                    const float4 v = zr[k + 1];
                    b.re = ds_make(v.x, v.y);
                    b.im = ds_make(v.z, v.w);
                } else {
                    if (cur >= 0) {
                        zr[cur] = make_float4(a.re.h, a.re.l, a.im.h, a.im.l);
                        zr[cur + 1] = make_float4(b.re.h, b.re.l, b.im.h, b.im.l);
                    }
                    const float4 v0 = zr[k], v1 = zr[k + 1];
                    a.re = ds_make(v0.x, v0.y);
                    a.im = ds_make(v0.z, v0.w);
                    b.re = ds_make(v1.x, v1.y);
                    b.im = ds_make(v1.z, v1.w);
                }
                cur = k;
            }
            RotDS g;
            g.c = ds_make(L.ch, L.cl);
            g.s.re = ds_make(L.srh, L.srl);
            g.s.im = ds_make(L.sih, L.sil);
            rot_right_ds(g, a, b);
        }
    }
    if (r >= m) return;
    if (cur >= 0) {
        zr[cur] = make_float4(a.re.h, a.re.l, a.im.h, a.im.l);
        zr[cur + 1] = make_float4(b.re.h, b.re.l, b.im.h, b.im.l);
    }
    for (int c = 0; c < m; ++c) {
        const float4 v = zr[c];
        Q[r + (int64_t)c * m] = zmake((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}

#if FEAST_QR_FP32
}  // namespace
#endif

#if FEAST_QR_FP32
#define schur_large_work_bytes schur_large_work_bytes_fp32
#define zeig_large_work_bytes zeig_large_work_bytes_fp32
#define schur_large schur_large_fp32
#endif
size_t schur_large_work_bytes(int m)
{
    // v (m) + w (m) + u (2m) complex, tau, absmax, rotations, barrier words,
    // then either the double-single copies of H and Q (m*m float4 each) or
    // the one-CTA kernel's rotation log (monotone in m, so that a block of a
    // larger problem fits the larger problem's work)
    const size_t mq = (size_t)(m < SQ_MAX ? m : SQ_MAX);
    const size_t big = 2 * sizeof(float4) * (size_t)m * m, small = sizeof(RotLog) * SQ_LOG * mq * mq + 16;
    return sizeof(zd) * (4 * (size_t)m) + 64 + sizeof(RotDS) * NSH * CH + sizeof(float2) * NSH +
           sizeof(float4) * NW * NW + 16 + 64 + 256 + (big > small ? big : small);
}

size_t zeig_large_work_bytes(int m)
{
    return sizeof(zd) * (size_t)m * m + schur_large_work_bytes(m);
}

int schur_large(cudaStream_t s, int m, zd *C, zd *Q, void *work, int *fail, int *timeout, int *stats, double *hn_out,
                double defl)
{
    if (m <= 0) return FEAST_OK;
    zd *v = (zd *)work;
    zd *wv = v + m;
    zd *u = wv + m;
    double *tau = (double *)(u + 2 * m);
    double *hmax = tau + 1;
    RotDS *rots = (RotDS *)(hmax + 7);
    float2 *shifts = (float2 *)(rots + NSH * CH);
    float4 *vwin = (float4 *)(shifts + NSH);
    int *ctl = (int *)(vwin + NW * NW);
    unsigned *bar = (unsigned *)(ctl + 4);
    float4 *Hds = (float4 *)(((uintptr_t)(bar + 16) + 255) & ~(uintptr_t)255);
    float4 *Qds = Hds + (size_t)m * m;
    k_eye<<<cdiv((size_t)m * m, 256) > 2048 ? 2048 : cdiv((size_t)m * m, 256), 256, 0, s>>>(m, Q, m);
    FEAST_LAUNCH_CHECK();
    // Hessenberg reduction C <- Q^H C Q: one cooperative launch (the
    // per-column kernels below when the grid form cannot be launched)
    unsigned *hbar = (unsigned *)(((uintptr_t)(wv + m) + 15) & ~(uintptr_t)15);   // (w is unused by it)
    int hgrid = 0;
    if (m >= 3) {
        // the FP32 build reduces in FP32 too when its multishift QR follows
        // (C and Q in complex64 in the double-single copies' space)
        const bool hf = FEAST_QR_FP32 && m > SQ_MAX;
        int dev = 0, sms = 0, per = 0;
        const size_t hsm = (hf ? sizeof(cf) : sizeof(zd)) * (size_t)m;
        FEAST_CUDA_TRY(cudaGetDevice(&dev));
        FEAST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (hf) {
            FEAST_CUDA_TRY(ensure_dyn_smem(k_hess_grid<cf>, hsm));
            FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hess_grid<cf>, HG_T, hsm));
        } else {
            FEAST_CUDA_TRY(ensure_dyn_smem(k_hess_grid<zd>, hsm));
            FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hess_grid<zd>, HG_T, hsm));
        }
        hgrid = (per >= 1) ? sms : 0;
        const int need = (2 * m + HG_R - 1) / HG_R;     // right-update slabs
        if (hgrid > need) hgrid = need;
        if (hgrid > 0) {
            FEAST_CUDA_TRY(cudaMemsetAsync(hbar, 0, 2 * sizeof(unsigned), s));
            GridSync hg{hbar, hbar + 1, timeout, TO_HESS};
            int mm = m, ldq = m;
            const unsigned gc = cdiv((size_t)m * m, 256) > 4096 ? 4096 : cdiv((size_t)m * m, 256);
            if (hf) {
                cf *Cf = (cf *)Hds, *Qf = (cf *)Qds;
                k_z2c<<<gc, 256, 0, s>>>((int64_t)m * m, C, Cf);
                FEAST_LAUNCH_CHECK();
                k_eye_c<<<gc, 256, 0, s>>>(m, Qf);
                FEAST_LAUNCH_CHECK();
                void *hargs[] = {&mm, &Cf, &Qf, &ldq, &hg};
                FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_hess_grid<cf>, dim3(hgrid), dim3(HG_T), hargs,
                                                           hsm, s));
                FEAST_LAUNCH_CHECK();
                k_c2z<<<gc, 256, 0, s>>>((int64_t)m * m, Cf, C);
                FEAST_LAUNCH_CHECK();
                k_c2z<<<gc, 256, 0, s>>>((int64_t)m * m, Qf, Q);
                FEAST_LAUNCH_CHECK();
            } else {
                void *hargs[] = {&mm, &C, &Q, &ldq, &hg};
                FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_hess_grid<zd>, dim3(hgrid), dim3(HG_T), hargs,
                                                           hsm, s));
                FEAST_LAUNCH_CHECK();
            }
        }
    }
    for (int j = 0; hgrid == 0 && j + 2 < m; ++j) {
        const int len = m - j - 1;
        k_house<<<1, 256, 0, s>>>(m, j, C, m, v, tau);
        FEAST_LAUNCH_CHECK();
        zd *blkC = C + (j + 1) + (int64_t)(j + 1) * m;
        k_vh_times<<<cdiv((size_t)len * 32, 256), 256, 0, s>>>(len, len, blkC, m, v, wv);
        FEAST_LAUNCH_CHECK();
        unsigned g1 = cdiv((size_t)len * len, 256);
        k_rank1_left<<<g1 > 4096 ? 4096 : g1, 256, 0, s>>>(len, len, blkC, m, v, wv, tau);
        FEAST_LAUNCH_CHECK();
        k_times_v2<<<cdiv((size_t)2 * m, TV_R), TV_R * TV_G, 0, s>>>(m, len, C + (int64_t)(j + 1) * m,
                                                                       Q + (int64_t)(j + 1) * m, m, v, u);
        FEAST_LAUNCH_CHECK();
        unsigned g2 = cdiv((size_t)2 * m * len, 256);
        k_rank1_right2<<<g2 > 4096 ? 4096 : g2, 256, 0, s>>>(m, len, C + (int64_t)(j + 1) * m,
                                                             Q + (int64_t)(j + 1) * m, m, u, v, tau);
        FEAST_LAUNCH_CHECK();
    }
    // norm for the deflation test
    FEAST_CUDA_TRY(cudaMemsetAsync(hmax, 0, sizeof(double), s));
    k_absmax<<<64, 256, 0, s>>>((int64_t)m * m, C, hmax);
    FEAST_LAUNCH_CHECK();
    double hn = 0.0;
    int htimeout = 0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&hn, hmax, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (hgrid > 0) FEAST_CUDA_TRY(cudaMemcpyAsync(&htimeout, timeout, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaMemsetAsync(bar, 0, 16, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    // the reduction's grid barrier gave up (or a wait before it did, and
    // the reduction stopped at its first barrier)
    if (htimeout) return note_timeout(htimeout);
    if (hn_out) *hn_out = hn;
    // deflation thresholds at double-single resolution (2^-44 relative),
    // or a few FP32 units in the FP32 build (or the caller's looser one)
    const double floor_rel = FEAST_QR_FP32 ? 1e-6 : 5.7e-14;
    const double tr = defl > floor_rel ? defl : floor_rel;
    float tol_rel = (float)tr, tol_abs = (float)(tr * (hn > 0.0 ? hn : 1e-300));
    if (m >= 2 && m <= SQ_MAX) {
        // one CTA, the matrix in shared memory; falls through to the grid
        // QR if its iteration budget or rotation log runs out
        RotLog *rlog = (RotLog *)Hds;
        int *sst = (int *)(rlog + (size_t)SQ_LOG * m * m);
        FEAST_CUDA_TRY(allow_dyn_smem(k_small_schur));
        k_small_schur<<<1, SQ_T, sq_smem_bytes(m), s>>>(m, C, rlog, SQ_LOG * m * m, sst, tol_rel, tol_abs);
        FEAST_LAUNCH_CHECK();
        int hs[3] = {0, 0, 0};
        FEAST_CUDA_TRY(cudaMemcpyAsync(hs, sst, sizeof(hs), cudaMemcpyDeviceToHost, s));
        FEAST_CUDA_TRY(cudaStreamSynchronize(s));
        if (hs[0] == 0) {
            FEAST_CUDA_TRY(allow_dyn_smem(k_apply_rotlog));
            k_apply_rotlog<<<cdiv(m, AR), AR, sizeof(float4) * AR * (size_t)m, s>>>(m, Q, rlog, sst);
            FEAST_LAUNCH_CHECK();
            if (stats) {
                k_add_stats<<<1, 1, 0, s>>>(stats, hs[2]);
                FEAST_LAUNCH_CHECK();
            }
            return FEAST_OK;
        }
    }
    // QR sweeps: cooperative grid, one CTA per SM at most
    int dev = 0, sms = 0, per = 0;
    FEAST_CUDA_TRY(cudaGetDevice(&dev));
    FEAST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t dyn = sizeof(AedShared);
    FEAST_CUDA_TRY(allow_dyn_smem(k_hqr));
    FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hqr, QT, dyn));
    if (per < 1) return FEAST_ECUDA;
    // at most one CTA per SM; the far-part passes have ~3 m independent
    // lines and a sweep at most NSH bulges, so a small projected problem
    // takes a proportionally small grid (and leaves the rest of the GPU to
    // other pencils of a batch)
    int grid = m / 8;
    if (grid < NSH) grid = NSH;
    if (grid > sms) grid = sms;
    GridSync gs{bar, bar + 1, timeout, TO_HQR};
    int mm = m, ldh = m;
    const unsigned gcv = cdiv((size_t)m * m, 256) > 4096 ? 4096 : cdiv((size_t)m * m, 256);
    k_to_ds<<<gcv, 256, 0, s>>>((int64_t)m * m, C, Hds);
    FEAST_LAUNCH_CHECK();
    k_to_ds<<<gcv, 256, 0, s>>>((int64_t)m * m, Q, Qds);
    FEAST_LAUNCH_CHECK();
    void *args[] = {&mm, &Hds, &Qds, &ldh, &rots, &shifts, &vwin, &ctl, &gs, &fail, &tol_rel, &tol_abs, &stats};
    FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_hqr, dim3(grid), dim3(QT), args, dyn, s));
    FEAST_LAUNCH_CHECK();
    k_from_ds<<<gcv, 256, 0, s>>>((int64_t)m * m, Hds, C);
    FEAST_LAUNCH_CHECK();
    k_from_ds<<<gcv, 256, 0, s>>>((int64_t)m * m, Qds, Q);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// A (m x m, overwritten), Bt (m x m upper triangular, overwritten by the
// solve), alpha/beta (beta = 1), V (m x m unit eigenvectors).
#if !FEAST_QR_FP32
int zeig_large(cudaStream_t s, int m, zd *A, zd *Bt, zd *alpha, zd *beta, zd *V, void *work,
               int *fail, int *timeout, int *stats, double defl)
{
    if (m <= 0) return FEAST_OK;
    zd *Q = (zd *)work;
    int e;
    // C = B~^{-1} A~  (upper-triangular solve with m right-hand sides)
    if ((e = trsm_upper_batched<zd>(s, m, m, 1, Bt, m, 0, A, m, 0))) return e;
    zd *C = A;
    double hn = 0.0;
    if ((e = schur_large(s, m, C, Q, (char *)work + sizeof(zd) * (size_t)m * m, fail, timeout, stats, &hn, defl)))
        return e;
    // eigenvalues and eigenvectors
    k_diag_out<<<cdiv(m, 128), 128, 0, s>>>(m, C, m, alpha, beta);
    FEAST_LAUNCH_CHECK();
    zd *Yh = Bt;  // B~ is no longer needed
    if ((e = schur_vectors(s, m, C, Yh, hn, V))) return e;   // V: transpose scratch until the product below
    if ((e = zgemm_batched(s, 0, m, m, m, zmake(1.0, 0.0), Q, m, 0, Yh, m, 0, zmake(0.0, 0.0), V, m, 0, 1)))
        return e;
    k_normalise_cols<<<cdiv((size_t)m * 32, 256), 256, 0, s>>>(m, V, m);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// Launch helpers for the warm-started solve (k_warm.cu).
int schur_vectors(cudaStream_t s, int m, const zd *T, zd *Y, double snorm, zd *scratch)
{
    k_transpose<<<dim3(cdiv(m, 32), cdiv(m, 32)), 256, 0, s>>>(m, T, m, scratch);
    FEAST_LAUNCH_CHECK();
    // one CTA per SM with ceil(m / SMs) warps: eigenvector k on CTA k mod
    // G, so every SM gets the same mix of long and short back-substitutions
    // (a grid of 8-warp CTAs a little larger than the SM count doubles the
    // work of the SMs that take two)
    int dev = 0, sms = 0;
    FEAST_CUDA_TRY(cudaGetDevice(&dev));
    FEAST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int G = sms < m ? sms : m;
    int wpc = (m + G - 1) / G;
    if (wpc > 32) {
        wpc = 32;
        G = (m + 31) / 32;
    }
    k_schur_vectors<<<G, 32 * wpc, 0, s>>>(m, scratch, m, Y, snorm);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int normalise_cols(cudaStream_t s, int m, zd *V)
{
    k_normalise_cols<<<cdiv((size_t)m * 32, 256), 256, 0, s>>>(m, V, m);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}
#endif  // !FEAST_QR_FP32

}  // namespace feast
