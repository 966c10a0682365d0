// Complex dense kernels (FP64 for the plain path, FP32 for the low-precision
// factors of the precision form): batched GEMM, formation
// of the shifted matrices z_j B - A (eq. 4.2), blocked right-looking LU with
// partial pivoting, blocked triangular solves with many right-hand sides,
// and the quadrature node-sum U = sum_j w_j X_j (eq. 4.1).
//
// GB300 runs FP64 at ~2 DFMA per clock per SM (1.05 TFLOP/s measured for
// the whole GPU), so these kernels are bound by the FP64 pipe, not by
// memory: a modest register tile (4 x 4 complex per thread) already keeps
// the pipe busy, and the work is spread over all 152 SMs through the batch
// (node) dimension and the tile grid.
#include "common.cuh"

namespace feast {

// ------------------------------------------------------------------ GEMM
namespace {
constexpr int GB_M = 64, GB_N = 64, GB_K = 8, GB_T = 256;

constexpr int GB_SMAX = 8;     // most K-slices of a tile summed in one (portable) cluster

__device__ __forceinline__ void atomic_cadd(double2 *p, double2 v)
{
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void atomic_cadd(float2 *p, float2 v)
{
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

__device__ __forceinline__ unsigned gb_cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void gb_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Load 2 (float2) or 4 (double2) words of shared memory from CTA `rank`.
__device__ __forceinline__ float2 gb_dsmem_load(const float2 *p, unsigned rank)
{
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double2 gb_dsmem_load(const double2 *p, unsigned rank)
{
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
    return v;
}

// splits > 1: blockIdx.z = batch * splits + s takes the s-th slice of K.
// Up to GB_SMAX slices the launch groups a tile's slices into one cluster
// (s = the CTA's rank in it) and CTA 0 sums the slices' tiles in rank order
// through distributed shared memory before it writes C, so the result does
// not depend on which slice finishes first; beyond that (long, skinny
// products) the slices add alpha * partial into C atomically, C pre-scaled
// by beta on the host side of the launch.
template <typename T>
__global__ void __launch_bounds__(GB_T) k_gemm(int conj_a, int64_t m, int64_t n, int64_t k,
                                               T alpha, const T *__restrict__ A, int64_t lda,
                                               int64_t sA, const T *__restrict__ B,
                                               int64_t ldb, int64_t sB, T beta,
                                               T *__restrict__ C, int64_t ldc, int64_t sC,
                                               int splits, int64_t kchunk, int tri)
{
    __shared__ T As[GB_K][GB_M + 1];
    __shared__ T Bs[GB_K][GB_N + 1];
    extern __shared__ __align__(16) unsigned char gb_red_raw[];   // splits > 1: this slice's tile
    const int b = blockIdx.z / splits, sp = blockIdx.z % splits;
    const int64_t i0 = (int64_t)blockIdx.x * GB_M, j0 = (int64_t)blockIdx.y * GB_N;
    if (tri == 3 && i0 >= j0 + GB_N) return;  // tile below the diagonal (uniform per CTA)
    int64_t kbeg = (int64_t)sp * kchunk;
    int64_t kend = (kbeg + kchunk < k) ? kbeg + kchunk : k;
    if (tri == 1 && kbeg < i0) kbeg = i0;            // op(A)(i, k) = 0 for k < i
    if (tri == 2 && kend > j0 + GB_N) kend = j0 + GB_N;  // B(k, j) = 0 for k > j
    A += (int64_t)b * sA;
    B += (int64_t)b * sB;
    C += (int64_t)b * sC;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = cx<T>(0, 0);

    for (int64_t k0 = kbeg; k0 < kend; k0 += GB_K) {
        // A tile: op(A)(i0 + r, k0 + kk)
        for (int e = threadIdx.x; e < GB_M * GB_K; e += GB_T) {
            int r, kk;
            if (!conj_a) { r = e % GB_M; kk = e / GB_M; }
            else         { kk = e % GB_K; r = e / GB_K; }
            int64_t gi = i0 + r, gk = k0 + kk;
            T v = cx<T>(0, 0);
            if (gi < m && gk < kend) v = conj_a ? cconj(A[gk + gi * lda]) : A[gi + gk * lda];
            As[kk][r] = v;
        }
        for (int e = threadIdx.x; e < GB_N * GB_K; e += GB_T) {
            int kk = e % GB_K, c = e / GB_K;
            int64_t gj = j0 + c, gk = k0 + kk;
            Bs[kk][c] = (gj < n && gk < kend) ? B[gk + gj * ldb] : cx<T>(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) cfma(acc[a][c], av[a], bv[c]);
        }
        __syncthreads();
    }
    if (splits > GB_SMAX) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int64_t gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * c;
                if (gi < m && gj < n) atomic_cadd(&C[gi + gj * ldc], cmul(alpha, acc[a][c]));
            }
        return;
    }
    if (splits > 1) {
        // every slice's tile into its own shared memory; CTA 0 adds the
        // others' in rank order (distributed shared memory), then all wait
        // until it has read them
        T *red = reinterpret_cast<T *>(gb_red_raw);
        const unsigned rank = gb_cluster_rank();
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[(a * 4 + c) * GB_T + threadIdx.x] = acc[a][c];
        gb_cluster_sync();
        if (rank == 0)
            for (int r = 1; r < splits; ++r)
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        acc[a][c] = cadd(acc[a][c], gb_dsmem_load(red + (a * 4 + c) * GB_T + threadIdx.x, r));
        gb_cluster_sync();
        if (rank != 0) return;
    }
    const bool beta0 = cis_zero(beta);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * c;
            if (gi < m && gj < n) {
                T v = cmul(alpha, acc[a][c]);
                if (!beta0) v = cadd(v, cmul(beta, C[gi + gj * ldc]));
                C[gi + gj * ldc] = v;
            }
        }
}
// C <- beta C (beta = 0 writes zeros, so stale NaNs do not survive)
template <typename T>
__global__ void k_scale(int64_t m, int64_t n, T beta, T *C, int64_t ldc, int64_t sC)
{
    T *Cb = C + (int64_t)blockIdx.y * sC;
    const bool zero = cis_zero(beta);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % m, c = e / m;
        T &x = Cb[r + c * ldc];
        x = zero ? cx<T>(0, 0) : cmul(beta, x);
    }
}
}  // namespace

template <typename T>
int gemm_batched(cudaStream_t s, int conj_a, int64_t m, int64_t n, int64_t k, T alpha,
                 const T *A, int64_t lda, int64_t sA, const T *B, int64_t ldb, int64_t sB,
                 T beta, T *C, int64_t ldc, int64_t sC, int batch, int tri)
{
    if (m <= 0 || n <= 0 || batch <= 0) return FEAST_OK;
    if (batch > 65535) return FEAST_EINVAL;
    if (tri < 0 || tri > 3 || (conj_a && (tri == 1 || tri == 2))) return FEAST_EINVAL;
    const unsigned tiles = cdiv(m, GB_M) * cdiv(n, GB_N) * (unsigned)batch;
    // split K when the output tiles cannot fill the GPU twice over (the
    // FP64 pipe is the bound, so every SM counts: a 64 x 64 tile with
    // K = 256 is ~1 ms of one SM's FP64 pipe), in slices of at least 32
    // (complex64: 128); up to GB_SMAX slices are summed in a fixed order
    // (one cluster per tile), more of them atomically (products with a
    // long K and only a tile or two of output)
    const bool fp64 = sizeof(T) == sizeof(zd);
    const int64_t kmin = fp64 ? 32 : 128;
    int splits = 1;
    if (tiles < 2 * 152 && k >= (fp64 ? 2 * kmin : 4 * kmin)) {
        const int64_t want = (2 * 152 + tiles - 1) / tiles;
        const int64_t many = k >= 512 ? (want < k / 128 ? want : k / 128) : 0;   // slices of >= 128
        int64_t few = want < k / kmin ? want : k / kmin;                         // slices of >= kmin
        if (few > GB_SMAX) few = GB_SMAX;
        splits = (int)(many > GB_SMAX ? many : few);
        if (splits * batch > 65535) splits = 65535 / batch;
        if (splits < 1) splits = 1;
    }
    int64_t kchunk = (k + splits - 1) / splits;
    kchunk = ((kchunk + GB_K - 1) / GB_K) * GB_K;
    dim3 grid(cdiv(m, GB_M), cdiv(n, GB_N), batch * splits);
    if (grid.y > 65535) return FEAST_EINVAL;
    if (splits == 1) {
        k_gemm<T><<<grid, GB_T, 0, s>>>(conj_a, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, 1, kchunk,
                                        tri);
        FEAST_LAUNCH_CHECK();
        return FEAST_OK;
    }
    if (splits > GB_SMAX) {
        // C <- beta C first; the slices then add alpha * partial atomically
        if (!(beta.x == 1 && beta.y == 0)) {
            unsigned gx = cdiv((size_t)m * n, 256);
            k_scale<T><<<dim3(gx > 4096 ? 4096 : gx, batch), 256, 0, s>>>(m, n, beta, C, ldc, sC);
            FEAST_LAUNCH_CHECK();
        }
        k_gemm<T><<<grid, GB_T, 0, s>>>(conj_a, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits,
                                        kchunk, tri);
        FEAST_LAUNCH_CHECK();
        return FEAST_OK;
    }
    const size_t red = sizeof(T) * 16 * GB_T;
    FEAST_CUDA_TRY(ensure_dyn_smem(k_gemm<T>, red));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = (unsigned)splits;
    cfg.gridDim = grid;
    cfg.blockDim = dim3(GB_T);
    cfg.dynamicSmemBytes = red;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FEAST_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gemm<T>, conj_a, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                      sC, splits, kchunk, tri));
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}
template int gemm_batched<double2>(cudaStream_t, int, int64_t, int64_t, int64_t, double2, const double2 *,
                                   int64_t, int64_t, const double2 *, int64_t, int64_t, double2, double2 *,
                                   int64_t, int64_t, int, int);
template int gemm_batched<float2>(cudaStream_t, int, int64_t, int64_t, int64_t, float2, const float2 *,
                                  int64_t, int64_t, const float2 *, int64_t, int64_t, float2, float2 *,
                                  int64_t, int64_t, int, int);

int zgemm_batched(cudaStream_t s, int conj_a, int64_t m, int64_t n, int64_t k, zd alpha,
                  const zd *A, int64_t lda, int64_t sA, const zd *B, int64_t ldb, int64_t sB,
                  zd beta, zd *C, int64_t ldc, int64_t sC, int batch, int tri)
{
    return gemm_batched<zd>(s, conj_a, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, tri);
}

// ------------------------------------------------------------------ z_j B - A
namespace {
__global__ void k_form_shifted(int64_t n, const zd *__restrict__ A, const zd *__restrict__ B,
                               int64_t ld, const zd *__restrict__ z, zd *__restrict__ F,
                               int64_t ldf, int64_t sF)
{
    const int j = blockIdx.y;
    const zd zj = z[j];
    const int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        zd bij = B ? B[r + c * ld] : zmake(r == c ? 1.0 : 0.0, 0.0);
        F[(int64_t)j * sF + r + c * ldf] = zsub(zmul(zj, bij), A[r + c * ld]);
    }
}
}  // namespace

int zform_shifted(cudaStream_t s, int64_t n, int q, const zd *A, const zd *B, int64_t ld,
                  const zd *z, zd *F, int64_t ldf, int64_t sF)
{
    unsigned gx = cdiv(n * n, 256);
    if (gx > 1024) gx = 1024;
    k_form_shifted<<<dim3(gx, q), 256, 0, s>>>(n, A, B, ld, z, F, ldf, sF);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// ------------------------------------------------------------------ LU
namespace {
constexpr int LU_NB = 32;     // panel width
constexpr int LU_PT = 512;    // panel threads
constexpr int LU_NBO = 256;   // outer block of the tensor-core LU

// Factor the panel [k0, k0 + nb) x [k0, n) of every batch member: pivot by
// largest modulus (ties -> smallest row), swap within the panel columns,
// scale, rank-1 update of the remaining panel columns.
template <typename T>
__global__ void __launch_bounds__(LU_PT) k_lu_panel(int64_t n, int64_t k0, int nb, T *F,
                                                   int64_t ldf, int64_t sF, int *piv, int64_t pstride,
                                                   int *info, int *row)
{
    typedef typename CxReal<T>::type R;
    const int b = blockIdx.x;
    T *Am = F + (int64_t)b * sF;
    __shared__ R s_val[LU_PT / 32];
    __shared__ int64_t s_idx[LU_PT / 32];
    __shared__ int64_t s_p;
    __shared__ T s_row[LU_NB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < nb; ++j) {
        const int64_t col = k0 + j;
        R best = -1;
        int64_t bi = col;
        for (int64_t i = col + threadIdx.x; i < n; i += LU_PT) {
            R v = cabs2(Am[i + col * ldf]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            R ov = __shfl_down_sync(0xffffffffu, best, off);
            int64_t oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            R bv = s_val[0];
            int64_t bx = s_idx[0];
            for (int w = 1; w < LU_PT / 32; ++w)
                if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bx)) { bv = s_val[w]; bx = s_idx[w]; }
            s_p = bx;
            piv[(int64_t)b * pstride + col] = (int)bx;
            if (bv == 0 && info) {
                // record the first failing block (1-based) and column
                if (atomicCAS(info, 0, b + 1) == 0 && row) *row = (int)col + 1;
            }
        }
        __syncthreads();
        const int64_t p = s_p;
        if (p != col && threadIdx.x < nb) {
            int64_t c = k0 + threadIdx.x;
            T t = Am[col + c * ldf];
            Am[col + c * ldf] = Am[p + c * ldf];
            Am[p + c * ldf] = t;
        }
        __syncthreads();
        if (threadIdx.x < nb) s_row[threadIdx.x] = Am[col + (k0 + threadIdx.x) * ldf];
        __syncthreads();
        const T d = s_row[j];
        if (!cis_zero(d)) {
            for (int64_t i = col + 1 + threadIdx.x; i < n; i += LU_PT) {
                T l = cdiv(Am[i + col * ldf], d);
                Am[i + col * ldf] = l;
                const T nl = cneg(l);
                for (int c = j + 1; c < nb; ++c) {
                    T &a = Am[i + (k0 + c) * ldf];
                    T v = a;
                    cfma(v, nl, s_row[c]);
                    a = v;
                }
            }
        }
        __syncthreads();
    }
}

// Apply the panel's row interchanges to the columns outside the panel.
template <typename T>
__global__ void k_laswp_outside(int64_t n, int64_t k0, int nb, T *F, int64_t ldf, int64_t sF,
                                const int *piv)
{
    const int b = blockIdx.y;
    T *Am = F + (int64_t)b * sF;
    const int *pv = piv + (int64_t)b * n;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= k0 && c < k0 + nb) continue;
        for (int j = 0; j < nb; ++j) {
            int64_t r = k0 + j, p = pv[r];
            if (p != r) {
                T t = Am[r + c * ldf];
                Am[r + c * ldf] = Am[p + c * ldf];
                Am[p + c * ldf] = t;
            }
        }
    }
}

// U12 = L11^{-1} A12 for the nb rows of the panel (L11 unit lower), one
// thread per column in [cbeg, cend).
template <typename T>
__global__ void k_trsm_u12(int64_t cbeg, int64_t cend, int64_t k0, int nb, T *F, int64_t ldf, int64_t sF)
{
    const int b = blockIdx.y;
    T *Am = F + (int64_t)b * sF;
    __shared__ T L[LU_NB][LU_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e % nb, c = e / nb;
        L[r][c] = Am[(k0 + r) + (k0 + c) * ldf];
    }
    __syncthreads();
    const int64_t c = cbeg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cend) return;
    T x[LU_NB];
#pragma unroll
    for (int r = 0; r < LU_NB; ++r)
        if (r < nb) x[r] = Am[(k0 + r) + c * ldf];
#pragma unroll
    for (int i = 0; i < LU_NB; ++i) {
        if (i >= nb) break;
#pragma unroll
        for (int r = i + 1; r < LU_NB; ++r)
            if (r < nb) cfma(x[r], cneg(L[r][i]), x[i]);
    }
#pragma unroll
    for (int r = 0; r < LU_NB; ++r)
        if (r < nb) Am[(k0 + r) + c * ldf] = x[r];
}
}  // namespace

template <typename T>
int getrf_batched(cudaStream_t s, int64_t n, int batch, T *F, int64_t ldf, int64_t sF, int *piv,
                  int *info, int *row)
{
    if (n <= 0 || batch <= 0) return FEAST_OK;
    for (int64_t k0 = 0; k0 < n; k0 += LU_NB) {
        int nb = (int)((n - k0) < LU_NB ? (n - k0) : LU_NB);
        k_lu_panel<T><<<batch, LU_PT, 0, s>>>(n, k0, nb, F, ldf, sF, piv, n, info, row);
        FEAST_LAUNCH_CHECK();
        unsigned gx = cdiv(n, 128);
        k_laswp_outside<T><<<dim3(gx, batch), 128, 0, s>>>(n, k0, nb, F, ldf, sF, piv);
        FEAST_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest > 0) {
            k_trsm_u12<T><<<dim3(cdiv(rest, 128), batch), 128, 0, s>>>(k0 + nb, n, k0, nb, F, ldf, sF);
            FEAST_LAUNCH_CHECK();
            int e = gemm_batched<T>(s, 0, rest, rest, nb, cx<T>(-1, 0), F + k0 + nb + k0 * ldf,
                                    ldf, sF, F + k0 + (k0 + nb) * ldf, ldf, sF, cx<T>(1, 0),
                                    F + (k0 + nb) + (k0 + nb) * ldf, ldf, sF, batch);
            if (e) return e;
        }
    }
    return FEAST_OK;
}
template int getrf_batched<double2>(cudaStream_t, int64_t, int, double2 *, int64_t, int64_t, int *, int *, int *);

// complex64 LU with the bulk of its flops on the tensor cores.  Two-level
// right-looking blocking: an outer block of LU_NBO columns is factored with
// the LU_NB-wide panel kernel as above, except that each inner rank-LU_NB
// update is confined to the outer block's columns (all rows below) and to
// the outer block's rows (columns beyond it); the trailing matrix then takes
// one rank-LU_NBO update A22 -= L21 U12 through the tcgen05 GEMM.  The
// factors and pivots are those of the one-level routine up to rounding.
size_t getrf_tc_scratch_floats(int64_t n, int batch)
{
    return tc_scratch_floats(n, LU_NBO, n, batch);
}

int getrf_batched_tc(cudaStream_t s, int64_t n, int batch, cf *F, int64_t ldf, int64_t sF, int *piv,
                     int *info, int *row, float *scratch, int *tc_err, TcTimer *tt)
{
    if (n <= 0 || batch <= 0) return FEAST_OK;
    const cf mone = cx<cf>(-1, 0), one = cx<cf>(1, 0);
    int e;
    for (int64_t k0 = 0; k0 < n; k0 += LU_NBO) {
        const int64_t nbo = (n - k0) < LU_NBO ? (n - k0) : LU_NBO;
        const int64_t kend = k0 + nbo;                  // first column after the outer block
        for (int64_t kk = k0; kk < kend; kk += LU_NB) {
            const int nb = (int)((kend - kk) < LU_NB ? (kend - kk) : LU_NB);
            k_lu_panel<cf><<<batch, LU_PT, 0, s>>>(n, kk, nb, F, ldf, sF, piv, n, info, row);
            FEAST_LAUNCH_CHECK();
            k_laswp_outside<cf><<<dim3(cdiv(n, 128), batch), 128, 0, s>>>(n, kk, nb, F, ldf, sF, piv);
            FEAST_LAUNCH_CHECK();
            const int64_t c1 = kk + nb;                 // first column right of the panel
            if (kend > c1) {
                // inside the outer block only: columns beyond it keep their
                // original values (row swaps included) until the block is done
                k_trsm_u12<cf><<<dim3(cdiv(kend - c1, 128), batch), 128, 0, s>>>(c1, kend, kk, nb, F, ldf, sF);
                FEAST_LAUNCH_CHECK();
                if ((e = gemm_batched<cf>(s, 0, n - c1, kend - c1, nb, mone, F + c1 + kk * ldf, ldf, sF,
                                          F + kk + c1 * ldf, ldf, sF, one, F + c1 + c1 * ldf, ldf, sF, batch)))
                    return e;
            }
        }
        const int64_t rest = n - kend;
        if (rest <= 0) break;
        // U12 = L11^{-1} A12 for the columns beyond the block, LU_NB rows at a time
        for (int64_t kk = k0; kk < kend; kk += LU_NB) {
            const int nb = (int)((kend - kk) < LU_NB ? (kend - kk) : LU_NB);
            k_trsm_u12<cf><<<dim3(cdiv(rest, 128), batch), 128, 0, s>>>(kend, n, kk, nb, F, ldf, sF);
            FEAST_LAUNCH_CHECK();
            const int64_t r1 = kk + nb;
            if (r1 < kend) {
                if ((e = gemm_batched<cf>(s, 0, kend - r1, rest, nb, mone, F + r1 + kk * ldf, ldf, sF,
                                          F + kk + kend * ldf, ldf, sF, one, F + r1 + kend * ldf, ldf, sF,
                                          batch)))
                    return e;
            }
        }
        // A22 -= L21 U12   (rest x rest, inner dimension nbo)
        if ((e = tc_cgemm(s, rest, rest, nbo, mone, F + kend + k0 * ldf, ldf, sF, F + k0 + kend * ldf, ldf, sF,
                          one, F + kend + kend * ldf, ldf, sF, batch, scratch, tc_err, tt)))
            return e;
    }
    return FEAST_OK;
}

// Factor only the leading panel (columns 0..nb-1, all rows) of each batch
// member; pivots at piv[b * pstride + k].
template <typename T>
int getrf_panel(cudaStream_t s, int64_t rows, int nb, int batch, T *F, int64_t ldf, int64_t sF,
                int *piv, int64_t pstride, int *info, int *row)
{
    if (rows <= 0 || nb <= 0 || batch <= 0) return FEAST_OK;
    k_lu_panel<T><<<batch, LU_PT, 0, s>>>(rows, 0, nb, F, ldf, sF, piv, pstride, info, row);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}
template int getrf_panel<double2>(cudaStream_t, int64_t, int, int, double2 *, int64_t, int64_t, int *,
                                  int64_t, int *, int *);
template int getrf_panel<float2>(cudaStream_t, int64_t, int, int, float2 *, int64_t, int64_t, int *,
                                 int64_t, int *, int *);
template int getrf_batched<float2>(cudaStream_t, int64_t, int, float2 *, int64_t, int64_t, int *, int *, int *);

int zgetrf_batched(cudaStream_t s, int64_t n, int batch, zd *F, int64_t ldf, int64_t sF,
                   int *piv, int *info, int *row)
{
    return getrf_batched<zd>(s, n, batch, F, ldf, sF, piv, info, row);
}

// ------------------------------------------------------------------ solves
namespace {
constexpr int SV_NB = 32;

// X rows [k0, k0+nb) <- T^{-1} X rows [k0, k0+nb) for the diagonal block T of
// the factor (lower = unit lower L, else upper U).  One thread per column.
template <typename C>
__global__ void k_trsv_diag(int64_t n, int64_t nrhs, int64_t k0, int nb, int lower,
                            const C *F, int64_t ldf, int64_t sF, C *X, int64_t ldx, int64_t sX)
{
    const int b = blockIdx.y;
    const C *Am = F + (int64_t)b * sF;
    C *Xb = X + (int64_t)b * sX;
    __shared__ C T[SV_NB][SV_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e % nb, c = e / nb;
        T[r][c] = Am[(k0 + r) + (k0 + c) * ldf];
    }
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    C x[SV_NB];
#pragma unroll
    for (int r = 0; r < SV_NB; ++r)
        if (r < nb) x[r] = Xb[(k0 + r) + c * ldx];
    if (lower) {
#pragma unroll
        for (int i = 0; i < SV_NB; ++i) {
            if (i >= nb) break;
#pragma unroll
            for (int r = i + 1; r < SV_NB; ++r)
                if (r < nb) cfma(x[r], cneg(T[r][i]), x[i]);
        }
    } else {
#pragma unroll
        for (int i = SV_NB - 1; i >= 0; --i) {
            if (i >= nb) continue;
            x[i] = cdiv(x[i], T[i][i]);
#pragma unroll
            for (int r = 0; r < SV_NB; ++r)
                if (r < i) cfma(x[r], cneg(T[r][i]), x[i]);
        }
    }
#pragma unroll
    for (int r = 0; r < SV_NB; ++r)
        if (r < nb) Xb[(k0 + r) + c * ldx] = x[r];
}

// Apply the interchanges piv[0..n) to each column of X in sequence.
template <typename T>
__global__ void k_laswp_rhs(int64_t n, int64_t nrhs, const int *piv, T *X, int64_t ldx,
                            int64_t sX)
{
    const int b = blockIdx.y;
    T *Xb = X + (int64_t)b * sX;
    const int *pv = piv + (int64_t)b * n;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nrhs) return;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = pv[k];
        if (p != k) {
            T t = Xb[k + c * ldx];
            Xb[k + c * ldx] = Xb[p + c * ldx];
            Xb[p + c * ldx] = t;
        }
    }
}

// Composition of the interchanges: perm[i] = original row that ends at i.
__global__ void k_piv_to_perm(int64_t n, const int *piv, int *perm)
{
    const int b = blockIdx.x;
    const int *pv = piv + (int64_t)b * n;
    int *pm = perm + (int64_t)b * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) pm[i] = (int)i;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int64_t k = 0; k < n; ++k) {
            int64_t p = pv[k];
            if (p != k) { int t = pm[k]; pm[k] = pm[p]; pm[p] = t; }
        }
}

template <typename T>
__global__ void k_gather_rows(int64_t n, int64_t nrhs, const int *perm, const T *R, int64_t ldr,
                              int64_t sR, T *X, int64_t ldx, int64_t sX)
{
    const int b = blockIdx.y;
    const int *pm = perm + (int64_t)b * n;
    const T *Rb = R + (int64_t)b * sR;
    T *Xb = X + (int64_t)b * sX;
    const int64_t total = n * nrhs;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        Xb[r + c * ldx] = Rb[pm[r] + c * ldr];
    }
}
}  // namespace

// Complex64 L U solve of already-permuted right-hand sides with the bulk of
// the flops on the tensor cores: outer blocks of LU_NBO rows, solved inside
// with the SV_NB-wide diagonal kernel and SIMT updates confined to the
// block, and one rank-LU_NBO tensor-core update (tc_cgemm) of the rows
// beyond the block per outer step.  scratch: tc_scratch_floats(n, LU_NBO,
// nrhs, batch) floats.
// The off-block panels of the factors as tensor-core left operands, in the
// order trsm_lu_tc uses them: forward (L) panels F[kend:, k0:kend] for
// k0 = 0, LU_NBO, ...; then backward (U) panels F[0:k0, k0:kend] for k0
// from the last block down.
size_t trsm_tc_cache_floats(int64_t n, int batch)
{
    size_t tot = 0;
    for (int64_t k0 = 0; k0 < n; k0 += LU_NBO) {
        const int64_t kend = (k0 + LU_NBO < n) ? k0 + LU_NBO : n;
        if (kend < n) tot += tc_prepA_floats(n - kend, kend - k0, batch);
        if (k0 > 0) tot += tc_prepA_floats(k0, kend - k0, batch);
    }
    return tot;
}

int trsm_tc_cache_fill(cudaStream_t s, int64_t n, int batch, const cf *F, int64_t ldf, int64_t sF, float *cache)
{
    int e;
    size_t off = 0;
    for (int64_t k0 = 0; k0 < n; k0 += LU_NBO) {
        const int64_t kend = (k0 + LU_NBO < n) ? k0 + LU_NBO : n;
        if (kend < n) {
            if ((e = tc_prepare_A(s, n - kend, kend - k0, F + kend + k0 * ldf, ldf, sF, batch, cache + off))) return e;
            off += tc_prepA_floats(n - kend, kend - k0, batch);
        }
    }
    const int64_t last = ((n - 1) / LU_NBO) * LU_NBO;
    for (int64_t k0 = last; k0 >= 0; k0 -= LU_NBO) {
        const int64_t kend = (k0 + LU_NBO < n) ? k0 + LU_NBO : n;
        if (k0 > 0) {
            if ((e = tc_prepare_A(s, k0, kend - k0, F + k0 * ldf, ldf, sF, batch, cache + off))) return e;
            off += tc_prepA_floats(k0, kend - k0, batch);
        }
    }
    return FEAST_OK;
}

int trsm_lu_tc(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const cf *F, int64_t ldf, int64_t sF, cf *X,
               int64_t ldx, int64_t sX, float *scratch, int *tc_err, const float *cache, TcTimer *tt)
{
    if (n <= 0 || nrhs <= 0 || batch <= 0) return FEAST_OK;
    size_t coff = 0;
    const cf mone = cx<cf>(-1, 0), one = cx<cf>(1, 0);
    dim3 g(cdiv(nrhs, 64), batch);
    int e;
    // forward: unit lower L
    for (int64_t k0 = 0; k0 < n; k0 += LU_NBO) {
        const int64_t kend = (k0 + LU_NBO < n) ? k0 + LU_NBO : n;
        for (int64_t kk = k0; kk < kend; kk += SV_NB) {
            const int nb = (int)((kend - kk) < SV_NB ? (kend - kk) : SV_NB);
            k_trsv_diag<cf><<<g, 64, 0, s>>>(n, nrhs, kk, nb, 1, F, ldf, sF, X, ldx, sX);
            FEAST_LAUNCH_CHECK();
            const int64_t r1 = kk + nb;
            if (r1 < kend &&
                (e = gemm_batched<cf>(s, 0, kend - r1, nrhs, nb, mone, F + r1 + kk * ldf, ldf, sF, X + kk, ldx, sX,
                                      one, X + r1, ldx, sX, batch)))
                return e;
        }
        if (kend < n) {
            if (cache) {
                e = tc_cgemm_prepA(s, n - kend, nrhs, kend - k0, mone, cache + coff, X + k0, ldx, sX, one, X + kend,
                                   ldx, sX, batch, scratch, tc_err, tt);
                coff += tc_prepA_floats(n - kend, kend - k0, batch);
            } else {
                e = tc_cgemm(s, n - kend, nrhs, kend - k0, mone, F + kend + k0 * ldf, ldf, sF, X + k0, ldx, sX, one,
                             X + kend, ldx, sX, batch, scratch, tc_err, tt);
            }
            if (e) return e;
        }
    }
    // backward: upper U
    const int64_t last = ((n - 1) / LU_NBO) * LU_NBO;
    for (int64_t k0 = last; k0 >= 0; k0 -= LU_NBO) {
        const int64_t kend = (k0 + LU_NBO < n) ? k0 + LU_NBO : n;
        const int64_t ilast = k0 + ((kend - k0 - 1) / SV_NB) * SV_NB;
        for (int64_t kk = ilast; kk >= k0; kk -= SV_NB) {
            const int nb = (int)((kend - kk) < SV_NB ? (kend - kk) : SV_NB);
            k_trsv_diag<cf><<<g, 64, 0, s>>>(n, nrhs, kk, nb, 0, F, ldf, sF, X, ldx, sX);
            FEAST_LAUNCH_CHECK();
            if (kk > k0 &&
                (e = gemm_batched<cf>(s, 0, kk - k0, nrhs, nb, mone, F + k0 + kk * ldf, ldf, sF, X + kk, ldx, sX,
                                      one, X + k0, ldx, sX, batch)))
                return e;
        }
        if (k0 > 0) {
            if (cache) {
                e = tc_cgemm_prepA(s, k0, nrhs, kend - k0, mone, cache + coff, X + k0, ldx, sX, one, X, ldx, sX,
                                   batch, scratch, tc_err, tt);
                coff += tc_prepA_floats(k0, kend - k0, batch);
            } else {
                e = tc_cgemm(s, k0, nrhs, kend - k0, mone, F + k0 * ldf, ldf, sF, X + k0, ldx, sX, one, X, ldx, sX,
                             batch, scratch, tc_err, tt);
            }
            if (e) return e;
        }
    }
    return FEAST_OK;
}

int zpiv_to_perm(cudaStream_t s, int64_t n, int batch, const int *piv, int *perm)
{
    k_piv_to_perm<<<batch, 256, 0, s>>>(n, piv, perm);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

template <typename T>
int gather_rows(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const int *perm, const T *R,
                int64_t ldr, int64_t sR, T *X, int64_t ldx, int64_t sX)
{
    unsigned gx = cdiv(n * nrhs, 256);
    if (gx > 2048) gx = 2048;
    k_gather_rows<T><<<dim3(gx, batch), 256, 0, s>>>(n, nrhs, perm, R, ldr, sR, X, ldx, sX);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}
template int gather_rows<double2>(cudaStream_t, int64_t, int64_t, int, const int *, const double2 *,
                                  int64_t, int64_t, double2 *, int64_t, int64_t);
template int gather_rows<float2>(cudaStream_t, int64_t, int64_t, int, const int *, const float2 *,
                                 int64_t, int64_t, float2 *, int64_t, int64_t);

int zgather_rows(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const int *perm,
                 const zd *R, int64_t ldr, zd *X, int64_t ldx, int64_t sX)
{
    return gather_rows<zd>(s, n, nrhs, batch, perm, R, ldr, 0, X, ldx, sX);
}

// Forward substitution with the unit-lower factor (in place).
template <typename T>
int trsm_lower_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const T *F, int64_t ldf,
                       int64_t sF, T *X, int64_t ldx, int64_t sX)
{
    if (n <= 0 || nrhs <= 0 || batch <= 0) return FEAST_OK;
    dim3 g(cdiv(nrhs, 64), batch);
    for (int64_t k0 = 0; k0 < n; k0 += SV_NB) {
        int nb = (int)((n - k0) < SV_NB ? (n - k0) : SV_NB);
        k_trsv_diag<T><<<g, 64, 0, s>>>(n, nrhs, k0, nb, 1, F, ldf, sF, X, ldx, sX);
        FEAST_LAUNCH_CHECK();
        int64_t rest = n - k0 - nb;
        if (rest > 0) {
            int e = gemm_batched<T>(s, 0, rest, nrhs, nb, cx<T>(-1, 0), F + (k0 + nb) + k0 * ldf,
                                    ldf, sF, X + k0, ldx, sX, cx<T>(1, 0), X + k0 + nb, ldx, sX,
                                    batch);
            if (e) return e;
        }
    }
    return FEAST_OK;
}

// Back substitution with the upper factor (in place).
template <typename T>
int trsm_upper_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const T *F, int64_t ldf,
                       int64_t sF, T *X, int64_t ldx, int64_t sX)
{
    if (n <= 0 || nrhs <= 0 || batch <= 0) return FEAST_OK;
    dim3 g(cdiv(nrhs, 64), batch);
    int64_t last = ((n - 1) / SV_NB) * SV_NB;
    for (int64_t k0 = last; k0 >= 0; k0 -= SV_NB) {
        int nb = (int)((n - k0) < SV_NB ? (n - k0) : SV_NB);
        k_trsv_diag<T><<<g, 64, 0, s>>>(n, nrhs, k0, nb, 0, F, ldf, sF, X, ldx, sX);
        FEAST_LAUNCH_CHECK();
        if (k0 > 0) {
            int e = gemm_batched<T>(s, 0, k0, nrhs, nb, cx<T>(-1, 0), F + k0 * ldf, ldf, sF,
                                    X + k0, ldx, sX, cx<T>(1, 0), X, ldx, sX, batch);
            if (e) return e;
        }
    }
    return FEAST_OK;
}

// L U solve of already-permuted right-hand sides.
template <typename T>
int trsm_lu_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const T *F, int64_t ldf,
                    int64_t sF, T *X, int64_t ldx, int64_t sX)
{
    int e = trsm_lower_batched<T>(s, n, nrhs, batch, F, ldf, sF, X, ldx, sX);
    if (e) return e;
    return trsm_upper_batched<T>(s, n, nrhs, batch, F, ldf, sF, X, ldx, sX);
}
template int trsm_upper_batched<double2>(cudaStream_t, int64_t, int64_t, int, const double2 *, int64_t,
                                         int64_t, double2 *, int64_t, int64_t);
template int trsm_upper_batched<float2>(cudaStream_t, int64_t, int64_t, int, const float2 *, int64_t,
                                        int64_t, float2 *, int64_t, int64_t);
template int trsm_lu_batched<double2>(cudaStream_t, int64_t, int64_t, int, const double2 *, int64_t,
                                      int64_t, double2 *, int64_t, int64_t);
template int trsm_lu_batched<float2>(cudaStream_t, int64_t, int64_t, int, const float2 *, int64_t,
                                     int64_t, float2 *, int64_t, int64_t);

int ztrsm_lu_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const zd *F,
                     int64_t ldf, int64_t sF, zd *X, int64_t ldx, int64_t sX)
{
    return trsm_lu_batched<zd>(s, n, nrhs, batch, F, ldf, sF, X, ldx, sX);
}

int zgetrs_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const zd *F,
                   int64_t ldf, int64_t sF, const int *piv, zd *X, int64_t ldx, int64_t sX)
{
    if (n <= 0 || nrhs <= 0 || batch <= 0) return FEAST_OK;
    k_laswp_rhs<zd><<<dim3(cdiv(nrhs, 64), batch), 64, 0, s>>>(n, nrhs, piv, X, ldx, sX);
    FEAST_LAUNCH_CHECK();
    return ztrsm_lu_batched(s, n, nrhs, batch, F, ldf, sF, X, ldx, sX);
}

// ------------------------------------------------------------------ node sum
namespace {
__global__ void k_node_sum(int64_t n, int64_t m, int q, const zd *__restrict__ w,
                           const zd *__restrict__ X, int64_t ldx, int64_t sX, zd *__restrict__ U,
                           int64_t ldu)
{
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % n, c = e / n;
        zd acc = zmake(0.0, 0.0);
        for (int j = 0; j < q; ++j) zfma(acc, w[j], X[(int64_t)j * sX + r + c * ldx]);
        U[r + c * ldu] = acc;
    }
}
}  // namespace

int znode_sum(cudaStream_t s, int64_t n, int64_t m, int q, const zd *w, const zd *X,
              int64_t ldx, int64_t sX, zd *U, int64_t ldu)
{
    unsigned gx = cdiv(n * m, 256);
    if (gx > 152 * 16) gx = 152 * 16;
    k_node_sum<<<gx, 256, 0, s>>>(n, m, q, w, X, ldx, sX, U, ldu);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
