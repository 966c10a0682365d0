// Internal helpers shared by the CUDA translation units of the GB300 FEAST
// library (never by the oracle).  Complex numbers are double2 (re, im) in
// FP64 and float2 in FP32; all matrices are column-major with an explicit
// leading dimension.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/feast_gb300.h"

namespace feast {

// ---------------------------------------------------------------- complex FP64
typedef double2 zd;

__host__ __device__ __forceinline__ zd zmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ zd zadd(zd a, zd b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zd zsub(zd a, zd b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zd zmul(zd a, zd b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ zd zconj(zd a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ zd zscale(zd a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double zabs2(zd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double zabs(zd a) { return hypot(a.x, a.y); }
// c += a * b
__host__ __device__ __forceinline__ void zfma(zd &c, zd a, zd b)
{
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
}
// c += conj(a) * b
__host__ __device__ __forceinline__ void zfma_conj(zd &c, zd a, zd b)
{
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(-a.y, b.x, c.y);
}
// a / b  (Smith's algorithm, avoids overflow in |b|^2)
__host__ __device__ __forceinline__ zd zdiv(zd a, zd b)
{
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}

// ---------------------------------------------------------------- complex FP32
typedef float2 cf;
__host__ __device__ __forceinline__ cf cmakef(float r, float i) { return make_float2(r, i); }

// Overloads shared by the templated kernels (T = double2 or float2).
template <typename T> struct CxReal;
template <> struct CxReal<double2> { typedef double type; };
template <> struct CxReal<float2> { typedef float type; };
template <typename T> __host__ __device__ __forceinline__ T cx(typename CxReal<T>::type r, typename CxReal<T>::type i)
{
    T v;
    v.x = r;
    v.y = i;
    return v;
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return zadd(a, b); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) { return zmul(a, b); }
__host__ __device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return zconj(a); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return zabs2(a); }
__host__ __device__ __forceinline__ void cfma(float2 &c, float2 a, float2 b)
{
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
}
__host__ __device__ __forceinline__ void cfma(double2 &c, double2 a, double2 b) { zfma(c, a, b); }
__host__ __device__ __forceinline__ float2 cdiv(float2 a, float2 b)
{
    if (fabsf(b.x) >= fabsf(b.y)) {
        float r = b.y / b.x, d = b.x + b.y * r;
        return make_float2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        float r = b.x / b.y, d = b.x * r + b.y;
        return make_float2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) { return zdiv(a, b); }
__host__ __device__ __forceinline__ bool cis_zero(float2 a) { return a.x == 0.f && a.y == 0.f; }
__host__ __device__ __forceinline__ bool cis_zero(double2 a) { return a.x == 0.0 && a.y == 0.0; }

// ---------------------------------------------------------------- status
// Per-context device-side status written by kernels (pivot failures,
// non-finite values) and read by the host at the one sync point per pass.
struct DevStatus {
    int lu_info;        // first node (1-based) with an exactly zero pivot, else 0
    int lu_row;         // its column (1-based)
    int nonfinite;      // non-zero if a NaN/Inf reached a residual
    int count;          // c(k)
    double err;         // e(k)
    int flag;           // 2 continue, 1 / 0 / -1 stopping criteria
    int qz_fail;        // pencils whose QZ iteration hit its iteration cap
    int timeout;        // TO_* bits of the bounded waits that gave up
    int qz_sweeps;      // QR sweeps of the last large projected eigensolve
    int qz_phases;      // chase phases (chunks) of those sweeps
    int qz_aed;         // early-deflation windows applied
};

// Records the failing CUDA call (error name, file, line) for
// feast_last_cuda_error; returns FEAST_ECUDA.
int note_cuda_error(cudaError_t e, const char *file, int line);
// Records which bounded waits gave up (TO_* bits) for feast_last_cuda_error;
// returns FEAST_ETIMEOUT.
int note_timeout(int bits);
#define FEAST_CUDA_TRY(expr)                                                         \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) return ::feast::note_cuda_error(_e, __FILE__, __LINE__); \
    } while (0)

// Every kernel launch of the library is followed by this check, which also
// counts the launch (feast_kernel_launches reports the total).
void count_launch();
#define FEAST_LAUNCH_CHECK()                                                         \
    do {                                                                             \
        ::feast::count_launch();                                                     \
        cudaError_t _e = cudaGetLastError();                                         \
        if (_e != cudaSuccess) return ::feast::note_cuda_error(_e, __FILE__, __LINE__); \
    } while (0)

static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit to everything the device
// allows beside its static shared memory.  The value depends only on the
// kernel and the device, so concurrent callers (the batch solver's worker
// threads) never lower each other's limit below what a launch needs.
template <typename K>
inline cudaError_t allow_dyn_smem(K kernel)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, (const void *)kernel)) != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

// Opt a launch with `bytes` of dynamic shared memory in above the 48 KB
// default when the kernel's static plus dynamic shared memory exceeds it.
template <typename K>
inline cudaError_t ensure_dyn_smem(K kernel, size_t bytes)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, (const void *)kernel);
    if (e != cudaSuccess) return e;
    if (bytes + fa.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
    return allow_dyn_smem(kernel);
}

// ---------------------------------------------------------------- bounded waits
// Where a bounded wait gave up: bits of DevStatus::timeout, set only by the
// wait that ran out (a wait that stops because another one already gave up
// adds nothing), so the host can name the first site.
enum : int {
    TO_HESS = 1 << 1,       // k_hess_grid grid barrier
    TO_HQR = 1 << 2,        // k_hqr grid barrier
    TO_CHOL = 1 << 3,       // k_chol_grid grid barrier
    TO_CGS2 = 1 << 4,       // k_cgs2_grid grid barrier
    TO_PCHOL = 1 << 5,      // k_pchol_grid grid barrier
    TO_TC_LOAD = 1 << 6,    // k_tc_cgemm2 producer (free stage)
    TO_TC_MMA = 1 << 7,     // k_tc_cgemm2 MMA issuer (loaded stage / free accumulator)
    TO_TC_EPI = 1 << 8,     // k_tc_cgemm2 epilogue (finished accumulator)
    TO_TC_DRAIN = 1 << 9,   // k_tc_cgemm2 final MMA completion
    TO_OZ = 1 << 10,        // k_oz_gemm (any of its mbarrier waits)
};
// Every wait polls until its condition holds, another wait has given up,
// or WAIT_NS of device time (%globaltimer) have passed; the iteration cap
// is a second bound in case the timer does not advance.
constexpr unsigned long long WAIT_NS = 4000000000ull;
constexpr long long SPIN_LIMIT = 1ll << 30;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct GridSync {
    unsigned *count;
    unsigned *gen;
    int *err;
    int site;       // TO_* bit raised when this barrier's wait runs out
};

// Sense-counting grid barrier for a cooperative launch, with a bounded spin:
// on timeout it raises *err and returns (every caller then bails out).
__device__ __forceinline__ bool grid_barrier(const GridSync &g)
{
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = g.gen;
        const unsigned my = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(g.count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(g.count, 0u);
            __threadfence();
            atomicAdd(g.gen, 1u);
        } else {
            long long it = 0;
            const unsigned long long t0 = global_ns();
            while (*vgen == my) {
                if (*(volatile int *)g.err) { ok = 0; break; }
                if (++it > SPIN_LIMIT || ((it & 255) == 0 && global_ns() - t0 > WAIT_NS)) {
                    ok = 0;
                    atomicOr(g.err, g.site);
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
        s_ok = ok && !*(volatile int *)g.err;
    }
    __syncthreads();
    return s_ok != 0;
}



// ---------------------------------------------------------------- kernels (FP64)
// Templated dense kernels (T = double2 or float2), instantiated in k_dense.cu.
// tri (structure the GEMM may skip): 0 none; 1 op(A) upper triangular
// (row tile i0 starts its K loop at i0); 2 B upper triangular (column tile
// j0 ends it at j0 + tile width); 3 only the upper triangle of C is wanted
// (tiles strictly below the diagonal are not computed).  1 and 2 need
// conj_a = 0.
template <typename T>
int gemm_batched(cudaStream_t s, int conj_a, int64_t m, int64_t n, int64_t k, T alpha,
                 const T *A, int64_t lda, int64_t sA, const T *B, int64_t ldb, int64_t sB,
                 T beta, T *C, int64_t ldc, int64_t sC, int batch, int tri = 0);
template <typename T>
int getrf_batched(cudaStream_t s, int64_t n, int batch, T *F, int64_t ldf, int64_t sF, int *piv,
                  int *info, int *row);
template <typename T>
int getrf_panel(cudaStream_t s, int64_t rows, int nb, int batch, T *F, int64_t ldf, int64_t sF,
                int *piv, int64_t pstride, int *info, int *row);
template <typename T>
int trsm_lu_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const T *F, int64_t ldf,
                    int64_t sF, T *X, int64_t ldx, int64_t sX);
template <typename T>
int trsm_upper_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const T *F, int64_t ldf,
                       int64_t sF, T *X, int64_t ldx, int64_t sX);
// X_b[i, :] = R_b[perm_b[i], :]   (sR = 0 shares one right-hand side)
template <typename T>
int gather_rows(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const int *perm, const T *R,
                int64_t ldr, int64_t sR, T *X, int64_t ldx, int64_t sX);

// Batched complex GEMM:  C_b = alpha * op(A_b) * B_b + beta * C_b, b = 0..batch-1,
// op(A) = A (conj_a = 0) or A^H (conj_a = 1).  op(A) is m x k, B k x n.
// Strides are in elements between consecutive batch members.
int zgemm_batched(cudaStream_t s, int conj_a, int64_t m, int64_t n, int64_t k, zd alpha,
                  const zd *A, int64_t lda, int64_t sA, const zd *B, int64_t ldb, int64_t sB,
                  zd beta, zd *C, int64_t ldc, int64_t sC, int batch, int tri = 0);

// M_j = z_j B - A for j = 0..q-1 into F (q blocks of ldf x n); B may be null
// (identity).
int zform_shifted(cudaStream_t s, int64_t n, int q, const zd *A, const zd *B, int64_t ld,
                  const zd *z, zd *F, int64_t ldf, int64_t sF);

// Batched LU with partial pivoting (modulus criterion) in place.
// info (may be null): set to 1 + the first block with an exact zero pivot;
// row (may be null): that pivot's column + 1.
int zgetrf_batched(cudaStream_t s, int64_t n, int batch, zd *F, int64_t ldf, int64_t sF,
                   int *piv, int *info, int *row);

// Batched solve with the LU factors: X_b = F_b^{-1} X_b in place
// (rows permuted by piv first).  X_b is n x nrhs.
int zgetrs_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const zd *F,
                   int64_t ldf, int64_t sF, const int *piv, zd *X, int64_t ldx, int64_t sX);

// U = sum_j w_j X_j  (n x m, node order j = 0..q-1).
int znode_sum(cudaStream_t s, int64_t n, int64_t m, int q, const zd *w, const zd *X,
              int64_t ldx, int64_t sX, zd *U, int64_t ldu);

// Thin QR by block classical Gram-Schmidt with re-orthogonalisation:
// V (n x m, overwritten by Q), R (m x m upper, real positive diagonal).
// timeout: flag raised if a grid barrier of the tall-panel form gives up
// oz (may be null): digit-plane scratch (rows >= oz_rows_bytes(n, m), cols
// >= oz_cols_bytes(m, 32)) to run the tall updates on the tensor cores.
struct OzScratch {
    void *rows, *cols;
    int *err;
};
// QR by Cholesky QR twice (k_chol.cu): V (n x m, ldv) <- Q, R (may be null)
// <- upper triangular with real positive diagonal.  Gram matrices and the
// products V R^{-1} on the tensor cores (oz.rows >= oz_rows_bytes(max(n, m),
// max(n, m)), oz.cols >= oz_cols_bytes(n, m)); Cholesky and triangular
// inverses FP64 (oz.rows null: every product an FP64 GEMM, through tmp,
// n x m).  *ok = 0 (V untouched) when a pivot shows cond(V) beyond
// reach (checked on the first factorisation); the caller then runs
// BCGS2.  work: zorth_chol_work_bytes(m).
// Ri (m x m, ld m) = R^{-1}, R upper triangular (ld ldr); recursive
// doubling over 32 x 32 diagonal blocks with batched FP64 GEMMs (k_chol.cu).
// T: tri_inverse_scratch_elems(m) entries.
size_t tri_inverse_scratch_elems(int m);
int tri_inverse(cudaStream_t s, int m, const zd *R, int64_t ldr, zd *Ri, zd *T);
size_t zorth_chol_work_bytes(int64_t m);
int zorth_chol(cudaStream_t s, int64_t n, int64_t m, zd *V, int64_t ldv, zd *R, int64_t ldr, void *work,
               const OzScratch &oz, int *ok, zd *tmp = nullptr);

int zorth(cudaStream_t s, int64_t n, int64_t m, zd *V, int64_t ldv, zd *R, int64_t ldr,
          zd *work, int *timeout, const OzScratch *oz = nullptr);
size_t zorth_work_elems(int64_t n, int64_t m);

// Batched projected eigensolve: alpha / beta eigenvalue pairs and unit right
// eigenvectors V of (A, B), B upper triangular.  m <= 64: QZ, one warp per
// pencil (A, B overwritten by the Schur form); m > 64: standard-form path
// of k_zeig.cu, pencil by pencil (A, B overwritten).  work: batch *
// zqz_work_bytes(m) bytes.  timeout (may be null): set if a grid barrier
// of the large path gave up.
size_t zqz_work_bytes(int m);
int zqz_batched(cudaStream_t s, int m, int batch, zd *A, int64_t lda, int64_t sA, zd *B,
                int64_t ldb, int64_t sB, zd *alpha, zd *beta, zd *V, int64_t ldv, int64_t sV,
                void *work, int *fail, int *timeout, int *stats = nullptr, double defl = 0.0);

// Large projected problems (k_zeig.cu): standard form, Hessenberg
// reduction and chunked QR; alpha = eigenvalue, beta = 1.
size_t zeig_large_work_bytes(int m);
// stats (may be null): stats[0] += QR sweeps, stats[1] += chase phases,
// stats[2] += early-deflation windows applied.
// defl: relative deflation tolerance of the QR (0: the double-single floor,
// 2^-44); a looser one when the eigenpairs are wanted to less accuracy.
int zeig_large(cudaStream_t s, int m, zd *A, zd *Bt, zd *alpha, zd *beta, zd *V, void *work,
               int *fail, int *timeout, int *stats = nullptr, double defl = 0.0);
// Schur form of a contiguous m x m matrix (k_zeig.cu): C <- T = Q^H C Q
// (upper triangle; Hessenberg reduction then the double-single QR), Q
// unitary.  work: schur_large_work_bytes(m).  hn_out (may be null): max
// |C_ij| of the Hessenberg matrix.
size_t schur_large_work_bytes(int m);
int schur_large(cudaStream_t s, int m, zd *C, zd *Q, void *work, int *fail, int *timeout, int *stats,
                double *hn_out, double defl = 0.0);
// Eigenvectors of the upper triangle of T (m x m), unit diagonal, by
// back-substitution; unit 2-norm columns.
// scratch: m x m (T transposed, for contiguous row reads).
int schur_vectors(cudaStream_t s, int m, const zd *T, zd *Y, double snorm, zd *scratch);
// The same Schur form with the QR in plain FP32 (k_zeig32.cu): Q unitary
// and T triangular to ~1e-6 relative -- a start for an FP64 polish.
// work: schur_large_work_bytes_fp32(m) (= schur_large_work_bytes(m)).
size_t schur_large_work_bytes_fp32(int m);
int schur_large_fp32(cudaStream_t s, int m, zd *C, zd *Q, void *work, int *fail, int *timeout, int *stats,
                     double *hn_out, double defl);
int normalise_cols(cudaStream_t s, int m, zd *V);

// SEARCH (k_search.cu): out = sum_j Re(y_j^H u_j) over p columns; the
// rank-revealing factorisation of an n x m block U (pivoted Cholesky of
// U^H U): *t = numerical rank at rank_tol, Q[:, :t] <- U[:, piv] R_t^{-1}
// (a basis of the selected columns' span, orthonormal to ~eps cond^2; U is
// left as it was).
int trace_real(cudaStream_t s, int64_t n, int p, const zd *Y, int64_t ldy, const zd *U, int64_t ldu, double *out);
// Block CIRR step 1 (k_cirr.cu): R[:, i h + c] = sum_j w_j ((z_j - centre) /
// scale)^i X_j[:, c] for i < g, c < h (X_j at stride sX, leading dim n).
int moment_sum(cudaStream_t s, int64_t n, int h, int q, int g, const zd *z, const zd *w, double cre, double cim,
               double scale, const zd *X, int64_t sX, zd *R, int64_t ldr);
size_t rrqr_work_bytes(int64_t n, int m);
int rrqr_basis(cudaStream_t s, int64_t n, int m, const zd *U, zd *Q, double rank_tol, void *work, int *timeout,
               int *t_out);

// Warm-started projected eigensolve (k_warm.cu).
struct WarmParams {
    int min_m;          // smallest m that tries it
    int min_tail;       // smallest trailing block given to the QR
    double tau;         // column of C counted converged: ||C[j+1:, j]|| <= tau max|C|
    double accept_tol;  // largest relative eigen-residual accepted
    double tail_defl;   // relative deflation tolerance of the tail QR (0: the floor)
    int cold_fp32;      // 1: no converged block assumed -- the whole matrix
                        // through the FP32 QR, its Schur vectors made unitary
                        // in FP64 (BCGS2), then the Newton step
};
struct WarmResult {
    int accepted;   // 1: alpha, beta, V hold the eigenpairs
    int k;          // converged leading columns found
    int tail;       // rows of the block given to the QR
    double resid;   // largest relative eigen-residual of the Newton step
};
size_t zeig_warm_work_bytes(int m);
// Events around the warm solve's FP64 product segments (GEMMs and
// triangular inverses), for the per-kernel roofline: pairs (begin, end) in
// ev[0 .. used), with the segments' algorithmic flops (complex MAC = 8).
struct GemmTimer {
    static constexpr int kMax = 10;
    cudaEvent_t ev[kMax];
    int used;
    double flops;
};
// A, Bt as zeig_large (both overwritten whether accepted or not).  qz_work:
// zeig_large_work_bytes(m) bytes.  gt (may be null): segment timer.
int zeig_warm(cudaStream_t s, int m, zd *A, zd *Bt, zd *alpha, zd *beta, zd *V, void *warm_work, void *qz_work,
              const WarmParams &prm, WarmResult *res, int *fail, int *timeout, int *stats, GemmTimer *gt = nullptr,
              const OzScratch *oz = nullptr);
// Line 16 on Ritz pairs in defect form (k_defect.cu):
// U = X rho(Lambda) + sum_j w_j M_j^{-1} (R D_j), R = A X - B X Lambda.
struct DefectScratch {
    cf *d32;     // q x m: 1 / (z_j - lambda_i) (1 for plain columns)
    zd *rho;     // m: rho(lambda_i) (0 for plain columns)
    int *plain;  // m: 1 when the column takes the plain right-hand side B x
    cf *S;       // n x m: R (or B X) rounded to complex64
};
int defect_prepare(cudaStream_t s, int64_t n, int m, int q, const zd *z, const zd *w, const zd *lam, double dmin,
                   const zd *AX, const zd *BX, DefectScratch &d);
// X_j (slot stride sX) = rows perm_j of S scaled by d_j (perm null: no interchange)
int defect_rhs(cudaStream_t s, int64_t n, int m, int q, const int *perm, const DefectScratch &d, cf *X, int64_t sX);
// U = sum_j w_j Y_j + X rho
int defect_sum(cudaStream_t s, int64_t n, int m, int q, const cf *Y, int64_t sY, const zd *w, const zd *X,
               const DefectScratch &d, zd *U);
// Vout[:, i] = Vin[:, perm[i]] (rows x m, leading dim rows).
int permute_cols(cudaStream_t s, int64_t rows, int m, const int *perm, const zd *Vin, zd *Vout);

// Composition of the LU interchanges: perm[b*n + i] = original row at i.
int zpiv_to_perm(cudaStream_t s, int64_t n, int batch, const int *piv, int *perm);
// X_b[i, :] = R[perm_b[i], :]
int zgather_rows(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const int *perm,
                 const zd *R, int64_t ldr, zd *X, int64_t ldx, int64_t sX);
// L then U solves of already-permuted right-hand sides (in place).
int ztrsm_lu_batched(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const zd *F,
                     int64_t ldf, int64_t sF, zd *X, int64_t ldx, int64_t sX);

// Residuals of eq. 5.1 for every Ritz pair.
int ritz_residuals(cudaStream_t s, int64_t n, int m, const zd *AX, const zd *BX, int64_t ld,
                   const zd *alpha, const zd *beta, zd *lam, double *res, DevStatus *st);
// Selection and stopping tests of GFEAST lines 7-15 (device side).
int stop_test(cudaStream_t s, int m, const feast_contour *c, const zd *lam, const double *res,
              double eta, double eps, int k, int max_iter, int c_prev, double e_prev, int converged_only,
              int *sel, int *idx, DevStatus *st);
// Accepted pairs to the front of Xc / lamc / resc.
int compact_pairs(cudaStream_t s, int64_t n, int m, const int *idx, const DevStatus *st,
                  const zd *X, int64_t ldx, const zd *lam, const double *res, zd *Xc, zd *lamc,
                  double *resc);

// Precision form (k_refine.cu).
int form_shifted32(cudaStream_t s, int64_t n, int q, const zd *A, const zd *B, int64_t ld, const zd *z, cf *M32);
int z2c(cudaStream_t s, int64_t count, const zd *x, cf *y);
int c2z(cudaStream_t s, int64_t count, const cf *x, zd *y);
int add_c32(cudaStream_t s, int64_t count, zd *x, const cf *c);
// out = ||x||^2 over count entries
int sumsq(cudaStream_t s, int64_t count, const zd *x, double *out);

// Banded pencils (k_band.cu): LAPACK general-band factor storage
// (ldab = 2 kl + ku + 1), unblocked-convention multipliers.
size_t gb_scratch_elems(int64_t kl, int64_t ku, int q);
size_t gb_piv_scratch(int64_t kl, int q);
template <typename T>
int gb_form(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const zd *A, const zd *B,
            int64_t ldin, int q, const zd *z, T *F);
template <typename T>
int gb_getrf(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, int q, T *F, int *piv, void *scratch,
             int *pivl, int *info, int *row);
// the largest dynamic shared memory a band solve of elements of es bytes
// needs (k_band.cu); it bounds the bandwidths the band path takes
size_t gb_solve_smem_bytes(int64_t kl, int64_t ku, size_t es);
constexpr size_t kSmemOptinMax = 227 * 1024;   // sm_100-family opt-in limit per CTA
template <typename T>
int gb_solve(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, int q, const T *F, const int *piv,
             int64_t nrhs, T *X, int64_t ldx, int64_t sX);
int gb_matmul(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const zd *M, int64_t ldin, int64_t m,
              const zd *X, zd *Y);
int gb_residual(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const zd *A, const zd *B,
                int64_t ldin, int q, const zd *z, int64_t m, const zd *RHS, const zd *X, zd *R,
                double *nrm2);
// B = I: the same residual with the band product A X_j in double-single
// arithmetic; Ads is A's band as packed (hi, lo) pairs (z2ds), Xds scratch
// for the split X (q n m entries).
int z2ds(cudaStream_t s, int64_t count, const zd *x, float4 *y);
int gb_residual_ds(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const float4 *Ads, int64_t ldin, int q,
                   const zd *z, int64_t m, const zd *RHS, const zd *X, float4 *Xds, zd *R, double *nrm2);

// CUDA events around the tensor-core GEMM launches of one phase (the
// set-up LU's trailing updates, or one pass's shifted solves) and their
// algorithmic flops (complex multiply-add = 8): each launch of k_tc_cgemm2
// records an event before and after itself while room is left.
struct TcTimer {
    static constexpr int kMax = 64;   // launches timed per phase
    cudaEvent_t ev[2 * kMax];
    int used;                         // events recorded
    double flops;
};
// Tensor-core complex64 GEMM (k_tc.cu): C_b = beta C_b + alpha A_b X_b on
// tcgen05 (kind::tf32, 3-pass split); scratch of tc_scratch_floats floats.
size_t tc_scratch_floats(int64_t m, int64_t k, int64_t n, int batch);
int tc_cgemm(cudaStream_t s, int64_t m, int64_t n, int64_t k, cf alpha, const cf *A, int64_t lda,
             int64_t sA, const cf *X, int64_t ldx, int64_t sX, cf beta, cf *C, int64_t ldc, int64_t sC,
             int batch, float *scratch, int *err, TcTimer *tt = nullptr);
// The same product with A's realified planes made beforehand
// (tc_prepare_A into tc_prepA_floats floats); scratch then only holds X's.
size_t tc_prepA_floats(int64_t m, int64_t k, int batch);
int tc_prepare_A(cudaStream_t s, int64_t m, int64_t k, const cf *A, int64_t lda, int64_t sA, int batch,
                 float *Aprep);
int tc_cgemm_prepA(cudaStream_t s, int64_t m, int64_t n, int64_t k, cf alpha, const float *Aprep, const cf *X,
                   int64_t ldx, int64_t sX, cf beta, cf *C, int64_t ldc, int64_t sC, int batch, float *scratch,
                   int *err, TcTimer *tt = nullptr);
// FP64-accurate complex GEMM on the bf16 tensor cores by exact base-64
// digit slicing (k_oz.cu): prepare digit planes of the left operand (rows)
// and the right operand (columns), then C = beta C + alpha_c A B with
// alpha_c = alpha * zcol[c / cblk] when zcol is given.
size_t oz_rows_bytes(int64_t M, int64_t K);
size_t oz_cols_bytes(int64_t K, int64_t N);
int oz_prepare_rows(cudaStream_t s, int64_t M, int64_t K, const zd *A, int64_t lda, void *work, int ct = 0);
int oz_prepare_cols(cudaStream_t s, int64_t K, int64_t N, const zd *B, int64_t ldb, void *work);
int oz_gemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, const void *Arows, const void *Bcols, zd alpha,
            const zd *zcol, int64_t cblk, zd beta, zd *C, int64_t ldc, int *err);
// R_j = BV - [xz] z_j X_j for every node j (X, R: n x (q m)); xz may be null.
int resid_init(cudaStream_t s, int64_t n, int64_t m, int q, const zd *BV, const zd *xz, const zd *z, zd *R);
// out[j] = ||x_j||_F^2 for q consecutive blocks of count entries.
int sumsq_blocks(cudaStream_t s, int64_t count, int q, const zd *x, double *out);

// Differentiation form (k_adjoint.cu): pair coefficients alpha_i, beta_i
// from c_i = v_{k_i}^H (B X)_i, and G_A = V_k diag(alpha) X^H, G_B likewise.
int adjoint_coef(cudaStream_t s, int64_t n, int cnt, const zd *V, int64_t ldv, const int *kidx, const zd *BX,
                 int64_t ldb, const zd *lam, zd *alpha, zd *beta);
int adjoint_grad(cudaStream_t s, int64_t n, int cnt, const zd *V, int64_t ldv, const int *kidx, const zd *X,
                 int64_t ldx, const zd *alpha, const zd *beta, zd *GA, zd *GB, int64_t ldg);

// complex64 LU whose trailing updates run on tc_cgemm (pivots and factors as
// getrf_batched<cf>); scratch of getrf_tc_scratch_floats floats.
size_t getrf_tc_scratch_floats(int64_t n, int batch);
// complex64 L U solve (permuted right-hand sides) whose off-block updates
// run on tc_cgemm; scratch as for getrf_batched_tc with nrhs <= n.
// cache (may be null): the factors' off-block panels prepared once by
// trsm_tc_cache_fill (trsm_tc_cache_floats floats), so that a solve only
// prepares its right-hand sides.
int trsm_lu_tc(cudaStream_t s, int64_t n, int64_t nrhs, int batch, const cf *F, int64_t ldf, int64_t sF, cf *X,
               int64_t ldx, int64_t sX, float *scratch, int *tc_err, const float *cache = nullptr,
               TcTimer *tt = nullptr);
size_t trsm_tc_cache_floats(int64_t n, int batch);
int trsm_tc_cache_fill(cudaStream_t s, int64_t n, int batch, const cf *F, int64_t ldf, int64_t sF, float *cache);
int getrf_batched_tc(cudaStream_t s, int64_t n, int batch, cf *F, int64_t ldf, int64_t sF, int *piv,
                     int *info, int *row, float *scratch, int *tc_err, TcTimer *tt = nullptr);

// Contour nodes / weights on the device.
int contour_nodes(cudaStream_t s, const feast_contour *c, zd *z, zd *w);

}  // namespace feast
