// C ABI of the GB300 FEAST library: context set-up (GFEAST lines 1-3 with a
// given start block), one pass of lines 5-17 per feast_iterate, the output
// of lines 13-15, and the standalone batched LU / solve / QZ entry points.
//
// All device memory is carved from one caller-provided workspace; the
// context record itself is the only host allocation.  Every step runs in
// this library's kernels on the caller's stream; the host only sequences
// launches and reads c(k), e(k) and the flag once per pass.
#include <algorithm>
#include <atomic>
#include <complex>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace feast;

namespace feast {
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static thread_local char g_cuda_error[256] = "";
int note_cuda_error(cudaError_t e, const char *file, int line)
{
    const char *base = strrchr(file, '/');
    snprintf(g_cuda_error, sizeof(g_cuda_error), "%s (%s:%d)", cudaGetErrorName(e), base ? base + 1 : file, line);
    return FEAST_ECUDA;
}
int note_timeout(int bits)
{
    static const char *const names[] = {"?", "k_hess_grid barrier", "k_hqr barrier", "k_chol_grid barrier",
                                        "k_cgs2_grid barrier", "k_pchol_grid barrier", "k_tc_cgemm2 producer",
                                        "k_tc_cgemm2 MMA", "k_tc_cgemm2 epilogue", "k_tc_cgemm2 drain",
                                        "k_oz_gemm"};
    int at = snprintf(g_cuda_error, sizeof(g_cuda_error), "bounded wait gave up (0x%x):", bits);
    for (int b = 0; b < 11 && at > 0 && at < (int)sizeof(g_cuda_error); ++b)
        if (bits & (1 << b))
            at += snprintf(g_cuda_error + at, sizeof(g_cuda_error) - at, " %s", names[b]);
    return FEAST_ETIMEOUT;
}
}  // namespace feast

struct feast_ctx {
    // problem
    int kind;
    int64_t n, kl, ku;
    int b_identity;
    int q, m0;          // q: nodes this context owns; m0: the active width (<= m0cap)
    int qall, j0;       // all nodes of the contour; the first node this context owns
    int m0cap;
    feast_contour contour;
    double eps, eta;
    int max_iter, prec, no_stop, converged_only;
    int projection;     // FEAST_OBLIQUE or FEAST_RAYLEIGH_RITZ
    cudaStream_t s;
    // device arrays
    zd *A, *B;          // n x n copies (B null when identity)
    zd *z, *w;          // this context's nodes and weights (zall + j0, wall + j0)
    zd *zall, *wall;    // every node and weight of the contour
    feast_collective_fn coll;   // node-sharded run: combines the ranks (null: all nodes here)
    void *coll_user;
    double *coll_buf;
    zd *F;              // q x n x n factors
    int *piv, *perm;    // q x n
    zd *Xs;             // q x n x m0 per-node solutions
    zd *U, *U1, *U2;    // n x m0
    zd *W;              // n x 2 m0 : [A U1 | B U1]
    zd *R1, *R2;        // m0 x m0
    zd *P;              // m0 x 2 m0 : [A~ | B~]
    zd *Q;              // m0 x 2 m0 : QZ working copy
    zd *Yv;             // m0 x m0 projected eigenvectors
    zd *alpha, *beta, *lam;
    zd *Xr;             // n x m0 Ritz vectors
    zd *AXBX;           // n x 2 m0 : [A X | B X]
    double *res;
    int *sel, *idx;
    zd *Xc[2], *lamc[2];
    double *resc[2];
    zd *Xo, *lamo;
    double *reso;
    zd *tmp;            // n x m0
    zd *orth_work;
    void *chol_work;    // Cholesky QR (dense precision form)
    void *search_work;  // SEARCH's rank-revealing factorisation
    void *qz_work;
    void *warm_work;    // warm-started projected eigensolve (m0 >= kWarmMinM)
    int *pair_perm;     // m0: order of the Ritz pairs (most converged next pass first)
    zd *ord_x, *ord_ab; // gather targets for X (n x m0) and [A X | B X] (n x 2 m0)
    DevStatus *st;
    // precision form
    cf *F32;            // q x n x n complex64 factors
    float *tcs;         // tensor-core LU operand scratch (complex64 dense)
    float *tcA;         // the factors' off-block panels as tensor-core operands (made once)
    float4 *Ads, *Xds;  // band A and the solutions as double-single pairs (banded precision form, B = I)
    void *ozA, *ozB;    // base-64 digit planes of A and B (refinement residual)
    void *ozX;          // digit planes of the q solution blocks, n x (q m0); right-operand scratch
    void *ozR;          // left-operand digit planes: U2^H, U1, A U1, B U1 (m0 x n or n x m0)
    OzScratch oz_orth;  // the same scratch, handed to the orthonormalisation
    cf *Xhi;            // q x n x m0 complex64 scratch (rounded residuals)
    cf *C32;            // q x n x m0 low-precision solves / corrections
    zd *R64;            // q x n x m0 residuals
    DefectScratch dfx;  // line 16 on Ritz pairs in defect form (precision form)
    double *nrm2;       // q + 1 squared norms
    int max_refine;
    double refine_tol;
    // banded pencils
    int64_t ldin, ldab;  // compact input / factor storage leading dims
    zd *Fb;             // q x ldab x n complex128 band factors (FP64)
    cf *Fb32;           // q x ldab x n complex64 band factors (precision form)
    void *gb_scratch;
    int *gb_pivl;
    int last_sweeps;
    double last_rel;
    float ms_refine;
    // host state
    double *zw_host;    // nodes and weights (2 q complex), for rho(lambda)
    int ritz_filter;    // line 16 of this pass filters the Ritz vectors
    int warm_ready;     // U1 comes from ordered Ritz vectors: line 6 may start warm
    WarmResult last_warm;
    int warm_tried;
    int cold_fp32;      // this pass: 1 FP32 QR + Newton accepted, -1 tried and not accepted
    int k, c_prev, done, cur;
    double e_prev;
    int out_count, out_flag, out_k;
    double out_err;
    cudaEvent_t ev[8];
    GemmTimer gt;       // the warm solve's FP64 product segments
    TcTimer tct;        // tensor-core GEMM launches: set-up LU updates, or one pass's solves
};

namespace {

// Projected problems this large take the warm-started solve (k_warm.cu)
// once a pass has ordered its Ritz pairs.
constexpr int kWarmMinM = 96;
constexpr int kWarmMinTail = 65;     // the QR's own size range (m > 64)
constexpr double kWarmTauMin = 1e-8; // converged column: strictly lower part <= tau max|C|
constexpr double kWarmAccMin = 1e-12;  // the cold double-single QR's own backward error (2^-44 of ||H||)
// A cold pass whose pairs are needed to at least this (relative eigen-
// residual) tries the FP32 QR polished by the Newton step first: from an
// FP32 Schur form (~1e-6 remainder) one Newton step reaches ~1e-10.
constexpr double kColdFp32AccMin = 1e-8;
constexpr int kZeigMinM = 8;         // smallest projected problem on the standard-form QR
// banded precision form: the n x m0 products go to the digit-sliced
// tensor-core GEMM from this width on (below it the FP64 GEMMs of the tall,
// skinny blocks were faster: at n = 16384, m0 = 64 the orthonormalisation
// took 9.8 ms per pass in FP64 and 16.8 ms on the digit slices)
constexpr int kBandOzMinM = 256;
constexpr double kZeigSmallEpsMin = 1e-10;   // ... when m0 <= 64: the strictest eps it serves

struct Carver {
    char *base;
    size_t off;
    bool dry;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = dry ? nullptr : reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

int validate(const feast_pencil *p, const feast_contour *c, const feast_options *o)
{
    if (!p || !c || !o) return FEAST_EINVAL;
    if (p->n < 1 || o->m0 < 1 || o->m0 > p->n || c->q < 1 || c->q > 4096) return FEAST_EINVAL;
    if (p->kind != FEAST_DENSE && p->kind != FEAST_BANDED) return FEAST_EINVAL;
    if (p->kind == FEAST_BANDED && (p->kl < 0 || p->ku < 0 || p->kl >= p->n || p->ku >= p->n ||
                                    p->ld < p->kl + p->ku + 1 || p->kl > 4096 || p->ku > 4096))
        return FEAST_EINVAL;
    if (o->prec != FEAST_FP64 && o->prec != FEAST_C64_REFINE) return FEAST_EINVAL;
    if (o->prec == FEAST_C64_REFINE && (o->max_refine < 0 || !(o->refine_tol > 0.0))) return FEAST_EINVAL;
    // the band solves keep a window of kl + ku + 2 right-hand-side rows and
    // one factor column in shared memory at the least: kl + ku up to ~7200
    // in FP64 (the precision form fits every band the limits above allow)
    if (p->kind == FEAST_BANDED &&
        gb_solve_smem_bytes(p->kl, p->ku, o->prec == FEAST_FP64 ? sizeof(zd) : sizeof(cf)) + 1024 > kSmemOptinMax)
        return FEAST_EINVAL;
    if (p->kind == FEAST_DENSE && p->ld < p->n) return FEAST_EINVAL;
    if (!(c->a > 0.0) || (c->kind == FEAST_ELLIPSE && !(c->b > 0.0))) return FEAST_EINVAL;
    if (c->kind != FEAST_CIRCLE && c->kind != FEAST_ELLIPSE) return FEAST_EINVAL;
    if (c->rule != FEAST_TRAPEZOID && c->rule != FEAST_GAUSS_LEGENDRE) return FEAST_EINVAL;
    if (o->max_iter < 1 || !(o->eta > 0.0)) return FEAST_EINVAL;
    if (o->projection != FEAST_OBLIQUE && o->projection != FEAST_RAYLEIGH_RITZ) return FEAST_EINVAL;
    if (!p->A || (!p->B && !p->b_is_identity) || !o->Y0) return FEAST_EINVAL;
    if (o->node_begin != 0 || o->node_end != 0) {
        // a range of nodes: the other ranks' partial sums come through the hook
        if (o->node_begin < 0 || o->node_end <= o->node_begin || o->node_end > c->q) return FEAST_EINVAL;
        if (!o->collective || !o->collective_buf || ((uintptr_t)o->collective_buf & 255u)) return FEAST_EINVAL;
    }
    return FEAST_OK;
}

void carve_defect(feast_ctx *c, Carver &cv)
{
    const size_t n = (size_t)c->n, m = (size_t)c->m0, q = (size_t)c->q;
    c->dfx.d32 = cv.take<cf>(q * m);
    c->dfx.rho = cv.take<zd>(m);
    c->dfx.plain = cv.take<int>(m);
    c->dfx.S = cv.take<cf>(n * m);
}

void carve(feast_ctx *c, Carver &cv)
{
    const size_t n = (size_t)c->n, m = (size_t)c->m0, q = (size_t)c->q;
    const size_t asz = (c->kind == FEAST_DENSE) ? n * n : (size_t)c->ldin * n;
    c->A = cv.take<zd>(asz);
    c->B = c->b_identity ? nullptr : cv.take<zd>(asz);
    c->zall = cv.take<zd>((size_t)c->qall);
    c->wall = cv.take<zd>((size_t)c->qall);
    c->z = c->zall ? c->zall + c->j0 : nullptr;
    c->w = c->wall ? c->wall + c->j0 : nullptr;
    if (c->kind == FEAST_BANDED) {
        const size_t fsz = q * (size_t)c->ldab * n;
        if (c->prec == FEAST_FP64) {
            c->Fb = cv.take<zd>(fsz);
            c->gb_scratch = cv.take<zd>(gb_scratch_elems(c->kl, c->ku, (int)q));
        } else {
            c->Fb32 = cv.take<cf>(fsz);
            c->gb_scratch = cv.take<cf>(gb_scratch_elems(c->kl, c->ku, (int)q));
            if (c->b_identity) {
                c->Ads = cv.take<float4>((size_t)c->ldin * n);
                c->Xds = cv.take<float4>(q * n * m);
            }
            c->C32 = cv.take<cf>(q * n * m);
            c->R64 = cv.take<zd>(q * n * m);
            c->nrm2 = cv.take<double>(q + 1);
            carve_defect(c, cv);
            if (m >= kBandOzMinM) {
                // digit planes for the n x m0 products (projection, Ritz
                // vectors, Cholesky QR, warm Newton step) on the tensor cores
                c->ozX = cv.take<char>(oz_cols_bytes((int64_t)n, (int64_t)(2 * m)));
                const size_t r1 = oz_rows_bytes((int64_t)m, (int64_t)n), r2 = oz_rows_bytes((int64_t)n, (int64_t)m);
                c->ozR = cv.take<char>(r1 > r2 ? r1 : r2);
            }
            // Cholesky QR twice (FP64 GEMMs below that width; BCGS2 as the
            // fallback when a pivot shows the block too ill-conditioned)
            c->chol_work = cv.take<char>(zorth_chol_work_bytes((int64_t)m));
        }
        c->gb_pivl = cv.take<int>(gb_piv_scratch(c->kl, (int)q));
    } else if (c->prec == FEAST_FP64) {
        c->F = cv.take<zd>(q * n * n);
    } else {
        c->F32 = cv.take<cf>(q * n * n);
        c->tcs = cv.take<float>(getrf_tc_scratch_floats((int64_t)n, (int)q));
        c->tcA = cv.take<float>(trsm_tc_cache_floats((int64_t)n, (int)q));
        c->ozA = cv.take<char>(oz_rows_bytes((int64_t)n, (int64_t)n));
        c->ozB = c->b_identity ? nullptr : cv.take<char>(oz_rows_bytes((int64_t)n, (int64_t)n));
        c->ozX = cv.take<char>(oz_cols_bytes((int64_t)n, (int64_t)(q * m)));
        {
            const size_t r1 = oz_rows_bytes((int64_t)m, (int64_t)n), r2 = oz_rows_bytes((int64_t)n, (int64_t)m);
            c->ozR = cv.take<char>(r1 > r2 ? r1 : r2);
        }
        c->Xhi = cv.take<cf>(q * n * m);
        c->chol_work = cv.take<char>(zorth_chol_work_bytes((int64_t)m));
        c->C32 = cv.take<cf>(q * n * m);
        c->R64 = cv.take<zd>(q * n * m);
        c->nrm2 = cv.take<double>(q + 1);
        carve_defect(c, cv);
    }
    c->piv = cv.take<int>(q * n);
    c->perm = cv.take<int>(q * n);
    c->Xs = cv.take<zd>(q * n * m);
    c->U = cv.take<zd>(n * m);
    c->U1 = cv.take<zd>(n * m);
    c->U2 = cv.take<zd>(n * m);
    c->W = cv.take<zd>(2 * n * m);
    c->R1 = cv.take<zd>(m * m);
    c->R2 = cv.take<zd>(m * m);
    c->P = cv.take<zd>(2 * m * m);
    c->Q = cv.take<zd>(2 * m * m);
    c->Yv = cv.take<zd>(m * m);
    c->alpha = cv.take<zd>(m);
    c->beta = cv.take<zd>(m);
    c->lam = cv.take<zd>(m);
    c->Xr = cv.take<zd>(n * m);
    c->AXBX = cv.take<zd>(2 * n * m);
    c->res = cv.take<double>(m);
    c->sel = cv.take<int>(m);
    c->idx = cv.take<int>(m);
    for (int i = 0; i < 2; ++i) {
        c->Xc[i] = cv.take<zd>(n * m);
        c->lamc[i] = cv.take<zd>(m);
        c->resc[i] = cv.take<double>(m);
    }
    c->Xo = cv.take<zd>(n * m);
    c->lamo = cv.take<zd>(m);
    c->reso = cv.take<double>(m);
    c->tmp = cv.take<zd>(n * m);
    c->orth_work = cv.take<zd>(zorth_work_elems((int64_t)n, (int64_t)m));
    c->qz_work = cv.take<char>(std::max(zqz_work_bytes((int)m), (zeig_large_work_bytes((int)m) + 255) & ~(size_t)255));
    c->search_work = cv.take<char>(rrqr_work_bytes((int64_t)n, (int)m));
    if ((int)m >= kWarmMinM) {
        c->warm_work = cv.take<char>(zeig_warm_work_bytes((int)m));
        c->pair_perm = cv.take<int>(m);
        c->ord_x = cv.take<zd>(n * m);
        c->ord_ab = cv.take<zd>(2 * n * m);
    }
    c->st = cv.take<DevStatus>(1);
}

void fill_ctx_params(feast_ctx *c, const feast_pencil *p, const feast_contour *ct,
                     const feast_options *o)
{
    c->kind = p->kind;
    c->n = p->n;
    c->kl = p->kind == FEAST_BANDED ? p->kl : 0;
    c->ku = p->kind == FEAST_BANDED ? p->ku : 0;
    c->ldin = c->kl + c->ku + 1;
    c->ldab = 2 * c->kl + c->ku + 1;
    c->b_identity = p->b_is_identity ? 1 : 0;
    c->qall = ct->q;
    const bool sharded = o->node_begin != 0 || o->node_end != 0;
    c->j0 = sharded ? o->node_begin : 0;
    c->q = sharded ? o->node_end - o->node_begin : ct->q;
    c->coll = sharded ? o->collective : nullptr;
    c->coll_user = sharded ? o->collective_user : nullptr;
    c->coll_buf = sharded ? (double *)o->collective_buf : nullptr;
    c->m0 = o->m0;
    c->m0cap = o->m0;
    c->contour = *ct;
    if (c->contour.kind == FEAST_CIRCLE) c->contour.b = c->contour.a;
    c->eps = o->eps;
    c->eta = o->eta;
    c->max_iter = o->max_iter;
    c->prec = o->prec;
    c->no_stop = o->no_stop;
    c->converged_only = o->converged_only;
    c->projection = o->projection;
    c->s = (cudaStream_t)o->stream;
    c->max_refine = o->max_refine;
    c->refine_tol = o->refine_tol;
}

const zd kOne = {1.0, 0.0}, kZero = {0.0, 0.0};

float ev_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
    return ms;
}

// Sum of the timed launches' durations (ms) of a TcTimer whose events have completed.
double tc_timer_ms(const TcTimer &t)
{
    double ms = 0.0;
    for (int i = 0; i + 1 < t.used; i += 2) ms += ev_ms(t.ev[i], t.ev[i + 1]);
    return ms;
}

// Node-sharded run: U (n x m0, this rank's partial quadrature sum over its
// own nodes) <- the sum of every rank's partial sum, through the caller's
// collective hook (a no-op when this context owns every node).
int collect_nodes(feast_ctx *c, zd *U)
{
    if (!c->coll) return FEAST_OK;
    const size_t nd = 2 * (size_t)c->n * (size_t)c->m0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->coll_buf, U, sizeof(double) * nd, cudaMemcpyDeviceToDevice, c->s));
    if (c->coll(c->coll_user, FEAST_COLL_SUM, c->coll_buf, (int64_t)nd, c->s)) return FEAST_ECUDA;
    FEAST_CUDA_TRY(cudaMemcpyAsync(U, c->coll_buf, sizeof(double) * nd, cudaMemcpyDeviceToDevice, c->s));
    return FEAST_OK;
}

// One host scalar through the hook (FEAST_COLL_SUM or FEAST_COLL_BCAST);
// synchronises the stream.
int collect_scalar(feast_ctx *c, int op, double *v)
{
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->coll_buf, v, sizeof(double), cudaMemcpyHostToDevice, c->s));
    if (c->coll(c->coll_user, op, c->coll_buf, 1, c->s)) return FEAST_ECUDA;
    FEAST_CUDA_TRY(cudaMemcpyAsync(v, c->coll_buf, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(c->s));
    return FEAST_OK;
}

// Y = B X (copy when B = I).  X, Y: n x m, leading dim n.
// Dense operands of the precision form: FP64-accurate products on the
// tensor cores (digit planes of the left operand made beforehand).
// products with the dense operators A, B on their digit planes
bool use_oz(const feast_ctx *c) { return c->kind == FEAST_DENSE && c->prec != FEAST_FP64; }
// the n x m0 and m0 x m0 products of the precision form (dense or band)
bool use_oz_small(const feast_ctx *c) { return c->prec != FEAST_FP64 && c->ozR && c->ozX; }

// Digit-plane scratch for the orthonormalisation's tall updates (precision form).
const OzScratch *orth_oz(feast_ctx *c)
{
    if (!use_oz_small(c)) return nullptr;
    c->oz_orth = OzScratch{c->ozR, c->ozX, &c->st->timeout};
    return &c->oz_orth;
}

// Y (M x N) = L X with L given by its digit planes (M x K), X (K x N, ldx).
int oz_mul(feast_ctx *c, const void *Lrows, int64_t M, int64_t K, const zd *X, int64_t ldx, int64_t N, zd *Y,
           int64_t ldy)
{
    int e;
    if ((e = oz_prepare_cols(c->s, K, N, X, ldx, c->ozX))) return e;
    return oz_gemm(c->s, M, N, K, Lrows, c->ozX, kOne, nullptr, 0, kZero, Y, ldy, &c->st->timeout);
}

int apply_B(feast_ctx *c, const zd *X, zd *Y, int64_t m)
{
    const int64_t n = c->n;
    if (c->b_identity) {
        FEAST_CUDA_TRY(cudaMemcpyAsync(Y, X, sizeof(zd) * n * m, cudaMemcpyDeviceToDevice, c->s));
        return FEAST_OK;
    }
    if (c->kind == FEAST_BANDED) return gb_matmul(c->s, n, c->kl, c->ku, c->B, c->ldin, m, X, Y);
    if (use_oz(c)) return oz_mul(c, c->ozB, n, n, X, n, m, Y, n);
    return zgemm_batched(c->s, 0, n, m, n, kOne, c->B, n, 0, X, n, 0, kZero, Y, n, 0, 1);
}

// Y = A X.
int apply_A(feast_ctx *c, const zd *X, zd *Y, int64_t m)
{
    const int64_t n = c->n;
    if (c->kind == FEAST_BANDED) return gb_matmul(c->s, n, c->kl, c->ku, c->A, c->ldin, m, X, Y);
    if (use_oz(c)) return oz_mul(c, c->ozA, n, n, X, n, m, Y, n);
    return zgemm_batched(c->s, 0, n, m, n, kOne, c->A, n, 0, X, n, 0, kZero, Y, n, 0, 1);
}

// X_j = RHS for every node (right-hand side shared by the band solves).
template <typename T>
int broadcast_rhs(feast_ctx *c, const T *rhs, T *X)
{
    const int64_t nm = c->n * c->m0;
    for (int j = 0; j < c->q; ++j)
        FEAST_CUDA_TRY(cudaMemcpyAsync(X + (int64_t)j * nm, rhs, sizeof(T) * nm, cudaMemcpyDeviceToDevice, c->s));
    return FEAST_OK;
}

// Shifted solves for banded pencils: X_j = (z_j B - A)^{-1} BV in FP64, or
// in complex64 with FP64-residual refinement (the band residual is cheap:
// 2 kl + ku + 1 products per entry).
int solve_band(feast_ctx *c, const zd *BV, double tol)
{
    const int64_t n = c->n, m = c->m0, q = c->q, nm = n * m, all = q * nm;
    cudaStream_t s = c->s;
    int e;
    if (c->prec == FEAST_FP64) {
        if ((e = broadcast_rhs<zd>(c, BV, c->Xs))) return e;
        return gb_solve<zd>(s, n, c->kl, c->ku, (int)q, c->Fb, c->piv, m, c->Xs, n, nm);
    }
    cf *rhs32 = c->C32;  // node 0's slot doubles as the rounded right-hand side
    if ((e = z2c(s, nm, BV, rhs32))) return e;
    for (int j = 1; j < q; ++j)
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->C32 + j * nm, rhs32, sizeof(cf) * nm, cudaMemcpyDeviceToDevice, s));
    if ((e = gb_solve<cf>(s, n, c->kl, c->ku, (int)q, c->Fb32, c->piv, m, c->C32, n, nm))) return e;
    if ((e = c2z(s, all, c->C32, c->Xs))) return e;
    c->last_sweeps = 0;
    c->last_rel = -1.0;
    c->ms_refine = 0.f;
    if (tol > 1e-6 || c->max_refine == 0) return FEAST_OK;
    cudaEvent_t e0 = c->ev[6], e1 = c->ev[7];
    FEAST_CUDA_TRY(cudaEventRecord(e0, s));
    if ((e = sumsq(s, nm, BV, c->nrm2 + q))) return e;
    double h[4096 + 1];
    for (int sweep = 0; sweep <= c->max_refine; ++sweep) {
        if (c->Ads) {
            if ((e = gb_residual_ds(s, n, c->kl, c->ku, c->Ads, c->ldin, (int)q, c->z, m, BV, c->Xs, c->Xds, c->R64,
                                    c->nrm2))) return e;
        } else if ((e = gb_residual(s, n, c->kl, c->ku, c->A, c->B, c->ldin, (int)q, c->z, m, BV, c->Xs, c->R64,
                                    c->nrm2))) {
            return e;
        }
        FEAST_CUDA_TRY(cudaMemcpyAsync(h, c->nrm2, sizeof(double) * (q + 1), cudaMemcpyDeviceToHost, s));
        FEAST_CUDA_TRY(cudaStreamSynchronize(s));
        double worst = 0.0;
        for (int j = 0; j < q; ++j) worst = h[j] > worst ? h[j] : worst;
        const double rel = h[q] > 0.0 ? sqrt(worst / h[q]) : 0.0;
        c->last_rel = rel;
        if (!(rel > tol) || sweep == c->max_refine) break;
        if ((e = z2c(s, all, c->R64, c->C32))) return e;
        if ((e = gb_solve<cf>(s, n, c->kl, c->ku, (int)q, c->Fb32, c->piv, m, c->C32, n, nm))) return e;
        if ((e = add_c32(s, all, c->Xs, c->C32))) return e;
        c->last_sweeps = sweep + 1;
    }
    FEAST_CUDA_TRY(cudaEventRecord(e1, s));
    FEAST_CUDA_TRY(cudaEventSynchronize(e1));
    c->ms_refine = ev_ms(e0, e1);
    return FEAST_OK;
}

// Shifted solves of the precision form: complex64 LU solves, then
// refinement sweeps X_j += M32_j^{-1} (R_j) with R_j = B V - M_j X_j formed
// FP64-accurately (its products A X and B X on the tensor cores, k_oz.cu)
// until max_j ||R_j||_F / ||B V||_F <= tol (or max_refine
// sweeps).  tol > 1e-6 (looser than what one complex64 solve reaches)
// skips the residual altogether.  Result: X_j (FP64) in c->Xs.
int solve_refine(feast_ctx *c, const zd *BV, double tol)
{
    const int64_t n = c->n, m = c->m0, q = c->q;
    const int64_t nm = n * m, all = q * nm;
    cudaStream_t s = c->s;
    int e;
    cf *rhs32 = c->Xhi;  // node 0's slot: rounded right-hand side before its gather
    if ((e = z2c(s, nm, BV, rhs32))) return e;
    if ((e = gather_rows<cf>(s, n, m, (int)q, c->perm, rhs32, n, 0, c->C32, n, nm))) return e;
    if ((e = trsm_lu_tc(s, n, m, (int)q, c->F32, n, n * n, c->C32, n, nm, c->tcs, &c->st->timeout, c->tcA,
                        &c->tct)))
        return e;
    if ((e = c2z(s, all, c->C32, c->Xs))) return e;
    c->last_sweeps = 0;
    c->last_rel = -1.0;
    c->ms_refine = 0.f;
    if (tol > 1e-6 || c->max_refine == 0) return FEAST_OK;
    cudaEvent_t e0 = c->ev[6], e1 = c->ev[7];
    FEAST_CUDA_TRY(cudaEventRecord(e0, s));
    if ((e = sumsq(s, nm, BV, c->nrm2 + q))) return e;
    double h[4096 + 1];
    for (int sweep = 0; sweep <= c->max_refine; ++sweep) {
        // R_j = B V - z_j (B X_j) + A X_j, FP64-accurate products on the tensor cores
        if ((e = resid_init(s, n, m, (int)q, BV, c->b_identity ? c->Xs : nullptr, c->z, c->R64))) return e;
        if ((e = oz_prepare_cols(s, n, q * m, c->Xs, n, c->ozX))) return e;
        if (!c->b_identity &&
            (e = oz_gemm(s, n, q * m, n, c->ozB, c->ozX, zmake(-1.0, 0.0), c->z, m, zmake(1.0, 0.0), c->R64, n,
                         &c->st->timeout)))
            return e;
        if ((e = oz_gemm(s, n, q * m, n, c->ozA, c->ozX, zmake(1.0, 0.0), nullptr, 0, zmake(1.0, 0.0), c->R64, n,
                         &c->st->timeout)))
            return e;
        if ((e = sumsq_blocks(s, nm, (int)q, c->R64, c->nrm2))) return e;
        FEAST_CUDA_TRY(cudaMemcpyAsync(h, c->nrm2, sizeof(double) * (q + 1), cudaMemcpyDeviceToHost, s));
        FEAST_CUDA_TRY(cudaStreamSynchronize(s));
        double worst = 0.0;
        for (int j = 0; j < q; ++j) worst = h[j] > worst ? h[j] : worst;
        const double rel = h[q] > 0.0 ? sqrt(worst / h[q]) : 0.0;
        c->last_rel = rel;
        if (!(rel > tol) || sweep == c->max_refine) break;  // also stops on NaN
        // correction: C_j = M32_j^{-1} R_j, X_j += C_j
        if ((e = z2c(s, all, c->R64, c->Xhi))) return e;
        if ((e = gather_rows<cf>(s, n, m, (int)q, c->perm, c->Xhi, n, nm, c->C32, n, nm))) return e;
        if ((e = trsm_lu_tc(s, n, m, (int)q, c->F32, n, n * n, c->C32, n, nm, c->tcs, &c->st->timeout, c->tcA))) return e;
        if ((e = add_c32(s, all, c->Xs, c->C32))) return e;
        c->last_sweeps = sweep + 1;
    }
    FEAST_CUDA_TRY(cudaEventRecord(e1, s));
    FEAST_CUDA_TRY(cudaEventSynchronize(e1));
    c->ms_refine = ev_ms(e0, e1);
    return FEAST_OK;
}

// U = sum_j w_j (z_j B - A)^{-1} B V   (eq. 4.1 - 4.2).  tol applies to the
// precision form only.
// X_j = M_j^{-1} RHS for every node j into c->Xs (stride n m0), the
// precision form refined to tol.
int solve_nodes(feast_ctx *c, const zd *rhs, double tol)
{
    const int64_t n = c->n, m = c->m0;
    if (c->kind == FEAST_BANDED) return solve_band(c, rhs, tol);
    if (c->prec != FEAST_FP64) return solve_refine(c, rhs, tol);
    int e;
    if ((e = zgather_rows(c->s, n, m, c->q, c->perm, rhs, n, c->Xs, n, n * m))) return e;
    return ztrsm_lu_batched(c->s, n, m, c->q, c->F, n, n * n, c->Xs, n, n * m);
}

int filter(feast_ctx *c, const zd *V, zd *Uout, double tol)
{
    const int64_t n = c->n, m = c->m0;
    int e;
    if ((e = apply_B(c, V, c->tmp, m))) return e;
    if ((e = solve_nodes(c, c->tmp, tol))) return e;
    if ((e = znode_sum(c->s, n, m, c->q, c->w, c->Xs, n, n * m, Uout, n))) return e;
    return collect_nodes(c, Uout);
}

// Line 16 of the precision form on the Ritz block X = c->Xr with Ritz
// values c->lam (k_defect.cu): U = X rho(Lambda) + sum_j w_j M_j^{-1}
// (R D_j), R = A X - B X Lambda from the products of line 9 (c->AXBX).
// The complex64 solves see only R, so no refinement sweeps are needed.
int filter_defect(feast_ctx *c, zd *Uout)
{
    const int64_t n = c->n, m = c->m0, q = c->q, nm = n * m;
    cudaStream_t s = c->s;
    int e;
    const double dmin = 1e-6 * fmin(c->contour.a, c->contour.b);
    if ((e = defect_prepare(s, n, (int)m, (int)q, c->z, c->w, c->lam, dmin, c->AXBX, c->AXBX + nm, c->dfx)))
        return e;
    if (c->kind == FEAST_BANDED) {
        if ((e = defect_rhs(s, n, (int)m, (int)q, nullptr, c->dfx, c->C32, nm))) return e;
        if ((e = gb_solve<cf>(s, n, c->kl, c->ku, (int)q, c->Fb32, c->piv, m, c->C32, n, nm))) return e;
    } else {
        if ((e = defect_rhs(s, n, (int)m, (int)q, c->perm, c->dfx, c->C32, nm))) return e;
        if ((e = trsm_lu_tc(s, n, m, (int)q, c->F32, n, n * n, c->C32, n, nm, c->tcs, &c->st->timeout, c->tcA,
                            &c->tct)))
            return e;
    }
    c->last_sweeps = 0;
    c->last_rel = -1.0;
    c->ms_refine = 0.f;
    if ((e = defect_sum(s, n, (int)m, (int)q, c->C32, nm, c->w, c->Xr, c->dfx, Uout))) return e;
    return collect_nodes(c, Uout);
}

// V = Q R in place (n x m0).  Dense precision form: Cholesky QR twice on
// the tensor-core products (k_chol.cu), BCGS2 if V is too ill-conditioned
// for it; otherwise BCGS2 (k_zorth.cu).  want_r false: only Q is needed (R
// may be left unset; it is scratch for BCGS2).
int orth_block(feast_ctx *c, zd *V, zd *R, bool want_r = true)
{
    const int64_t n = c->n, m = c->m0;
    int e;
    if (c->chol_work) {
        int ok = 0;
        const OzScratch *oz = orth_oz(c);
        const OzScratch none{nullptr, nullptr, &c->st->timeout};
        if ((e = zorth_chol(c->s, n, m, V, n, want_r ? R : nullptr, m, c->chol_work, oz ? *oz : none, &ok,
                            c->tmp)))
            return e;
        if (ok) return FEAST_OK;
    }
    return zorth(c->s, n, m, V, n, R, m, c->orth_work, &c->st->timeout, orth_oz(c));
}

// U1 R1 = U ; W[:, m0:] = B U1 ; U2 R2 = B U1   (GFEAST lines 2, 17; the
// Rayleigh-Ritz projection has no test basis to build)
int orthonormalise(feast_ctx *c, const zd *Usrc)
{
    const int64_t n = c->n, m = c->m0;
    int e;
    if (Usrc != c->U1)
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->U1, Usrc, sizeof(zd) * n * m, cudaMemcpyDeviceToDevice, c->s));
    if ((e = orth_block(c, c->U1, c->R1, false))) return e;   // (only U1's span and order are used)
    zd *BU1 = c->W + n * m;
    if ((e = apply_B(c, c->U1, BU1, m))) return e;
    if (c->projection == FEAST_RAYLEIGH_RITZ) return FEAST_OK;
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->U2, BU1, sizeof(zd) * n * m, cudaMemcpyDeviceToDevice, c->s));
    return orth_block(c, c->U2, c->R2);
}

}  // namespace

extern "C" {

int feast_workspace_size(const feast_pencil *pencil, const feast_contour *contour,
                         const feast_options *opts, size_t *bytes)
{
    int e = validate(pencil, contour, opts);
    if (e) return e;
    if (!bytes) return FEAST_EINVAL;
    feast_ctx c;
    memset(&c, 0, sizeof(c));
    fill_ctx_params(&c, pencil, contour, opts);
    Carver cv{nullptr, 0, true};
    carve(&c, cv);
    *bytes = cv.off + 256;
    return FEAST_OK;
}

int feast_setup(feast_ctx **out, const feast_pencil *pencil, const feast_contour *contour,
                const feast_options *opts, void *workspace, size_t workspace_bytes,
                feast_iter_info *info)
{
    if (!out) return FEAST_EINVAL;
    *out = nullptr;
    int e = validate(pencil, contour, opts);
    if (e) return e;
    size_t need = 0;
    feast_workspace_size(pencil, contour, opts, &need);
    if (!workspace || workspace_bytes < need) return FEAST_ENOMEM;
    if (((uintptr_t)workspace & 255u) != 0) return FEAST_EINVAL;
    feast_ctx *c = (feast_ctx *)calloc(1, sizeof(feast_ctx));
    if (!c) return FEAST_ENOMEM;
    fill_ctx_params(c, pencil, contour, opts);
    Carver cv{(char *)workspace, 0, false};
    carve(c, cv);
    for (int i = 0; i < 8; ++i)
        if (cudaEventCreate(&c->ev[i]) != cudaSuccess) { feast_destroy(c); return FEAST_ECUDA; }
    for (int i = 0; i < GemmTimer::kMax; ++i)
        if (cudaEventCreate(&c->gt.ev[i]) != cudaSuccess) { feast_destroy(c); return FEAST_ECUDA; }
    if (c->kind == FEAST_DENSE && c->prec != FEAST_FP64)
        for (int i = 0; i < 2 * TcTimer::kMax; ++i)
            if (cudaEventCreate(&c->tct.ev[i]) != cudaSuccess) { feast_destroy(c); return FEAST_ECUDA; }
    const int64_t n = c->n;
    cudaStream_t s = c->s;
#define TRY(x) do { int _r = (x); if (_r) { feast_destroy(c); return _r; } } while (0)
#define CTRY(x) do { if ((x) != cudaSuccess) { feast_destroy(c); return FEAST_ECUDA; } } while (0)
    CTRY(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
    const int64_t rowsA = (c->kind == FEAST_DENSE) ? n : c->ldin;
    CTRY(cudaMemcpy2DAsync(c->A, rowsA * sizeof(zd), pencil->A, pencil->ld * sizeof(zd), rowsA * sizeof(zd), n,
                           cudaMemcpyDeviceToDevice, s));
    if (!c->b_identity)
        CTRY(cudaMemcpy2DAsync(c->B, rowsA * sizeof(zd), pencil->B, pencil->ld * sizeof(zd), rowsA * sizeof(zd), n,
                               cudaMemcpyDeviceToDevice, s));
    CTRY(cudaEventRecord(c->ev[0], s));
    TRY(contour_nodes(s, &c->contour, c->zall, c->wall));
    c->zw_host = (double *)malloc(sizeof(double) * 4 * (size_t)c->qall);
    if (!c->zw_host) {
        feast_destroy(c);
        return FEAST_EINVAL;
    }
    CTRY(cudaMemcpyAsync(c->zw_host, c->zall, sizeof(zd) * c->qall, cudaMemcpyDeviceToHost, s));
    CTRY(cudaMemcpyAsync(c->zw_host + 2 * c->qall, c->wall, sizeof(zd) * c->qall, cudaMemcpyDeviceToHost, s));
    // z_j B - A and its LU factors (factored once, reused every pass)
    if (c->kind == FEAST_BANDED) {
        if (c->prec == FEAST_FP64) {
            TRY(gb_form<zd>(s, n, c->kl, c->ku, c->A, c->B, c->ldin, c->q, c->z, c->Fb));
            TRY(gb_getrf<zd>(s, n, c->kl, c->ku, c->q, c->Fb, c->piv, c->gb_scratch, c->gb_pivl,
                             &c->st->lu_info, &c->st->lu_row));
        } else {
            TRY(gb_form<cf>(s, n, c->kl, c->ku, c->A, c->B, c->ldin, c->q, c->z, c->Fb32));
            if (c->Ads) TRY(z2ds(s, c->ldin * n, c->A, c->Ads));
            TRY(gb_getrf<cf>(s, n, c->kl, c->ku, c->q, c->Fb32, c->piv, c->gb_scratch, c->gb_pivl,
                             &c->st->lu_info, &c->st->lu_row));
        }
    } else if (c->prec == FEAST_FP64) {
        TRY(zform_shifted(s, n, c->q, c->A, c->B, n, c->z, c->F, n, n * n));
        TRY(zgetrf_batched(s, n, c->q, c->F, n, n * n, c->piv, &c->st->lu_info, &c->st->lu_row));
    } else {
        TRY(form_shifted32(s, n, c->q, c->A, c->B, n, c->z, c->F32));
        TRY(oz_prepare_rows(s, n, n, c->A, n, c->ozA));
        if (!c->b_identity) TRY(oz_prepare_rows(s, n, n, c->B, n, c->ozB));
        c->tct.used = 0;
        c->tct.flops = 0.0;
        TRY(getrf_batched_tc(s, n, c->q, c->F32, n, n * n, c->piv, &c->st->lu_info, &c->st->lu_row, c->tcs,
                             &c->st->timeout, &c->tct));
        TRY(trsm_tc_cache_fill(s, n, c->q, c->F32, n, n * n, c->tcA));
    }
    if (c->kind == FEAST_DENSE) TRY(zpiv_to_perm(s, n, c->q, c->piv, c->perm));
    CTRY(cudaEventRecord(c->ev[1], s));
    if (c->coll) {
        // every rank learns whether any rank's factors failed before the
        // first collective of the subspace build
        DevStatus hl;
        CTRY(cudaMemcpyAsync(&hl, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
        CTRY(cudaStreamSynchronize(s));
        double bad = (hl.timeout ? 1000.0 : 0.0) + (hl.lu_info ? 1.0 : 0.0);
        TRY(collect_scalar(c, FEAST_COLL_SUM, &bad));
        if (bad > 0.0) {
            if (info) {
                memset(info, 0, sizeof(*info));
                info->flag = 2;
                info->bad_node = hl.lu_info ? hl.lu_info + c->j0 : 0;
            }
            feast_destroy(c);
            return bad >= 1000.0 ? note_timeout(hl.timeout) : FEAST_ESINGULAR;
        }
    }
    // first subspace U = Q Y0, then U1, U2
    TRY(filter(c, (const zd *)opts->Y0, c->U, 1.0));
    TRY(orthonormalise(c, c->U));
    CTRY(cudaEventRecord(c->ev[2], s));
    DevStatus hs;
    CTRY(cudaMemcpyAsync(&hs, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CTRY(cudaStreamSynchronize(s));
    if (info) {
        memset(info, 0, sizeof(*info));
        info->ms_lu = ev_ms(c->ev[0], c->ev[1]);
        info->ms_solve = ev_ms(c->ev[1], c->ev[2]);
        // the LU's trailing updates on the tensor cores (k_tc_cgemm2 launches only)
        info->ms_tc_gemm = tc_timer_ms(c->tct);
        info->tc_gemm_flop = c->tct.used >= 2 ? c->tct.flops : 0.0;
        info->flag = 2;
        info->bad_node = hs.lu_info ? hs.lu_info + c->j0 : 0;
    }
    if (hs.lu_info) {
        feast_destroy(c);
        return FEAST_ESINGULAR;
    }
    if (hs.timeout) {
        feast_destroy(c);
        return note_timeout(hs.timeout);
    }
    c->k = 0;
    c->c_prev = 0;
    c->e_prev = 0.0;
    c->done = 0;
    c->cur = 0;
    *out = c;
    return FEAST_OK;
#undef TRY
#undef CTRY
}

// Ritz pairs ordered by the residual they are expected to have after the
// next filter application, r_i / |rho(lambda_i)| (r_i of eq. 5.1, rho the
// filter of eq. 4.1: an eigenvector x gives sum_j w_j (z_j B - A)^{-1} B x
// = rho(lambda) x, so a pair's residual shrinks by |rho(lambda_{m0+1})| /
// |rho(lambda_i)| per pass).  The columns of X and [A X | B X] are gathered
// on the device, lambda and r re-uploaded; lines 7-15 of this pass have
// already used them, line 16 uses the new order.
static int order_pairs(feast_ctx *c)
{
    const int m = c->m0, q = c->qall;   // the whole contour's filter rho
    const int64_t n = c->n;
    cudaStream_t s = c->s;
    std::vector<double> lam(2 * (size_t)m), res(m), key(m), lam2(2 * (size_t)m), res2(m);
    std::vector<int> perm(m);
    FEAST_CUDA_TRY(cudaMemcpyAsync(lam.data(), c->lam, sizeof(zd) * m, cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaMemcpyAsync(res.data(), c->res, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    const double *zh = c->zw_host, *wh = c->zw_host + 2 * q;
    for (int i = 0; i < m; ++i) {
        const std::complex<double> l(lam[2 * i], lam[2 * i + 1]);
        std::complex<double> r(0.0, 0.0);
        for (int j = 0; j < q; ++j)
            r += std::complex<double>(wh[2 * j], wh[2 * j + 1]) / (std::complex<double>(zh[2 * j], zh[2 * j + 1]) - l);
        const double a = std::abs(r);
        key[i] = (a > 0.0) ? res[i] / a : 1e300;
        if (!(key[i] == key[i])) key[i] = 1e300;
    }
    for (int i = 0; i < m; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return key[x] < key[y]; });
    for (int i = 0; i < m; ++i) {
        lam2[2 * i] = lam[2 * perm[i]];
        lam2[2 * i + 1] = lam[2 * perm[i] + 1];
        res2[i] = res[perm[i]];
    }
    // (pageable host-to-device copies are staged before cudaMemcpyAsync
    // returns, so the vectors may go out of scope)
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->pair_perm, perm.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->lam, lam2.data(), sizeof(zd) * m, cudaMemcpyHostToDevice, s));
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->res, res2.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    int e;
    if ((e = permute_cols(s, n, m, c->pair_perm, c->Xr, c->ord_x))) return e;
    if ((e = permute_cols(s, n, m, c->pair_perm, c->AXBX, c->ord_ab))) return e;
    if ((e = permute_cols(s, n, m, c->pair_perm, c->AXBX + n * m, c->ord_ab + n * m))) return e;
    std::swap(c->Xr, c->ord_x);
    std::swap(c->AXBX, c->ord_ab);
    c->ritz_filter = 1;
    return FEAST_OK;
}

// Rayleigh-Ritz: B~ = U1^H B U1 is a full matrix, while both projected
// solvers take B~ upper triangular (as the oblique projection's R2).  With
// B~ = Q_b R_b the pencil (Q_b^H A~, R_b) has the same eigenpairs.  Works on
// c->Q = [A~ | B~]; R2 (no test basis under Rayleigh-Ritz) holds R_b.
int triangularise_bt(feast_ctx *c)
{
    const int64_t m = c->m0;
    cudaStream_t s = c->s;
    zd *At = c->Q, *Bt = c->Q + m * m;
    int e;
    if ((e = zorth(s, m, m, Bt, m, c->R2, m, c->orth_work, &c->st->timeout, nullptr))) return e;
    // A~ <- Q_b^H A~ (through the residual buffer as scratch: m <= n)
    if ((e = zgemm_batched(s, 1, m, m, m, kOne, Bt, m, 0, c->P, m, 0, kZero, c->AXBX, m, 0, 1))) return e;
    FEAST_CUDA_TRY(cudaMemcpyAsync(At, c->AXBX, sizeof(zd) * m * m, cudaMemcpyDeviceToDevice, s));
    FEAST_CUDA_TRY(cudaMemcpyAsync(Bt, c->R2, sizeof(zd) * m * m, cudaMemcpyDeviceToDevice, s));
    return FEAST_OK;
}

static int iterate_impl(feast_ctx *c, feast_iter_info *info);

int feast_iterate(feast_ctx *c, feast_iter_info *info)
{
    try {   // no C++ exception (a host allocation) may cross the C boundary
        return iterate_impl(c, info);
    } catch (...) {
        return FEAST_ENOMEM;
    }
}

static int iterate_impl(feast_ctx *c, feast_iter_info *info)
{
    if (!c) return FEAST_EINVAL;
    if (c->done && !c->no_stop) return FEAST_EDONE;
    const int64_t n = c->n, m = c->m0;
    cudaStream_t s = c->s;
    int e;
    c->k += 1;
    FEAST_CUDA_TRY(cudaEventRecord(c->ev[0], s));
    // line 5: [A~ | B~] = T^H [A U1 | B U1] with the test basis T = U2
    // (oblique, eq. 3.10) or T = U1 (Rayleigh-Ritz, Algorithm FEAST); B U1 is
    // already in W[:, m0:]
    const bool rr = c->projection == FEAST_RAYLEIGH_RITZ;
    const zd *Tb = rr ? c->U1 : c->U2;
    if ((e = apply_A(c, c->U1, c->W, m))) return e;
    if (use_oz_small(c)) {
        if ((e = oz_prepare_rows(s, m, n, Tb, n, c->ozR, 1))) return e;
        if ((e = oz_mul(c, c->ozR, m, n, c->W, n, 2 * m, c->P, m))) return e;
    } else if ((e = zgemm_batched(s, 1, m, 2 * m, n, kOne, Tb, n, 0, c->W, n, 0, kZero, c->P, m, 0, 1))) {
        return e;
    }
    FEAST_CUDA_TRY(cudaEventRecord(c->ev[1], s));
    // line 6: projected eigenpairs, x_i = U1 y_i
    FEAST_CUDA_TRY(cudaMemsetAsync(&c->st->qz_sweeps, 0, 3 * sizeof(int), s));
    c->last_warm = WarmResult{};
    c->gt.used = 0;
    c->gt.flops = 0.0;
    c->warm_tried = c->warm_ready;
    c->cold_fp32 = 0;
    // the projected solve is held to 1e-3 of the accuracy already reached
    // (eta before any pair is accepted)
    const double eref = (c->c_prev > 0 && c->e_prev > 0.0) ? c->e_prev : c->eta;
    // (a pass at max_iter returns its pairs whatever the tests say: full
    // accuracy, as at any pass that may stop)
    const bool final_pass = c->k >= c->max_iter && !c->no_stop;
    const double acc = final_pass ? kWarmAccMin : fmax(kWarmAccMin, 1e-3 * eref);
    if (c->warm_ready) {
        // the previous pass filtered its |rho|-ordered Ritz vectors: C is
        // block upper triangular up to a remainder of the size of its
        // residuals.  A converged column's remainder enters the Newton step
        // squared over an eigenvalue gap (~1e-3 of max|C| and up):
        // tau^2 / 1e-3 <= tol
        const double tau = fmin(1e-5, fmax(kWarmTauMin, sqrt(1e-3 * acc)));
        // the tail QR deflates at 1e-3 of the acceptance tolerance, and at
        // most at 1e-2 eps: its backward error (~ the deflation times
        // max|C|) then stays far below the residual a stop needs
        const WarmParams prm{kWarmMinM, kWarmMinTail, tau, acc, fmin(1e-3 * acc, 1e-2 * c->eps), 0};
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->Q, c->P, sizeof(zd) * 2 * m * m, cudaMemcpyDeviceToDevice, s));
        // (the Newton step's defect-form products on the digit-sliced
        // tensor-core GEMM where the context has its scratch)
        if ((e = zeig_warm(s, (int)m, c->Q, c->Q + m * m, c->alpha, c->beta, c->Yv, c->warm_work, c->qz_work, prm,
                           &c->last_warm, &c->st->qz_fail, &c->st->timeout, &c->st->qz_sweeps, &c->gt, orth_oz(c))))
            return e;
        if (!c->last_warm.accepted) FEAST_CUDA_TRY(cudaMemsetAsync(&c->st->qz_fail, 0, sizeof(int), s));
    }
    if (!c->last_warm.accepted && !rr && c->warm_work && acc >= kColdFp32AccMin) {
        // cold, but the pairs are needed only to acc: the Schur form of the
        // whole matrix by the FP32 QR (its rotation chains are shorter),
        // made exact by the FP64 Newton step -- whose error, the square of
        // the FP32 remainder over an eigenvalue gap, is far below acc
        // (its products on the digit-sliced tensor-core GEMM where the
        // context has the scratch: ~48-bit per row and column, far beyond acc)
        const WarmParams prm{kWarmMinM, kWarmMinTail, kWarmTauMin, acc, 0.0, 1};
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->Q, c->P, sizeof(zd) * 2 * m * m, cudaMemcpyDeviceToDevice, s));
        if ((e = zeig_warm(s, (int)m, c->Q, c->Q + m * m, c->alpha, c->beta, c->Yv, c->warm_work, c->qz_work, prm,
                           &c->last_warm, &c->st->qz_fail, &c->st->timeout, &c->st->qz_sweeps, &c->gt, orth_oz(c))))
            return e;
        c->cold_fp32 = c->last_warm.accepted ? 1 : -1;
        if (!c->last_warm.accepted) FEAST_CUDA_TRY(cudaMemsetAsync(&c->st->qz_fail, 0, sizeof(int), s));
    }
    if (!c->last_warm.accepted) {
        // before any pair has been accepted the stop cannot fire at this
        // pass (lines 13-14 need a fixed non-zero count), so unless it is
        // the last pass (max_iter) its eigenpairs are needed only far
        // beyond their residuals (>= eta): the QR deflates at 1e-8.  Any
        // pass that may stop deflates at the double-single floor, so that
        // its pairs reach eps.
        const double defl = (c->c_prev > 0 || final_pass) ? 0.0 : 1e-8;
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->Q, c->P, sizeof(zd) * 2 * m * m, cudaMemcpyDeviceToDevice, s));
        if (rr && (e = triangularise_bt(c))) return e;
        // B~ is upper triangular here (R2, or made so for Rayleigh-Ritz):
        // the standard-form QR on the FP32 pipe (double-single) from m =
        // kZeigMinM up (GB300's FP64 pipe made the FP64 QZ ~50 ms at m0 =
        // 64); a small problem keeps the FP64 QZ when eps is within ~1000x
        // of the double-single QR's backward error (2^-44 of ||C||), so
        // that e(k) can still fall below eps
        if (m > 64 || (m >= kZeigMinM && c->eps >= kZeigSmallEpsMin))
            e = zeig_large(s, (int)m, c->Q, c->Q + m * m, c->alpha, c->beta, c->Yv, c->qz_work, &c->st->qz_fail,
                           &c->st->timeout, &c->st->qz_sweeps, defl);
        else
            e = zqz_batched(s, (int)m, 1, c->Q, m, 0, c->Q + m * m, m, 0, c->alpha, c->beta, c->Yv, m, 0,
                            c->qz_work, &c->st->qz_fail, &c->st->timeout, &c->st->qz_sweeps, defl);
        if (e) return e;
    }
    FEAST_CUDA_TRY(cudaEventRecord(c->ev[2], s));
    if (use_oz_small(c)) {
        // x_i = U1 y_i, A x_i = (A U1) y_i, B x_i = (B U1) y_i with Y's digits made once
        if ((e = oz_prepare_cols(s, m, m, c->Yv, m, c->ozX))) return e;
        const zd *lhs[3] = {c->U1, c->W, c->W + n * m};
        zd *dst[3] = {c->Xr, c->AXBX, c->AXBX + n * m};
        for (int t = 0; t < 3; ++t) {
            if ((e = oz_prepare_rows(s, n, m, lhs[t], n, c->ozR))) return e;
            if ((e = oz_gemm(s, n, m, m, c->ozR, c->ozX, kOne, nullptr, 0, kZero, dst[t], n, &c->st->timeout)))
                return e;
        }
    } else {
        if ((e = zgemm_batched(s, 0, n, m, m, kOne, c->U1, n, 0, c->Yv, m, 0, kZero, c->Xr, n, 0, 1))) return e;
        // A x_i = (A U1) y_i, B x_i = (B U1) y_i
        if ((e = zgemm_batched(s, 0, n, m, m, kOne, c->W, n, n * m, c->Yv, m, 0, kZero, c->AXBX, n, n * m, 2)))
            return e;
    }
    // lines 7-12: residuals (eq. 5.1), selection, c(k), e(k); lines 13-15
    if ((e = ritz_residuals(s, n, (int)m, c->AXBX, c->AXBX + n * m, n, c->alpha, c->beta, c->lam, c->res, c->st))) return e;
    if ((e = stop_test(s, (int)m, &c->contour, c->lam, c->res, c->eta, c->eps, c->k, c->max_iter, c->c_prev,
                       c->e_prev, c->converged_only, c->sel, c->idx, c->st))) return e;
    if ((e = compact_pairs(s, n, (int)m, c->idx, c->st, c->Xr, n, c->lam, c->res, c->Xc[c->cur], c->lamc[c->cur],
                           c->resc[c->cur]))) return e;
    // the precision form always filters the Ritz pairs (defect form); the
    // pairs are ordered when the next pass may solve warm
    c->ritz_filter = (c->prec != FEAST_FP64);
    if (!rr && c->pair_perm && m >= kWarmMinM && (e = order_pairs(c))) return e;
    FEAST_CUDA_TRY(cudaEventRecord(c->ev[3], s));
    // lines 16-17, issued before the flag is read back so that the whole pass
    // is one stream-ordered sequence; when a stop fires the new subspace is
    // simply not used (the stopped pairs were compacted above).
    // line 16.  Precision form: on the Ritz pairs in defect form (no
    // refinement sweeps; the solves see only the residual block).  FP64: on
    // U1, or on the |rho|-ordered Ritz vectors when the next pass may solve
    // warm (the same subspace, x_i = U1 y_i, in a basis whose leading
    // columns converge first).
    // (a pass at max_iter stops whatever the tests say: no next subspace)
    const bool last = c->k >= c->max_iter && !c->no_stop;
    c->tct.used = 0;
    c->tct.flops = 0.0;
    if (!last) {
        if (c->prec != FEAST_FP64) e = filter_defect(c, c->U);
        else e = filter(c, c->ritz_filter ? c->Xr : c->U1, c->U, 1.0);
        if (e) return e;
    }
    // (the warm solve relies on B~ = R2 being upper triangular: oblique only)
    c->warm_ready = !rr && c->ritz_filter && c->pair_perm && m >= kWarmMinM;
    FEAST_CUDA_TRY(cudaEventRecord(c->ev[4], s));
    if (!last && (e = orthonormalise(c, c->U))) return e;
    FEAST_CUDA_TRY(cudaEventRecord(c->ev[5], s));
    DevStatus hs;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&hs, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    if (c->coll) {
        // node-sharded: lines 5-15 ran on every rank from the same summed
        // subspace, but rounding may differ between ranks; all ranks stop
        // (or fail) together, with rank 0's flag
        double bad = (hs.timeout || hs.nonfinite || hs.qz_fail) ? 1.0 : 0.0;
        if ((e = collect_scalar(c, FEAST_COLL_SUM, &bad))) return e;
        if (bad > 0.0 && !(hs.timeout || hs.nonfinite || hs.qz_fail)) return FEAST_ENOCONV;
        double f = (double)hs.flag;
        if (bad == 0.0) {
            if ((e = collect_scalar(c, FEAST_COLL_BCAST, &f))) return e;
            hs.flag = (int)f;
        }
    }
    if (hs.timeout) return note_timeout(hs.timeout);
    if (hs.nonfinite) return FEAST_ENONFINITE;
    if (hs.qz_fail) return FEAST_ENOCONV;
    if (hs.flag != 2 && !c->done) {
        c->done = 1;
        c->out_flag = hs.flag;
        // line 14 returns the previous iterate
        const int src = (hs.flag == 0) ? (c->cur ^ 1) : c->cur;
        c->out_count = (hs.flag == 0) ? c->c_prev : hs.count;
        c->out_err = (hs.flag == 0) ? c->e_prev : hs.err;
        c->out_k = (hs.flag == 0) ? c->k - 1 : c->k;
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->Xo, c->Xc[src], sizeof(zd) * n * m, cudaMemcpyDeviceToDevice, s));
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->lamo, c->lamc[src], sizeof(zd) * m, cudaMemcpyDeviceToDevice, s));
        FEAST_CUDA_TRY(cudaMemcpyAsync(c->reso, c->resc[src], sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    }
    c->c_prev = hs.count;
    c->e_prev = hs.err;
    c->cur ^= 1;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->k = c->k;
        info->count = hs.count;
        info->err = hs.err;
        info->flag = hs.flag;
        info->ms_proj = ev_ms(c->ev[0], c->ev[1]) + ev_ms(c->ev[2], c->ev[3]);
        info->ms_qz = ev_ms(c->ev[1], c->ev[2]);
        info->ms_solve = ev_ms(c->ev[3], c->ev[4]);
        info->ms_qr = ev_ms(c->ev[4], c->ev[5]);
        info->ms_refine = c->prec == FEAST_FP64 ? 0.0 : c->ms_refine;
        info->refine_sweeps_max = c->prec == FEAST_FP64 ? 0 : c->last_sweeps;
        info->qz_sweeps = hs.qz_sweeps;
        info->qz_phases = hs.qz_phases;
        info->qz_warm = c->last_warm.accepted && !c->cold_fp32;
        info->qz_cold_fp32 = c->cold_fp32;
        info->qz_rows = c->last_warm.accepted ? c->last_warm.tail : (int)m;
        info->qz_warm_resid = c->last_warm.resid;
        info->qz_warm_k = c->warm_tried ? c->last_warm.k : -1;
        double gms = 0.0;
        for (int i = 0; i + 1 < c->gt.used; i += 2) gms += ev_ms(c->gt.ev[i], c->gt.ev[i + 1]);
        info->ms_warm_gemm = gms;
        info->warm_gemm_flop = c->gt.used >= 2 ? c->gt.flops : 0.0;
        // this pass's shifted solves: the k_tc_cgemm2 launches only
        info->ms_tc_gemm = tc_timer_ms(c->tct);
        info->tc_gemm_flop = c->tct.used >= 2 ? c->tct.flops : 0.0;
    }
    return FEAST_OK;
}

int feast_eigs(feast_ctx *c, int *count, double *lambda, void *X, int64_t ldx, double *resid,
               double *err, int *flag)
{
    if (!c || !count || !lambda || !err || !flag) return FEAST_EINVAL;
    if (!c->done) return FEAST_EINVAL;
    const int64_t n = c->n;
    cudaStream_t s = c->s;
    const int cnt = c->out_count;
    if (cnt > 0) {
        FEAST_CUDA_TRY(cudaMemcpyAsync(lambda, c->lamo, sizeof(zd) * cnt, cudaMemcpyDeviceToHost, s));
        if (resid) FEAST_CUDA_TRY(cudaMemcpyAsync(resid, c->reso, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        if (X) {
            if (ldx < n) return FEAST_EINVAL;
            FEAST_CUDA_TRY(cudaMemcpy2DAsync(X, ldx * sizeof(zd), c->Xo, n * sizeof(zd), n * sizeof(zd), cnt,
                                             cudaMemcpyDeviceToDevice, s));
        }
    }
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    *count = cnt;
    *err = c->out_err;
    *flag = c->out_flag;
    return FEAST_OK;
}

int feast_get(const feast_ctx *c, int what, void *dst)
{
    if (!c || !dst) return FEAST_EINVAL;
    const size_t n = (size_t)c->n, m = (size_t)c->m0;
    const void *src = nullptr;
    size_t bytes = 0;
    switch (what) {
    case 0: src = c->U1; bytes = n * m * sizeof(zd); break;
    case 1: src = c->U2; bytes = n * m * sizeof(zd); break;
    case 2: src = c->R2; bytes = m * m * sizeof(zd); break;
    case 3: src = c->P; bytes = m * m * sizeof(zd); break;
    case 4: src = c->P + m * m; bytes = m * m * sizeof(zd); break;
    case 5: src = c->Xr; bytes = n * m * sizeof(zd); break;
    case 6: src = c->lam; bytes = m * sizeof(zd); break;
    case 7: src = c->W; bytes = n * m * sizeof(zd); break;
    case 8: src = c->W + n * m; bytes = n * m * sizeof(zd); break;
    case 9: src = c->zall; bytes = (size_t)c->qall * sizeof(zd); break;
    case 10: src = c->wall; bytes = (size_t)c->qall * sizeof(zd); break;
    case 11: src = c->res; bytes = m * sizeof(double); break;
    case 12: src = c->sel; bytes = m * sizeof(int); break;
    default: return FEAST_EINVAL;
    }
    FEAST_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->s));
    return FEAST_OK;
}

int feast_filter(feast_ctx *c, const void *V, void *U)
{
    if (!c || !V || !U) return FEAST_EINVAL;
    return filter(c, (const zd *)V, (zd *)U, c->refine_tol);
}

int feast_set_subspace(feast_ctx *c, const void *U1)
{
    if (!c || !U1) return FEAST_EINVAL;
    const int64_t n = c->n, m = c->m0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->U1, U1, sizeof(zd) * n * m, cudaMemcpyDeviceToDevice, c->s));
    c->warm_ready = 0;  // an arbitrary basis: the next projected solve starts cold
    zd *BU1 = c->W + n * m;
    int e = apply_B(c, c->U1, BU1, m);
    if (e) return e;
    if (c->projection == FEAST_RAYLEIGH_RITZ) return FEAST_OK;
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->U2, BU1, sizeof(zd) * n * m, cudaMemcpyDeviceToDevice, c->s));
    return orth_block(c, c->U2, c->R2);
}

int feast_search(feast_ctx *c, const void *Ypool, int npool, double alpha, int p, double rank_tol, int *t,
                 int *s0)
{
    if (!c || !Ypool || !t || !s0) return FEAST_EINVAL;
    if (c->coll) return FEAST_EINVAL;   // SEARCH runs on a context that owns every node
    const int64_t n = c->n;
    const int cap = c->m0cap;
    if (p < 1 || p > cap || npool < p || !(alpha > 1.0) || !(rank_tol > 0.0 && rank_tol < 1.0)) return FEAST_EINVAL;
    cudaStream_t s = c->s;
    int e;
    c->m0 = cap;  // filter at the full width the workspace holds
    const zd *Y = (const zd *)Ypool;
    zd *Ucur = c->Xr, *V = c->W, *Uf = c->U;
    const double ftol = (c->prec == FEAST_FP64) ? 1.0 : c->refine_tol;
    // U[:, at:at+w] = Q Y[:, from:from+w] (zero-padded block through the quadrature)
    auto filt = [&](int from, int w, int at) -> int {
        FEAST_CUDA_TRY(cudaMemsetAsync(V, 0, sizeof(zd) * n * cap, s));
        FEAST_CUDA_TRY(cudaMemcpyAsync(V, Y + (size_t)from * n, sizeof(zd) * n * w, cudaMemcpyDeviceToDevice, s));
        int r = filter(c, V, Uf, ftol);
        if (r) return r;
        FEAST_CUDA_TRY(cudaMemcpyAsync(Ucur + (size_t)at * n, Uf, sizeof(zd) * n * w, cudaMemcpyDeviceToDevice, s));
        return FEAST_OK;
    };
    // line 1
    if ((e = filt(0, p, 0))) return e;
    int used = p, have = p;
    // line 2: s0 = ceil(Re trace(Y_0^H U) / p)
    double *dtr = c->nrm2 ? c->nrm2 : (double *)c->res;
    if ((e = trace_real(s, n, p, Y, n, Ucur, n, dtr))) return e;
    double tr = 0.0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&tr, dtr, sizeof(double), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    const int est = (int)ceil(tr / p);
    int sd = est > p ? est : p;
    if (sd > n) sd = (int)n;
    int r = 0;
    for (;;) {
        if (sd > cap) return FEAST_ENOCONV;   // the workspace's width is too small
        if (sd > have) {                      // lines 3-5
            if (used + (sd - have) > npool) return FEAST_EINVAL;
            if ((e = filt(used, sd - have, have))) return e;
            used += sd - have;
            have = sd;
        }
        // lines 9-10: rank-revealing factorisation.  On full rank the block
        // stays as filtered columns (the span of U1, on the scale of the
        // columns that join it next, so the relative rank test compares like
        // with like); on a deficiency its selected columns' orthonormal basis
        // is U1.
        if ((e = rrqr_basis(s, n, sd, Ucur, Uf, rank_tol, c->search_work, &c->st->timeout, &r))) return e;
        if (r <= 0) return FEAST_ENOCONV;
        if (r < sd) {
            if ((e = zorth(s, n, r, Uf, n, c->R1, r, c->orth_work, &c->st->timeout, nullptr))) return e;
            break;
        }
        have = sd;
        sd = (int)ceil(alpha * r);
        if (sd > n) sd = (int)n;
        if (sd == r) return FEAST_ENOCONV;   // full rank over the whole space
    }
    // Algorithm 6, line 1: the search's basis is U1; line 2: B U1 = U2 R2
    c->m0 = r;
    if ((e = feast_set_subspace(c, Uf))) return e;
    c->k = 0;
    c->c_prev = 0;
    c->e_prev = 0.0;
    c->done = 0;
    c->cur = 0;
    c->warm_ready = 0;
    c->ritz_filter = 0;
    DevStatus hs;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&hs, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.timeout) return note_timeout(hs.timeout);
    *t = r;
    *s0 = est;
    return FEAST_OK;
}

int feast_cirr(feast_ctx *c, const void *Y, int h, int g, feast_iter_info *info)
{
    if (!c || !Y || !info || h < 1 || g < 1) return FEAST_EINVAL;
    if (c->projection != FEAST_RAYLEIGH_RITZ || c->coll) return FEAST_EINVAL;
    const int64_t n = c->n, t = (int64_t)h * g;
    if (t > c->m0cap) return FEAST_EINVAL;
    cudaStream_t s = c->s;
    int e;
    // step 1: X_j = M_j^{-1} Y at width h, then the moment block (width t)
    c->m0 = h;
    FEAST_CUDA_TRY(cudaMemcpyAsync(c->tmp, Y, sizeof(zd) * n * h, cudaMemcpyDeviceToDevice, s));
    e = solve_nodes(c, c->tmp, (c->prec == FEAST_FP64) ? 1.0 : c->refine_tol);
    if (!e)
        e = moment_sum(s, n, h, c->q, g, c->z, c->w, c->contour.center_re, c->contour.center_im,
                       fmax(c->contour.a, c->contour.b), c->Xs, n * h, c->U, n);
    c->m0 = (int)t;
    if (e) return e;
    // step 2: an orthonormal basis of the moment block (QR; the SVD's U spans
    // the same space), and B U1 for the projection
    if ((e = orthonormalise(c, c->U))) return e;
    // steps 3-5: one Rayleigh-Ritz pass; the stop of line 15 keeps the
    // selected pairs for feast_eigs
    c->k = 0;
    c->c_prev = 0;
    c->e_prev = 0.0;
    c->done = 0;
    c->cur = 0;
    c->warm_ready = 0;
    c->ritz_filter = 0;
    const int mi = c->max_iter, ns = c->no_stop;
    c->max_iter = 1;
    c->no_stop = 0;
    e = feast_iterate(c, info);
    c->max_iter = mi;
    c->no_stop = ns;
    return e;
}

void feast_destroy(feast_ctx *c)
{
    if (!c) return;
    for (int i = 0; i < 8; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    for (int i = 0; i < GemmTimer::kMax; ++i)
        if (c->gt.ev[i]) cudaEventDestroy(c->gt.ev[i]);
    for (int i = 0; i < 2 * TcTimer::kMax; ++i)
        if (c->tct.ev[i]) cudaEventDestroy(c->tct.ev[i]);
    free(c->zw_host);
    free(c);
}

// ------------------------------------------------------------ ragged batch
// Many independent pencils (uneven n, m0, contours) solved concurrently:
// nworkers host threads, each with its own CUDA stream and its own slice of
// the workspace, take pencils from a shared counter and run set-up and the
// whole GFEAST loop on them.  The kernels of different pencils overlap on
// the GPU; per pencil the sequence of launches is the single-pencil one.
size_t feast_batch_workspace_size(int count, const feast_pencil *pencils,
                                  const feast_contour *contours, const feast_options *opts,
                                  int nworkers)
{
    if (count <= 0 || !pencils || !contours || !opts || nworkers <= 0) return 0;
    size_t mx = 0;
    for (int i = 0; i < count; ++i) {
        size_t b = 0;
        if (feast_workspace_size(pencils + i, contours + i, opts + i, &b) != FEAST_OK) return 0;
        mx = b > mx ? b : mx;
    }
    mx = (mx + 255) & ~(size_t)255;
    const int w = nworkers < count ? nworkers : count;
    return mx * (size_t)w;
}

int feast_solve_batch(int count, const feast_pencil *pencils, const feast_contour *contours,
                      const feast_options *opts, void *workspace, size_t workspace_bytes,
                      int nworkers, feast_batch_item *items, double *lambda, double *resid)
{
    if (count > 0 && opts && (opts->node_begin != 0 || opts->node_end != 0)) return FEAST_EINVAL;
    if (count <= 0 || !pencils || !contours || !opts || !workspace || !items || !lambda || nworkers <= 0)
        return FEAST_EINVAL;
    const size_t need = feast_batch_workspace_size(count, pencils, contours, opts, nworkers);
    if (need == 0) return FEAST_EINVAL;
    if (workspace_bytes < need || ((uintptr_t)workspace & 255u)) return FEAST_ENOMEM;
    const int w = nworkers < count ? nworkers : count;
    const size_t slice = need / (size_t)w;
    std::vector<size_t> off;
    try {
        off.assign((size_t)count + 1, 0);
    } catch (...) {
        return FEAST_ENOMEM;
    }
    for (int i = 0; i < count; ++i) off[i + 1] = off[i] + (size_t)opts[i].m0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FEAST_ECUDA;
    std::atomic<int> next{0};
    std::atomic<int> worst{FEAST_OK};
    auto worker = [&](int wid) {
        if (cudaSetDevice(dev) != cudaSuccess) { worst = FEAST_ECUDA; return; }
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { worst = FEAST_ECUDA; return; }
        void *ws = (char *)workspace + slice * (size_t)wid;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= count) break;
            feast_batch_item &it = items[i];
            memset(&it, 0, sizeof(it));
            feast_options o = opts[i];
            o.stream = st;
            o.no_stop = 0;
            feast_ctx *ctx = nullptr;
            feast_iter_info info;
            memset(&info, 0, sizeof(info));
            int e = feast_setup(&ctx, pencils + i, contours + i, &o, ws, slice, &info);
            it.ms_setup = info.ms_lu + info.ms_solve;
            while (e == FEAST_OK) {
                e = feast_iterate(ctx, &info);
                if (e == FEAST_OK) {
                    it.ms_pass += info.ms_proj + info.ms_qz + info.ms_solve + info.ms_qr;
                    it.ms_solve += info.ms_solve;
                    it.ms_qz += info.ms_qz;
                }
                if (e == FEAST_OK && info.flag != 2) break;
            }
            if (e == FEAST_OK) {
                int cnt = 0, flag = 0;
                double err = 0.0;
                e = feast_eigs(ctx, &cnt, lambda + 2 * off[i], nullptr, pencils[i].n,
                               resid ? resid + off[i] : nullptr, &err, &flag);
                it.count = cnt;
                it.flag = flag;
                it.err = err;
                it.k = info.k;
            }
            it.status = e;
            if (e != FEAST_OK) worst = e;
            feast_destroy(ctx);
        }
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    try {
        pool.reserve((size_t)w);
        for (int t = 0; t < w; ++t) pool.emplace_back(worker, t);
    } catch (...) {
        // the workers already running take the whole batch; none running:
        // nothing was solved
        if (pool.empty()) return FEAST_ENOMEM;
    }
    for (auto &th : pool) th.join();
    return worst.load();
}

unsigned long long feast_kernel_launches(void) { return g_launches.load(); }

const char *feast_last_cuda_error(void) { return g_cuda_error; }

const char *feast_strerror(int status)
{
    switch (status) {
    case FEAST_OK: return "ok";
    case FEAST_EINVAL: return "invalid argument";
    case FEAST_ENOMEM: return "workspace too small or host allocation failed";
    case FEAST_ECUDA: return "CUDA runtime error";
    case FEAST_ESINGULAR: return "a shifted matrix has an exact zero pivot";
    case FEAST_ENONFINITE: return "non-finite value in a residual";
    case FEAST_ETIMEOUT: return "bounded device wait timed out";
    case FEAST_ENOCONV: return "projected QZ did not converge";
    case FEAST_EDONE: return "the iteration has already stopped";
    default: return "unknown status";
    }
}

int feast_zgetrf_batched(int64_t n, int batch, void *M, int64_t ld, int64_t stride, int *piv,
                         int *info, void *stream)
{
    if (n < 0 || batch < 0 || ld < n || stride < ld * n || !M || !piv || !info) return FEAST_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    FEAST_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    return zgetrf_batched(s, n, batch, (zd *)M, ld, stride, piv, info, nullptr);
}

int feast_zgetrs_batched(int64_t n, int64_t nrhs, int batch, const void *M, int64_t ld,
                         int64_t stride, const int *piv, void *X, int64_t ldx, int64_t sx,
                         void *stream)
{
    if (n < 0 || nrhs < 0 || batch < 0 || ld < n || ldx < n || !M || !piv || !X) return FEAST_EINVAL;
    return zgetrs_batched((cudaStream_t)stream, n, nrhs, batch, (const zd *)M, ld, stride, piv, (zd *)X,
                          ldx, sx);
}

size_t feast_cgemm_tc_scratch_bytes(int64_t m, int64_t n, int64_t k, int batch)
{
    if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return 0;
    return sizeof(float) * tc_scratch_floats(m, k, n, batch) + 256;
}

int feast_cgemm_tc(int64_t m, int64_t n, int64_t k, float alpha_re, float alpha_im, const void *A,
                   int64_t lda, int64_t sA, const void *X, int64_t ldx, int64_t sX, float beta_re,
                   float beta_im, void *C, int64_t ldc, int64_t sC, int batch, void *scratch,
                   size_t scratch_bytes, int *err, void *stream)
{
    if (m < 0 || n < 0 || k < 0 || batch < 0 || !A || !X || !C || !scratch || !err) return FEAST_EINVAL;
    if (lda < m || ldx < k || ldc < m) return FEAST_EINVAL;
    if (scratch_bytes < feast_cgemm_tc_scratch_bytes(m, n, k, batch)) return FEAST_ENOMEM;
    float *sc = (float *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
    cudaStream_t s = (cudaStream_t)stream;
    FEAST_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    return tc_cgemm(s, m, n, k, make_float2(alpha_re, alpha_im), (const cf *)A, lda, sA, (const cf *)X, ldx, sX,
                    make_float2(beta_re, beta_im), (cf *)C, ldc, sC, batch, sc, err);
}

static int grad_abs2_impl(feast_ctx *r, feast_ctx *l, void *gA, void *gB, int64_t ldg, double *L, int *count);

int feast_grad_abs2(feast_ctx *r, feast_ctx *l, void *gA, void *gB, int64_t ldg, double *L, int *count)
{
    try {
        return grad_abs2_impl(r, l, gA, gB, ldg, L, count);
    } catch (...) {
        return FEAST_ENOMEM;
    }
}

static int grad_abs2_impl(feast_ctx *r, feast_ctx *l, void *gA, void *gB, int64_t ldg, double *L, int *count)
{
    if (!r || !l || !gA || !gB || !L || !count) return FEAST_EINVAL;
    if (!r->done || !l->done) return FEAST_EINVAL;
    if (r->kind != FEAST_DENSE || l->kind != FEAST_DENSE || r->n != l->n || ldg < r->n) return FEAST_EINVAL;
    const int64_t n = r->n;
    const int cnt = r->out_count;
    *count = 0;
    *L = 0.0;
    if (l->out_count != cnt) return FEAST_ENOCONV;   // the two runs disagree on the inside count
    cudaStream_t s = r->s;
    std::vector<zd> lam(cnt > 0 ? cnt : 1), mu(cnt > 0 ? cnt : 1);
    if (cnt > 0) {
        FEAST_CUDA_TRY(cudaMemcpyAsync(lam.data(), r->lamo, sizeof(zd) * cnt, cudaMemcpyDeviceToHost, s));
        FEAST_CUDA_TRY(cudaMemcpyAsync(mu.data(), l->lamo, sizeof(zd) * cnt, cudaMemcpyDeviceToHost, s));
        FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // pair each right eigenvalue with the nearest unused conjugate of a left one
    std::vector<int> kidx(cnt > 0 ? cnt : 1);
    std::vector<char> used(cnt > 0 ? cnt : 1, 0);
    double L2 = 0.0;
    for (int i = 0; i < cnt; ++i) {
        int best = -1;
        double bd = 0.0;
        for (int k = 0; k < cnt; ++k) {
            if (used[k]) continue;
            const double dx = mu[k].x - lam[i].x, dy = -mu[k].y - lam[i].y;
            const double d = dx * dx + dy * dy;
            if (best < 0 || d < bd) { best = k; bd = d; }
        }
        used[best] = 1;
        kidx[i] = best;
        L2 += lam[i].x * lam[i].x + lam[i].y * lam[i].y;
    }
    int *dk = r->idx;              // scratch once the run is done
    zd *BX = r->AXBX, *alpha = r->lamc[0], *beta = r->lamc[1];
    int e;
    if (cnt > 0) {
        FEAST_CUDA_TRY(cudaMemcpyAsync(dk, kidx.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
        if ((e = apply_B(r, r->Xo, BX, cnt))) return e;
        if ((e = adjoint_coef(s, n, cnt, l->Xo, n, dk, BX, n, r->lamo, alpha, beta))) return e;
    }
    if ((e = adjoint_grad(s, n, cnt, l->Xo, n, dk, r->Xo, n, alpha, beta, (zd *)gA, (zd *)gB, ldg))) return e;
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    *count = cnt;
    *L = L2;
    return FEAST_OK;
}

size_t feast_zgemm_oz_work_bytes(int64_t m, int64_t n, int64_t k)
{
    if (m <= 0 || n <= 0 || k <= 0) return 0;
    return oz_rows_bytes(m, k) + oz_cols_bytes(k, n) + 1024;
}

int feast_zgemm_oz(int64_t m, int64_t n, int64_t k, double alpha_re, double alpha_im, const void *A, int64_t lda,
                   const void *B, int64_t ldb, double beta_re, double beta_im, void *C, int64_t ldc, void *work,
                   size_t work_bytes, int *err, void *stream)
{
    if (m < 0 || n < 0 || k < 0 || !A || !B || !C || !work || !err) return FEAST_EINVAL;
    if (lda < m || ldb < k || ldc < m) return FEAST_EINVAL;
    if (((uintptr_t)work & 255u) != 0) return FEAST_EINVAL;
    if (m == 0 || n == 0) return FEAST_OK;
    if (work_bytes < feast_zgemm_oz_work_bytes(m, n, k)) return FEAST_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    FEAST_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    char *wa = (char *)work;
    char *wb = wa + ((oz_rows_bytes(m, k) + 255) & ~(size_t)255);
    int e;
    if ((e = oz_prepare_rows(s, m, k, (const zd *)A, lda, wa))) return e;
    if ((e = oz_prepare_cols(s, k, n, (const zd *)B, ldb, wb))) return e;
    return oz_gemm(s, m, n, k, wa, wb, zmake(alpha_re, alpha_im), nullptr, 0, zmake(beta_re, beta_im), (zd *)C, ldc,
                   err);
}

size_t feast_zqz_work_bytes(int m, int batch)
{
    if (m < 0 || batch < 0) return 0;
    return (size_t)batch * zqz_work_bytes(m);
}

int feast_zqz_batched(int m, int batch, void *A, void *B, void *alpha, void *beta, void *V,
                      void *work, int *status, void *stream)
{
    if (m < 0 || batch < 0 || !A || !B || !alpha || !beta || !V || !work || !status) return FEAST_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    FEAST_CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(int), s));
    int e = zqz_batched(s, m, batch, (zd *)A, m, (int64_t)m * m, (zd *)B, m, (int64_t)m * m, (zd *)alpha,
                        (zd *)beta, (zd *)V, m, (int64_t)m * m, work, status, status + 1);
    return e;
}

}  // extern "C"
