// Tensor-core (tcgen05, kind::tf32) complex64 GEMM for sm_103a.
//
//   C_b = beta C_b + alpha A_b X_b     (A: m x k, X: k x n, C: m x n complex64,
//                                       column-major, interleaved re/im)
//
// Complex arithmetic as one real GEMM: every complex row i of A becomes two
// real rows of A' (length 2k, K contiguous):
//   A'(2i,   2p) =  Re A(i,p)   A'(2i,   2p+1) = -Im A(i,p)
//   A'(2i+1, 2p) =  Im A(i,p)   A'(2i+1, 2p+1) =  Re A(i,p)
// and X (column-major, interleaved) already is the real K-major operand
// X'(2p + c, j).  Then D' = A' X' holds Re(AX)(i,j) in row 2i and Im in
// row 2i+1, so one tcgen05 accumulator tile of 128 real rows covers 64
// complex rows.  For ~FP32 accuracy each operand is split into a TF32 head
// and a TF32 tail (3 products: hh + ht + th).
//
// Per CTA: one 128 x BN tile of D'.  Warp 0 (one lane) feeds a STAGES-deep
// ring of 128B-swizzled shared-memory tiles with TMA (cp.async.bulk.tensor,
// completion on an mbarrier); warp 1 (one lane) issues tcgen05.mma into a
// TMEM accumulator and frees each stage with tcgen05.commit; all four warps
// then read their 32 TMEM lanes (tcgen05.ld), pair re/im rows across
// neighbouring lanes and write C.  Every mbarrier wait has an iteration cap;
// on expiry the kernel raises an error word and finishes without hanging.
#include "tcgen05.cuh"

namespace feast {

namespace {
using namespace tc;

constexpr int TC_BM = 128;          // real rows per tile (= 64 complex rows)
constexpr int TC_BK = 32;           // fp32 per 128-byte swizzle row
constexpr int TC_STAGES = 3;
template <int BN>
__global__ void __launch_bounds__(128) k_tc_cgemm(const __grid_constant__ CUtensorMap tAh,
                                                  const __grid_constant__ CUtensorMap tAt,
                                                  const __grid_constant__ CUtensorMap tXh,
                                                  const __grid_constant__ CUtensorMap tXt, int mr,
                                                  int n, int kr, float2 *C, int64_t ldc, int64_t sC,
                                                  float2 alpha, float2 beta, int *err)
{
    constexpr int A_BYTES = TC_BM * TC_BK * 4;          // 16 KiB
    constexpr int B_BYTES = BN * TC_BK * 4;
    constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bz = blockIdx.z;
    const int row0 = blockIdx.x * TC_BM;                 // real row
    const int col0 = blockIdx.y * BN;
    const int kb_n = (kr + TC_BK - 1) / TC_BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer
        for (int kb = 0; kb < kb_n; ++kb) {
            const int s = kb % TC_STAGES;
            const uint32_t ph = (uint32_t)((kb / TC_STAGES) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1u)) { s_fail = 1; break; }
            unsigned char *st = base + s * STAGE;
            mbar_expect_tx(&full[s], STAGE);
            const int kx = kb * TC_BK;
            tma_load_3d(st, &tAh, &full[s], kx, row0, bz);
            tma_load_3d(st + A_BYTES, &tAt, &full[s], kx, row0, bz);
            tma_load_3d(st + 2 * A_BYTES, &tXh, &full[s], kx, col0, bz);
            tma_load_3d(st + 2 * A_BYTES + B_BYTES, &tXt, &full[s], kx, col0, bz);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: D = M=128 x N=BN, K=8 per instruction, 4 per stage
        const uint32_t idesc = idesc_f32acc(2u, TC_BM, BN);
        bool ok = true;
        for (int kb = 0; kb < kb_n && ok; ++kb) {
            const int s = kb % TC_STAGES;
            const uint32_t ph = (uint32_t)((kb / TC_STAGES) & 1);
            if (!mbar_wait(&full[s], ph)) { s_fail = 1; ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            unsigned char *st = base + s * STAGE;
            const uint64_t ah = sdesc<128>(st), at = sdesc<128>(st + A_BYTES);
            const uint64_t xh = sdesc<128>(st + 2 * A_BYTES), xt = sdesc<128>(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 8; ++kk) {
                const uint64_t adv = (uint64_t)((kk * 8 * 4) >> 4);   // 32 bytes per step
                const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
                mma_tf32(tmem, ah + adv, xh + adv, idesc, acc0);
                mma_tf32(tmem, ah + adv, xt + adv, idesc, 1u);
                mma_tf32(tmem, at + adv, xh + adv, idesc, 1u);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    // epilogue: all warps wait for the accumulator
    bool good = mbar_wait(&done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!good || s_fail) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else {
        const int r = row0 + warp * 32 + lane;            // real row of this lane
        const int ci = r >> 1;                             // complex row
        const bool im_row = (r & 1) != 0;
        float2 *Cb = C + (int64_t)bz * sC;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            tmem_ld32(taddr, v);
            // even lane (Re row) stores columns 0..15 of this chunk, odd lane
            // (Im row) stores 16..31; each needs its partner's values
            const int half = im_row ? 1 : 0;
            float dre[16], dim[16];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float mine = __uint_as_float(v[j]);
                const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
                if ((j >> 4) == half) {
                    dre[j & 15] = im_row ? other : mine;
                    dim[j & 15] = im_row ? mine : other;
                }
            }
            // the 16 old values first (independent loads in flight), then the update
            const bool rd = (beta.x != 0.f || beta.y != 0.f);
            float2 old[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = col0 + c0 + half * 16 + i;
                old[i] = (rd && r < mr && col < n) ? Cb[ci + (int64_t)col * ldc] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = col0 + c0 + half * 16 + i;
                if (r < mr && col < n) {
                    float2 res;
                    res.x = alpha.x * dre[i] - alpha.y * dim[i] + beta.x * old[i].x - beta.y * old[i].y;
                    res.y = alpha.x * dim[i] + alpha.y * dre[i] + beta.x * old[i].y + beta.y * old[i].x;
                    Cb[ci + (int64_t)col * ldc] = res;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// A (m x k complex, column-major, ld) -> head / tail of A' (2m x 2k real,
// row-major with leading dim ldr), batched.
__global__ void k_realify_split(int m, int k, const float2 *A, int64_t lda, int64_t sA, float *head,
                                float *tail, int64_t ldr, int64_t sR)
{
    const int b = blockIdx.y;
    const float2 *Ab = A + (int64_t)b * sA;
    float *H = head + (int64_t)b * sR, *Tt = tail + (int64_t)b * sR;
    const int64_t total = (int64_t)m * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), p = (int)(e / m);
        const float2 a = Ab[i + (int64_t)p * lda];
        const float v[4] = {a.x, -a.y, a.y, a.x};   // (2i,2p) (2i,2p+1) (2i+1,2p) (2i+1,2p+1)
        const int64_t o[4] = {(int64_t)(2 * i) * ldr + 2 * p, (int64_t)(2 * i) * ldr + 2 * p + 1,
                              (int64_t)(2 * i + 1) * ldr + 2 * p, (int64_t)(2 * i + 1) * ldr + 2 * p + 1};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float h = __uint_as_float(__float_as_uint(v[t]) & 0xFFFFE000u);  // TF32 head (truncated)
            H[o[t]] = h;
            Tt[o[t]] = v[t] - h;
        }
    }
}

// X (k x n complex, column-major, ld) -> head / tail (same layout, as reals)
__global__ void k_split_tf32(int64_t rows2, int n, const float *X, int64_t ldx2, int64_t sX, float *head,
                             float *tail, int64_t ldh2, int64_t sH)
{
    const int b = blockIdx.y;
    const float *Xb = X + (int64_t)b * sX;
    float *H = head + (int64_t)b * sH, *Tt = tail + (int64_t)b * sH;
    const int64_t total = rows2 * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % rows2, c = e / rows2;
        const float v = Xb[r + c * ldx2];
        const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        H[r + c * ldh2] = h;
        Tt[r + c * ldh2] = v - h;
    }
}

}  // namespace

namespace tc {
PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    // looked up once (thread-safe static initialisation)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

int make_map_3d(CUtensorMap *map, CUtensorMapDataType dt, int elem_bytes, const void *base, int64_t inner,
                int64_t rows, int64_t planes, int64_t ld_bytes, int64_t plane_bytes, int box_inner,
                int box_rows, CUtensorMapSwizzle swz)
{
    auto enc = get_encode();
    if (!enc) return FEAST_ECUDA;
    (void)elem_bytes;
    if (((uintptr_t)base & 15) || (ld_bytes & 15) || (plane_bytes & 15)) return FEAST_EINVAL;
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)ld_bytes, (cuuint64_t)(plane_bytes > 0 ? plane_bytes : ld_bytes * rows)};
    cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FEAST_OK : FEAST_EINVAL;
}
}  // namespace tc

namespace {
// 3-D fp32 tensor map {inner, rows, batch}, box {32, box_rows, 1}, 128-byte swizzle.
int make_map(CUtensorMap *map, const float *base, int64_t inner, int64_t rows, int64_t batch,
             int64_t ld_bytes, int64_t batch_bytes, int box_rows)
{
    return tc::make_map_3d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, inner, rows, batch, ld_bytes, batch_bytes,
                           TC_BK, box_rows, CU_TENSOR_MAP_SWIZZLE_128B);
}
}  // namespace

constexpr int TC_BN = 128;

size_t tc_scratch_floats(int64_t m, int64_t k, int64_t n, int batch)
{
    const int64_t kr = ((2 * k + TC_BK - 1) / TC_BK) * TC_BK;
    const int64_t mr = 2 * m;
    return (size_t)batch * (2 * (size_t)mr * kr + 2 * (size_t)kr * n);
}

size_t tc_prepA_floats(int64_t m, int64_t k, int batch)
{
    const int64_t kr = ((2 * k + TC_BK - 1) / TC_BK) * TC_BK;
    return (size_t)batch * 2 * (size_t)(2 * m) * kr;
}

// The left operand's realified head / tail planes (A' of the file comment),
// made once when A is reused by many products (the LU factors' off-block
// panels in every shifted solve).
int tc_prepare_A(cudaStream_t s, int64_t m, int64_t k, const cf *A, int64_t lda, int64_t sA, int batch,
                 float *Aprep)
{
    if (m <= 0 || k <= 0 || batch <= 0) return FEAST_OK;
    const int64_t kr = ((2 * k + TC_BK - 1) / TC_BK) * TC_BK;
    const int64_t mr = 2 * m;
    float *Ah = Aprep, *At = Ah + (size_t)batch * mr * kr;
    if (kr != 2 * k) FEAST_CUDA_TRY(cudaMemsetAsync(Ah, 0, sizeof(float) * 2 * (size_t)batch * mr * kr, s));
    unsigned g = cdiv((size_t)m * k, 256);
    k_realify_split<<<dim3(g > 4096 ? 4096 : g, batch), 256, 0, s>>>((int)m, (int)k, A, lda, sA, Ah, At, kr,
                                                                     mr * kr);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// C_b = beta C_b + alpha A_b X_b with A given by tc_prepare_A's planes;
// scratch: the right operand's planes (2 * batch * kr * n floats).
int tc_cgemm_prepA(cudaStream_t s, int64_t m, int64_t n, int64_t k, cf alpha, const float *Aprep, const cf *X,
                   int64_t ldx, int64_t sX, cf beta, cf *C, int64_t ldc, int64_t sC, int batch, float *scratch,
                   int *err)
{
    if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return FEAST_OK;
    const int64_t kr = ((2 * k + TC_BK - 1) / TC_BK) * TC_BK;
    const int64_t mr = 2 * m;
    const float *Ah = Aprep, *At = Ah + (size_t)batch * mr * kr;
    float *Xh = scratch, *Xt = Xh + (size_t)batch * kr * n;
    if (kr != 2 * k) FEAST_CUDA_TRY(cudaMemsetAsync(Xh, 0, sizeof(float) * 2 * (size_t)batch * kr * n, s));
    unsigned g2 = cdiv((size_t)2 * k * n, 256);
    k_split_tf32<<<dim3(g2 > 4096 ? 4096 : g2, batch), 256, 0, s>>>(2 * k, (int)n, (const float *)X, 2 * ldx,
                                                                    2 * sX, Xh, Xt, kr, kr * n);
    FEAST_LAUNCH_CHECK();
    CUtensorMap mAh, mAt, mXh, mXt;
    int e;
    if ((e = make_map(&mAh, (float *)Ah, kr, mr, batch, kr * 4, mr * kr * 4, TC_BM))) return e;
    if ((e = make_map(&mAt, (float *)At, kr, mr, batch, kr * 4, mr * kr * 4, TC_BM))) return e;
    if ((e = make_map(&mXh, Xh, kr, n, batch, kr * 4, kr * n * 4, TC_BN))) return e;
    if ((e = make_map(&mXt, Xt, kr, n, batch, kr * 4, kr * n * 4, TC_BN))) return e;
    const size_t smem = (size_t)TC_STAGES * (2 * TC_BM * TC_BK * 4 + 2 * TC_BN * TC_BK * 4) + 1024;
    FEAST_CUDA_TRY(allow_dyn_smem(k_tc_cgemm<TC_BN>));
    dim3 grid(cdiv(mr, TC_BM), cdiv(n, TC_BN), batch);
    k_tc_cgemm<TC_BN><<<grid, 128, smem, s>>>(mAh, mAt, mXh, mXt, (int)mr, (int)n, (int)kr, C, ldc, sC, alpha,
                                              beta, err);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// C_b = beta C_b + alpha A_b X_b on tensor cores (see the file comment).
// scratch: tc_scratch_floats(m, k, n, batch) floats (16-byte aligned).
int tc_cgemm(cudaStream_t s, int64_t m, int64_t n, int64_t k, cf alpha, const cf *A, int64_t lda,
             int64_t sA, const cf *X, int64_t ldx, int64_t sX, cf beta, cf *C, int64_t ldc, int64_t sC,
             int batch, float *scratch, int *err)
{
    if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return FEAST_OK;
    int e;
    if ((e = tc_prepare_A(s, m, k, A, lda, sA, batch, scratch))) return e;
    return tc_cgemm_prepA(s, m, n, k, alpha, scratch, X, ldx, sX, beta, C, ldc, sC, batch,
                          scratch + tc_prepA_floats(m, k, batch), err);
}

}  // namespace feast
