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
// The GEMM runs as one persistent launch of two-CTA clusters (tcgen05
// cta_group::2, 256 x 256 tiles of D'), described at k_tc_cgemm2 below.
// Every mbarrier wait has an iteration cap; on expiry the kernel raises an
// error word and finishes without hanging.
#include <mutex>

#include "tcgen05.cuh"

namespace feast {

namespace {
using namespace tc;

// K of the realified operands is padded to a multiple of TC_BK (the layout of
// the prepared left-operand planes that callers cache).
constexpr int TC_BK = 32;
// ---------------------------------------------------------------------------
// Persistent two-CTA form (tcgen05 cta_group::2).  A cluster of two CTAs on
// neighbouring SMs computes 256 x 256 tiles of D': each CTA stages 128 rows
// of A' and 128 of the tile's 256 columns of X' (K-major, 64-byte swizzle,
// K2_BK = 16 fp32 per stage, K2_STAGES deep), the even CTA's MMA thread
// issues M = 256, N = 256 instructions that read both CTAs' tiles and write
// each CTA's 128 accumulator rows into its own tensor memory.  Every TMA
// load of a stage completes on the even CTA's full barrier; the MMA commit
// that frees a stage arrives on both CTAs' empty barriers.  Two 256-column
// accumulators per CTA (all 512 TMEM columns) let the epilogue warps read
// tile i back and write C while the MMAs of tile i + 1 run.  Tiles are
// taken in a fixed round-robin order over (batch, row pair, column tile),
// identical in both CTAs.  Warp roles (192 threads): warp 0 lane 0 TMA
// producer, warp 1 lane 0 MMA issuer (even CTA), warps 2-5 epilogue (TMEM
// lane quarter = warp % 4).  Every wait is bounded; a wait that gives up
// raises *err, and every other wait gives up as soon as it sees *err.
constexpr int K2_BM = 128;          // real rows per CTA (256 per pair)
constexpr int K2_BN = 256;          // columns per tile (128 staged per CTA)
constexpr int K2_BK = 16;           // fp32 per 64-byte swizzle row
constexpr int K2_STAGES = 6;
constexpr int K2_THREADS = 192;
constexpr int K2_TILE_BYTES = K2_BM * K2_BK * 4;        // 8 KiB: one plane of A' or X' per CTA
constexpr int K2_STAGE_BYTES = 4 * K2_TILE_BYTES;      // Ah, At, Xh, Xt
constexpr size_t K2_SMEM = (size_t)K2_STAGES * K2_STAGE_BYTES + 1024;

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Shared-memory address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(const void *p, uint32_t rank)
{
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
    return out;
}
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Bounded wait that also gives up once any thread has raised *err (unless
// it waits for this CTA's own copies or MMAs in flight: those are waited
// out, up to the time bound); a wait that runs out itself raises the
// site's bit in *err.
constexpr unsigned long long DRAIN_NS = 200000000ull;   // bound of a wait for this CTA's own work in flight
__device__ __forceinline__ bool wait2(uint64_t *bar, uint32_t parity, int *err, int site, bool stop_on_err = true)
{
    const unsigned long long limit = stop_on_err ? WAIT_NS : DRAIN_NS;
    const uint32_t a = smem_u32(bar);
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < SPIN; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023) == 1023) {
            if (stop_on_err && *(volatile const int *)err) return false;
            if (global_ns() - t0 > limit) break;
        }
    }
    atomicOr(err, site);
    return false;
}
// TMA tile load into this CTA's shared memory, completion counted on the
// mbarrier at cluster address bar_cluster (here: the even CTA's).
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cluster, int x,
                                                 int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar_cluster)
        : "memory");
}
__device__ __forceinline__ void mma_tf32_pair(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                              uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// Arrive on the barrier at this offset in both CTAs of the pair once every
// tcgen05 operation issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

__global__ void __launch_bounds__(K2_THREADS, 1)
    k_tc_cgemm2(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAt,
                const __grid_constant__ CUtensorMap tXh, const __grid_constant__ CUtensorMap tXt, int mr, int n,
                int kr, int batch, float2 *C, int64_t ldc, int64_t sC, float2 alpha, float2 beta, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[K2_STAGES], empty[K2_STAGES], tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const int mt = (mr + 2 * K2_BM - 1) / (2 * K2_BM), nt = (n + K2_BN - 1) / K2_BN;
    const long long tiles = (long long)batch * mt * nt;
    const int kb_n = kr / K2_BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < K2_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);         // one arrival per epilogue warp of both CTAs
        }
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    cluster_sync();                           // the peer's barriers exist before anyone signals them
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // TMA producer (both CTAs): this CTA's 128 rows of A', 128 columns of X'
        const uint32_t full0 = map_to_rank(&full[0], 0);
        long long it = 0;
        bool ok = true;
        for (long long t = pair; t < tiles && ok; t += npairs) {
            const int b = (int)(t / ((long long)mt * nt));
            const int rem = (int)(t % ((long long)mt * nt));
            const int row0 = (rem / nt) * 2 * K2_BM + (int)rank * K2_BM;
            const int col0 = (rem % nt) * K2_BN + (int)rank * (K2_BN / 2);
            for (int kb = 0; kb < kb_n; ++kb, ++it) {
                const int s = (int)(it % K2_STAGES);
                const uint32_t ph = (uint32_t)((it / K2_STAGES) & 1);
                if (!wait2(&empty[s], ph ^ 1u, err, TO_TC_LOAD)) { ok = false; break; }
                unsigned char *st = base + s * K2_STAGE_BYTES;
                const uint32_t fb = full0 + (uint32_t)(s * sizeof(uint64_t));
                if (rank == 0) mbar_expect_tx(&full[s], 2 * K2_STAGE_BYTES);
                const int kx = kb * K2_BK;
                tma_load_3d_pair(st, &tAh, fb, kx, row0, b);
                tma_load_3d_pair(st + K2_TILE_BYTES, &tAt, fb, kx, row0, b);
                tma_load_3d_pair(st + 2 * K2_TILE_BYTES, &tXh, fb, kx, col0, b);
                tma_load_3d_pair(st + 3 * K2_TILE_BYTES, &tXt, fb, kx, col0, b);
            }
        }
        if (!ok && rank == 0) {
            // let the loads already issued land before the CTA can exit
            for (int s = 0; s < K2_STAGES; ++s) {
                const long long last = it - 1 - ((it - 1 - s) % K2_STAGES + K2_STAGES) % K2_STAGES;
                if (last >= 0) wait2(&full[s], (uint32_t)((last / K2_STAGES) & 1), err, TO_TC_LOAD, false);
            }
        }
    } else if (warp == 1 && lane == 0 && rank == 0) {
        // MMA issuer: M = 256 (both CTAs' rows), N = 256, K = 8 per instruction
        const uint32_t idesc = idesc_f32acc(2u, 2 * K2_BM, K2_BN);
        long long it = 0;
        int tl = 0;
        bool ok = true;
        for (long long t = pair; t < tiles && ok; t += npairs, ++tl) {
            const int ab = tl & 1;
            const uint32_t aph = (uint32_t)((tl >> 1) & 1);
            if (!wait2(&tempty[ab], aph ^ 1u, err, TO_TC_MMA)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = tmem + (uint32_t)(ab * K2_BN);
            for (int kb = 0; kb < kb_n; ++kb, ++it) {
                const int s = (int)(it % K2_STAGES);
                const uint32_t ph = (uint32_t)((it / K2_STAGES) & 1);
                if (!wait2(&full[s], ph, err, TO_TC_MMA)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                unsigned char *st = base + s * K2_STAGE_BYTES;
                const uint64_t ah = sdesc<64>(st), at = sdesc<64>(st + K2_TILE_BYTES);
                const uint64_t xh = sdesc<64>(st + 2 * K2_TILE_BYTES), xt = sdesc<64>(st + 3 * K2_TILE_BYTES);
#pragma unroll
                for (int kk = 0; kk < K2_BK / 8; ++kk) {
                    const uint64_t adv = (uint64_t)((kk * 8 * 4) >> 4);   // 32 bytes per K = 8 step
                    const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
                    mma_tf32_pair(d, ah + adv, xh + adv, idesc, acc0);
                    mma_tf32_pair(d, ah + adv, xt + adv, idesc, 1u);
                    mma_tf32_pair(d, at + adv, xh + adv, idesc, 1u);
                }
                mma_commit_pair(&empty[s]);
            }
            if (ok) mma_commit_pair(&tfull[ab]);
        }
        // every MMA this thread issued has completed before the CTA can
        // release its tensor memory (also on the path that gave up)
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&drain))
                     : "memory");
        wait2(&drain, 0, err, TO_TC_DRAIN, false);
    } else if (warp >= 2) {
        // epilogue: TMEM lanes 32 (warp % 4) .. +31 of this CTA's 128 rows
        const int quarter = warp & 3;
        const uint32_t tempty0 = map_to_rank(&tempty[0], 0);
        const bool rd = (beta.x != 0.f || beta.y != 0.f);
        int tl = 0;
        for (long long t = pair; t < tiles; t += npairs, ++tl) {
            const int ab = tl & 1;
            const uint32_t aph = (uint32_t)((tl >> 1) & 1);
            if (!wait2(&tfull[ab], aph, err, TO_TC_EPI)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int b = (int)(t / ((long long)mt * nt));
            const int rem = (int)(t % ((long long)mt * nt));
            const int r = (rem / nt) * 2 * K2_BM + (int)rank * K2_BM + quarter * 32 + lane;   // real row
            const int ci = r >> 1;
            const bool im_row = (r & 1) != 0;
            const int half = im_row ? 1 : 0;
            const int colt = (rem % nt) * K2_BN;
            float2 *Cb = C + (int64_t)b * sC;
#pragma unroll 1
            for (int c0 = 0; c0 < K2_BN; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * K2_BN + c0), v);
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
                float2 old[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = colt + c0 + half * 16 + i;
                    old[i] = (rd && r < mr && col < n) ? Cb[ci + (int64_t)col * ldc] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = colt + c0 + half * 16 + i;
                    if (r < mr && col < n) {
                        float2 res;
                        res.x = alpha.x * dre[i] - alpha.y * dim[i] + beta.x * old[i].x - beta.y * old[i].y;
                        res.y = alpha.x * dim[i] + alpha.y * dre[i] + beta.x * old[i].y + beta.y * old[i].x;
                        Cb[ci + (int64_t)col * ldc] = res;
                    }
                }
            }
            // this warp's quarter of accumulator ab is read (tcgen05.ld
            // waited): free it for the tile after next
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                                 tempty0 + (uint32_t)(ab * sizeof(uint64_t)))
                             : "memory");
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    cluster_sync();                           // no CTA leaves while its peer may still signal it
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
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


// 3-D fp32 tensor map {inner, rows, batch}, box {16, 128, 1}, 64-byte swizzle
// (one stage of the two-CTA kernel).
int make_map2(CUtensorMap *map, const float *base, int64_t inner, int64_t rows, int64_t batch, int64_t ld_bytes,
              int64_t batch_bytes)
{
    return tc::make_map_3d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, inner, rows, batch, ld_bytes, batch_bytes,
                           K2_BK, K2_BM, CU_TENSOR_MAP_SWIZZLE_64B);
}

// Clusters of two k_tc_cgemm2 CTAs that fit on the current device at once
// (one CTA per SM), looked up once per device.
int k2_pairs(int *out)
{
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    FEAST_CUDA_TRY(cudaGetDevice(&dev));
    FEAST_CUDA_TRY(cudaFuncSetAttribute((const void *)k_tc_cgemm2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)K2_SMEM));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && cached[dev] > 0) {
        *out = cached[dev];
        return FEAST_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(K2_THREADS);
    cfg.dynamicSmemBytes = K2_SMEM;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    FEAST_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, (const void *)k_tc_cgemm2, &cfg));
    if (n < 1) return FEAST_ECUDA;
    if (dev >= 0 && dev < 64) cached[dev] = n;
    *out = n;
    return FEAST_OK;
}

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
                   int *err, TcTimer *tt)
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
    if ((e = make_map2(&mAh, (float *)Ah, kr, mr, batch, kr * 4, mr * kr * 4))) return e;
    if ((e = make_map2(&mAt, (float *)At, kr, mr, batch, kr * 4, mr * kr * 4))) return e;
    if ((e = make_map2(&mXh, Xh, kr, n, batch, kr * 4, kr * n * 4))) return e;
    if ((e = make_map2(&mXt, Xt, kr, n, batch, kr * 4, kr * n * 4))) return e;
    int pairs = 0;
    if ((e = k2_pairs(&pairs))) return e;
    const long long tiles = (long long)batch * ((mr + 2 * K2_BM - 1) / (2 * K2_BM)) * ((n + K2_BN - 1) / K2_BN);
    if (tiles < pairs) pairs = (int)tiles;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * pairs);
    cfg.blockDim = dim3(K2_THREADS);
    cfg.dynamicSmemBytes = K2_SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const bool timed = tt && tt->used + 2 <= 2 * TcTimer::kMax;
    if (timed) FEAST_CUDA_TRY(cudaEventRecord(tt->ev[tt->used++], s));
    FEAST_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_cgemm2, mAh, mAt, mXh, mXt, (int)mr, (int)n, (int)kr, batch, C, ldc,
                                      sC, alpha, beta, err));
    FEAST_LAUNCH_CHECK();
    if (timed) {
        FEAST_CUDA_TRY(cudaEventRecord(tt->ev[tt->used++], s));
        tt->flops += 8.0 * (double)m * (double)n * (double)k * (double)batch;
    }
    return FEAST_OK;
}

// C_b = beta C_b + alpha A_b X_b on tensor cores (see the file comment).
// scratch: tc_scratch_floats(m, k, n, batch) floats (16-byte aligned).
int tc_cgemm(cudaStream_t s, int64_t m, int64_t n, int64_t k, cf alpha, const cf *A, int64_t lda,
             int64_t sA, const cf *X, int64_t ldx, int64_t sX, cf beta, cf *C, int64_t ldc, int64_t sC,
             int batch, float *scratch, int *err, TcTimer *tt)
{
    if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return FEAST_OK;
    int e;
    if ((e = tc_prepare_A(s, m, k, A, lda, sA, batch, scratch))) return e;
    return tc_cgemm_prepA(s, m, n, k, alpha, scratch, X, ldx, sX, beta, C, ldc, sC, batch,
                          scratch + tc_prepA_floats(m, k, batch), err, tt);
}

}  // namespace feast
