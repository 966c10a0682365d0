// FP64-accurate complex GEMM on the bf16 tensor cores (tcgen05, kind::f16)
// by exact integer slicing, for the refinement residual of the precision
// form (and any FP64 product that tolerates ~2^-47 relative to |A||B|).
//
//   C = beta C + alpha_c A B       A: M x K, B: K x N complex128, column-major
//
// Complex as real: A' (2M x 2K) has rows 2i = [Re a_ik, -Im a_ik]_k and
// 2i+1 = [Im a_ik, Re a_ik]_k; B' (2K x N) is B's columns read as
// interleaved reals.  Every row of A' is scaled by a power of two 2^-e_i so
// its entries lie in (-1, 1) and written in base 64 with OZ_S signed digits
// (digit 1 in [-64, 64], later digits in [-32, 32]):
//     A' = diag(2^e) sum_s 64^-s A_s ,   likewise B' = (sum_t 64^-t B_t) diag(2^f).
// Digits are small integers, exact in bf16, and a digit product is exact in
// the FP32 accumulator; so is any sum of products of one weight class
// g = s + t over a K-chunk of OZ_KC terms while it stays below 2^24 (the
// leading classes always do; a late class can pass it only by a factor
// ~1.3 at worst, and rounds then at a weight below 2^-60).  The kernel keeps
// one tensor-memory accumulator per class g = 2..9 (all products with
// s + t <= OZ_S + 1; the rest weigh < 2^-60), reads the classes out after
// each K-chunk, combines them on the integer pipe into two exact int64
// partials and adds acc += sum_g 64^-(g-2) S_g in FP64 with two roundings;
// finally C gets alpha_c 2^(e_i + f_j - 12) acc.
// Representation and truncation error: ~2^-48 relative to
// max_k |A'_ik| * max_k |B'_kj| per entry, K-fold at most.
//
// Per CTA: one 128 x 64 tile of A'B'.  Warp 4 (one lane) streams K-stages of
// 32 bf16 (64-byte swizzle rows) of all OZ_S slices of both operands with
// TMA into a two-deep ring; warp 5 (one lane) issues the 36 slice products
// per K-step of 16 into the eight accumulators (8 x 64 = all 512 TMEM
// columns) and commits each stage and each K-chunk; warps 0-3 own TMEM
// lanes 0-127 and run the chunk read-outs and the final write.  All waits
// are bounded; on expiry the CTA raises *err and finishes.
#include "tcgen05.cuh"

namespace feast {

namespace {
using namespace tc;

constexpr int OZ_S = 8;                      // digits per operand entry
constexpr int OZ_NG = OZ_S;                  // weight classes g = 2 .. OZ_S + 1
constexpr int OZ_BM = 128;                   // rows of A' per tile
constexpr int OZ_BN = 64;                    // columns per tile
constexpr int OZ_BK = 32;                    // bf16 per stage row (64 bytes)
constexpr int OZ_STAGES = 2;
constexpr int OZ_KC = 2048;                  // K per exact chunk (real K)
constexpr int OZ_GM = 8;                     // row tiles per raster group
constexpr int OZ_THREADS = 192;
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2; // 8 KiB per slice
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2; // 4 KiB per slice
constexpr int OZ_STAGE = OZ_S * (OZ_A_TILE + OZ_B_TILE);

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    // exact: |digit| <= 64
    const uint32_t a = __float_as_uint(lo) >> 16, b = __float_as_uint(hi) >> 16;
    return a | (b << 16);
}

// x as a double, exactly, for |x| < 2^51: 1.5 2^52 + x has x in its low
// significand bits
__device__ __forceinline__ double exact_double(long long x)
{
    return __longlong_as_double(x + 0x4338000000000000LL) - 6755399441055744.0;
}

// A row or column with an Inf or NaN entry: its products are NaN (its
// digits are zero, and the epilogue writes NaN).
constexpr int OZ_NONFINITE = -0x40000000;

// The larger of |Re v|, |Im v| as IEEE bits (non-negative doubles order like
// their bits), folded into mx; bad is set for a non-finite entry.
__device__ __forceinline__ void fold_mag(zd v, unsigned long long &mx, bool &bad)
{
    const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffull;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffull;
    const unsigned long long m = a > b ? a : b;
    bad = bad || m >= 0x7ff0000000000000ull;
    mx = m > mx ? m : mx;
}

// Warp-wide: the exponent e with max < 2^e (frexp's; 0 for zero), or
// OZ_NONFINITE, in every lane.
__device__ __forceinline__ int warp_exponent(unsigned long long mx, bool bad)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    if (__any_sync(0xffffffffu, bad)) return OZ_NONFINITE;
    if (mx == 0) return 0;
    const int bexp = (int)(mx >> 52);
    return bexp ? bexp - 1022 : 64 - __clzll((long long)mx) - 1074;   // (subnormal max)
}

// e_i with max_k max(|Re a_ik|, |Im a_ik|) < 2^e_i (0 for a zero row); one
// warp per row.  ct: the operand is the conjugate transpose of the stored
// matrix, a_ik = conj(A[k + i lda]).
__global__ void k_oz_rowexp(int64_t M, int64_t K, const zd *__restrict__ A, int64_t lda, int ct,
                            int *__restrict__ e)
{
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= M) return;
    unsigned long long mx = 0;
    bool bad = false;
    for (int64_t k = lane; k < K; k += 32) fold_mag(ct ? A[k + i * lda] : A[i + k * lda], mx, bad);
    const int ex = warp_exponent(mx, bad);
    if (lane == 0) e[i] = ex;
}

// f_j for column j of B (one warp per column).
__global__ void k_oz_colexp(int64_t K, int64_t N, const zd *__restrict__ B, int64_t ldb, int *__restrict__ f)
{
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= N) return;
    unsigned long long mx = 0;
    bool bad = false;
    for (int64_t k = lane; k < K; k += 32) fold_mag(B[k + j * ldb], mx, bad);
    const int ex = warp_exponent(mx, bad);
    if (lane == 0) f[j] = ex;
}

// Digits of one real value v (IEEE bits b) scaled by 2^-e into (-1, 1):
// with N_s = rint(64^s v 2^-e) (round half to even), digit s is
// N_s - 64 N_(s-1) -- the same digits as the recursion t = 64 r, d = rint(t),
// r = t - d, whose steps are all exact (a subtracted multiple of 64 is even,
// so it commutes with the rounding).  Each N_s comes from the 53-bit
// significand by an integer shift with round-half-even, so the slicing runs
// on the integer pipe, not the FP64 one (1/64 of the FP32 rate on this part),
// and is exact for subnormal rows too.  (v is finite: rows and columns with
// an Inf or NaN are not sliced.)
__device__ __forceinline__ void digits(unsigned long long b, int e, float (&d)[OZ_S])
{
    const int ex = (int)(b >> 52) & 0x7ff;
    const unsigned long long mant = (b & 0xfffffffffffffull) | (ex ? (1ull << 52) : 0ull);
    const int base = (ex ? ex : 1) - 1075 - e;   // |v| 2^-e = mant 2^base < 1
    const bool neg = (b >> 63) != 0;
    long long prev = 0;
#pragma unroll
    for (int s = 1; s <= OZ_S; ++s) {
        const int rs = -(base + 6 * s);
        unsigned long long q;
        if (rs <= 0) {
            q = mant << (-rs);                       // (a subnormal row: no bits below the point)
        } else if (rs >= 64) {
            q = 0;                                   // below 2^-11
        } else {
            q = mant >> rs;
            const unsigned long long rem = mant & ((1ull << rs) - 1), half = 1ull << (rs - 1);
            q += (rem > half || (rem == half && (q & 1))) ? 1ull : 0ull;
        }
        const long long N = neg ? -(long long)q : (long long)q;
        d[s - 1] = (float)(int)(N - 64 * prev);      // |digit| <= 64: exact
        prev = N;
    }
}

// A' digit planes: plane s is (2M x kp) bf16, row-major; thread per
// (real row, complex column).  Columns K .. kp/2 - 1 are zero padding.
__global__ void k_oz_slice_rows(int64_t M, int64_t K, const zd *__restrict__ A, int64_t lda, int ct,
                                const int *__restrict__ e, uint32_t *__restrict__ planes, int64_t kp)
{
    const int64_t half = kp / 2;
    const int64_t total = 2 * M * half;
    const int64_t plane = 2 * M * kp / 2;   // in 32-bit words
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rr = x / half, kc = x % half;
        const int64_t i = rr >> 1;
        float d0[OZ_S], d1[OZ_S];
        const int ei = e[i];
        if (kc < K && ei != OZ_NONFINITE) {
            const zd v = ct ? A[kc + i * lda] : A[i + kc * lda];
            const unsigned long long sgn = 1ull << 63;
            const unsigned long long a = (unsigned long long)__double_as_longlong(v.x);
            const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) ^ (ct ? sgn : 0ull);
            if ((rr & 1) == 0) { digits(a, ei, d0); digits(b ^ sgn, ei, d1); }
            else { digits(b, ei, d0); digits(a, ei, d1); }
        } else {
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) { d0[s] = 0.f; d1[s] = 0.f; }
        }
        const int64_t o = rr * half + kc;
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) planes[(int64_t)s * plane + o] = pack_bf16x2(d0[s], d1[s]);
    }
}

// B' digit planes: plane s is (N x kp) bf16, row j = column j of B as
// interleaved reals; thread per (column, complex row).
__global__ void k_oz_slice_cols(int64_t K, int64_t N, const zd *__restrict__ B, int64_t ldb,
                                const int *__restrict__ f, uint32_t *__restrict__ planes, int64_t kp)
{
    const int64_t half = kp / 2;
    const int64_t total = N * half;
    const int64_t plane = N * half;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = x / half, kc = x % half;
        float d0[OZ_S], d1[OZ_S];
        const int fj = f[j];
        if (kc < K && fj != OZ_NONFINITE) {
            const zd v = B[kc + j * ldb];
            digits((unsigned long long)__double_as_longlong(v.x), fj, d0);
            digits((unsigned long long)__double_as_longlong(v.y), fj, d1);
        } else {
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) { d0[s] = 0.f; d1[s] = 0.f; }
        }
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) planes[(int64_t)s * plane + x] = pack_bf16x2(d0[s], d1[s]);
    }
}

struct OzOut {
    zd *C;
    int64_t ldc;
    zd alpha;
    const zd *zcol;     // optional per-column-block factor (alpha_c = alpha * zcol[c / cblk])
    int64_t cblk;
    zd beta;
};

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int mr, int n,
              int kr, const int *__restrict__ ea, const int *__restrict__ fb, OzOut out, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[OZ_STAGES], empty[OZ_STAGES], chunk_full, tmem_empty;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // raster: OZ_GM row tiles side by side share each column tile's operands in L2
    const int Mt = (mr + OZ_BM - 1) / OZ_BM, Nt = (n + OZ_BN - 1) / OZ_BN;
    const int L = blockIdx.x;
    const int grp = L / (OZ_GM * Nt);
    const int gbase = grp * OZ_GM;
    const int gsz = (Mt - gbase) < OZ_GM ? (Mt - gbase) : OZ_GM;
    const int rem = L - grp * OZ_GM * Nt;
    const int rt = gbase + rem % gsz, ct = rem / gsz;
    const int row0 = rt * OZ_BM, col0 = ct * OZ_BN;
    const int kb_n = (kr + OZ_BK - 1) / OZ_BK;
    constexpr int KB_CHUNK = OZ_KC / OZ_BK;
    const int nchunk = (kb_n + KB_CHUNK - 1) / KB_CHUNK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&chunk_full, 1);
        mbar_init(&tmem_empty, 128);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        if (lane == 0) {
            // producer
            int issued = 0;
            for (int kb = 0; kb < kb_n; ++kb) {
                const int s = kb % OZ_STAGES;
                const uint32_t ph = (uint32_t)((kb / OZ_STAGES) & 1);
                if (!mbar_wait(&empty[s], ph ^ 1u) || *(volatile int *)&s_fail) { s_fail = 1; break; }
                unsigned char *st = base + s * OZ_STAGE;
                mbar_expect_tx(&full[s], OZ_STAGE);
                const int kx = kb * OZ_BK;
#pragma unroll 1
                for (int sl = 0; sl < OZ_S; ++sl) {
                    tma_load_3d(st + sl * OZ_A_TILE, &tA, &full[s], kx, row0, sl);
                    tma_load_3d(st + OZ_S * OZ_A_TILE + sl * OZ_B_TILE, &tB, &full[s], kx, col0, sl);
                }
                issued = kb + 1;
            }
            // on failure, let the copies already issued land before the CTA exits
            if (s_fail)
                for (int kb = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); kb < issued; ++kb)
                    mbar_wait(&full[kb % OZ_STAGES], (uint32_t)((kb / OZ_STAGES) & 1));
        }
    } else if (warp == 5) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f32acc(1u, OZ_BM, OZ_BN);
            bool ok = true;
            for (int kb = 0; kb < kb_n && ok; ++kb) {
                const int s = kb % OZ_STAGES;
                const uint32_t ph = (uint32_t)((kb / OZ_STAGES) & 1);
                const int chunk = kb / KB_CHUNK;
                const bool first = (kb % KB_CHUNK) == 0;
                if (first && chunk > 0) {
                    // the read-out of the previous chunk must be done
                    if (!mbar_wait(&tmem_empty, (uint32_t)((chunk - 1) & 1))) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                }
                if (!mbar_wait(&full[s], ph) || *(volatile int *)&s_fail) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                unsigned char *st = base + s * OZ_STAGE;
                const uint32_t a0 = smem_u32(st), b0 = smem_u32(st + OZ_S * OZ_A_TILE);
                const uint64_t adesc = sdesc<64>(st), bdesc = sdesc<64>(st + OZ_S * OZ_A_TILE);
                (void)a0;
                (void)b0;
#pragma unroll
                for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
                    for (int sa = 0; sa < OZ_S; ++sa) {
#pragma unroll
                        for (int sb = 0; sb < OZ_S - sa; ++sb) {
                            const int g = sa + sb;
                            const uint64_t ad = adesc + (uint64_t)((sa * OZ_A_TILE + kk * 32) >> 4);
                            const uint64_t bd = bdesc + (uint64_t)((sb * OZ_B_TILE + kk * 32) >> 4);
                            const uint32_t acc = (first && kk == 0 && sa == 0) ? 0u : 1u;
                            mma_f16(tmem + (uint32_t)(g * OZ_BN), ad, bd, idesc, acc);
                        }
                    }
                }
                mma_commit(&empty[s]);
                if ((kb % KB_CHUNK) == KB_CHUNK - 1 || kb == kb_n - 1) mma_commit(&chunk_full);
            }
            if (!ok) s_fail = 1;
        }
    } else {
        // read-out warps 0-3: TMEM lanes 32 * warp ..
        double acc[OZ_BN];
#pragma unroll
        for (int j = 0; j < OZ_BN; ++j) acc[j] = 0.0;
        bool good = true;
        for (int c = 0; c < nchunk; ++c) {
            if (!mbar_wait(&chunk_full, (uint32_t)(c & 1)) || *(volatile int *)&s_fail) { good = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // acc += sum_g 64^-g S_g = 2^-18 (hi + 2^-24 lo) with the exact
            // integers hi = sum_(g<4) 64^(3-g) S_g, lo = sum_(g>=4) 64^(7-g) S_g
            // (|hi|, |lo| < 2^45): two roundings per chunk instead of eight,
            // and the class sums combined on the integer pipe
            static_assert(OZ_NG == 8, "the read-out pairs eight weight classes");
            const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
            for (int cg = 0; cg < OZ_BN / 8; ++cg) {
                int p[4][8];   // p_q = 64 S_2q + S_(2q+1) (|p_q| < 2^31)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t va[8], vb[8];
                    tmem_ld8x2(tw + (uint32_t)(2 * q * OZ_BN + cg * 8), tw + (uint32_t)((2 * q + 1) * OZ_BN + cg * 8),
                               va, vb);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        p[q][j] = __float2int_rn(__uint_as_float(va[j])) * 64 + __float2int_rn(__uint_as_float(vb[j]));
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const long long hi = (long long)p[0][j] * 4096 + p[1][j];
                    const long long lo = (long long)p[2][j] * 4096 + p[3][j];
                    const double t = fma(exact_double(lo), 0x1p-24, exact_double(hi));
                    acc[cg * 8 + j] = fma(t, 0x1p-18, acc[cg * 8 + j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&tmem_empty);
        }
        if (!good) {
            if (lane == 0) s_fail = 1;
        } else {
            const int r = row0 + warp * 32 + lane;           // real row
            const bool im_row = (r & 1) != 0;
            const int64_t ci = r >> 1;
            const int er = (r < mr) ? ea[ci] : 0;
            // pair the Re / Im rows (neighbouring lanes); the even lane writes
            // columns 0..31 of the tile, the odd lane 32..63, eight at a time
            // with the old values loaded first
            const int hsel = im_row ? 1 : 0;
            const bool rd = (out.beta.x != 0.0 || out.beta.y != 0.0);
            // (a real alpha and a unit beta, the common cases, skip the complex products)
            const bool real_alpha = out.zcol == nullptr && out.alpha.y == 0.0;
            const bool unit_beta = out.beta.x == 1.0 && out.beta.y == 0.0;
#pragma unroll
            for (int g8 = 0; g8 < OZ_BN / 2; g8 += 8) {
                zd d[8], o[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const double m0v = acc[g8 + i], m1v = acc[32 + g8 + i];
                    const double o0 = __shfl_xor_sync(0xffffffffu, m0v, 1);
                    const double o1 = __shfl_xor_sync(0xffffffffu, m1v, 1);
                    const double mine = hsel ? m1v : m0v, other = hsel ? o1 : o0;
                    d[i] = zmake(im_row ? other : mine, im_row ? mine : other);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int col = col0 + hsel * 32 + g8 + i;
                    o[i] = (rd && r < mr && col < n) ? out.C[ci + (int64_t)col * out.ldc] : zmake(0.0, 0.0);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int col = col0 + hsel * 32 + g8 + i;
                    if (r < mr && col < n && (er == OZ_NONFINITE || fb[col] == OZ_NONFINITE)) {
                        out.C[ci + (int64_t)col * out.ldc] = zmake(__longlong_as_double(0x7ff8000000000000LL),
                                                                   __longlong_as_double(0x7ff8000000000000LL));
                    } else if (r < mr && col < n) {
                        // d 2^(e_i + f_j - 12): a power of two built from its bits, or
                        // (a result near the ends of the range) ldexp, one rounding
                        const int ex = er + fb[col] - 12;
                        zd res = (ex >= -1022 && ex <= 1023)
                                     ? zscale(d[i], __longlong_as_double((long long)(ex + 1023) << 52))
                                     : zmake(ldexp(d[i].x, ex), ldexp(d[i].y, ex));
                        if (real_alpha) {
                            if (out.alpha.x != 1.0) res = zscale(res, out.alpha.x);
                        } else {
                            zd al = out.alpha;
                            if (out.zcol) al = zmul(al, out.zcol[col / out.cblk]);
                            res = zmul(al, res);
                        }
                        if (rd) res = zadd(res, unit_beta ? o[i] : zmul(out.beta, o[i]));
                        out.C[ci + (int64_t)col * out.ldc] = res;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) atomicOr(err, TO_OZ);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

int64_t oz_kp(int64_t K) { return ((2 * K + 63) / 64) * 64; }
}  // namespace

size_t oz_rows_bytes(int64_t M, int64_t K) { return (size_t)OZ_S * 2 * M * oz_kp(K) * 2 + 256 + 4 * (size_t)M; }
size_t oz_cols_bytes(int64_t K, int64_t N) { return (size_t)OZ_S * N * oz_kp(K) * 2 + 256 + 4 * (size_t)N; }

// Digit planes of the left operand (M x K): A itself, or with ct the
// conjugate transpose of the stored K x M matrix A; at `work`,
// oz_rows_bytes(M, K).
int oz_prepare_rows(cudaStream_t s, int64_t M, int64_t K, const zd *A, int64_t lda, void *work, int ct)
{
    if (M <= 0 || K <= 0) return FEAST_OK;
    const int64_t kp = oz_kp(K);
    uint32_t *planes = (uint32_t *)work;
    int *e = (int *)((char *)work + (size_t)OZ_S * 2 * M * kp * 2 + 256);
    k_oz_rowexp<<<cdiv((size_t)M * 32, 256), 256, 0, s>>>(M, K, A, lda, ct, e);
    FEAST_LAUNCH_CHECK();
    const int64_t total = 2 * M * (kp / 2);
    k_oz_slice_rows<<<cdiv(total, 256) > 16384 ? 16384 : cdiv(total, 256), 256, 0, s>>>(M, K, A, lda, ct, e, planes,
                                                                                         kp);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// Digit planes of the right operand B (K x N): at `work`, oz_cols_bytes(K, N).
int oz_prepare_cols(cudaStream_t s, int64_t K, int64_t N, const zd *B, int64_t ldb, void *work)
{
    if (N <= 0 || K <= 0) return FEAST_OK;
    const int64_t kp = oz_kp(K);
    uint32_t *planes = (uint32_t *)work;
    int *f = (int *)((char *)work + (size_t)OZ_S * N * kp * 2 + 256);
    k_oz_colexp<<<cdiv((size_t)N * 32, 256), 256, 0, s>>>(K, N, B, ldb, f);
    FEAST_LAUNCH_CHECK();
    const int64_t total = N * (kp / 2);
    k_oz_slice_cols<<<cdiv(total, 256) > 16384 ? 16384 : cdiv(total, 256), 256, 0, s>>>(K, N, B, ldb, f, planes, kp);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// C = beta C + alpha_c A B from prepared digit planes (A: M x K rows work,
// B: K x N cols work).  alpha_c = alpha * zcol[c / cblk] when zcol is set.
int oz_gemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, const void *Arows, const void *Bcols, zd alpha,
            const zd *zcol, int64_t cblk, zd beta, zd *C, int64_t ldc, int *err)
{
    if (M <= 0 || N <= 0 || K <= 0) return FEAST_OK;
    const int64_t kp = oz_kp(K);
    const int64_t mr = 2 * M;
    const int *ea = (const int *)((const char *)Arows + (size_t)OZ_S * mr * kp * 2 + 256);
    const int *fb = (const int *)((const char *)Bcols + (size_t)OZ_S * N * kp * 2 + 256);
    CUtensorMap mA, mB;
    int e;
    if ((e = make_map_3d(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Arows, kp, mr, OZ_S, kp * 2, mr * kp * 2, OZ_BK,
                         OZ_BM, CU_TENSOR_MAP_SWIZZLE_64B)))
        return e;
    if ((e = make_map_3d(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Bcols, kp, N, OZ_S, kp * 2, N * kp * 2, OZ_BK,
                         OZ_BN, CU_TENSOR_MAP_SWIZZLE_64B)))
        return e;
    const size_t smem = (size_t)OZ_STAGES * OZ_STAGE + 1024;
    FEAST_CUDA_TRY(allow_dyn_smem(k_oz_gemm));
    const int64_t tiles = ((mr + OZ_BM - 1) / OZ_BM) * ((N + OZ_BN - 1) / OZ_BN);
    if (tiles > 0x7fffffff) return FEAST_EINVAL;
    OzOut o{C, ldc, alpha, zcol, cblk > 0 ? cblk : 1, beta};
    k_oz_gemm<<<(unsigned)tiles, OZ_THREADS, smem, s>>>(mA, mB, (int)mr, (int)N, (int)(2 * K), ea, fb, o, err);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
