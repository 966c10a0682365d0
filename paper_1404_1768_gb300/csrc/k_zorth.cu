// Orthonormalisation of the search and test spaces (GFEAST lines 2 and 17:
// U = U1 R1, B U1 = U2 R2) in FP64.
//
// Block classical Gram-Schmidt with re-orthogonalisation (BCGS2, the
// two-pass form of Barlow & Smoktunowicz): each block of 32 columns is
// projected against the finished columns by two GEMM pairs, and inside the
// block a one-CTA kernel runs column-wise CGS2.  Loss of orthogonality stays
// at rounding level for condition numbers up to ~1/eps, which covers the
// FEAST subspaces (their weakest directions carry filter values down to
// ~1e-10).  R comes out upper triangular with a real positive diagonal.
#include "common.cuh"

namespace feast {

namespace {
constexpr int OB = 32;      // block width
constexpr int OT = 256;     // intra-block threads (32 complex partial sums each)

__device__ __forceinline__ zd warp_sum(zd v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    return v;
}

// Column-wise CGS2 of the n x w panel V (w <= 32) in place; T (w x w, leading
// dim ldt) receives the upper-triangular factor with V_in = V_out T.
__global__ void __launch_bounds__(OT) k_cgs2_intra(int64_t n, int w, zd *V, int64_t ldv, zd *T,
                                                   int64_t ldt)
{
    __shared__ zd red[OT / 32][OB];
    __shared__ zd coef[OB];
    __shared__ double s_nrm;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < w * w; e += OT) T[(e % w) + (e / w) * ldt] = zmake(0.0, 0.0);
    __syncthreads();
    for (int i = 0; i < w; ++i) {
        zd *vi = V + (int64_t)i * ldv;
        for (int pass = 0; pass < 2 && i > 0; ++pass) {
            zd part[OB];
#pragma unroll
            for (int p = 0; p < OB; ++p) part[p] = zmake(0.0, 0.0);
            for (int64_t r = threadIdx.x; r < n; r += OT) {
                zd x = vi[r];
#pragma unroll
                for (int p = 0; p < OB; ++p)
                    if (p < i) zfma_conj(part[p], V[r + (int64_t)p * ldv], x);
            }
#pragma unroll
            for (int p = 0; p < OB; ++p) {
                if (p < i) {
                    zd v = warp_sum(part[p]);
                    if (lane == 0) red[wid][p] = v;
                }
            }
            __syncthreads();
            if (threadIdx.x < i) {
                zd acc = zmake(0.0, 0.0);
                for (int ww = 0; ww < OT / 32; ++ww) acc = zadd(acc, red[ww][threadIdx.x]);
                coef[threadIdx.x] = acc;
                T[threadIdx.x + (int64_t)i * ldt] = zadd(T[threadIdx.x + (int64_t)i * ldt], acc);
            }
            __syncthreads();
            for (int64_t r = threadIdx.x; r < n; r += OT) {
                zd x = vi[r];
                for (int p = 0; p < i; ++p) {
                    zd c = coef[p];
                    zfma(x, zmake(-c.x, -c.y), V[r + (int64_t)p * ldv]);
                }
                vi[r] = x;
            }
            __syncthreads();
        }
        double nrm = 0.0;
        for (int64_t r = threadIdx.x; r < n; r += OT) nrm += zabs2(vi[r]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
        if (lane == 0) red[wid][0].x = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = 0.0;
            for (int ww = 0; ww < OT / 32; ++ww) acc += red[ww][0].x;
            s_nrm = sqrt(acc);
            T[i + (int64_t)i * ldt] = zmake(s_nrm, 0.0);
        }
        __syncthreads();
        const double nv = s_nrm;
        if (nv > 0.0) {
            const double inv = 1.0 / nv;
            for (int64_t r = threadIdx.x; r < n; r += OT) vi[r] = zscale(vi[r], inv);
        }
        __syncthreads();
    }
}
}  // namespace

size_t zorth_work_elems(int64_t n, int64_t m)
{
    (void)n;
    return (size_t)m * OB + 2 * (size_t)OB * OB;
}

int zorth(cudaStream_t s, int64_t n, int64_t m, zd *V, int64_t ldv, zd *R, int64_t ldr,
          zd *work)
{
    if (m <= 0) return FEAST_OK;
    if (m > n) return FEAST_EINVAL;
    zd *S2 = work;
    zd *T1 = S2 + (size_t)m * OB;
    zd *T2 = T1 + (size_t)OB * OB;
    FEAST_CUDA_TRY(cudaMemset2DAsync(R, (size_t)ldr * sizeof(zd), 0, (size_t)m * sizeof(zd), (size_t)m, s));
    const zd one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0), zero = zmake(0.0, 0.0);
    for (int64_t c0 = 0; c0 < m; c0 += OB) {
        const int w = (int)((m - c0) < OB ? (m - c0) : OB);
        zd *Vk = V + c0 * ldv;
        zd *Rd = R + c0 + c0 * ldr;
        if (c0 == 0) {
            k_cgs2_intra<<<1, OT, 0, s>>>(n, w, Vk, ldv, Rd, ldr);
            FEAST_LAUNCH_CHECK();
            continue;
        }
        zd *Ro = R + c0 * ldr;  // R[0:c0, c0:c0+w]
        int e;
        // pass 1: S1 = Q^H Vk (into R), Vk -= Q S1, Vk = W1 T1
        if ((e = zgemm_batched(s, 1, c0, w, n, one, V, ldv, 0, Vk, ldv, 0, zero, Ro, ldr, 0, 1))) return e;
        if ((e = zgemm_batched(s, 0, n, w, c0, mone, V, ldv, 0, Ro, ldr, 0, one, Vk, ldv, 0, 1))) return e;
        k_cgs2_intra<<<1, OT, 0, s>>>(n, w, Vk, ldv, T1, OB);
        FEAST_LAUNCH_CHECK();
        // pass 2: S2 = Q^H W1, W1 -= Q S2, W1 = Qk T2
        if ((e = zgemm_batched(s, 1, c0, w, n, one, V, ldv, 0, Vk, ldv, 0, zero, S2, m, 0, 1))) return e;
        if ((e = zgemm_batched(s, 0, n, w, c0, mone, V, ldv, 0, S2, m, 0, one, Vk, ldv, 0, 1))) return e;
        k_cgs2_intra<<<1, OT, 0, s>>>(n, w, Vk, ldv, T2, OB);
        FEAST_LAUNCH_CHECK();
        // R[0:c0, blk] = S1 + S2 T1,  R[blk, blk] = T2 T1
        if ((e = zgemm_batched(s, 0, c0, w, w, one, S2, m, 0, T1, OB, 0, one, Ro, ldr, 0, 1))) return e;
        if ((e = zgemm_batched(s, 0, w, w, w, one, T2, OB, 0, T1, OB, 0, zero, Rd, ldr, 0, 1))) return e;
    }
    return FEAST_OK;
}

}  // namespace feast
