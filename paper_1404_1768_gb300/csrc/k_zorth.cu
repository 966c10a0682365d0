// Orthonormalisation of the search and test spaces (GFEAST lines 2 and 17:
// U = U1 R1, B U1 = U2 R2) in FP64.
//
// Block classical Gram-Schmidt with re-orthogonalisation (BCGS2, the
// two-pass form of Barlow & Smoktunowicz): each block of 32 columns is
// projected against the finished columns by two GEMM pairs, and inside the
// block column-wise CGS2 runs either on one CTA (short panels) or on a
// cooperative grid that splits the panel's rows over the SMs, each CTA
// keeping its slab in shared memory and the column dot products reduced
// across CTAs in a fixed order (so results do not depend on timing).
// Loss of orthogonality stays
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

// Grid-wide column-wise CGS2 of the n x w panel V (w <= 32).  CTA b owns
// rows [b*rp, min(n, (b+1)*rp)) and keeps them in shared memory (row-major,
// row pitch OB+1 to spread the banks).  Each column takes two projection
// passes and a normalisation, each of which is a CTA-local partial sum, a
// grid barrier and a fixed-order sum of the partials (part, two buffers
// used alternately so a buffer is rewritten only after every CTA has passed
// the barrier that follows its last read).  CTA 0 writes T.
__global__ void __launch_bounds__(OT) k_cgs2_grid(int64_t n, int w, zd *V, int64_t ldv, zd *T,
                                                  int64_t ldt, int rp, zd *part, GridSync g)
{
    extern __shared__ zd slab[];
    __shared__ zd red[OT / 32][OB];
    __shared__ zd coef[OB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rp;
    const int rows = (int)((n - r0) < rp ? ((n - r0) > 0 ? (n - r0) : 0) : rp);
    constexpr int P = OB + 1;
    for (int e = threadIdx.x; e < rows * w; e += OT) {
        const int r = e % rows, p = e / rows;
        slab[r * P + p] = __ldcg(V + r0 + r + (int64_t)p * ldv);
    }
    if (blockIdx.x == 0)
        for (int e = threadIdx.x; e < w * w; e += OT) T[(e % w) + (e / w) * ldt] = zmake(0.0, 0.0);
    __syncthreads();
    int buf = 0;
    for (int i = 0; i < w; ++i) {
        for (int pass = 0; pass < 2 && i > 0; ++pass) {
            // partial dots  V(:, p)^H V(:, i)  over this CTA's rows, p = lane
            zd acc = zmake(0.0, 0.0);
            if (lane < i)
                for (int r = wid; r < rows; r += OT / 32) zfma_conj(acc, slab[r * P + lane], slab[r * P + i]);
            red[wid][lane] = acc;
            __syncthreads();
            zd *pb = part + (size_t)buf * OB * G;
            if (threadIdx.x < OB) {
                zd sum = zmake(0.0, 0.0);
                for (int ww = 0; ww < OT / 32; ++ww) sum = zadd(sum, red[ww][threadIdx.x]);
                __stcg(pb + (size_t)blockIdx.x * OB + threadIdx.x, sum);
            }
            if (!grid_barrier(g)) return;
            // fixed-order sum over the CTAs: lane picks p, warp wid a stride of CTAs
            zd tot = zmake(0.0, 0.0);
            if (lane < i)
                for (int b = wid; b < G; b += OT / 32) tot = zadd(tot, __ldcg(pb + (size_t)b * OB + lane));
            red[wid][lane] = tot;
            __syncthreads();
            if (threadIdx.x < i) {
                zd c = zmake(0.0, 0.0);
                for (int ww = 0; ww < OT / 32; ++ww) c = zadd(c, red[ww][threadIdx.x]);
                coef[threadIdx.x] = c;
                if (blockIdx.x == 0)
                    T[threadIdx.x + (int64_t)i * ldt] = zadd(T[threadIdx.x + (int64_t)i * ldt], c);
            }
            __syncthreads();
            for (int r = threadIdx.x; r < rows; r += OT) {
                zd x = slab[r * P + i];
                for (int p = 0; p < i; ++p) {
                    const zd c = coef[p];
                    zfma(x, zmake(-c.x, -c.y), slab[r * P + p]);
                }
                slab[r * P + i] = x;
            }
            buf ^= 1;
            __syncthreads();
        }
        // norm of column i
        double nrm = 0.0;
        for (int r = threadIdx.x; r < rows; r += OT) nrm += zabs2(slab[r * P + i]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
        if (lane == 0) red[wid][0].x = nrm;
        __syncthreads();
        zd *pb = part + (size_t)buf * OB * G;
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int ww = 0; ww < OT / 32; ++ww) s += red[ww][0].x;
            __stcg(pb + (size_t)blockIdx.x * OB, zmake(s, 0.0));
        }
        if (!grid_barrier(g)) return;
        if (threadIdx.x < 32) {
            double s = 0.0;
            for (int b = threadIdx.x; b < G; b += 32) s += __ldcg(pb + (size_t)b * OB).x;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (threadIdx.x == 0) {
                red[0][0].x = sqrt(s);
                if (blockIdx.x == 0) T[i + (int64_t)i * ldt] = zmake(red[0][0].x, 0.0);
            }
        }
        __syncthreads();
        const double nv = red[0][0].x;
        if (nv > 0.0) {
            const double inv = 1.0 / nv;
            for (int r = threadIdx.x; r < rows; r += OT) slab[r * P + i] = zscale(slab[r * P + i], inv);
        }
        buf ^= 1;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < rows * w; e += OT) {
        const int r = e % rows, p = e / rows;
        V[r0 + r + (int64_t)p * ldv] = slab[r * P + p];
    }
}

constexpr int GMAX = 256;           // most CTAs of the grid form
constexpr int RP_MIN = 32;          // fewest rows a CTA of the grid form takes

struct IntraPlan {
    int grid = 0;                   // 0: one-CTA kernel
    int rp = 0;
    size_t smem = 0;
};

// The grid form pays for ~3 grid barriers per column; it is used when the
// panel is tall enough that one SM's FP64 rate would dominate instead.
int plan_intra(int64_t n, IntraPlan &pl)
{
    pl = IntraPlan{};
    if (n < 4 * RP_MIN) return FEAST_OK;
    int dev = 0, sms = 0, smem_max = 0;
    FEAST_CUDA_TRY(cudaGetDevice(&dev));
    FEAST_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FEAST_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int G = (int)((n + RP_MIN - 1) / RP_MIN);
    if (G > sms) G = sms;
    if (G > GMAX) G = GMAX;
    const int rp = (int)((n + G - 1) / G);
    const size_t smem = (size_t)rp * (OB + 1) * sizeof(zd);
    if (smem + 8192 > (size_t)smem_max) return FEAST_OK;
    FEAST_CUDA_TRY(allow_dyn_smem(k_cgs2_grid));
    int per = 0;
    FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cgs2_grid, OT, smem));
    if (per < 1 || G > per * sms) return FEAST_OK;
    pl.grid = (int)((n + rp - 1) / rp);
    pl.rp = rp;
    pl.smem = smem;
    return FEAST_OK;
}

int run_intra(cudaStream_t s, const IntraPlan &pl, int64_t n, int w, zd *V, int64_t ldv, zd *T,
              int64_t ldt, zd *part, GridSync g)
{
    if (!pl.grid) {
        k_cgs2_intra<<<1, OT, 0, s>>>(n, w, V, ldv, T, ldt);
        FEAST_LAUNCH_CHECK();
        return FEAST_OK;
    }
    int rp = pl.rp;
    void *args[] = {&n, &w, &V, &ldv, &T, &ldt, &rp, &part, &g};
    FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_cgs2_grid, dim3(pl.grid), dim3(OT), args, pl.smem, s));
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}
}  // namespace

size_t zorth_work_elems(int64_t n, int64_t m)
{
    (void)n;
    return (size_t)m * OB + 2 * (size_t)OB * OB + 2 * (size_t)GMAX * OB + 1;
}

int zorth(cudaStream_t s, int64_t n, int64_t m, zd *V, int64_t ldv, zd *R, int64_t ldr,
          zd *work, int *timeout, const OzScratch *oz)
{
    if (m <= 0) return FEAST_OK;
    if (m > n) return FEAST_EINVAL;
    zd *S2 = work;
    zd *T1 = S2 + (size_t)m * OB;
    zd *T2 = T1 + (size_t)OB * OB;
    zd *part = T2 + (size_t)OB * OB;
    unsigned *bar = (unsigned *)(part + 2 * (size_t)GMAX * OB);
    IntraPlan pl;
    int e = plan_intra(n, pl);
    if (e) return e;
    GridSync gs{bar, bar + 1, timeout, TO_CGS2};
    if (pl.grid) FEAST_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    FEAST_CUDA_TRY(cudaMemset2DAsync(R, (size_t)ldr * sizeof(zd), 0, (size_t)m * sizeof(zd), (size_t)m, s));
    const zd one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0), zero = zmake(0.0, 0.0);
    for (int64_t c0 = 0; c0 < m; c0 += OB) {
        const int w = (int)((m - c0) < OB ? (m - c0) : OB);
        zd *Vk = V + c0 * ldv;
        zd *Rd = R + c0 + c0 * ldr;
        if (c0 == 0) {
            if ((e = run_intra(s, pl, n, w, Vk, ldv, Rd, ldr, part, gs))) return e;
            continue;
        }
        zd *Ro = R + c0 * ldr;  // R[0:c0, c0:c0+w]
        // pass 1: S1 = Q^H Vk (into R), Vk -= Q S1, Vk = W1 T1
        // (with oz: the tall updates V_k -= Q S on the tensor cores, Q's
        // digit planes made once per block)
        if (oz && (e = oz_prepare_rows(s, n, c0, V, ldv, oz->rows))) return e;
        if ((e = zgemm_batched(s, 1, c0, w, n, one, V, ldv, 0, Vk, ldv, 0, zero, Ro, ldr, 0, 1))) return e;
        if (oz) {
            if ((e = oz_prepare_cols(s, c0, w, Ro, ldr, oz->cols))) return e;
            if ((e = oz_gemm(s, n, w, c0, oz->rows, oz->cols, mone, nullptr, 0, one, Vk, ldv, oz->err))) return e;
        } else if ((e = zgemm_batched(s, 0, n, w, c0, mone, V, ldv, 0, Ro, ldr, 0, one, Vk, ldv, 0, 1))) {
            return e;
        }
        if ((e = run_intra(s, pl, n, w, Vk, ldv, T1, OB, part, gs))) return e;
        // pass 2: S2 = Q^H W1, W1 -= Q S2, W1 = Qk T2
        if ((e = zgemm_batched(s, 1, c0, w, n, one, V, ldv, 0, Vk, ldv, 0, zero, S2, m, 0, 1))) return e;
        if (oz) {
            if ((e = oz_prepare_cols(s, c0, w, S2, m, oz->cols))) return e;
            if ((e = oz_gemm(s, n, w, c0, oz->rows, oz->cols, mone, nullptr, 0, one, Vk, ldv, oz->err))) return e;
        } else if ((e = zgemm_batched(s, 0, n, w, c0, mone, V, ldv, 0, S2, m, 0, one, Vk, ldv, 0, 1))) {
            return e;
        }
        if ((e = run_intra(s, pl, n, w, Vk, ldv, T2, OB, part, gs))) return e;
        // R[0:c0, blk] = S1 + S2 T1,  R[blk, blk] = T2 T1
        if ((e = zgemm_batched(s, 0, c0, w, w, one, S2, m, 0, T1, OB, 0, one, Ro, ldr, 0, 1))) return e;
        if ((e = zgemm_batched(s, 0, w, w, w, one, T2, OB, 0, T1, OB, 0, zero, Rd, ldr, 0, 1))) return e;
    }
    return FEAST_OK;
}

}  // namespace feast
