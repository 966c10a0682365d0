// Banded pencils (e.g. the 5-point convection-diffusion operator, half
// bandwidth = grid width): formation of z_j B - A in LAPACK general-band
// storage, node-batched blocked band LU with partial pivoting, band solves
// with many right-hand sides, band products and the refinement residual.
//
// Factor storage per node: ldab = 2 kl + ku + 1 rows, kv = kl + ku; entry
// (i, c) lives at F[kv + i - c + c * ldab] for c - kv <= i <= c + kl.  The
// multipliers follow the unblocked convention (each column's multipliers
// are stored as they were when that column was eliminated; later row
// interchanges are not applied to them), so L stays inside kl subdiagonals
// and the solve interleaves interchanges and eliminations column by column.
//
// The LU is blocked by panels of NB columns.  A panel (NB + kl rows) is
// copied to a dense scratch, factored there with the dense panel kernel,
// its interchanges are applied to the columns right of it, U12 = L11^{-1}
// A12 and the trailing update A22 -= L21 U12 (kl x kv, band-masked) follow,
// and the panel is written back with its multipliers converted to the
// unblocked convention.  The solves are sequential along the band (one
// column per step) but parallel over nodes and over chunks of right-hand
// sides; each CTA keeps a sliding window of kl + 1 (forward) or kv + 1
// (backward) rows of its right-hand sides in shared memory.
#include "common.cuh"

namespace feast {

namespace {
constexpr int GB_NB = 32;     // panel width
constexpr int GB_CW = 8;      // right-hand sides per solve CTA (at most; fewer for wide bands)
constexpr int GB_ST = 256;    // solve threads (>= kl and >= kv handled by striding)
constexpr int GB_JC = 32;     // solve steps per staged chunk (at most: one warp's lanes)

__host__ __device__ __forceinline__ int64_t bidx(int64_t kv, int64_t ldab, int64_t i, int64_t c)
{
    return kv + i - c + c * ldab;
}

__device__ __forceinline__ float2 shfl_cx(float2 v, int src)
{
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ double2 shfl_cx(double2 v, int src)
{
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// F_j = z_j B - A in factor storage; rows 0..kl-1 of each column (fill) = 0.
template <typename T>
__global__ void k_gb_form(int64_t n, int64_t kl, int64_t ku, const zd *A, const zd *B, int64_t ldin,
                          const zd *z, T *F, int64_t ldab, int64_t sF)
{
    typedef typename CxReal<T>::type R;
    const int j = blockIdx.y;
    const zd zj = z[j];
    const int64_t kv = kl + ku, total = ldab * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % ldab, c = e / ldab;
        const int64_t i = r - kv + c;  // matrix row of this slot
        zd v = zmake(0.0, 0.0);
        if (r >= kl && i >= 0 && i < n) {
            const int64_t s = ku + i - c + c * ldin;  // compact storage slot
            zd bij = B ? B[s] : zmake(i == c ? 1.0 : 0.0, 0.0);
            v = zsub(zmul(zj, bij), A[s]);
        }
        F[(int64_t)j * sF + e] = cx<T>((R)v.x, (R)v.y);
    }
}

// Dense scratch of the panel: D(r, cc) = F(k0 + r, k0 + cc), zero outside
// the band or the matrix.  D: rows x NB per node (leading dim ldd).
template <typename T>
__global__ void k_gb_gather(int64_t n, int64_t kl, int64_t ku, int64_t k0, int rows, int nb,
                            const T *F, int64_t ldab, int64_t sF, T *D, int ldd, int64_t sD)
{
    const int b = blockIdx.y;
    const T *Fb = F + (int64_t)b * sF;
    T *Db = D + (int64_t)b * sD;
    const int64_t kv = kl + ku;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ldd * GB_NB; e += gridDim.x * blockDim.x) {
        const int r = e % ldd, cc = e / ldd;
        const int64_t i = k0 + r, c = k0 + cc;
        T v = cx<T>(0, 0);
        if (r < rows && cc < nb && i - c <= kl && c - i <= kv) v = Fb[bidx(kv, ldab, i, c)];
        Db[r + (int64_t)cc * ldd] = v;
    }
}

// Apply the panel's interchanges to the columns right of it (band-limited).
template <typename T>
__global__ void k_gb_swap_right(int64_t n, int64_t kl, int64_t ku, int64_t k0, int nb, T *F,
                                int64_t ldab, int64_t sF, const int *pivl, int ldp)
{
    const int b = blockIdx.y;
    T *Fb = F + (int64_t)b * sF;
    const int *pv = pivl + (int64_t)b * ldp;
    const int64_t kv = kl + ku;
    const int64_t c = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || c >= k0 + nb + kv) return;
    for (int j = 0; j < nb; ++j) {
        const int64_t r = k0 + j, p = k0 + pv[j];
        if (p != r && c - r <= kv) {
            T t = Fb[bidx(kv, ldab, r, c)];
            Fb[bidx(kv, ldab, r, c)] = Fb[bidx(kv, ldab, p, c)];
            Fb[bidx(kv, ldab, p, c)] = t;
        }
    }
}

// U12 = L11^{-1} A12 (L11 unit lower from the factored scratch D); U12 is
// written to the band storage and to a dense scratch (nb x kv, ld GB_NB).
template <typename T>
__global__ void k_gb_u12(int64_t n, int64_t kl, int64_t ku, int64_t k0, int nb, T *F, int64_t ldab,
                         int64_t sF, const T *D, int ldd, int64_t sD, T *U, int64_t sU)
{
    const int b = blockIdx.y;
    T *Fb = F + (int64_t)b * sF;
    const T *Db = D + (int64_t)b * sD;
    T *Ub = U + (int64_t)b * sU;
    __shared__ T L[GB_NB][GB_NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) L[e % nb][e / nb] = Db[(e % nb) + (e / nb) * ldd];
    __syncthreads();
    const int64_t kv = kl + ku;
    const int cc = blockIdx.x * blockDim.x + threadIdx.x;   // 0 .. kv-1
    const int64_t c = k0 + nb + cc;
    if (cc >= kv) return;
    T x[GB_NB];
#pragma unroll
    for (int r = 0; r < GB_NB; ++r) {
        x[r] = cx<T>(0, 0);
        const int64_t i = k0 + r;
        if (r < nb && c < n && c - i <= kv) x[r] = Fb[bidx(kv, ldab, i, c)];
    }
#pragma unroll
    for (int i = 0; i < GB_NB; ++i) {
        if (i >= nb) break;
#pragma unroll
        for (int r = i + 1; r < GB_NB; ++r)
            if (r < nb) cfma(x[r], cneg(L[r][i]), x[i]);
    }
#pragma unroll
    for (int r = 0; r < GB_NB; ++r) {
        Ub[r + (int64_t)cc * GB_NB] = (r < nb && c < n) ? x[r] : cx<T>(0, 0);
        const int64_t i = k0 + r;
        if (r < nb && c < n && c - i <= kv) Fb[bidx(kv, ldab, i, c)] = x[r];
    }
}

// A22 -= L21 U12 on the band: rows k0+nb .. k0+nb+kl-1, columns
// k0+nb .. k0+nb+kv-1, in-band entries only.  L21 = D rows nb.., U12 scratch.
template <typename T>
__global__ void k_gb_update(int64_t n, int64_t kl, int64_t ku, int64_t k0, int nb, int rows, T *F,
                            int64_t ldab, int64_t sF, const T *D, int ldd, int64_t sD, const T *U,
                            int64_t sU)
{
    const int b = blockIdx.z;
    T *Fb = F + (int64_t)b * sF;
    const T *Lb = D + (int64_t)b * sD + nb;      // row nb of D
    const T *Ub = U + (int64_t)b * sU;
    const int64_t kv = kl + ku;
    __shared__ T Ls[GB_NB][32 + 1];
    __shared__ T Us[GB_NB][32 + 1];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8
    const int lrows = rows - nb;                              // rows of L21
    for (int e = threadIdx.x; e < 32 * GB_NB; e += blockDim.x) {
        int r = e % 32, k = e / 32;
        Ls[k][r] = (r0 + r < lrows && k < nb) ? Lb[(r0 + r) + (int64_t)k * ldd] : cx<T>(0, 0);
        int c = e % 32;
        Us[k][c] = (c0 + c < kv && k < nb) ? Ub[k + (int64_t)(c0 + c) * GB_NB] : cx<T>(0, 0);
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
        const int lr = r0 + rr;
        const int64_t i = k0 + nb + lr, c = k0 + nb + c0 + tx;
        if (lr >= lrows || c0 + tx >= kv || c >= n || i >= n) continue;
        if (i - c > kl || c - i > kv) continue;
        T acc = cx<T>(0, 0);
#pragma unroll 8
        for (int k = 0; k < GB_NB; ++k) cfma(acc, Ls[k][rr], Us[k][tx]);
        T &dst = Fb[bidx(kv, ldab, i, c)];
        dst = cadd(dst, cneg(acc));
    }
}

// Write the factored panel back: U part as is, multipliers converted to the
// unblocked convention (undo the later interchanges of the panel), global
// pivots recorded.
template <typename T>
__global__ void k_gb_writeback(int64_t n, int64_t kl, int64_t ku, int64_t k0, int nb, int rows, T *F,
                               int64_t ldab, int64_t sF, const T *D, int ldd, int64_t sD,
                               const int *pivl, int ldp, int *piv)
{
    const int b = blockIdx.x;
    T *Fb = F + (int64_t)b * sF;
    const T *Db = D + (int64_t)b * sD;
    const int *pv = pivl + (int64_t)b * ldp;
    const int64_t kv = kl + ku;
    extern __shared__ unsigned char sm_raw[];
    T *col = reinterpret_cast<T *>(sm_raw);   // rows entries
    for (int j = 0; j < nb; ++j) {
        const int64_t c = k0 + j;
        for (int r = threadIdx.x; r < rows; r += blockDim.x) col[r] = Db[r + (int64_t)j * ldd];
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = nb - 1; t > j; --t) {
                const int p = pv[t];
                if (p != t) { T tmp = col[t]; col[t] = col[p]; col[p] = tmp; }
            }
            piv[(int64_t)b * n + c] = (int)(k0 + pv[j]);
        }
        __syncthreads();
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
            const int64_t i = k0 + r;
            if (i - c <= kl && c - i <= kv) Fb[bidx(kv, ldab, i, c)] = col[r];
        }
        __syncthreads();
    }
}

// Asynchronous global -> shared copies of B bytes (B = 4, 8 or 16); an
// invalid source writes zeros instead (nothing is read).  The staging of
// the next chunk's factor columns runs under the current chunk's solves.
template <int B>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(B), "r"(valid ? B : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Forward pass of the solve (unblocked convention: for j = 0..n-1, swap
// rows j and piv[j], then rows j+1 .. j+kl -= l_j x_j), taken jc steps at a
// time.  Within a chunk the interchanges commute to the front: the chunk is
// x <- L'_{jc-1} .. L'_0 P_{jc-1} .. P_0 x with L'_i's column = the later
// interchanges of the chunk applied to l_i (they touch only rows below
// i).  So a chunk is (1) its interchanges on the right-hand sides, (2) a
// unit lower triangular solve on its jc rows (one warp per right-hand
// side, a lane per row, the solved value passed by shuffles), (3) one
// rank-jc update of the kl rows below it.  CTA = (chunk of cw <= GB_CW
// right-hand sides, node); the right-hand sides live in a circular window
// of WL = kl + 1 + jcm rows in shared memory, the chunk's multipliers
// (jcm + kl rows x jcm columns, column-major) and pivots beside it, in
// nbuf = 2 buffers when they fit (the next chunk's copied in meanwhile).
template <typename T, int CW>
__global__ void __launch_bounds__(GB_ST) k_gb_fwd(int64_t n, int64_t kl, int64_t ku, int64_t nrhs,
                                                  const T *F, int64_t ldab, int64_t sF, const int *piv, T *X,
                                                  int64_t ldx, int64_t sX, int jcm, int nbuf)
{
    constexpr int cw = CW;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int WL = (int)(kl + 1 + jcm), LR = (int)(jcm + kl), kv = (int)(kl + ku);
    T *W = reinterpret_cast<T *>(sm_raw);      // cw columns of WL slots: row r of column cc at W[cc * WL + r % WL]
    T *const Lb0 = W + (size_t)WL * cw;         // LR x jcm: Lb[jj * LR + rho] = L'(j0 + rho, j0 + jj)
    T *const Lb1 = Lb0 + (size_t)(nbuf - 1) * LR * jcm;
    int *const pb0 = reinterpret_cast<int *>(Lb0 + (size_t)nbuf * LR * jcm);   // the chunk's pivots (global rows)
    int *const pb1 = pb0 + (nbuf - 1) * jcm;
    const int b = blockIdx.y;
    const T *Fb = F + (int64_t)b * sF;
    const int *pv = piv + (int64_t)b * n;
    T *Xb = X + (int64_t)b * sX;
    const int64_t c0 = (int64_t)blockIdx.x * cw;
    const int ncol = (int)((nrhs - c0) < cw ? (nrhs - c0) : cw);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto stage = [&](int64_t js, T *Lb, int *ps) {
        const int jcs = (int)((n - js) < jcm ? (n - js) : jcm);
        for (int e = threadIdx.x; e < LR * jcs; e += GB_ST) {
            const int jj = e / LR, rho = e % LR;
            const int64_t r = js + rho, c = js + jj;
            const bool in = rho > jj && rho <= jj + kl && r < n;
            cp_async<sizeof(T)>(Lb + jj * LR + rho, in ? (const void *)(Fb + bidx(kv, ldab, r, c)) : (const void *)Fb,
                                in);
        }
        if (threadIdx.x < jcs) cp_async<4>(ps + threadIdx.x, pv + js + threadIdx.x, true);
    };
    for (int e = threadIdx.x; e < WL * cw; e += GB_ST) {
        const int r = e % WL, cc = e / WL;
        const bool in = r < n && cc < ncol;
        cp_async<sizeof(T)>(W + cc * WL + r, in ? (const void *)(Xb + r + (c0 + cc) * ldx) : (const void *)Xb, in);
    }
    stage(0, Lb0, pb0);
    cp_async_commit();
    int k = 0;
    for (int64_t j0 = 0; j0 < n; j0 += jcm, ++k) {
        const int jc = (int)((n - j0) < jcm ? (n - j0) : jcm);
        const int s0 = (int)(j0 % WL);
        T *Lb = (k & 1) ? Lb1 : Lb0;
        const int *ps = (k & 1) ? pb1 : pb0;
        cp_async_wait_all();
        __syncthreads();
        if (threadIdx.x < cw) {
            // (1) the chunk's interchanges, in order, on this right-hand side
            const int cc = threadIdx.x;
            for (int jj = 0; jj < jc; ++jj) {
                const int p = (int)(ps[jj] - j0);
                if (p != jj) {
                    int sa = s0 + jj, sb = s0 + p;
                    if (sa >= WL) sa -= WL;
                    if (sb >= WL) sb -= WL;
                    const T t = W[cc * WL + sa];
                    W[cc * WL + sa] = W[cc * WL + sb];
                    W[cc * WL + sb] = t;
                }
            }
        } else if (threadIdx.x >= 32 && threadIdx.x < 32 + jc) {
            // L'_jj: the later interchanges of the chunk on column jj
            const int jj = threadIdx.x - 32;
            T *col = Lb + jj * LR;
            for (int jp = jj + 1; jp < jc; ++jp) {
                const int p = (int)(ps[jp] - j0);
                if (p != jp) {
                    const T t = col[jp];
                    col[jp] = col[p];
                    col[p] = t;
                }
            }
        }
        __syncthreads();
        const bool more = j0 + jcm < n;
        if (nbuf == 2 && more) {
            stage(j0 + jcm, (k & 1) ? Lb0 : Lb1, (k & 1) ? pb0 : pb1);
            cp_async_commit();
        }
        // (2) unit lower triangular solve on the chunk's rows
        if (wid < cw) {
            int sl = s0 + lane;
            if (sl >= WL) sl -= WL;
            T x = (lane < jc) ? W[wid * WL + sl] : cx<T>(0, 0);
            for (int jj = 0; jj + 1 < jc; ++jj) {
                const T xj = shfl_cx(x, jj);
                if (lane > jj && lane < jc) cfma(x, cneg(Lb[jj * LR + lane]), xj);
            }
            if (lane < jc) {
                W[wid * WL + sl] = x;
                if (wid < ncol) Xb[j0 + lane + (c0 + wid) * ldx] = x;
            }
        }
        __syncthreads();
        // (3) rows j0 + jc .. j0 + jc + kl - 1 -= L'(those rows, chunk) x(chunk):
        // a thread per row and all cw right-hand sides (one multiplier load
        // per cw products; the x values are broadcast)
        for (int t = threadIdx.x; t < kl; t += GB_ST) {
            const int64_t r = j0 + jc + t;
            if (r >= n) continue;
            int sr = s0 + jc + t;
            while (sr >= WL) sr -= WL;
            T acc[CW];
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) acc[cc] = W[cc * WL + sr];
            int sj = s0;
            for (int jj = 0; jj < jc; ++jj) {
                const T l = cneg(Lb[jj * LR + jc + t]);
#pragma unroll
                for (int cc = 0; cc < CW; ++cc) cfma(acc[cc], l, W[cc * WL + sj]);
                if (++sj == WL) sj = 0;
            }
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) W[cc * WL + sr] = acc[cc];
        }
        __syncthreads();
        // rows j0 .. j0+jc-1 are final; their slots take rows j0+WL ..
        for (int e = threadIdx.x; e < jc * cw; e += GB_ST) {
            const int jj = e / cw, cc = e % cw;
            const int64_t r = j0 + jj + WL;
            int sl = s0 + jj;
            if (sl >= WL) sl -= WL;
            const bool in = r < n && cc < ncol;
            cp_async<sizeof(T)>(W + cc * WL + sl, in ? (const void *)(Xb + r + (c0 + cc) * ldx) : (const void *)Xb,
                                in);
        }
        if (nbuf == 1 && more) stage(j0 + jcm, Lb0, pb0);   // (its buffer is free only now)
        cp_async_commit();
    }
    cp_async_wait_all();
}

// Backward pass: for j = n-1..0: x_j /= U(j,j); rows j-kv .. j-1 -= U(:, j) x_j,
// taken jc columns at a time: an upper triangular solve on the chunk's rows
// (a warp per right-hand side), then one rank-jc update of the kv rows
// above it.  Window of WL = kv + 1 + jcm rows; the chunk's columns of U
// (diagonal included) staged column-major, Us[jj * (kv + 1) + t] =
// U(j - t, j) with j = j1 - jj, in nbuf buffers as in the forward pass.
template <typename T, int CW>
__global__ void __launch_bounds__(GB_ST) k_gb_bwd(int64_t n, int64_t kl, int64_t ku, int64_t nrhs,
                                                  const T *F, int64_t ldab, int64_t sF, T *X,
                                                  int64_t ldx, int64_t sX, int jcm, int nbuf)
{
    constexpr int cw = CW;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int kv = (int)(kl + ku), WL = kv + 1 + jcm, UL = kv + 1;
    T *W = reinterpret_cast<T *>(sm_raw);      // cw columns of WL slots: row r of column cc at W[cc * WL + r % WL]
    T *const Ub0 = W + (size_t)WL * cw;
    T *const Ub1 = Ub0 + (size_t)(nbuf - 1) * jcm * UL;
    const int b = blockIdx.y;
    const T *Fb = F + (int64_t)b * sF;
    T *Xb = X + (int64_t)b * sX;
    const int64_t c0 = (int64_t)blockIdx.x * cw;
    const int ncol = (int)((nrhs - c0) < cw ? (nrhs - c0) : cw);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto stage = [&](int64_t js, T *Us) {
        const int jcs = (int)((js + 1) < jcm ? (js + 1) : jcm);
        for (int e = threadIdx.x; e < jcs * UL; e += GB_ST) {
            const int jj = e / UL, t = e % UL;
            const int64_t c = js - jj, r = c - t;
            const bool in = r >= 0;
            cp_async<sizeof(T)>(Us + jj * UL + t, in ? (const void *)(Fb + bidx(kv, ldab, r, c)) : (const void *)Fb,
                                in);
        }
    };
    for (int e = threadIdx.x; e < WL * cw; e += GB_ST) {
        const int t = e % WL, cc = e / WL;
        const int64_t r = n - 1 - t;
        if (r >= 0) {
            const bool in = cc < ncol;
            cp_async<sizeof(T)>(W + cc * WL + (int)(r % WL), in ? (const void *)(Xb + r + (c0 + cc) * ldx)
                                                                : (const void *)Xb, in);
        }
    }
    stage(n - 1, Ub0);
    cp_async_commit();
    int k = 0;
    for (int64_t j1 = n - 1; j1 >= 0; j1 -= jcm, ++k) {
        const int jc = (int)((j1 + 1) < jcm ? (j1 + 1) : jcm);
        const int s1 = (int)(j1 % WL);        // slot of row j1; row j1 - d at s1 - d (mod WL)
        const T *Us = (k & 1) ? Ub1 : Ub0;
        const bool more = j1 - jcm >= 0;
        cp_async_wait_all();
        __syncthreads();
        if (nbuf == 2 && more) {
            stage(j1 - jcm, (k & 1) ? Ub0 : Ub1);
            cp_async_commit();
        }
        // upper triangular solve on rows j1 - jc + 1 .. j1 (lane d: row j1 - d)
        if (wid < cw) {
            int sl = s1 - lane;
            if (sl < 0) sl += WL;
            T x = (lane < jc) ? W[wid * WL + sl] : cx<T>(0, 0);
            for (int jj = 0; jj < jc; ++jj) {
                if (lane == jj) x = cdiv(x, Us[jj * UL]);
                const T xj = shfl_cx(x, jj);
                const int t = lane - jj;
                if (t > 0 && t <= kv && lane < jc) cfma(x, cneg(Us[jj * UL + t]), xj);
            }
            if (lane < jc) {
                W[wid * WL + sl] = x;
                if (wid < ncol) Xb[j1 - lane + (c0 + wid) * ldx] = x;
            }
        }
        __syncthreads();
        // rows above the chunk: r = j1 - jc - tt, tt = 0 .. kv-1, a thread
        // per row and all cw right-hand sides
        for (int tt = threadIdx.x; tt < kv; tt += GB_ST) {
            const int64_t r = j1 - jc - tt;
            if (r < 0) continue;
            int sr = s1 - jc - tt;
            while (sr < 0) sr += WL;
            T acc[CW];
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) acc[cc] = W[cc * WL + sr];
            int sj = s1;
            for (int jj = 0; jj < jc; ++jj) {
                const int t = jc - jj + tt;       // (j1 - jj) - r
                if (t <= kv) {
                    const T u = cneg(Us[jj * UL + t]);
#pragma unroll
                    for (int cc = 0; cc < CW; ++cc) cfma(acc[cc], u, W[cc * WL + sj]);
                }
                if (--sj < 0) sj = WL - 1;
            }
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) W[cc * WL + sr] = acc[cc];
        }
        __syncthreads();
        // rows j1-jc+1 .. j1 are final; their slots take rows j - WL
        for (int e = threadIdx.x; e < jc * cw; e += GB_ST) {
            const int jj = e / cw, cc = e % cw;
            const int64_t r = j1 - jj - WL;
            int sl = s1 - jj;
            if (sl < 0) sl += WL;
            if (r >= 0) {
                const bool in = cc < ncol;
                cp_async<sizeof(T)>(W + cc * WL + sl, in ? (const void *)(Xb + r + (c0 + cc) * ldx) : (const void *)Xb,
                                    in);
            }
        }
        if (nbuf == 1 && more) stage(j1 - jcm, Ub0);
        cp_async_commit();
    }
    cp_async_wait_all();
}

// Y = op X with op = A (which 0) or z_j B - A style combinations done by the
// caller; plain band product Y[:, c] = M X[:, c], M in compact storage.
__global__ void k_gb_matmul(int64_t n, int64_t kl, int64_t ku, const zd *M, int64_t ldin,
                            int64_t m, const zd *X, int64_t ldx, zd *Y, int64_t ldy)
{
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, c = e / n;
        const int64_t j0 = i - kl > 0 ? i - kl : 0, j1 = i + ku < n - 1 ? i + ku : n - 1;
        zd acc = zmake(0.0, 0.0);
        for (int64_t j = j0; j <= j1; ++j) zfma(acc, M[ku + i - j + j * ldin], X[j + c * ldx]);
        Y[i + c * ldy] = acc;
    }
}

// The whole band LU of one node in one cluster of GL_C CTAs (complex64;
// one launch for all nodes): for each panel of nb columns, every CTA of the
// cluster (1) copies the panel's nb + kl rows into its shared memory and
// (2) factors it there with partial pivoting (pivot: largest |.|^2, the
// first on ties) -- the same arithmetic in the same order in every CTA, so
// their panels agree bit for bit and nothing is exchanged; then each CTA
// takes its own slice of the kv columns right of the panel: (3) the
// panel's interchanges, (4) U12 = L11^{-1} A12 (a warp per column, in
// shared memory), (5) A22 -= L21 U12 on the band (a warp per 32 rows x 4
// columns); (6) CTA 0 writes the panel back with its multipliers in the
// unblocked convention.  A cluster barrier closes each panel.  The same
// factors as the multi-launch form; the clusters (nodes) never wait for
// one another.
constexpr int GL_T = 256;
constexpr int GL_C = 8;          // CTAs per node (a portable cluster)
constexpr int GL_NB = 32;
__device__ __forceinline__ unsigned gl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void gl_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <typename T>
__global__ void __launch_bounds__(GL_T) k_gb_lu_fused(int64_t n, int kl, int ku, T *F, int64_t ldab, int64_t sF,
                                                     int *piv, int nbp, int *info, int *row)
{
    typedef typename CxReal<T>::type R;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int kv = kl + ku, ldd = nbp + kl;
    const int rank = (int)gl_rank(), kvs = (kv + GL_C - 1) / GL_C;
    const int cb = rank * kvs, ce = (cb + kvs < kv) ? cb + kvs : kv;   // this CTA's columns cc in [cb, ce)
    const int nc = ce > cb ? ce - cb : 0, ldu = kvs + 1;
    T *D = reinterpret_cast<T *>(sm_raw);      // ldd x nbp panel, column-major
    T *U = D + (size_t)ldd * nbp;               // nbp x kvs slice of U12, row-major: U[k * ldu + cc - cb]
    int *ps = reinterpret_cast<int *>(U + (size_t)nbp * ldu);  // local pivots of the panel
    __shared__ R s_val[GL_T / 32];
    __shared__ int s_idx[GL_T / 32];
    __shared__ int s_p;
    const int b = blockIdx.x / GL_C;
    T *Fb = F + (int64_t)b * sF;
    int *pvb = piv + (int64_t)b * n;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const T zero = cx<T>(0, 0);
    for (int64_t k0 = 0; k0 < n; k0 += nbp) {
        const int nb = (int)((n - k0) < nbp ? (n - k0) : nbp);
        const int rows = (int)((n - k0) < ldd ? (n - k0) : ldd);
        // (1) gather (asynchronous copies, all in flight at once)
        for (int e = tid; e < ldd * nb; e += GL_T) {
            const int r = e % ldd, cc = e / ldd;
            const int64_t i = k0 + r, c = k0 + cc;
            const bool in = r < rows && i - c <= kl && c - i <= kv;
            cp_async<sizeof(T)>(D + cc * ldd + r, in ? (const void *)(Fb + bidx(kv, ldab, i, c)) : (const void *)Fb, in);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        // every CTA holds the panel before CTA 0 can write it back (step 6)
        gl_cluster_sync();
        // (2) panel LU
        for (int j = 0; j < nb; ++j) {
            const T *dj = D + j * ldd;
            R best = -1;
            int bi = j;
            for (int r = j + tid; r < rows; r += GL_T) {
                const R v = cabs2(dj[r]);
                if (v > best) { best = v; bi = r; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const R ov = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
            __syncthreads();
            // every warp reduces the warp partials itself (a shuffle tree in
            // the same order everywhere)
            R bv = (lane < GL_T / 32) ? s_val[lane] : (R)-1;
            int p = (lane < GL_T / 32) ? s_idx[lane] : j;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const R ov = __shfl_xor_sync(0xffffffffu, bv, off);
                const int oi = __shfl_xor_sync(0xffffffffu, p, off);
                if (ov > bv || (ov == bv && oi < p)) { bv = ov; p = oi; }
            }
            if (tid == 0) {
                ps[j] = p;
                if (bv == 0 && rank == 0 && info && atomicCAS(info, 0, b + 1) == 0 && row) *row = (int)(k0 + j) + 1;
            }
            if (p != j && tid < nb) {
                const T t = D[tid * ldd + j];
                D[tid * ldd + j] = D[tid * ldd + p];
                D[tid * ldd + p] = t;
            }
            __syncthreads();
            const T d = D[j * ldd + j];
            if (!cis_zero(d)) {
                for (int r = j + 1 + tid; r < rows; r += GL_T) D[j * ldd + r] = cdiv(D[j * ldd + r], d);
                __syncthreads();
                // rows j+1 .. rows-1 by lane, columns j+1 .. nb-1 by warp
                for (int r = j + 1 + lane; r < rows; r += 32) {
                    const T l = cneg(D[j * ldd + r]);
                    for (int cc = j + 1 + wid; cc < nb; cc += GL_T / 32) {
                        T v = D[cc * ldd + r];
                        cfma(v, l, D[cc * ldd + j]);
                        D[cc * ldd + r] = v;
                    }
                }
            }
            __syncthreads();
        }
        if (rank == 0 && tid < nb) pvb[k0 + tid] = (int)(k0 + ps[tid]);
        // (3) the interchanges on this CTA's columns right of the panel
        for (int cc = cb + tid; cc < ce; cc += GL_T) {
            const int64_t c = k0 + nb + cc;
            if (c >= n) continue;
            for (int j = 0; j < nb; ++j) {
                const int64_t r = k0 + j, p = k0 + ps[j];
                if (p != r && c - r <= kv) {
                    T &x = Fb[bidx(kv, ldab, r, c)], &y = Fb[bidx(kv, ldab, p, c)];
                    const T t = x;
                    x = y;
                    y = t;
                }
            }
        }
        __syncthreads();
        // (4) U12 = L11^{-1} A12 on this CTA's columns, in shared memory
        // (rows padded to kvs + 1)
        for (int e = tid; e < nbp * nc; e += GL_T) {
            const int r = e % nbp, cl = e / nbp;
            const int64_t c = k0 + nb + cb + cl;
            const bool in = r < nb && c < n && c - (k0 + r) <= kv;
            cp_async<sizeof(T)>(U + r * ldu + cl, in ? (const void *)(Fb + bidx(kv, ldab, k0 + r, c)) : (const void *)Fb,
                                in);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        // a warp per column, a lane per row, the solved value by shuffles
        for (int cl = wid; cl < nc; cl += GL_T / 32) {
            T x = (lane < nb) ? U[lane * ldu + cl] : zero;
            for (int i = 0; i + 1 < nb; ++i) {
                const T xi = shfl_cx(x, i);
                if (lane > i && lane < nb) cfma(x, cneg(D[i * ldd + lane]), xi);
            }
            if (lane < nb) U[lane * ldu + cl] = x;
        }
        __syncthreads();
        for (int e = tid; e < nb * nc; e += GL_T) {
            const int r = e % nb, cl = e / nb;
            const int64_t c = k0 + nb + cb + cl;
            if (c < n && c - (k0 + r) <= kv) Fb[bidx(kv, ldab, k0 + r, c)] = U[r * ldu + cl];
        }
        // (5) A22 -= L21 U12: rows k0+nb+t (t < rows-nb <= kl), this CTA's
        // columns k0+nb+cc -- all inside the band; a warp per 32 rows x 4
        // columns, a lane per row
        {
            const int R2 = rows - nb;
            const int rt = (R2 + 31) / 32, ct = (nc + 3) / 4;
            for (int task = wid; task < rt * ct; task += GL_T / 32) {
                const int t = (task % rt) * 32 + lane, c4 = (task / rt) * 4;
                if (t >= R2) continue;
                const int64_t i = k0 + nb + t;
                // the destinations first: their loads run under the products
                T old[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t c = k0 + nb + cb + c4 + u;
                    old[u] = (c4 + u < nc && c < n) ? Fb[bidx(kv, ldab, i, c)] : zero;
                }
                T acc[4] = {zero, zero, zero, zero};
                for (int k = 0; k < nb; ++k) {
                    const T l = D[k * ldd + nb + t];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (c4 + u < nc) cfma(acc[u], l, U[k * ldu + c4 + u]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t c = k0 + nb + cb + c4 + u;
                    if (c4 + u < nc && c < n) Fb[bidx(kv, ldab, i, c)] = cadd(old[u], cneg(acc[u]));
                }
            }
        }
        __syncthreads();   // (step 5 reads L21 from the panel that step 6 rewrites)
        // (6) the panel back (CTA 0), multipliers in the unblocked convention
        // (the panel's later interchanges undone on each column)
        if (rank == 0) {
            if (tid < nb) {
                T *col = D + tid * ldd;
                for (int t = nb - 1; t > tid; --t) {
                    const int p = ps[t];
                    if (p != t) {
                        const T v = col[t];
                        col[t] = col[p];
                        col[p] = v;
                    }
                }
            }
            __syncthreads();
            for (int e = tid; e < rows * nb; e += GL_T) {
                const int r = e % rows, cc = e / rows;
                const int64_t i = k0 + r, c = k0 + cc;
                if (i - c <= kl && c - i <= kv) Fb[bidx(kv, ldab, i, c)] = D[cc * ldd + r];
            }
        }
        // every CTA's updates (and the panel) are in memory before any
        // CTA gathers the next panel
        gl_cluster_sync();
    }
}

// R_j = RHS - (z_j B - A) X_j for every node (FP64).  B null -> identity.
__global__ void k_gb_residual(int64_t n, int64_t kl, int64_t ku, const zd *A, const zd *B,
                              int64_t ldin, const zd *z, int64_t m, const zd *RHS, const zd *X,
                              zd *R, double *nrm2)
{
    __shared__ double red[32];
    const int jn = blockIdx.y;
    const zd zj = z[jn];
    const zd *Xj = X + (int64_t)jn * n * m;
    zd *Rj = R + (int64_t)jn * n * m;
    const int64_t total = n * m;
    double part = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, c = e / n;
        const int64_t j0 = i - kl > 0 ? i - kl : 0, j1 = i + ku < n - 1 ? i + ku : n - 1;
        zd acc = RHS[i + c * n];
        for (int64_t j = j0; j <= j1; ++j) {
            const int64_t s = ku + i - j + j * ldin;
            zd bij = B ? B[s] : zmake(i == j ? 1.0 : 0.0, 0.0);
            zd mij = zsub(zmul(zj, bij), A[s]);
            zfma(acc, zmake(-mij.x, -mij.y), Xj[j + c * n]);
        }
        Rj[i + c * n] = acc;
        part += zabs2(acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        atomicAdd(nrm2 + jn, s);
    }
}

// ---------------------------------------------- double-single band residual
// Unevaluated float pairs (hi, lo) with error-free products (FMA) and sums;
// the explicit _rn intrinsics keep the compiler from contracting the error
// terms away.  ~48 significant bits.
struct BDS {
    float h, l;
};
__device__ __forceinline__ void bds_mac(BDS &acc, float ah, float al, float xh, float xl)
{
    float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    float s = __fadd_rn(acc.h, p);
    float bb = __fsub_rn(s, acc.h);
    float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    float t = __fadd_rn(acc.l, __fadd_rn(err, e));
    float h = __fadd_rn(s, t);
    acc.l = __fsub_rn(t, __fsub_rn(h, s));
    acc.h = h;
}

// Complex FP64 values as double-single pairs, packed (hi.re, hi.im, lo.re,
// lo.im): the band of A once at set-up, the solutions X_j before each
// residual.
__global__ void k_z2ds(int64_t count, const zd *__restrict__ x, float4 *__restrict__ y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const zd v = x[e];
        const float hr = (float)v.x, hm = (float)v.y;
        y[e] = make_float4(hr, hm, (float)(v.x - (double)hr), (float)(v.y - (double)hm));
    }
}

// R_j = RHS - z_j X_j + A X_j for B = I (M_j = z_j I - A), the band product
// A X_j in double-single arithmetic on the FP32 pipe (the FP64 pipe is 64x
// slower); nrm2[j] += ||R_j||_F^2.  Thread per (row, column) of one node:
// a warp's A loads are one column of the band (coalesced), its X loads one
// broadcast element.
__global__ void k_gb_residual_ds(int64_t n, int64_t kl, int64_t ku, const float4 *__restrict__ Ads, int64_t ldin,
                                 const zd *__restrict__ z, int64_t m, const zd *__restrict__ RHS,
                                 const zd *__restrict__ X, const float4 *__restrict__ Xds, zd *__restrict__ R,
                                 double *__restrict__ nrm2)
{
    __shared__ double red[32];
    const int jn = blockIdx.y;
    const zd zj = z[jn];
    const zd *Xj = X + (int64_t)jn * n * m;
    const float4 *Dj = Xds + (int64_t)jn * n * m;
    zd *Rj = R + (int64_t)jn * n * m;
    const int64_t total = n * m;
    double part = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, c = e / n;
        const int64_t j0 = i - kl > 0 ? i - kl : 0, j1 = i + ku < n - 1 ? i + ku : n - 1;
        BDS re{0.f, 0.f}, im{0.f, 0.f};
        const float4 *xc = Dj + c * n;
        for (int64_t j = j0; j <= j1; ++j) {
            const float4 a = Ads[ku + i - j + j * ldin];
            const float4 x = xc[j];
            // (a.re + i a.im)(x.re + i x.im), each part hi + lo
            bds_mac(re, a.x, a.z, x.x, x.z);
            bds_mac(re, -a.y, -a.w, x.y, x.w);
            bds_mac(im, a.x, a.z, x.y, x.w);
            bds_mac(im, a.y, a.w, x.x, x.z);
        }
        const zd x = Xj[i + c * n];
        const zd rhs = RHS[i + c * n];
        const zd zx = zmul(zj, x);
        const zd acc = zmake(rhs.x - zx.x + ((double)re.h + (double)re.l),
                             rhs.y - zx.y + ((double)im.h + (double)im.l));
        Rj[i + c * n] = acc;
        part += zabs2(acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
        atomicAdd(nrm2 + jn, s);
    }
}
}  // namespace

size_t gb_scratch_elems(int64_t kl, int64_t ku, int q)
{
    // dense panel (NB + kl) x NB and U12 NB x kv per node
    return (size_t)q * ((size_t)(GB_NB + kl) * GB_NB + (size_t)GB_NB * (kl + ku));
}
size_t gb_piv_scratch(int64_t kl, int q) { return (size_t)q * (GB_NB + kl); }

template <typename T>
int gb_form(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const zd *A, const zd *B,
            int64_t ldin, int q, const zd *z, T *F)
{
    const int64_t ldab = 2 * kl + ku + 1;
    unsigned gx = cdiv(ldab * n, 256);
    if (gx > 2048) gx = 2048;
    k_gb_form<T><<<dim3(gx, q), 256, 0, s>>>(n, kl, ku, A, B, ldin, z, F, ldab, ldab * n);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

// Shared memory of the one-launch band LU (per CTA) for a panel width nbp.
static size_t gb_lu_fused_smem(int64_t kl, int64_t ku, int nbp, size_t es)
{
    const int64_t kvs = (kl + ku + GL_C - 1) / GL_C;
    return ((size_t)(nbp + kl) * nbp + (size_t)nbp * (kvs + 1)) * es + (size_t)nbp * sizeof(int);
}

template <typename T>
int gb_getrf(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, int q, T *F, int *piv, void *scratch,
             int *pivl, int *info, int *row)
{
    const int64_t ldab = 2 * kl + ku + 1, kv = kl + ku, sF = ldab * n;
    if constexpr (sizeof(T) == sizeof(cf)) {
        // complex64: the whole LU of each node in one cluster when its
        // panel and its slice of U12 fit shared memory (the widest panel
        // that does) and the band is narrow enough that the cluster's
        // share of the trailing updates (kl x kv x nb per panel) stays
        // near the panel's own latency; wider bands spread their updates
        // over the whole GPU below
        for (int nbp = GL_NB; nbp >= 8 && kv <= 512; nbp /= 2) {
            const size_t sm = gb_lu_fused_smem(kl, ku, nbp, sizeof(T));
            if (sm + 1024 > kSmemOptinMax) continue;
            FEAST_CUDA_TRY(ensure_dyn_smem(k_gb_lu_fused<T>, sm));
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = GL_C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3((unsigned)(q * GL_C));
            cfg.blockDim = dim3(GL_T);
            cfg.dynamicSmemBytes = sm;
            cfg.stream = s;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            FEAST_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gb_lu_fused<T>, n, (int)kl, (int)ku, F, ldab, sF, piv, nbp,
                                              info, row));
            FEAST_LAUNCH_CHECK();
            return FEAST_OK;
        }
    }
    const int ldd = (int)(GB_NB + kl);
    T *D = (T *)scratch;
    const int64_t sD = (int64_t)ldd * GB_NB;
    T *U = D + (size_t)q * sD;
    const int64_t sU = (int64_t)GB_NB * kv;
    for (int64_t k0 = 0; k0 < n; k0 += GB_NB) {
        const int nb = (int)((n - k0) < GB_NB ? (n - k0) : GB_NB);
        const int rows = (int)((n - k0) < ldd ? (n - k0) : ldd);
        k_gb_gather<T><<<dim3(cdiv((size_t)ldd * GB_NB, 256), q), 256, 0, s>>>(n, kl, ku, k0, rows, nb, F, ldab, sF,
                                                                             D, ldd, sD);
        FEAST_LAUNCH_CHECK();
        // dense panel factorization of the scratch (rows x nb, pivots local)
        int e = getrf_panel<T>(s, rows, nb, q, D, ldd, sD, pivl, ldd, info, row);
        if (e) return e;
        if (kv > 0) {
            k_gb_swap_right<T><<<dim3(cdiv(kv, 128), q), 128, 0, s>>>(n, kl, ku, k0, nb, F, ldab, sF, pivl, ldd);
            FEAST_LAUNCH_CHECK();
            k_gb_u12<T><<<dim3(cdiv(kv, 64), q), 64, 0, s>>>(n, kl, ku, k0, nb, F, ldab, sF, D, ldd, sD, U, sU);
            FEAST_LAUNCH_CHECK();
            if (rows > nb) {
                dim3 g(cdiv(rows - nb, 32), cdiv(kv, 32), q);
                k_gb_update<T><<<g, 256, 0, s>>>(n, kl, ku, k0, nb, rows, F, ldab, sF, D, ldd, sD, U, sU);
                FEAST_LAUNCH_CHECK();
            }
        }
        FEAST_CUDA_TRY(ensure_dyn_smem(k_gb_writeback<T>, (size_t)rows * sizeof(T)));
        k_gb_writeback<T><<<q, 256, (size_t)rows * sizeof(T), s>>>(n, kl, ku, k0, nb, rows, F, ldab, sF, D,
                                                                  ldd, sD, pivl, ldd, piv);
        FEAST_LAUNCH_CHECK();
    }
    return FEAST_OK;
}

// Dynamic shared memory of the band solves (forward, backward) for elements
// of es bytes: the staged factor columns and right-hand-side chunks.
static size_t gb_fwd_smem(int64_t kl, size_t es, int cw, int jcm, int nbuf)
{
    return ((size_t)(kl + 1 + jcm) * cw + (size_t)nbuf * jcm * (jcm + kl)) * es + (size_t)nbuf * jcm * sizeof(int) + 16;
}
static size_t gb_bwd_smem(int64_t kl, int64_t ku, size_t es, int cw, int jcm, int nbuf)
{
    const int64_t kv = kl + ku;
    return ((size_t)(kv + 1 + jcm) * cw + (size_t)nbuf * jcm * (kv + 1)) * es;
}

// Staging of the band solves: the most right-hand sides per CTA (cw), then
// the deepest factor staging (jcm) whose shared memory fits, with the next
// chunk's factor columns double-buffered (nbuf = 2) while a chunk of at
// least 8 steps fits that way.  Wide bands trade all three for the band
// itself: cw = jcm = nbuf = 1 holds a window of kv + 2 rows and one factor
// column.
struct GbPlan {
    int cw, jcm, nbuf;
    size_t smf, smb;
};
static GbPlan gb_plan(int64_t kl, int64_t ku, size_t es)
{
    const size_t lim = kSmemOptinMax - 1024;
    for (int nbuf = 2; nbuf >= 1; --nbuf)
        for (int cw = GB_CW; cw >= 1; cw /= 2)
            for (int jcm = GB_JC; jcm >= (nbuf == 2 ? 8 : 1); jcm /= 2) {
                const size_t f = gb_fwd_smem(kl, es, cw, jcm, nbuf), b = gb_bwd_smem(kl, ku, es, cw, jcm, nbuf);
                if (f <= lim && b <= lim) return GbPlan{cw, jcm, nbuf, f, b};
            }
    // (does not fit: the caller refuses the band)
    return GbPlan{1, 1, 1, gb_fwd_smem(kl, es, 1, 1, 1), gb_bwd_smem(kl, ku, es, 1, 1, 1)};
}

size_t gb_solve_smem_bytes(int64_t kl, int64_t ku, size_t es)
{
    const GbPlan p = gb_plan(kl, ku, es);
    return p.smf > p.smb ? p.smf : p.smb;
}

template <typename T, int CW>
static int gb_solve_cw(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, int q, const T *F, const int *piv,
                       int64_t nrhs, T *X, int64_t ldx, int64_t sX, const GbPlan &pl)
{
    const int64_t ldab = 2 * kl + ku + 1, sF = ldab * n;
    dim3 g(cdiv(nrhs, CW), q);
    FEAST_CUDA_TRY(ensure_dyn_smem(k_gb_fwd<T, CW>, pl.smf));
    FEAST_CUDA_TRY(ensure_dyn_smem(k_gb_bwd<T, CW>, pl.smb));
    k_gb_fwd<T, CW><<<g, GB_ST, pl.smf, s>>>(n, kl, ku, nrhs, F, ldab, sF, piv, X, ldx, sX, pl.jcm, pl.nbuf);
    FEAST_LAUNCH_CHECK();
    k_gb_bwd<T, CW><<<g, GB_ST, pl.smb, s>>>(n, kl, ku, nrhs, F, ldab, sF, X, ldx, sX, pl.jcm, pl.nbuf);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

template <typename T>
int gb_solve(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, int q, const T *F, const int *piv,
             int64_t nrhs, T *X, int64_t ldx, int64_t sX)
{
    const GbPlan pl = gb_plan(kl, ku, sizeof(T));
    if (pl.smf > kSmemOptinMax - 1024 || pl.smb > kSmemOptinMax - 1024) return FEAST_EINVAL;
    switch (pl.cw) {
    case 8: return gb_solve_cw<T, 8>(s, n, kl, ku, q, F, piv, nrhs, X, ldx, sX, pl);
    case 4: return gb_solve_cw<T, 4>(s, n, kl, ku, q, F, piv, nrhs, X, ldx, sX, pl);
    case 2: return gb_solve_cw<T, 2>(s, n, kl, ku, q, F, piv, nrhs, X, ldx, sX, pl);
    default: return gb_solve_cw<T, 1>(s, n, kl, ku, q, F, piv, nrhs, X, ldx, sX, pl);
    }
}

int gb_matmul(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const zd *M, int64_t ldin, int64_t m,
              const zd *X, zd *Y)
{
    unsigned gx = cdiv(n * m, 256);
    if (gx > 4096) gx = 4096;
    k_gb_matmul<<<gx, 256, 0, s>>>(n, kl, ku, M, ldin, m, X, n, Y, n);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int gb_residual(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const zd *A, const zd *B,
                int64_t ldin, int q, const zd *z, int64_t m, const zd *RHS, const zd *X, zd *R,
                double *nrm2)
{
    FEAST_CUDA_TRY(cudaMemsetAsync(nrm2, 0, sizeof(double) * q, s));
    unsigned gx = cdiv(n * m, 256);
    if (gx > 1024) gx = 1024;
    k_gb_residual<<<dim3(gx, q), 256, 0, s>>>(n, kl, ku, A, B, ldin, z, m, RHS, X, R, nrm2);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

template int gb_form<double2>(cudaStream_t, int64_t, int64_t, int64_t, const zd *, const zd *, int64_t, int,
                              const zd *, double2 *);
template int gb_form<float2>(cudaStream_t, int64_t, int64_t, int64_t, const zd *, const zd *, int64_t, int,
                             const zd *, float2 *);
template int gb_getrf<double2>(cudaStream_t, int64_t, int64_t, int64_t, int, double2 *, int *, void *, int *,
                               int *, int *);
template int gb_getrf<float2>(cudaStream_t, int64_t, int64_t, int64_t, int, float2 *, int *, void *, int *,
                              int *, int *);
template int gb_solve<double2>(cudaStream_t, int64_t, int64_t, int64_t, int, const double2 *, const int *,
                               int64_t, double2 *, int64_t, int64_t);
template int gb_solve<float2>(cudaStream_t, int64_t, int64_t, int64_t, int, const float2 *, const int *,
                              int64_t, float2 *, int64_t, int64_t);

int z2ds(cudaStream_t s, int64_t count, const zd *x, float4 *y)
{
    unsigned g = cdiv(count, 256);
    if (g > 4096) g = 4096;
    k_z2ds<<<g, 256, 0, s>>>(count, x, y);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

int gb_residual_ds(cudaStream_t s, int64_t n, int64_t kl, int64_t ku, const float4 *Ads, int64_t ldin, int q,
                   const zd *z, int64_t m, const zd *RHS, const zd *X, float4 *Xds, zd *R, double *nrm2)
{
    int e;
    if ((e = z2ds(s, (int64_t)q * n * m, X, Xds))) return e;
    FEAST_CUDA_TRY(cudaMemsetAsync(nrm2, 0, sizeof(double) * q, s));
    unsigned gx = cdiv(n * m, 256);
    if (gx > 1024) gx = 1024;
    k_gb_residual_ds<<<dim3(gx, q), 256, 0, s>>>(n, kl, ku, Ads, ldin, z, m, RHS, X, Xds, R, nrm2);
    FEAST_LAUNCH_CHECK();
    return FEAST_OK;
}

}  // namespace feast
