// Sparse pencils onto the banded path: a bandwidth-reducing ordering of the
// pencil's joint pattern (reverse Cuthill-McKee: Cuthill & McKee 1969, the
// reversal of George 1971, pseudo-peripheral start nodes of Gibbs, Poole &
// Stockmeyer 1976), then a scatter of each CSR matrix into the compact band
// storage of the permuted matrix.  A symmetric permutation P A P^T,
// P B P^T keeps the eigenvalues of the pencil and permutes its eigenvectors,
// so the whole GFEAST path then runs on the band LU (k_band.cu).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace feast {
namespace {

// Breadth-first level structure from root over the unvisited part of the
// graph (stamp[v] = s marks v as reached by this search).  Returns the
// number of levels; `last` receives the nodes of the last level and `all`
// (if given) every node reached.
int bfs_levels(int64_t root, const std::vector<int64_t> &xadj, const std::vector<int64_t> &adj,
               const std::vector<char> &done, std::vector<int64_t> &stamp, int64_t s, std::vector<int64_t> &last,
               std::vector<int64_t> *all = nullptr)
{
    std::vector<int64_t> cur{root}, next;
    stamp[root] = s;
    if (all) all->assign(1, root);
    int levels = 0;
    while (!cur.empty()) {
        ++levels;
        last = cur;
        next.clear();
        for (int64_t v : cur)
            for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p) {
                const int64_t w = adj[p];
                if (!done[w] && stamp[w] != s) {
                    stamp[w] = s;
                    next.push_back(w);
                    if (all) all->push_back(w);
                }
            }
        cur.swap(next);
    }
    return levels;
}

__global__ void k_csr_to_band(int64_t n, const int64_t *__restrict__ rowptr, const int64_t *__restrict__ col,
                              const zd *__restrict__ val, const int64_t *__restrict__ iperm, int64_t kl, int64_t ku,
                              zd *__restrict__ band, int *__restrict__ outside)
{
    const int64_t ldab = kl + ku + 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ip = iperm[i];
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const int64_t j = col[p];
            if (j < 0 || j >= n) { atomicAdd(outside, 1); continue; }
            const int64_t jp = iperm[j], d = ip - jp;
            if (d > kl || -d > ku) { atomicAdd(outside, 1); continue; }
            zd &b = band[(ku + d) + jp * ldab];   // one thread per row: duplicates add in order
            b = zmake(b.x + val[p].x, b.y + val[p].y);
        }
    }
}

}  // namespace
}  // namespace feast

using namespace feast;

extern "C" {

static int csr_rcm(int64_t n, const int64_t *a_rowptr, const int64_t *a_col, const int64_t *b_rowptr,
                   const int64_t *b_col, int64_t *perm, int64_t *kl_out, int64_t *ku_out);

int feast_csr_rcm(int64_t n, const int64_t *a_rowptr, const int64_t *a_col, const int64_t *b_rowptr,
                  const int64_t *b_col, int64_t *perm, int64_t *kl_out, int64_t *ku_out)
{
    try {   // no C++ exception may cross the C boundary
        return csr_rcm(n, a_rowptr, a_col, b_rowptr, b_col, perm, kl_out, ku_out);
    } catch (...) {
        return FEAST_ENOMEM;
    }
}

static int csr_rcm(int64_t n, const int64_t *a_rowptr, const int64_t *a_col, const int64_t *b_rowptr,
                   const int64_t *b_col, int64_t *perm, int64_t *kl_out, int64_t *ku_out)
{
    if (n < 1 || !a_rowptr || !a_col || !perm || !kl_out || !ku_out || (!b_rowptr) != (!b_col)) return FEAST_EINVAL;
    const int64_t *rp[2] = {a_rowptr, b_rowptr};
    const int64_t *ci[2] = {a_col, b_col};
    // symmetrised joint pattern, self loops dropped
    std::vector<std::vector<int64_t>> nb((size_t)n);
    for (int t = 0; t < 2; ++t) {
        if (!rp[t]) continue;
        if (rp[t][0] != 0) return FEAST_EINVAL;
        for (int64_t i = 0; i < n; ++i) {
            if (rp[t][i + 1] < rp[t][i]) return FEAST_EINVAL;
            for (int64_t p = rp[t][i]; p < rp[t][i + 1]; ++p) {
                const int64_t j = ci[t][p];
                if (j < 0 || j >= n) return FEAST_EINVAL;
                if (j == i) continue;
                nb[i].push_back(j);
                nb[j].push_back(i);
            }
        }
    }
    std::vector<int64_t> xadj((size_t)n + 1, 0), adj;
    for (int64_t i = 0; i < n; ++i) {
        std::sort(nb[i].begin(), nb[i].end());
        nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
        xadj[i + 1] = xadj[i] + (int64_t)nb[i].size();
    }
    adj.reserve((size_t)xadj[n]);
    for (int64_t i = 0; i < n; ++i) adj.insert(adj.end(), nb[i].begin(), nb[i].end());
    nb.clear();
    auto deg = [&](int64_t v) { return xadj[v + 1] - xadj[v]; };
    std::vector<char> done((size_t)n, 0);
    std::vector<int64_t> stamp((size_t)n, -1), order, last;
    order.reserve((size_t)n);
    int64_t s = 0;
    for (int64_t seed = 0; seed < n; ++seed) {
        if (done[seed]) continue;
        // the component's node of least degree, then a pseudo-peripheral
        // node: move to a least-degree node of the last level while the
        // eccentricity grows
        int64_t r = seed;
        {
            std::vector<int64_t> lev, comp;
            bfs_levels(seed, xadj, adj, done, stamp, s++, lev, &comp);
            for (int64_t v : comp)
                if (deg(v) < deg(r) || (deg(v) == deg(r) && v < r)) r = v;
        }
        int ecc = bfs_levels(r, xadj, adj, done, stamp, s++, last);
        for (int it = 0; it < 32; ++it) {
            int64_t x = last[0];
            for (int64_t v : last)
                if (deg(v) < deg(x) || (deg(v) == deg(x) && v < x)) x = v;
            std::vector<int64_t> lx;
            const int e = bfs_levels(x, xadj, adj, done, stamp, s++, lx);
            if (e <= ecc) break;
            r = x;
            ecc = e;
            last.swap(lx);
        }
        // Cuthill-McKee from r: neighbours in increasing degree (then index)
        size_t head = order.size();
        order.push_back(r);
        done[r] = 1;
        std::vector<int64_t> cand;
        while (head < order.size()) {
            const int64_t v = order[head++];
            cand.clear();
            for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p)
                if (!done[adj[p]]) cand.push_back(adj[p]);
            std::sort(cand.begin(), cand.end(), [&](int64_t a, int64_t b) {
                return deg(a) < deg(b) || (deg(a) == deg(b) && a < b);
            });
            for (int64_t w : cand) {
                done[w] = 1;
                order.push_back(w);
            }
        }
    }
    // reverse: perm[new] = old
    for (int64_t k = 0; k < n; ++k) perm[k] = order[(size_t)(n - 1 - k)];
    std::vector<int64_t> iperm((size_t)n);
    for (int64_t k = 0; k < n; ++k) iperm[perm[k]] = k;
    int64_t kl = 0, ku = 0;
    for (int t = 0; t < 2; ++t) {
        if (!rp[t]) continue;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t p = rp[t][i]; p < rp[t][i + 1]; ++p) {
                const int64_t d = iperm[i] - iperm[ci[t][p]];
                kl = std::max(kl, d);
                ku = std::max(ku, -d);
            }
    }
    *kl_out = kl;
    *ku_out = ku;
    return FEAST_OK;
}

int feast_csr_to_band(int64_t n, const int64_t *rowptr, const int64_t *col, const void *val, const int64_t *iperm,
                      int64_t kl, int64_t ku, void *band, int *status, void *stream)
{
    if (n < 1 || !rowptr || !col || !val || !iperm || !band || !status || kl < 0 || ku < 0) return FEAST_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    FEAST_CUDA_TRY(cudaMemsetAsync(band, 0, sizeof(zd) * (size_t)(kl + ku + 1) * (size_t)n, s));
    FEAST_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    unsigned g = cdiv((size_t)n, 256);
    if (g > 152 * 16) g = 152 * 16;
    k_csr_to_band<<<g, 256, 0, s>>>(n, rowptr, col, (const zd *)val, iperm, kl, ku, (zd *)band, status);
    FEAST_LAUNCH_CHECK();
    int h = 0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    return h ? FEAST_EINVAL : FEAST_OK;
}

}  // extern "C"
