// feast_zqz_batched_noalloc: the batched projected-pencil eigensolve of
// feast_zqz_batched for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or unsafe --
// inside a CUDA graph that is being captured (allocation calls are not
// capturable), inside another library's callback that must not block on the
// allocator, or in a process whose device memory is fully reserved by a
// pool it does not own.  Such a caller can pass only its inputs and
// outputs.  This entry point therefore takes its scratch space (the
// back-substitution workspace of the QZ kernel, one m x m complex block per
// pencil) from a fixed array compiled into this library, not from the
// caller.
//
// Limits and sharing rules:
//   * the array holds NOALLOC_ELEMS complex128 values (4 MiB); a call needs
//     batch * m * m of them and m <= 64 -- anything larger is rejected with
//     FEAST_EINVAL before any work is queued;
//   * every GPU that loads the library carries the array until the process
//     exits;
//   * all calls on a device share the one array and it keeps whatever the
//     last call left in it.  The kernel writes every scratch element it
//     reads, so nothing has to be cleared between calls, but two calls
//     whose work overlaps on the GPU (different streams, or different host
//     threads) would overwrite each other's scratch: serialise them;
//   * the first call in a CUDA context looks up the array's device address
//     (with that context current) and remembers it together with the
//     context's unique ID; make that first call outside any stream capture.
//     A later call in another context (a new primary context after
//     cudaDeviceReset, or a context the caller created) sees a different ID
//     and looks the address up again, so no call ever hands a kernel an
//     address from a context that is gone.
#include <cuda.h>
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t NOALLOC_ELEMS = 64 * 64 * 64;   // 64 pencils of 64 x 64
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_ELEMS];

std::mutex g_noalloc_mutex;

// The driver's context queries, reached through the runtime (the library
// links the CUDA runtime only).
typedef CUresult (*ctx_get_current_fn)(CUcontext *);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long *);
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;

struct ScratchAddr {
    unsigned long long ctx_id;  // 0: none cached
    void *ptr;
};
ScratchAddr g_noalloc_addr[MAX_DEVICES] = {};

// ID of the context current on this thread (unique for the process's
// lifetime, unlike the CUcontext handle, which may be reused), or 0.
unsigned long long current_ctx_id()
{
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current context (host code may
// not use the symbol itself as a device pointer).
int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FEAST_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return FEAST_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_ctx_get_current) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !f1 ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f2)
            return FEAST_ECUDA;
        g_ctx_get_id = (ctx_get_id_fn)f2;
        g_ctx_get_current = (ctx_get_current_fn)f1;
    }
    unsigned long long id = current_ctx_id();
    if (id != 0 && g_noalloc_addr[dev].ctx_id == id && g_noalloc_addr[dev].ptr) {
        *out = g_noalloc_addr[dev].ptr;
        return FEAST_OK;
    }
    // first call in this context: the lookup also makes the runtime's
    // context current when none was yet
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FEAST_ECUDA;
    id = current_ctx_id();
    if (id == 0) return FEAST_ECUDA;
    g_noalloc_addr[dev] = ScratchAddr{id, p};
    *out = p;
    return FEAST_OK;
}

}  // namespace

extern "C" {

int feast_zqz_batched_noalloc(int m, int batch, void *A, void *B, void *alpha, void *beta,
                              void *V, int *status, void *stream)
{
    if (m < 0 || batch < 0 || !A || !B || !alpha || !beta || !V || !status) return FEAST_EINVAL;
    if (m > 64) return FEAST_EINVAL;
    if ((size_t)batch * (size_t)m * (size_t)m > NOALLOC_ELEMS) return FEAST_EINVAL;
    void *scratch = nullptr;
    int e = noalloc_scratch(&scratch);
    if (e) return e;
    cudaStream_t s = (cudaStream_t)stream;
    FEAST_CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(int), s));
    return feast::zqz_batched(s, m, batch, (feast::zd *)A, m, (int64_t)m * m, (feast::zd *)B, m,
                              (int64_t)m * m, (feast::zd *)alpha, (feast::zd *)beta,
                              (feast::zd *)V, m, (int64_t)m * m, scratch, status, status + 1);
}

}  // extern "C"
