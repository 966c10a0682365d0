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
//   * the first call on a device looks up the array's device address (with
//     that device current) and remembers it; make that first call outside
//     any stream capture.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t NOALLOC_ELEMS = 64 * 64 * 64;   // 64 pencils of 64 x 64
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_ELEMS];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (host code may
// not use the symbol itself as a device pointer).
int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FEAST_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return FEAST_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FEAST_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
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
