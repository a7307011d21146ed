// moa_inner_bf16x3_noalloc: the split-BF16x3 (add, mul) inner product for
// callers that may not allocate device memory — for example code being
// captured into a CUDA graph, a serving loop with a fixed memory budget
// that must not stall on the allocator, or a callback that may not re-enter
// an allocator.  The scratch it needs (the bf16 hi/mid/lo planes of both
// operands) lives in one fixed file-scope device array instead of the
// library's stream-ordered workspace.
//
// The array belongs to this file's module: every GPU that loads the library
// holds MOA_NOALLOC_SCRATCH_BYTES for it until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a
// shadow variable), so the first call on each device looks the address up
// with cudaGetSymbolAddress while that device is current and caches it.
// That first call should happen before any stream capture begins.
//
// All calls share the one array and a call leaves its planes behind; nothing
// needs clearing because every plane element a call reads (padding included)
// is written earlier in the same call.  Calls that may overlap on the GPU
// race on the array and must be serialised by the caller.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tc.h"

namespace moa {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MOA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
moa_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MOA_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return MOA_ERR_INTERNAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MOA_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MOA_OK;
}

moa_status extents(int rank, const int64_t *shape, int64_t *n) {
    int64_t c = 1;
    for (int k = 0; k < rank; ++k) {
        if (shape[k] < 0) return MOA_ERR_OVERFLOW;
        if (shape[k] != 0 && c > INT64_MAX / shape[k]) return MOA_ERR_OVERFLOW;
        c *= shape[k];
    }
    *n = c;
    return MOA_OK;
}

}  // namespace
}  // namespace moa

using namespace moa;

extern "C" moa_status moa_inner_bf16x3_noalloc(int rankA, const int64_t *shapeA, const float *A, int rankB,
                                               const int64_t *shapeB, const float *B, float *out, moa_stream stream) {
    // same validation as moa_inner for (add, mul), FP32 -> FP32, MOA_FORM_BF16X3
    if (rankA < 1 || rankB < 1 || rankA > 8 || rankB > 8) return MOA_ERR_RANK;
    if (!shapeA || !shapeB) return MOA_ERR_NULL;
    int64_t nA, nB, M, N;
    moa_status st;
    if ((st = extents(rankA, shapeA, &nA)) != MOA_OK) return st;
    if ((st = extents(rankB, shapeB, &nB)) != MOA_OK) return st;
    if (shapeA[rankA - 1] != shapeB[0]) return MOA_ERR_SHAPE_MISMATCH;
    if ((st = extents(rankA - 1, shapeA, &M)) != MOA_OK) return st;
    if ((st = extents(rankB - 1, shapeB + 1, &N)) != MOA_OK) return st;
    const int64_t K = shapeA[rankA - 1];
    if (M != 0 && N > INT64_MAX / M) return MOA_ERR_OVERFLOW;
    if (M == 0 || N == 0) return MOA_OK;
    if (!out || (K > 0 && (!A || !B))) return MOA_ERR_NULL;
    if ((uintptr_t)A % 4 || (uintptr_t)B % 4 || (uintptr_t)out % 4) return MOA_ERR_ALIGNMENT;
    cudaStream_t s = (cudaStream_t)stream;
    // scratch needed: three bf16 planes of A (M x Kp) and of B (K x Np)
    const int64_t lim = (int64_t)MOA_NOALLOC_SCRATCH_BYTES / 6;
    const int64_t Kp = (K + 7) / 8 * 8, Np = (N + 7) / 8 * 8;
    if (K > 0 && (M > lim / Kp || K > lim / Np || M * Kp + K * Np > lim)) return MOA_ERR_SCRATCH_LIMIT;
    const void *used[3] = {K > 0 ? A : nullptr, K > 0 ? B : nullptr, out};
    if ((st = check_device_ptrs(used, 3)) != MOA_OK) return st;
    if (K == 0) return launch_fill32((uint32_t *)out, 0u, M * N, s) == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
    void *scratch = nullptr;
    if ((st = scratch_address(&scratch)) != MOA_OK) return st;
    return tc_inner_bf16x3_scratch(A, B, out, M, N, K, scratch, s);
}
