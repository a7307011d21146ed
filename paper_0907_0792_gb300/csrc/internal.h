// Host-side interface between the C ABI (api.cu) and the kernel files.
// Every launcher takes the psi-flattened problem (Fig. 1: M result rows of N
// elements, contraction length K) and device pointers, enqueues on `stream`
// and returns a cudaError_t (cudaSuccess when the launch was accepted).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "moa.h"

namespace moa {

// Workspace: scratch device memory owned by the library, one buffer per
// (device, stream, slot), grown with stream-ordered allocation (api.cu).
// Slot 0 serves the inner and outer products, slot 1 the transposed operands
// of moa_inner_axes, slot 2 the device copies of moa_inner_host's operands,
// slot 3 the digit planes of B that moa_inner_host's Ozaki row blocks share.
void *workspace_get(cudaStream_t stream, size_t bytes, moa_status *st, int slot = 0);

// MOA_OK when every non-null pointer of ptrs[0..n) lies in device (or
// managed) memory of the current device; MOA_ERR_NOT_DEVICE otherwise (host
// memory, another GPU's memory, or an address the CUDA runtime does not
// know).  The tensor maps and kernels of the library address A, B and out as
// memory of the device they run on.
moa_status check_device_ptrs(const void *const *ptrs, int n);

// timing.cu — while moa_kernel_timing is on, a GemmTimer around a GEMM
// launch records a CUDA event pair on the launch stream (nothing otherwise).
class GemmTimer {
  public:
    explicit GemmTimer(cudaStream_t s);
    void done();  // call right after the launch
    ~GemmTimer();

  private:
    cudaStream_t stream_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// outer.cu — Eq. (1) over the flattened operands (C is M x N, M = |A|, N = |B|).
cudaError_t launch_outer(int op, moa_dtype dtype, moa_dtype out_dtype, const void *A, const void *B, void *C,
                         int64_t M, int64_t N, cudaStream_t stream);

// fill.cu helpers: fill `count` elements of `elem_bytes` bytes with a pattern.
cudaError_t launch_fill32(uint32_t *p, uint32_t value, int64_t count, cudaStream_t stream);
cudaError_t launch_fill64(uint64_t *p, uint64_t value, int64_t count, cudaStream_t stream);

// semiring.cu — CUDA-core tiled inner product, Eq. (2), D = A (M x K) . B (K x N).
// kind selects the element type / operator pair.
enum SemiringKind {
    SR_F64_PLUS_TIMES = 0,
    SR_F32_PLUS_TIMES = 1,
    SR_F32_MIN_PLUS = 2,
    SR_F32_MAX_PLUS = 3,
    SR_F32_MIN_TIMES = 4,
    SR_F32_MAX_TIMES = 5,
    SR_I32_PLUS_TIMES = 6,
    SR_F32_MIN_MINUS = 7,
    SR_F32_MAX_MINUS = 8,
    SR_F32_MAX_MIN = 9,   // widest (bottleneck) paths
    SR_F32_MIN_MAX = 10,  // minimax paths
    SR_F32_MIN_MIN = 11,
    SR_F32_MAX_MAX = 12,
};
// With `run_if`, every CTA returns at once unless *run_if is non-zero (a
// flag an earlier kernel on the stream sets).
cudaError_t launch_semiring(SemiringKind kind, const void *A, const void *B, void *D, int64_t M, int64_t N, int64_t K,
                            cudaStream_t stream, const uint32_t *run_if = nullptr);

// transpose.cu — out (rank axes, output axis k = input axis perm[k]) from
// in (row-major, extents `shape`), elements of elem_bytes (1, 2, 4, 8).
cudaError_t launch_transpose(size_t elem_bytes, int rank, const int64_t *shape, const int *perm, const void *in,
                             void *out, cudaStream_t stream);

// skinny.cu — (add, mul) with a result of at most kSkinnyMaxM rows, FP64 or
// FP32: a stream over B (the shape of the method's own measurement).
constexpr int64_t kSkinnyMaxM = 8;
bool skinny_applies(int64_t M, int64_t N, int64_t K);
cudaError_t launch_skinny(bool f64, const void *A, const void *B, void *D, int64_t M, int64_t N, int64_t K,
                          cudaStream_t stream);

// bits.cu — (or, and) on packed bits.  A, B, D use the MOA_B1_U32 stream
// layout; ws is scratch of bits_workspace_bytes(M, N, K) bytes (may be NULL
// when that is 0).
size_t bits_workspace_bytes(int64_t M, int64_t N, int64_t K);
cudaError_t launch_or_and(const uint32_t *A, const uint32_t *B, uint32_t *D, int64_t M, int64_t N, int64_t K,
                          void *ws, cudaStream_t stream);

// bits_tc.cu — (or, and) by exact counting on the FP8 pair-MMA kernel, for
// results with more than 128 rows and a multiple of 32 (> 128) columns.
bool or_and_tc_applies(int64_t M, int64_t N, int64_t K);
size_t or_and_tc_workspace_bytes(int64_t M, int64_t N, int64_t K);
cudaError_t launch_or_and_tc(const uint32_t *A, const uint32_t *B, uint32_t *D, int64_t M, int64_t N, int64_t K,
                             void *ws, cudaStream_t stream);

// batch.cu — read and clear the grouped kernel's status word (bounded waits).
cudaError_t batch_read_and_clear_status(uint32_t *flags);

}  // namespace moa
