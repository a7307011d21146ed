// Generalized inner product over Booleans, Eq. (2) with (reduce, combine) =
// (or, and), on tensor cores by exact counting:
//     D[i, j] = OR_p (A[i, p] AND B[p, j]) = [ sum_p A[i, p] * B[p, j] > 0 ]
// with the Booleans as e4m3 0 / 1.  Every partial sum is an integer below
// 2^24, so the FP32 accumulation in TMEM is exact whatever its order, and
// the comparison with 0 gives the same bits as the definition.
//
// Pre-pass: the packed bit streams of A (M x K) and B (K x N) are expanded
// into e4m3 bytes, A row-major [M][Kp] and B transposed [N][Kp] (the K-major
// operands of the block-scaled pair GEMM, whose scales are all 1).  The
// GEMM's epilogue writes the result bits directly (one word per 32 columns of
// a row), so N must be a multiple of 32.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.h"

namespace moa {
namespace {

constexpr uint8_t kOne = 0x38;  // 1.0 in e4m3

MOA_DEV uint32_t bit_at(const uint32_t *__restrict__ w, int64_t e) { return (__ldg(w + (e >> 5)) >> (e & 31)) & 1u; }

// 16 bytes (16 consecutive k of one row) per thread.
__global__ void unpack_a_kernel(const uint32_t *__restrict__ A, int64_t M, int64_t K, int64_t Kp,
                                uint8_t *__restrict__ A8) {
    const int64_t groups = Kp / 16, total = M * groups;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / groups, k0 = (idx - i * groups) * 16;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (k0 + t < K && bit_at(A, i * K + k0 + t)) w[t / 4] |= (uint32_t)kOne << (8 * (t % 4));
        *reinterpret_cast<uint4 *>(A8 + i * Kp + k0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// B transposed: 16 consecutive k of one column n per thread, consecutive
// threads on consecutive columns.
__global__ void unpack_bt_kernel(const uint32_t *__restrict__ B, int64_t K, int64_t N, int64_t Kp,
                                 uint8_t *__restrict__ Bt8) {
    const int64_t groups = Kp / 16, total = N * groups;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = idx / N, n = idx - g * N, k0 = g * 16;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (k0 + t < K && bit_at(B, (k0 + t) * N + n)) w[t / 4] |= (uint32_t)kOne << (8 * (t % 4));
        *reinterpret_cast<uint4 *>(Bt8 + n * Kp + k0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct Layout {
    int64_t Kp, KB, MB, TN;
    size_t a8, bt8, sfa, sfb, total;  // byte offsets
};

Layout layout(int64_t M, int64_t N, int64_t K) {
    Layout l;
    l.Kp = (K + 15) / 16 * 16;
    l.KB = (K + 127) / 128;
    l.MB = (M + 127) / 128;
    l.TN = (N + pair_fp8_tile_n() - 1) / pair_fp8_tile_n();
    l.a8 = 0;
    l.bt8 = (size_t)(M * l.Kp + 15) / 16 * 16;
    l.sfa = l.bt8 + (size_t)(N * l.Kp + 15) / 16 * 16;
    l.sfb = l.sfa + (size_t)(l.MB * l.KB * 128) * 4;
    l.total = l.sfb + (size_t)(l.TN * l.KB * 256) * 4;
    return l;
}

}  // namespace

bool or_and_tc_applies(int64_t M, int64_t N, int64_t K) {
    return M > 128 && N > 128 && N % 32 == 0 && K >= 16 && K < (1ll << 24) && M < (1ll << 31) && N < (1ll << 31) &&
           pair_mma_enabled();
}

size_t or_and_tc_workspace_bytes(int64_t M, int64_t N, int64_t K) { return layout(M, N, K).total + 16; }

cudaError_t launch_or_and_tc(const uint32_t *A, const uint32_t *B, uint32_t *D, int64_t M, int64_t N, int64_t K, void *ws,
                             cudaStream_t s) {
    const Layout l = layout(M, N, K);
    uint8_t *base = (uint8_t *)(((uintptr_t)ws + 15) & ~(uintptr_t)15);
    uint8_t *a8 = base + l.a8, *bt8 = base + l.bt8;
    uint32_t *sfa = (uint32_t *)(base + l.sfa), *sfb = (uint32_t *)(base + l.sfb);
    cudaError_t e = cudaMemsetAsync(sfa, 0x7f, l.total - l.sfa, s);  // every scale 2^0
    if (e != cudaSuccess) return e;
    const int64_t ta = M * (l.Kp / 16), tb = N * (l.Kp / 16);
    unpack_a_kernel<<<(unsigned)std::min<int64_t>((ta + 255) / 256, 152 * 16), 256, 0, s>>>(A, M, K, l.Kp, a8);
    unpack_bt_kernel<<<(unsigned)std::min<int64_t>((tb + 255) / 256, 152 * 16), 256, 0, s>>>(B, K, N, l.Kp, bt8);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return tc_gemm_pair_fp8_launch(a8, l.Kp, bt8, l.Kp, (int)M, (int)N, (int)K, sfa, sfb, nullptr, N, s, D);
}

}  // namespace moa
