// FP8 (e4m3) form of the (add, mul) inner product (Eq. 2, matrix-multiply
// case): quantisation pre-pass and dispatch.  A is scaled per 1 x 128 block along the
// contraction (row i, k-block kb), B per 128 x 128 tile (k-block kb, column
// block nb), each by a power of two s = 2^(E - 8) where max|x| = m 2^E,
// m in [1/2, 1): the block maximum maps into [128, 256), inside e4m3's range
// (largest finite 448), and x / s is one exact scaling followed by one
// round-to-nearest-even conversion to e4m3 (saturating).  The tcgen05 kernel
// (tc_gemm.cu, MODE_FP8) multiplies each k-block's exact FP32 partial sum by
// sA * sB, also exact; the block-scaled pair kernel (tc_gemm_pair.cu,
// MODE_FP8) applies the same scales inside each MMA (UE8M0 scale factors of
// A's rows and B's columns) and accumulates the whole contraction in TMEM.
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc.h"

namespace moa {

moa_status tc_gemm_fp8(const uint8_t *A, int64_t lda, const uint8_t *B, int64_t ldb, const float *scale_a,
                       const float *scale_b, float *D, int64_t ldd, int64_t M, int64_t N, int64_t K, cudaStream_t s);

namespace {

MOA_DEV float block_scale(float amax, float *inv) {
    if (!(amax > 0.0f)) {
        *inv = 1.0f;
        return 1.0f;
    }
    int E;
    frexpf(amax, &E);
    *inv = ldexpf(1.0f, 8 - E);
    return ldexpf(1.0f, E - 8);
}

MOA_DEV uint8_t to_e4m3(float x) { return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3); }

// One warp per (row, k-block) of A: 128 elements, 4 per lane.
__global__ void quant_a_kernel(const float *__restrict__ A, int64_t M, int64_t K, int64_t Kp, int64_t KB,
                               uint8_t *__restrict__ A8, float *__restrict__ sA) {
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    const int lane = threadIdx.x % 32;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < M * KB; w += nw) {
        const int64_t row = w / KB, kb = w - row * KB;
        const int64_t k0 = kb * 128 + lane * 4;
        float x[4];
        float amax = 0.0f;
        const float *src = A + row * K + k0;
        if (k0 + 4 <= K && ((uintptr_t)src & 15) == 0) {  // one 16-byte load
            const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
            x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = (k0 + i < K) ? __ldg(src + i) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) amax = fmaxf(amax, fabsf(x[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        float inv;
        const float sc = block_scale(amax, &inv);
        if (k0 < Kp) {
            uint32_t packed = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) packed |= (uint32_t)to_e4m3(__fmul_rn(x[i], inv)) << (8 * i);
            *reinterpret_cast<uint32_t *>(A8 + row * Kp + k0) = packed;
        }
        if (lane == 0) sA[row * KB + kb] = sc;
    }
}

// One block per 128 x 128 tile of B.  Thread t owns columns 4 (t % 32) .. +3
// of rows t / 32, t / 32 + 8, ...: one 16-byte load per row when aligned, the
// 64 values kept in registers between the maximum and the quantisation, and
// one packed 4-byte store per row.
__global__ void __launch_bounds__(256) quant_b_kernel(const float *__restrict__ B, int64_t K, int64_t N, int64_t Np,
                                                      int64_t NB, uint8_t *__restrict__ B8, float *__restrict__ sB) {
    __shared__ float red[8];
    const int64_t kb = blockIdx.y, nb = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t n0 = nb * 128 + (t % 32) * 4;
    const bool vec = (N % 4 == 0) && (((uintptr_t)B & 15) == 0) && (n0 + 4 <= N);
    float x[16][4];
    float amax = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int64_t k = kb * 128 + t / 32 + 8 * i;
        if (k < K && vec) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(B + k * N + n0));
            x[i][0] = v.x, x[i][1] = v.y, x[i][2] = v.z, x[i][3] = v.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) x[i][c] = (k < K && n0 + c < N) ? __ldg(B + k * N + n0 + c) : 0.0f;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) amax = fmaxf(amax, fabsf(x[i][c]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (t % 32 == 0) red[t / 32] = amax;
    __syncthreads();
    amax = red[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) amax = fmaxf(amax, red[i]);
    float inv;
    const float sc = block_scale(amax, &inv);
    if (n0 < Np) {  // Np is a multiple of 16, so n0 .. n0 + 3 are all inside a padded row
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int64_t k = kb * 128 + t / 32 + 8 * i;
            if (k >= K) break;
            uint32_t packed = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (n0 + c < N) packed |= (uint32_t)to_e4m3(__fmul_rn(x[i][c], inv)) << (8 * c);
            *reinterpret_cast<uint32_t *>(B8 + k * Np + n0) = packed;
        }
    }
    if (t == 0) sB[kb * NB + nb] = sc;
}

// The same quantisation of B, written transposed: Bt [N][Kp] (K-major), the
// operand layout of the block-scaled pair GEMM.  One block per 128 x 128
// tile; thread t owns column t % 128 and 64 consecutive k of it (loads
// coalesced across a warp along the row of B), and writes its 64 codes as
// four 16-byte stores into the column's row of Bt.
__global__ void __launch_bounds__(256) quant_bt_kernel(const float *__restrict__ B, int64_t K, int64_t N, int64_t Kp,
                                                       int64_t NB, uint8_t *__restrict__ Bt, float *__restrict__ sB) {
    __shared__ float red[8];
    const int64_t kb = blockIdx.y, nb = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t n = nb * 128 + (t & 127);
    const int64_t k0 = kb * 128 + (int64_t)(t >> 7) * 64;
    float x[64];
    float amax = 0.0f;
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        const int64_t k = k0 + i;
        x[i] = (k < K && n < N) ? __ldg(B + k * N + n) : 0.0f;
        amax = fmaxf(amax, fabsf(x[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (t % 32 == 0) red[t / 32] = amax;
    __syncthreads();
    amax = red[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) amax = fmaxf(amax, red[i]);
    float inv;
    const float sc = block_scale(amax, &inv);
    if (n < N) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            if (k0 + 16 * h >= Kp) break;
            uint32_t w[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                w[b] = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) w[b] |= (uint32_t)to_e4m3(__fmul_rn(x[16 * h + 4 * b + c], inv)) << (8 * c);
            }
            *reinterpret_cast<uint4 *>(Bt + n * Kp + k0 + 16 * h) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    if (t == 0) sB[kb * NB + nb] = sc;
}

// Scale factors of the block-scaled pair GEMM: UE8M0 byte = the exponent
// field of the power-of-two FP32 scale (both have bias 127), repeated in the
// four bytes of a word (one per 32-deep k-step of the 128-deep k-block), in
// the kernel's TMEM-word order (tc.h, tc_gemm_pair_fp8_launch).
MOA_DEV uint32_t ue8m0_word(float scale) { return ((__float_as_uint(scale) >> 23) & 255u) * 0x01010101u; }

__global__ void pack_sfa_kernel(const float *__restrict__ sA, int64_t M, int64_t KB, uint32_t *__restrict__ out,
                                int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % 128);
        const int64_t blk = i / 128, rb = blk / KB, kb = blk - rb * KB;
        const int64_t row = rb * 128 + 32 * (w % 4) + w / 4;
        out[i] = row < M ? ue8m0_word(sA[row * KB + kb]) : 0x7f7f7f7fu;
    }
}

__global__ void pack_sfb_kernel(const float *__restrict__ sB, int64_t N, int64_t KB, int64_t NB, int T,
                                uint32_t *__restrict__ out, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % 256);
        const int64_t blk = i / 256, tn = blk / KB, kb = blk - tn * KB;
        const int j = 4 * (w / 128) + w % 4, l = (w % 128) / 4;
        const int64_t col = tn * T + 32 * j + l;
        out[i] = (32 * j < T && col < N) ? ue8m0_word(sB[kb * NB + col / 128]) : 0x7f7f7f7fu;
    }
}

}  // namespace

size_t fp8_workspace_bytes(int64_t M, int64_t N, int64_t K) {
    const int64_t Kp = (K + 15) / 16 * 16, Np = (N + 15) / 16 * 16, KB = (K + 127) / 128, NB = (N + 127) / 128;
    const int64_t bbytes = K * Np > N * Kp ? K * Np : N * Kp;  // B as given or transposed
    const int64_t T = pair_fp8_tile_n(), MB = (M + 127) / 128, TN = (N + T - 1) / T;
    const int64_t words = MB * KB * 128 + TN * KB * 256;  // packed scale factors of the pair GEMM
    return (size_t)(M * Kp + bbytes) + (size_t)(M * KB + KB * NB) * 4 + (size_t)words * 4 + 96;
}

moa_status tc_inner_fp8(const float *A, const float *B, float *D, int64_t M, int64_t N, int64_t K, cudaStream_t s) {
    const int64_t Kp = (K + 15) / 16 * 16, Np = (N + 15) / 16 * 16, KB = (K + 127) / 128, NB = (N + 127) / 128;
    moa_status st;
    uint8_t *ws = (uint8_t *)workspace_get(s, fp8_workspace_bytes(M, N, K), &st);
    if (st != MOA_OK) return st;
    uint8_t *a8 = ws, *b8 = ws + M * Kp;
    const int64_t bbytes = K * Np > N * Kp ? K * Np : N * Kp;
    float *sa = (float *)(((uintptr_t)(b8 + bbytes) + 15) & ~(uintptr_t)15);
    float *sb = sa + M * KB;
    // the block-scaled pair GEMM (256 x 224 tiles, B transposed) for large
    // products; the single-CTA kernel with scaled register accumulation else
    const bool pair = M > 128 && N > 128 && M < (1ll << 31) && N < (1ll << 31) && K < (1ll << 31) && pair_mma_enabled();
    {
        int64_t warps = M * KB;
        int64_t blocks = (warps * 32 + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        quant_a_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, M, K, Kp, KB, a8, sa);
        if (KB > 65535) return MOA_ERR_OVERFLOW;
        if (pair)
            quant_bt_kernel<<<dim3((unsigned)NB, (unsigned)KB), 256, 0, s>>>(B, K, N, Kp, NB, b8, sb);
        else
            quant_b_kernel<<<dim3((unsigned)NB, (unsigned)KB), 256, 0, s>>>(B, K, N, Np, NB, b8, sb);
        if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    }
    if (pair) {
        const int64_t T = pair_fp8_tile_n(), MB = (M + 127) / 128, TN = (N + T - 1) / T;
        uint32_t *sfa = reinterpret_cast<uint32_t *>(((uintptr_t)(sb + KB * NB) + 15) & ~(uintptr_t)15);  // TMA: 16-B base
        uint32_t *sfb = sfa + MB * KB * 128;
        pack_sfa_kernel<<<(unsigned)std::min<int64_t>((MB * KB * 128 + 255) / 256, 152 * 8), 256, 0, s>>>(sa, M, KB, sfa,
                                                                                                        MB * KB * 128);
        pack_sfb_kernel<<<(unsigned)std::min<int64_t>((TN * KB * 256 + 255) / 256, 152 * 8), 256, 0, s>>>(
            sb, N, KB, NB, (int)T, sfb, TN * KB * 256);
        if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
        return tc_gemm_pair_fp8_launch(a8, Kp, b8, Kp, (int)M, (int)N, (int)K, sfa, sfb, D, N, s) == cudaSuccess
                   ? MOA_OK
                   : MOA_ERR_CUDA;
    }
    return tc_gemm_fp8(a8, Kp, b8, Np, sa, sb, D, N, M, N, K, s);
}

}  // namespace moa
