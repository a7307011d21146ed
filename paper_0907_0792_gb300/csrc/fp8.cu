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

// Scale factors of the block-scaled pair GEMM: UE8M0 byte = the exponent
// field of the power-of-two FP32 scale (both have bias 127), repeated in the
// four bytes of a word (one per 32-deep k-step of the 128-deep k-block), in
// the kernel's TMEM-word order (tc.h, tc_gemm_pair_fp8_launch).
MOA_DEV uint32_t ue8m0_word(float scale) { return ((__float_as_uint(scale) >> 23) & 255u) * 0x01010101u; }

// Eight threads per (row, k-block) of A: 16 elements each (four 16-byte
// loads when aligned), the block maximum by three shuffles inside the
// group, one 16-byte store of codes per thread.  With `sfa`, the scale is
// also written as the pair GEMM's scale word.
__global__ void __launch_bounds__(256) quant_a_kernel(const float *__restrict__ A, int64_t M, int64_t K, int64_t Kp,
                                                      int64_t KB, uint8_t *__restrict__ A8, float *__restrict__ sA,
                                                      uint32_t *__restrict__ sfa) {
    const int sub = threadIdx.x % 8;
    for (int64_t blk = (int64_t)blockIdx.x * 32 + threadIdx.x / 8; blk < M * KB; blk += (int64_t)gridDim.x * 32) {
        const int64_t row = blk / KB, kb = blk - row * KB;
        const int64_t k0 = kb * 128 + sub * 16;
        const float *src = A + row * K + k0;
        float x[16];
        if (k0 + 16 <= K && ((uintptr_t)src & 15) == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + i);
                x[4 * i] = v.x, x[4 * i + 1] = v.y, x[4 * i + 2] = v.z, x[4 * i + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) x[i] = (k0 + i < K) ? __ldg(src + i) : 0.0f;
        }
        float amax = 0.0f;
#pragma unroll
        for (int i = 0; i < 16; ++i) amax = fmaxf(amax, fabsf(x[i]));
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        float inv;
        const float sc = block_scale(amax, &inv);
        if (k0 < Kp) {  // Kp is a multiple of 16: all 16 codes lie inside the padded row
            uint32_t w[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                w[b] = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) w[b] |= (uint32_t)to_e4m3(__fmul_rn(x[4 * b + c], inv)) << (8 * c);
            }
            *reinterpret_cast<uint4 *>(A8 + row * Kp + k0) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (sub == 0) {
            sA[row * KB + kb] = sc;
            if (sfa) sfa[((row / 128) * KB + kb) * 128 + (row % 32) * 4 + (row % 128) / 32] = ue8m0_word(sc);
        }
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
// operand layout of the block-scaled pair GEMM, with the scale also written
// as that GEMM's scale word of every column.  One block per 128 x 128 tile;
// thread t owns column t % 128 and 64 consecutive k of it (loads coalesced
// across a warp along the row of B), and writes its 64 codes as four
// 16-byte stores into the column's row of Bt.
__global__ void __launch_bounds__(256) quant_bt_kernel(const float *__restrict__ B, int64_t K, int64_t N, int64_t Kp,
                                                       int64_t NB, uint8_t *__restrict__ Bt, float *__restrict__ sB,
                                                       uint32_t *__restrict__ sfb, int T, int64_t KB) {
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
    if (t < 128 && n < N) {  // this column's scale word of the pair GEMM (tile T columns wide)
        const int64_t tn = n / T;
        const int j = (int)(n - tn * T) / 32, l = (int)(n % 32);
        sfb[(tn * KB + kb) * 256 + (j / 4) * 128 + l * 4 + j % 4] = ue8m0_word(sc);
    }
}

// Byte rows X (rows x cols, row stride cols) -> rows x colsp (colsp a
// multiple of 16, zero past cols): one 16-byte store per thread.
__global__ void __launch_bounds__(256) pad_rows_u8(const uint8_t *__restrict__ X, int64_t rows, int64_t cols,
                                                   int64_t colsp, uint8_t *__restrict__ out) {
    const int64_t groups = colsp / 16, total = rows * groups;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / groups, c = (idx - r * groups) * 16;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int b = 0; b < 16; ++b)
            if (c + b < cols) w[b / 4] |= (uint32_t)__ldg(X + r * cols + c + b) << (8 * (b % 4));
        *reinterpret_cast<uint4 *>(out + r * colsp + c) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Bt [N][Kp] = B [K][N] transposed (bytes; zero for k >= K): 64 x 64 tiles
// through shared memory, reads along B's rows, writes along Bt's rows.
__global__ void __launch_bounds__(256) transpose_u8(const uint8_t *__restrict__ B, int64_t K, int64_t N, int64_t Kp,
                                                    uint8_t *__restrict__ Bt) {
    __shared__ uint8_t tile[64][65];
    const int64_t k0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    const int tx = threadIdx.x % 64, ty = threadIdx.x / 64;  // 64 x 4
    for (int i = ty; i < 64; i += 4) {
        const int64_t k = k0 + i, n = n0 + tx;
        tile[i][tx] = (k < K && n < N) ? __ldg(B + k * N + n) : (uint8_t)0;
    }
    __syncthreads();
    for (int i = ty; i < 64; i += 4) {
        const int64_t n = n0 + i, k = k0 + tx;
        if (n < N && k < Kp) Bt[n * Kp + k] = tile[tx][i];
    }
}

// Caller scales (FP32, taken as the power of two of their exponent field)
// -> the pair GEMM's UE8M0 words: A's [row][k-block] and B's [k-block][column
// block of 128], in the word order of tc_gemm_pair_fp8_launch (tc.h).
__global__ void scale_words_kernel(const float *__restrict__ scale_a, const float *__restrict__ scale_b, int64_t M,
                                   int64_t N, int64_t KB, int64_t NB, int T, uint32_t *__restrict__ sfa,
                                   uint32_t *__restrict__ sfb) {
    const int64_t na = M * KB, nb = N * KB;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < na) {
            const int64_t row = i / KB, kb = i - row * KB;
            sfa[((row / 128) * KB + kb) * 128 + (row % 32) * 4 + (row % 128) / 32] = ue8m0_word(scale_a[i]);
        } else {
            const int64_t e = i - na, n = e / KB, kb = e - n * KB;
            const int64_t tn = n / T;
            const int j = (int)(n - tn * T) / 32, l = (int)(n % 32);
            sfb[(tn * KB + kb) * 256 + (j / 4) * 128 + l * 4 + j % 4] = ue8m0_word(scale_b[kb * NB + n / 128]);
        }
    }
}

// The same scales as FP32 powers of two (exponent field kept, sign and
// mantissa dropped) for the single-CTA kernel, so both kernels apply the same
// factors.
__global__ void pow2_scales_kernel(const float *__restrict__ src, int64_t n, float *__restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __uint_as_float(__float_as_uint(src[i]) & 0x7F800000u);
}

}  // namespace

// e4m3 operands as given: A [M][K] and B [K][N] bytes, with unit scales, or
// with the caller's scales scale_a [M][ceil(K/128)] and scale_b
// [ceil(K/128)][ceil(N/128)] (FP32 device arrays).  The block-scaled pair GEMM
// takes A K-major (padded rows when K % 16 != 0) and B transposed, with the
// scale words 2^0 or built from the caller's scales; the single-CTA FP8
// kernel takes B as given (padded rows) with scale tables.
moa_status tc_inner_e4m3(const uint8_t *A, const uint8_t *B, float *D, int64_t M, int64_t N, int64_t K, cudaStream_t s,
                         const float *scale_a, const float *scale_b) {
    const int64_t Kp = (K + 15) / 16 * 16, Np = (N + 15) / 16 * 16, KB = (K + 127) / 128, NB = (N + 127) / 128;
    if (KB > 65535) return MOA_ERR_OVERFLOW;
    const bool pair = M > 128 && N > 128 && M < (1ll << 31) && N < (1ll << 31) && K < (1ll << 31) && pair_mma_enabled();
    const bool a_direct = K % 16 == 0 && (uintptr_t)A % 16 == 0;
    const bool b_direct = !pair && N % 16 == 0 && (uintptr_t)B % 16 == 0;
    const int64_t T = pair_fp8_tile_n(), MB = (M + 127) / 128, TN = (N + T - 1) / T;
    const size_t abytes = a_direct ? 0 : (size_t)(M * Kp), bbytes = b_direct ? 0 : (size_t)(pair ? N * Kp : K * Np);
    const size_t words = pair ? (size_t)(MB * KB * 128 + TN * KB * 256) : (size_t)(M * KB + KB * NB);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    moa_status st;
    uint8_t *ws = (uint8_t *)workspace_get(s, up(abytes) + up(bbytes) + words * 4 + 256, &st);
    if (st != MOA_OK) return st;
    const uint8_t *a8 = a_direct ? A : ws;
    uint8_t *b8 = ws + up(abytes);
    uint32_t *scales = (uint32_t *)(ws + up(abytes) + up(bbytes));
    if (!a_direct) {
        const int64_t total = M * (Kp / 16);
        pad_rows_u8<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(A, M, K, Kp, ws);
    }
    if (pair) {
        transpose_u8<<<dim3((unsigned)((N + 63) / 64), (unsigned)((Kp + 63) / 64)), 256, 0, s>>>(B, K, N, Kp, b8);
        if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
        if (cudaMemsetAsync(scales, 0x7f, words * 4, s) != cudaSuccess) return MOA_ERR_CUDA;  // UE8M0 127 = 2^0
        uint32_t *sfa = scales, *sfb = scales + MB * KB * 128;
        if (scale_a) {
            const int64_t n = (M + N) * KB;
            scale_words_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
                scale_a, scale_b, M, N, KB, NB, (int)T, sfa, sfb);
            if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
        }
        return tc_gemm_pair_fp8_launch(a8, Kp, b8, Kp, (int)M, (int)N, (int)K, sfa, sfb, D, N, s) == cudaSuccess
                   ? MOA_OK
                   : MOA_ERR_CUDA;
    }
    const uint8_t *bb = B;
    if (!b_direct) {
        const int64_t total = K * (Np / 16);
        pad_rows_u8<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(B, K, N, Np, b8);
        bb = b8;
    }
    if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    float *sa = (float *)scales, *sb = sa + M * KB;
    if (scale_a) {
        pow2_scales_kernel<<<(unsigned)std::min<int64_t>((M * KB + 255) / 256, 152 * 16), 256, 0, s>>>(scale_a, M * KB, sa);
        pow2_scales_kernel<<<(unsigned)std::min<int64_t>((KB * NB + 255) / 256, 152 * 16), 256, 0, s>>>(scale_b, KB * NB, sb);
        if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    } else if (launch_fill32(scales, 0x3f800000u, (int64_t)words, s) != cudaSuccess) {  // FP32 1.0
        return MOA_ERR_CUDA;
    }
    return tc_gemm_fp8(a8, Kp, bb, Np, sa, sb, D, N, M, N, K, s);
}

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
    const int64_t T = pair_fp8_tile_n(), MB = (M + 127) / 128, TN = (N + T - 1) / T;
    uint32_t *sfa = reinterpret_cast<uint32_t *>(((uintptr_t)(sb + KB * NB) + 15) & ~(uintptr_t)15);  // TMA: 16-B base
    uint32_t *sfb = sfa + MB * KB * 128;
    if (KB > 65535) return MOA_ERR_OVERFLOW;
    if (pair && cudaMemsetAsync(sfa, 0x7f, (size_t)(MB * KB * 128 + TN * KB * 256) * 4, s) != cudaSuccess)
        return MOA_ERR_CUDA;  // words no row or column writes: scale 1
    {
        int64_t blocks = (M * KB + 31) / 32;
        if (blocks > 152 * 16) blocks = 152 * 16;
        quant_a_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, M, K, Kp, KB, a8, sa, pair ? sfa : nullptr);
        if (pair)
            quant_bt_kernel<<<dim3((unsigned)NB, (unsigned)KB), 256, 0, s>>>(B, K, N, Kp, NB, b8, sb, sfb, (int)T, KB);
        else
            quant_b_kernel<<<dim3((unsigned)NB, (unsigned)KB), 256, 0, s>>>(B, K, N, Np, NB, b8, sb);
        if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    }
    if (pair)
        return tc_gemm_pair_fp8_launch(a8, Kp, b8, Kp, (int)M, (int)N, (int)K, sfa, sfb, D, N, s) == cudaSuccess
                   ? MOA_OK
                   : MOA_ERR_CUDA;
    return tc_gemm_fp8(a8, Kp, b8, Np, sa, sb, D, N, M, N, K, s);
}

}  // namespace moa
