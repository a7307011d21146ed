// Generalized inner product over Booleans, Eq. (2) with (reduce, combine) =
// (or, and):  D[i, j] = OR_p ( A[i, p] AND B[p, j] ), on packed bits.
//
// The paper's row organisation (Fig. 1: row i of the result accumulates row p
// of B whenever A[i, p] contributes) becomes word-parallel here: one 32-bit
// word of B's row p carries 32 columns, so
//     D_word(i, w) |= B_word(p, w) & mask(A[i, p])
// applies the semiring to 32 (i, p, j) triples with one LOP3.  A CTA owns a
// 64-row x 32-word (1024-column) tile of D; B rows are staged in shared
// memory 32 contraction steps at a time (one A word per row).
//
// Layout: the ABI's bit stream (element e = bit e%32 of word e/32).  When K
// and N are multiples of 32 every row of A, B and D starts on a word and the
// kernel reads the stream directly; otherwise rows are first re-packed into
// word-aligned rows in scratch memory and D is re-packed back afterwards.
#include "common.cuh"
#include "internal.h"

namespace moa {
namespace {

constexpr int BM = 64;   // rows of D per CTA
constexpr int BW = 32;   // words of D per CTA (1024 columns)
constexpr int NT = 256;  // threads: word w = tid % 32, rows (tid / 32) * 8 .. + 7
constexpr int RPT = BM / (NT / BW);

__global__ void __launch_bounds__(NT) or_and_kernel(const uint32_t *__restrict__ A, const uint32_t *__restrict__ B,
                                                    uint32_t *__restrict__ D, int64_t M, int64_t KW, int64_t NW,
                                                    int64_t K) {
    __shared__ uint32_t Bs[32][BW + 1];
    __shared__ uint32_t As[BM];
    const int tid = threadIdx.x;
    const int w = tid % BW, g = tid / BW;
    const int64_t m0 = (int64_t)blockIdx.y * BM, w0 = (int64_t)blockIdx.x * BW;
    uint32_t acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = 0u;

    for (int64_t kw = 0; kw < KW; ++kw) {
        // stage 32 rows of B (contraction steps 32*kw .. 32*kw+31) and one A word per row
        for (int e = tid; e < 32 * BW; e += NT) {
            const int pr = e / BW, wc = e % BW;
            const int64_t p = kw * 32 + pr, col = w0 + wc;
            Bs[pr][wc] = (p < K && col < NW) ? B[p * NW + col] : 0u;
        }
        if (tid < BM) {
            const int64_t m = m0 + tid;
            As[tid] = (m < M) ? A[m * KW + kw] : 0u;
        }
        __syncthreads();
        uint32_t a[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) a[r] = As[g * RPT + r];
#pragma unroll 8
        for (int pr = 0; pr < 32; ++pr) {
            const uint32_t b = Bs[pr][w];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const uint32_t mask = (uint32_t)((int32_t)(a[r] << (31 - pr)) >> 31);  // all ones iff bit pr set
                acc[r] |= b & mask;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int64_t m = m0 + g * RPT + r, col = w0 + w;
        if (m < M && col < NW) D[m * NW + col] = acc[r];
    }
}

// Bit stream -> word-aligned rows: row r of `rows` x `len` bits becomes
// words (r, 0 .. ceil(len/32)-1), unused high bits zero.
__global__ void repack_rows(const uint32_t *__restrict__ S, uint32_t *__restrict__ R, int64_t rows, int64_t len) {
    const int64_t wpr = (len + 31) / 32, total = rows * wpr;
    const int64_t stream_words = (rows * len + 31) / 32;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / wpr, w = q - r * wpr;
        const int64_t e = r * len + w * 32;  // first bit of this word in the stream
        const int64_t sw = e / 32;
        const int sh = (int)(e % 32);
        const uint32_t lo = S[sw];
        const uint32_t hi = (sw + 1 < stream_words) ? S[sw + 1] : 0u;
        uint32_t v = __funnelshift_r(lo, hi, sh);
        const int64_t valid = len - w * 32;
        if (valid < 32) v &= (1u << valid) - 1u;
        R[q] = v;
    }
}

// Word-aligned rows -> bit stream (inverse of repack_rows).
__global__ void unpack_rows(const uint32_t *__restrict__ R, uint32_t *__restrict__ S, int64_t rows, int64_t len) {
    const int64_t wpr = (len + 31) / 32, nbits = rows * len;
    const int64_t stream_words = (nbits + 31) / 32;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < stream_words;
         q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0u;
        for (int b = 0; b < 32; ++b) {
            const int64_t e = q * 32 + b;
            if (e >= nbits) break;
            const int64_t r = e / len, c = e - r * len;
            v |= ((R[r * wpr + c / 32] >> (c % 32)) & 1u) << b;
        }
        S[q] = v;
    }
}

inline int64_t grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

}  // namespace

size_t bits_workspace_bytes(int64_t M, int64_t N, int64_t K) {
    if (K % 32 == 0 && N % 32 == 0) return 0;
    const int64_t KW = (K + 31) / 32, NW = (N + 31) / 32;
    return (size_t)(M * KW + K * NW + M * NW) * sizeof(uint32_t);
}

cudaError_t launch_or_and(const uint32_t *A, const uint32_t *B, uint32_t *D, int64_t M, int64_t N, int64_t K, void *ws,
                          cudaStream_t s) {
    const int64_t KW = (K + 31) / 32, NW = (N + 31) / 32;
    const uint32_t *a = A, *b = B;
    uint32_t *d = D;
    const bool aligned = (K % 32 == 0 && N % 32 == 0);
    if (!aligned) {
        uint32_t *wa = (uint32_t *)ws, *wb = wa + M * KW, *wd = wb + K * NW;
        if (M * KW > 0) repack_rows<<<(unsigned)grid_for(M * KW), 256, 0, s>>>(A, wa, M, K);
        if (K * NW > 0) repack_rows<<<(unsigned)grid_for(K * NW), 256, 0, s>>>(B, wb, K, N);
        a = wa, b = wb, d = wd;
    }
    const int64_t gx = (NW + BW - 1) / BW, gy = (M + BM - 1) / BM;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    or_and_kernel<<<dim3((unsigned)gx, (unsigned)gy), NT, 0, s>>>(a, b, d, M, KW, NW, K);
    if (!aligned) unpack_rows<<<(unsigned)grid_for((M * N + 31) / 32), 256, 0, s>>>(d, D, M, N);
    return cudaGetLastError();
}

}  // namespace moa
