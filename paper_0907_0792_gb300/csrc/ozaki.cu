// Ozaki-sliced FP64 (add, mul) inner product (Eq. 2 in its matrix-multiply
// case) on bf16 tensor cores: an error-free splitting of each FP64 operand
// into fixed-point digit slices (Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), with
// power-of-two scales per row of A and per column of B.
//
//   row i of A:    e_i with max_k |A[i,k]| < 2^e_i,  A[i,k] = 2^e_i * a'  (|a'| < 1)
//   column j of B: f_j with max_k |B[k,j]| < 2^f_j,  B[k,j] = 2^f_j * b'
//   a' ~ sum_{s<S} d_s 2^-(s+1)beta, d_s integers in [-(2^beta - 1), 2^beta - 1]
//   (the digits of |a'| truncated to S*beta fractional bits, signed like a')
//   D[i,j] ~ 2^(e_i + f_j) * sum_{s+u<S} 2^-(s+u+2)beta * (A_s . B_u)[i,j]
//
// With beta = 7 every digit is an integer of magnitude <= 127, exact in bf16,
// and a 1024-long partial sum of digit products stays below 2^24, so each
// chunk the tensor cores accumulate in FP32 is exact.  The pairs with
// s + u >= S are dropped (their weight is below 2^-(S+1)beta).  S slices keep
// S * 7 bits of every operand relative to its row / column maximum; S grows
// as the contraction shortens (a short sum can be dominated by entries far
// below their row or column maximum, and it costs little to slice deeper).
//
// Pre-pass (this file, memory bound): |A| row maxima and |B| column maxima as
// FP64 bit patterns (integer max of the magnitude bits; finite inputs), then
// the digit planes [S][rows][cols padded to 8] in bf16, computed with integer
// operations on the FP64 fields.  The slice-pair GEMM is tc_gemm_ozaki.
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "tc.h"

namespace moa {

moa_status tc_gemm_ozaki(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, int S, int beta,
                         int lsb, int chunk_kblocks, const uint64_t *row_max, const uint64_t *col_max, double *D,
                         int64_t ldd, int64_t M, int64_t N, int64_t K, void *scratch, cudaStream_t s);

namespace {

constexpr int kMaxSlices = 10;
constexpr int kBeta = 7;
constexpr int kChunkKBlocks = 16;  // 16 x 64 = 1024 products per exact FP32 chunk

MOA_DEV uint64_t mag_bits(double x) { return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull; }

// one warp per row: max |A[i, :]| as magnitude bits
__global__ void row_max_kernel(const double *__restrict__ A, int64_t M, int64_t K, uint64_t *__restrict__ out) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t i = warp; i < M; i += nwarps) {
        uint64_t m = 0;
        for (int64_t k = lane; k < K; k += 32) m = max(m, mag_bits(__ldg(A + i * K + k)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)m, o));
        if (lane == 0) out[i] = m;
    }
}

// column maxima of B: each thread a column, each block a slice of rows, combined with atomicMax
__global__ void col_max_kernel(const double *__restrict__ B, int64_t K, int64_t N, int64_t rows_per_block,
                               uint64_t *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int64_t k0 = (int64_t)blockIdx.y * rows_per_block;
    const int64_t k1 = min(K, k0 + rows_per_block);
    uint64_t m = 0;
    for (int64_t k = k0; k < k1; ++k) m = max(m, mag_bits(__ldg(B + k * N + j)));
    if (m) atomicMax((unsigned long long *)(out + j), (unsigned long long)m);
}

MOA_DEV int scale_exp(uint64_t maxbits) {
    const int be = (int)((maxbits >> 52) & 0x7FF);
    if (be == 0) return maxbits == 0 ? 0 : -1022;
    return be - 1022;
}

// Digit s of |x| * 2^-e (|x| < 2^e): floor(|x| 2^(-e + (s+1) beta)) mod 2^beta,
// from the FP64 fields (|x| = mant * 2^ex).
MOA_DEV int digit(uint64_t mant, int ex, int e, int s) {
    const int t = ex - e + (s + 1) * kBeta;  // |x| 2^(-e + (s+1) beta) = mant * 2^t
    uint64_t v;
    if (t >= 0) v = t >= 64 ? 0 : (mant << t);
    else v = (-t) >= 64 ? 0 : (mant >> (-t));
    return (int)(v & ((1u << kBeta) - 1u));
}

// X rows x cols (row stride cols) -> S digit planes [S][rows][colsp];
// row_scale: the exponent comes from maxbits[row], else from maxbits[col].
template <bool ROW_SCALE>
__global__ void __launch_bounds__(256) slice_kernel(const double *__restrict__ X, int64_t rows, int64_t cols,
                                                     int64_t colsp, const uint64_t *__restrict__ maxbits, int S,
                                                     __nv_bfloat16 *__restrict__ out) {
    const int64_t plane = rows * colsp;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const int er = ROW_SCALE ? scale_exp(maxbits[r]) : 0;
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < colsp; c += (int64_t)gridDim.x * blockDim.x) {
            uint64_t mant = 0;
            int ex = 0, e = 0;
            bool neg = false;
            if (c < cols) {
                const double x = __ldg(X + r * cols + c);
                const uint64_t b = (uint64_t)__double_as_longlong(x);
                const int be = (int)((b >> 52) & 0x7FF);
                mant = be ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : (b & 0xFFFFFFFFFFFFFull);
                ex = (be ? be : 1) - 1075;
                e = ROW_SCALE ? er : scale_exp(maxbits[c]);
                neg = (b >> 63) != 0;
            }
            __nv_bfloat16 *dst = out + r * colsp + c;
#pragma unroll
            for (int s = 0; s < kMaxSlices; ++s) {
                if (s >= S) break;
                const int d = mant ? digit(mant, ex, e, s) : 0;
                dst[s * plane] = __int2bfloat16_rn(neg ? -d : d);
            }
        }
    }
}

int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

}  // namespace

// Slices per operand for a contraction of length K (MOA_OZAKI_SLICES overrides, 4..10).
int ozaki_slices(int64_t K) {
    static const int forced = [] {  // read once, thread-safe
        const char *e = std::getenv("MOA_OZAKI_SLICES");
        const int v = e ? std::atoi(e) : 0;
        return (v < 4 || v > kMaxSlices) ? 0 : v;
    }();
    if (forced) return forced;
    return K <= 256 ? 10 : (K <= 2048 ? 9 : 8);
}

size_t ozaki_workspace_bytes(int64_t M, int64_t N, int64_t K) {
    return (size_t)ozaki_slices(K) * (size_t)(M * round8(K) + K * round8(N)) * 2 + (size_t)(M + N) * 8 +
           pair_ozaki_scratch_bytes() + 256;
}

moa_status tc_inner_ozaki(const double *A, const double *B, double *D, int64_t M, int64_t N, int64_t K,
                          cudaStream_t s) {
    // the int32 sum of one weight class (at most S pairs of K digit products
    // below 127^2) must stay below 2^31
    if ((double)ozaki_slices(K) * (double)K * 127.0 * 127.0 >= 2147483648.0) return MOA_ERR_UNSUPPORTED;
    const int64_t Kp = round8(K), Np = round8(N);
    moa_status st;
    uint8_t *ws = (uint8_t *)workspace_get(s, ozaki_workspace_bytes(M, N, K), &st);
    if (st != MOA_OK) return st;
    const int S = ozaki_slices(K);
    __nv_bfloat16 *a = (__nv_bfloat16 *)ws;
    __nv_bfloat16 *b = a + (int64_t)S * M * Kp;
    uint64_t *rmax = (uint64_t *)(((uintptr_t)(b + (int64_t)S * K * Np) + 15) & ~(uintptr_t)15);
    uint64_t *cmax = rmax + M;
    void *rs = (void *)(((uintptr_t)(cmax + N) + 15) & ~(uintptr_t)15);  // running sums of the pair GEMM
    // scales
    {
        int64_t warps = M < 152 * 32 ? M : 152 * 32;
        row_max_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(A, M, K, rmax);
        if (cudaMemsetAsync(cmax, 0, (size_t)N * 8, s) != cudaSuccess) return MOA_ERR_CUDA;
        const int64_t gx = (N + 255) / 256;
        int64_t gy = (152 * 8 + gx - 1) / gx;
        if (gy > K) gy = K;
        const int64_t rpb = (K + gy - 1) / gy;
        gy = (K + rpb - 1) / rpb;
        col_max_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(B, K, N, rpb, cmax);
    }
    // digit planes
    {
        const int64_t gxa = Kp >= 1024 ? 4 : (Kp + 255) / 256;
        slice_kernel<true><<<dim3((unsigned)gxa, (unsigned)(M < 4096 ? M : 4096)), 256, 0, s>>>(A, M, K, Kp, rmax, S, a);
        const int64_t gxb = Np >= 1024 ? 4 : (Np + 255) / 256;
        slice_kernel<false><<<dim3((unsigned)gxb, (unsigned)(K < 4096 ? K : 4096)), 256, 0, s>>>(B, K, N, Np, cmax, S, b);
        if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    }
    // accumulator units 2^-lsb with lsb = (S + 1) beta: every kept pair weight 2^(lsb - (s+u+2) beta) >= 1
    const int lsb = (S + 1) * kBeta;
    return tc_gemm_ozaki(a, Kp, b, Np, S, kBeta, lsb, kChunkKBlocks, rmax, cmax, D, N, M, N, K, rs, s);
}

}  // namespace moa
