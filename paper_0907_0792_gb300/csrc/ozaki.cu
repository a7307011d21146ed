// Ozaki-sliced FP64 (add, mul) inner product (Eq. 2 in its matrix-multiply
// case) on bf16 tensor cores: an error-free splitting of each FP64 operand
// into fixed-point digit slices (Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), with
// power-of-two scales per row of A and per column of B.
//
//   row i of A:    e_i with max_k |A[i,k]| < 2^(e_i - 1),  A[i,k] = 2^e_i * a'
//                  (|a'| < 1/2)
//   column j of B: f_j likewise,  B[k,j] = 2^f_j * b'
//   a' ~ sum_{s<S} d_s 2^-(s+1)beta, the S * beta fractional bits of |a'|
//        (truncated) written in balanced base 2^beta: d_s in [-2^(beta-1),
//        2^(beta-1) - 1] for s > 0 and d_0 in [0, 2^(beta-1)], signed like a'
//   D[i,j] ~ 2^(e_i + f_j) * sum_{s+u<S} 2^-(s+u+2)beta * (A_s . B_u)[i,j]
//
// With beta = 8 every digit is an integer of magnitude <= 128, exact in bf16,
// every digit product is at most 2^14, and a 1024-long partial sum stays at
// or below 2^24, so each chunk the tensor cores accumulate in FP32 is exact.
// The balanced digits carry 8 bits each where unsigned 7-bit digits carried
// 7 at the same product bound, so 7 slices keep 55 bits of every operand
// relative to its row / column maximum (28 slice products) where 8 slices of
// 7 bits needed 36 products for 56 bits.  The pairs with s + u >= S are
// dropped (their weight is at most 2^-(S+2)beta * 2^14).  S grows as the
// contraction shortens (a short sum can be dominated by entries far below
// their row or column maximum, and it costs little to slice deeper; the
// truncation errors of a long sum partly cancel): 10 slices up to K = 64, 8
// up to K = 256, 7 below K = 4096, 6 from K = 4096 (21 slice products; 47
// bits of every operand).
//
// Pre-pass (this file, memory bound): |A| row maxima and |B| column maxima as
// FP64 bit patterns (integer max of the magnitude bits; finite inputs), then
// the digit planes [S][rows][cols padded to 8] in bf16, computed with integer
// operations on the FP64 fields.  The slice-pair GEMM is tc_gemm_ozaki.
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "tc.h"
#include "ozaki_epi.cuh"

namespace moa {

moa_status tc_gemm_ozaki(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, int S, int beta,
                         int lsb, int chunk_kblocks, int acc_pairs, const uint64_t *row_max, const uint64_t *col_max,
                         double *D, int64_t ldd, int64_t M, int64_t N, int64_t K, void *scratch, cudaStream_t s);

namespace {

constexpr int kMaxSlices = 10;
constexpr int kBeta = 8;
constexpr int kChunkKBlocks = 16;  // 16 x 64 = 1024 products (each at most 2^14) per exact FP32 chunk

MOA_DEV uint64_t mag_bits(double x) { return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull; }

// one warp per row: max |A[i, :]| as magnitude bits; the grid also zeroes
// the N column maxima that col_max_kernel, launched next, combines into
__global__ void row_max_kernel(const double *__restrict__ A, int64_t M, int64_t K, uint64_t *__restrict__ out,
                               uint64_t *__restrict__ col_zero, int64_t N) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = tid; j < N; j += nthreads) col_zero[j] = 0;
    const int64_t warp = tid / 32;
    const int lane = threadIdx.x % 32;
    const int64_t nwarps = nthreads / 32;
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

// The S balanced digits of one element, signed like it: |x| = mant 2^ex,
// scaled by 2^-e (|x| < 2^(e-1)).  The unsigned base-2^beta digits u_s of
// the truncated |x| 2^-e (u_s = floor(|x| 2^(-e + (s+1) beta)) mod 2^beta,
// u_0 < 2^(beta-1)) are rewritten from the lowest up: a digit of 2^(beta-1)
// or more becomes u - 2^beta with a carry of one into the next higher digit.
template <int S>
MOA_DEV void balanced_digits(uint64_t mant, int ex, int e, bool neg, int (&d)[S]) {
    int carry = 0;
#pragma unroll
    for (int s = S - 1; s >= 0; --s) {
        const int t = ex - e + (s + 1) * kBeta;  // |x| 2^(-e + (s+1) beta) = mant * 2^t
        uint64_t v;
        if (t >= 0) v = t >= 64 ? 0 : (mant << t);
        else v = (-t) >= 64 ? 0 : (mant >> (-t));
        int u = (int)(v & ((1u << kBeta) - 1u)) + carry;
        carry = 0;
        if (s > 0 && u >= (1 << (kBeta - 1))) {
            u -= 1 << kBeta;
            carry = 1;
        }
        d[s] = neg ? -u : u;
    }
}

// X rows x cols (row stride cols) -> S digit planes [S][rows][colsp];
// row_scale: the exponent comes from maxbits[row], else from maxbits[col].
// Four consecutive columns per thread (colsp is a multiple of 8): one or two
// 16-byte loads when the row allows (VEC), one 8-byte store per plane.
template <bool ROW_SCALE, bool VEC, int S>
__global__ void __launch_bounds__(256) slice_kernel(const double *__restrict__ X, int64_t rows, int64_t cols,
                                                     int64_t colsp, const uint64_t *__restrict__ maxbits,
                                                     __nv_bfloat16 *__restrict__ out) {
    const int64_t plane = rows * colsp, groups = colsp / 4;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const int er = ROW_SCALE ? ozaki::scale_exponent(maxbits[r]) : 0;
        const double *src = X + r * cols;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c0 = 4 * g;
            double x[4];
            if constexpr (VEC) {  // cols % 4 == 0 and 16-byte aligned rows: the group is all in or all out
                if (c0 < cols) {
                    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(src + c0));
                    const double2 v1 = __ldg(reinterpret_cast<const double2 *>(src + c0 + 2));
                    x[0] = v0.x, x[1] = v0.y, x[2] = v1.x, x[3] = v1.y;
                } else {
                    x[0] = x[1] = x[2] = x[3] = 0.0;
                }
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) x[t] = c0 + t < cols ? __ldg(src + c0 + t) : 0.0;
            }
            uint32_t pk[S][2];  // four bf16 digits per plane, packed in two words
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint64_t b = (uint64_t)__double_as_longlong(x[t]);
                const int be = (int)((b >> 52) & 0x7FF);
                const uint64_t mant = be ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : (b & 0xFFFFFFFFFFFFFull);
                const int ex = (be ? be : 1) - 1075;
                const int e = ROW_SCALE ? er : (c0 + t < cols ? ozaki::scale_exponent(__ldg(maxbits + c0 + t)) : 0);
                int d[S];
                balanced_digits<S>(mant, ex, e, (b >> 63) != 0, d);
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    const uint32_t h = (uint32_t)__bfloat16_as_ushort(__int2bfloat16_rn(d[q]));
                    if (t % 2 == 0) pk[q][t / 2] = h;
                    else pk[q][t / 2] |= h << 16;
                }
            }
            __nv_bfloat16 *dst = out + r * colsp + c0;
#pragma unroll
            for (int q = 0; q < S; ++q) *reinterpret_cast<uint2 *>(dst + q * plane) = make_uint2(pk[q][0], pk[q][1]);
        }
    }
}

template <bool ROW_SCALE, int S>
void run_slices_s(const double *X, int64_t rows, int64_t cols, int64_t colsp, const uint64_t *maxbits,
                  __nv_bfloat16 *out, cudaStream_t s) {
    const int64_t groups = colsp / 4;
    const int64_t gx = groups >= 256 * 4 ? 4 : (groups + 255) / 256;
    const dim3 grid((unsigned)gx, (unsigned)(rows < 4096 ? rows : 4096));
    if (cols % 4 == 0 && (uintptr_t)X % 16 == 0)
        slice_kernel<ROW_SCALE, true, S><<<grid, 256, 0, s>>>(X, rows, cols, colsp, maxbits, out);
    else
        slice_kernel<ROW_SCALE, false, S><<<grid, 256, 0, s>>>(X, rows, cols, colsp, maxbits, out);
}

template <bool ROW_SCALE>
bool run_slices(const double *X, int64_t rows, int64_t cols, int64_t colsp, const uint64_t *maxbits, int S,
                __nv_bfloat16 *out, cudaStream_t s) {
    switch (S) {
    case 4: run_slices_s<ROW_SCALE, 4>(X, rows, cols, colsp, maxbits, out, s); return true;
    case 5: run_slices_s<ROW_SCALE, 5>(X, rows, cols, colsp, maxbits, out, s); return true;
    case 6: run_slices_s<ROW_SCALE, 6>(X, rows, cols, colsp, maxbits, out, s); return true;
    case 7: run_slices_s<ROW_SCALE, 7>(X, rows, cols, colsp, maxbits, out, s); return true;
    case 8: run_slices_s<ROW_SCALE, 8>(X, rows, cols, colsp, maxbits, out, s); return true;
    case 9: run_slices_s<ROW_SCALE, 9>(X, rows, cols, colsp, maxbits, out, s); return true;
    case 10: run_slices_s<ROW_SCALE, 10>(X, rows, cols, colsp, maxbits, out, s); return true;
    }
    return false;
}

int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

}  // namespace

// k-blocks of 64 per chunk of the contraction: 16 up to K = 6144, 8 above
// (MOA_OZAKI_CHUNK overrides, 1..16); an accumulator takes 16 / chunk slice
// pairs of a chunk, so it holds at most 1024 products of 2^14.  Measured on
// one box, effective FP64 TFLOP/s, chunk 8 / 16: n = 2048 35.7 / 37.1, 3072
// 46.1 / 47.9, 4096 59.6 / 61.6, 6144 69.0 / 70.3; at 8192 (power capped)
// chunk 8 72.3 against 69.7 for 16, since the shorter chunk's smaller working
// set cuts DRAM traffic and leaves more of the power budget to the SMs
// (earlier, with 7 slices: 16 51.5-52.0, 8 54.3-54.5, 4 52.0-52.4).
int ozaki_chunk(int64_t K) {
    static const int forced = [] {
        const char *e = std::getenv("MOA_OZAKI_CHUNK");
        const int v = e ? std::atoi(e) : 0;
        return (v < 1 || v > kChunkKBlocks) ? 0 : v;
    }();
    return forced ? forced : (K <= 6144 ? 16 : 8);
}

// Slices per operand for a contraction of length K (MOA_OZAKI_SLICES overrides, 4..10).
int ozaki_slices(int64_t K) {
    static const int forced = [] {  // read once, thread-safe
        const char *e = std::getenv("MOA_OZAKI_SLICES");
        const int v = e ? std::atoi(e) : 0;
        return (v < 4 || v > kMaxSlices) ? 0 : v;
    }();
    if (forced) return forced;
    return K <= 64 ? 10 : (K <= 256 ? 8 : (K < 4096 ? 7 : 6));
}

extern "C" int moa_ozaki_slices(int64_t K) { return K < 0 ? 0 : ozaki_slices(K); }

size_t ozaki_workspace_bytes(int64_t M, int64_t N, int64_t K) {
    return (size_t)ozaki_slices(K) * (size_t)(M * round8(K) + K * round8(N)) * 2 + (size_t)(M + N) * 8 +
           pair_ozaki_scratch_bytes() + 256;
}

moa_status tc_inner_ozaki(const double *A, const double *B, double *D, int64_t M, int64_t N, int64_t K,
                          cudaStream_t s) {
    // the int32 sum of one weight class (at most S pairs of K digit products
    // of magnitude at most 2^14) must stay below 2^31
    if ((double)ozaki_slices(K) * (double)K * 16384.0 >= 2147483648.0) return MOA_ERR_UNSUPPORTED;
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
        row_max_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(A, M, K, rmax, cmax, N);
        const int64_t gx = (N + 255) / 256;
        int64_t gy = (152 * 8 + gx - 1) / gx;
        if (gy > K) gy = K;
        const int64_t rpb = (K + gy - 1) / gy;
        gy = (K + rpb - 1) / rpb;
        col_max_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(B, K, N, rpb, cmax);
    }
    // digit planes
    if (!run_slices<true>(A, M, K, Kp, rmax, S, a, s) || !run_slices<false>(B, K, N, Np, cmax, S, b, s))
        return MOA_ERR_INTERNAL;
    if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    // accumulator units 2^-lsb with lsb = (S + 1) beta: every kept pair weight 2^(lsb - (s+u+2) beta) >= 1
    const int lsb = (S + 1) * kBeta;
    const int chunk = ozaki_chunk(K);
    return tc_gemm_ozaki(a, Kp, b, Np, S, kBeta, lsb, chunk, kChunkKBlocks / chunk, rmax, cmax, D, N, M, N, K, rs, s);
}

// The same product in two steps, for a caller that runs several blocks of
// result rows against one B (moa_inner_host): B's column maxima and digit
// planes once, then per block of rows A's maxima, planes and the GEMM.
size_t ozaki_b_bytes(int64_t K, int64_t N) {
    return (size_t)ozaki_slices(K) * (size_t)(K * round8(N)) * 2 + (size_t)N * 8 + 256;
}
size_t ozaki_rows_bytes(int64_t M, int64_t K) {
    return (size_t)ozaki_slices(K) * (size_t)(M * round8(K)) * 2 + (size_t)M * 8 + pair_ozaki_scratch_bytes() + 256;
}

moa_status ozaki_prepare_b(const double *B, int64_t K, int64_t N, void *ws, OzakiB *ob, cudaStream_t s) {
    if ((double)ozaki_slices(K) * (double)K * 16384.0 >= 2147483648.0) return MOA_ERR_UNSUPPORTED;
    const int S = ozaki_slices(K);
    const int64_t Np = round8(N);
    __nv_bfloat16 *b = (__nv_bfloat16 *)ws;
    uint64_t *cmax = (uint64_t *)(((uintptr_t)(b + (int64_t)S * K * Np) + 15) & ~(uintptr_t)15);
    if (launch_fill64(cmax, 0ull, N, s) != cudaSuccess) return MOA_ERR_CUDA;
    const int64_t gx = (N + 255) / 256;
    int64_t gy = (152 * 8 + gx - 1) / gx;
    if (gy > K) gy = K;
    const int64_t rpb = (K + gy - 1) / gy;
    gy = (K + rpb - 1) / rpb;
    col_max_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(B, K, N, rpb, cmax);
    if (!run_slices<false>(B, K, N, Np, cmax, S, b, s)) return MOA_ERR_INTERNAL;
    if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    *ob = OzakiB{b, cmax, S, K, N};
    return MOA_OK;
}

moa_status ozaki_rows(const double *A, int64_t M, const OzakiB &ob, double *D, void *ws, cudaStream_t s) {
    const int64_t K = ob.K, N = ob.N, Kp = round8(K);
    const int S = ob.S;
    __nv_bfloat16 *a = (__nv_bfloat16 *)ws;
    uint64_t *rmax = (uint64_t *)(((uintptr_t)(a + (int64_t)S * M * Kp) + 15) & ~(uintptr_t)15);
    void *rs = (void *)(((uintptr_t)(rmax + M) + 15) & ~(uintptr_t)15);
    const int64_t warps = M < 152 * 32 ? M : 152 * 32;
    row_max_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(A, M, K, rmax, nullptr, 0);
    if (!run_slices<true>(A, M, K, Kp, rmax, S, a, s)) return MOA_ERR_INTERNAL;
    if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    const int lsb = (S + 1) * kBeta;
    const int chunk = ozaki_chunk(K);
    return tc_gemm_ozaki(a, Kp, ob.planes, round8(N), S, kBeta, lsb, chunk, kChunkKBlocks / chunk, rmax, ob.cmax, D, N,
                         M, N, K, rs, s);
}

}  // namespace moa
