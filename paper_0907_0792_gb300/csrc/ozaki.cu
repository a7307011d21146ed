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

constexpr int kBeta = 8;

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

// B's column maxima into out (zeroed before): about eight blocks per SM
void launch_col_max(const double *B, int64_t K, int64_t N, uint64_t *out, cudaStream_t s) {
    const int64_t gx = (N + 255) / 256;
    int64_t gy = (152 * 8 + gx - 1) / gx;
    if (gy > K) gy = K;
    const int64_t rpb = (K + gy - 1) / gy;
    gy = (K + rpb - 1) / rpb;
    col_max_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(B, K, N, rpb, out);
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

// The same digits from one fixed-point word, for S <= 7 (the S beta
// fractional bits of |x| 2^-e fit 64 bits): F = floor(|x| 2^(S beta - e)).
// Adding 2^(beta-1) at every digit position below the top turns the balanced
// digits into the plain base-2^beta digits of the sum (each in [0, 2^beta)),
// the top one keeping the carry as is, so every digit is one byte of F + C.
// A byte b becomes an exact float as the bits of 2^23 + b, and the digit is
// then +-(2^23 + b - 2^23 - 2^(beta-1)) (+-(2^23 + b - 2^23) for the top),
// an exact FMA whose zero is +0 as in the integer form.
template <int S>
MOA_DEV void balanced_digits_f(uint64_t bits, int e, float (&f)[S]) {
    static_assert(S >= 2 && S <= 7, "the fractional bits must fit one 64-bit word");
    const int be = (int)((bits >> 52) & 0x7FF);
    const uint64_t mant = be ? ((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : (bits & 0xFFFFFFFFFFFFFull);
    const int t = (be ? be : 1) - 1075 - e + S * kBeta;
    const uint64_t F = t >= 0 ? (t >= 64 ? 0 : mant << t) : ((-t) >= 64 ? 0 : mant >> (-t));
    constexpr uint64_t C = 0x8080808080808080ull >> (8 * (9 - S));  // 2^(beta-1) in the S - 1 low digits
    const uint64_t G = F + C;
    const uint32_t w[2] = {(uint32_t)G, (uint32_t)(G >> 32)};
    const float sg = (bits >> 63) ? -1.0f : 1.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int p = S - 1 - s;  // byte of digit s
        const float m = __int_as_float((int)__byte_perm(w[p / 4], 0x4B000000u, 0x7540u | (unsigned)(p % 4)));
        const float off = s == 0 ? 8388608.0f : 8388608.0f + (float)(1 << (kBeta - 1));
        f[s] = fmaf(m, sg, -sg * off);
    }
}

MOA_DEV uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t w;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
    return w;
}

// The digit planes of four consecutive elements with scale exponents e[t],
// packed two bf16 digits to a word (column c0 + 2u in the low half of word u).
template <int S>
MOA_DEV void digits4(const double (&x)[4], const int (&e)[4], uint32_t (&pk)[S][2]) {
    if constexpr (S <= 7) {
        float f[4][S];
#pragma unroll
        for (int t = 0; t < 4; ++t) balanced_digits_f<S>((uint64_t)__double_as_longlong(x[t]), e[t], f[t]);
#pragma unroll
        for (int q = 0; q < S; ++q) {
            pk[q][0] = pack_bf16x2(f[0][q], f[1][q]);
            pk[q][1] = pack_bf16x2(f[2][q], f[3][q]);
        }
    } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint64_t b = (uint64_t)__double_as_longlong(x[t]);
            const int be = (int)((b >> 52) & 0x7FF);
            const uint64_t mant = be ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : (b & 0xFFFFFFFFFFFFFull);
            const int ex = (be ? be : 1) - 1075;
            int d[S];
            balanced_digits<S>(mant, ex, e[t], (b >> 63) != 0, d);
#pragma unroll
            for (int q = 0; q < S; ++q) {
                const uint32_t h = (uint32_t)__bfloat16_as_ushort(__int2bfloat16_rn(d[q]));
                if (t % 2 == 0) pk[q][t / 2] = h;
                else pk[q][t / 2] |= h << 16;
            }
        }
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
            int e[4];
#pragma unroll
            for (int t = 0; t < 4; ++t)
                e[t] = ROW_SCALE ? er : (c0 + t < cols ? ozaki::scale_exponent(__ldg(maxbits + c0 + t)) : 0);
            uint32_t pk[S][2];  // four bf16 digits per plane, packed in two words
            digits4<S>(x, e, pk);
            __nv_bfloat16 *dst = out + r * colsp + c0;
#pragma unroll
            for (int q = 0; q < S; ++q) *reinterpret_cast<uint2 *>(dst + q * plane) = make_uint2(pk[q][0], pk[q][1]);
        }
    }
}

// Rows of A short enough for the registers of TPR threads (colsp <= 32 TPR):
// each thread loads its kRowGroups groups of four columns of the row at once,
// the row's |A| maximum is reduced over the TPR threads (warp shuffles, then
// shared memory across the row's warps), and the digit planes are written
// from the same registers, so the row leaves DRAM once and no separate
// maximum pass runs.  The grid also zeroes the N column maxima that
// col_max_kernel combines into.  Rows are 16-byte aligned with cols % 4 == 0.
constexpr int kRowGroups = 8;

template <int TPR, int S>
__global__ void __launch_bounds__(256, 2) row_slice_kernel(const double *__restrict__ X, int64_t rows, int64_t cols,
                                                            int64_t colsp, uint64_t *__restrict__ rmax,
                                                            uint64_t *__restrict__ col_zero, int64_t ncz,
                                                            __nv_bfloat16 *__restrict__ out) {
    static_assert(TPR >= 32 && TPR <= 256 && (TPR & (TPR - 1)) == 0, "a power of two from a warp to the CTA");
    constexpr int RPC = 256 / TPR, WPR = TPR / 32;
    __shared__ uint64_t red[8];
    {
        const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
        for (int64_t j = tid; j < ncz; j += nthreads) col_zero[j] = 0;
    }
    const int sub = threadIdx.x / TPR, lt = threadIdx.x % TPR, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t groups = colsp / 4, plane = rows * colsp;
    for (int64_t r0 = (int64_t)blockIdx.x * RPC; r0 < rows; r0 += (int64_t)gridDim.x * RPC) {
        const int64_t r = r0 + sub;
        const bool live = r < rows;
        const double *src = X + r * cols;
        double x[kRowGroups][4];
#pragma unroll
        for (int i = 0; i < kRowGroups; ++i) {
            const int64_t c0 = 4 * (lt + (int64_t)i * TPR);
            if (live && c0 < cols) {
                const double2 v0 = __ldg(reinterpret_cast<const double2 *>(src + c0));
                const double2 v1 = __ldg(reinterpret_cast<const double2 *>(src + c0 + 2));
                x[i][0] = v0.x, x[i][1] = v0.y, x[i][2] = v1.x, x[i][3] = v1.y;
            } else {
                x[i][0] = x[i][1] = x[i][2] = x[i][3] = 0.0;
            }
        }
        uint64_t m = 0;
#pragma unroll
        for (int i = 0; i < kRowGroups; ++i)
#pragma unroll
            for (int t = 0; t < 4; ++t) m = max(m, mag_bits(x[i][t]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)m, o));
        if constexpr (WPR > 1) {
            if (lane == 0) red[warp] = m;
            __syncthreads();
            m = red[sub * WPR];
#pragma unroll
            for (int w = 1; w < WPR; ++w) m = max(m, red[sub * WPR + w]);
            __syncthreads();
        }
        if (!live) continue;
        if (lt == 0) rmax[r] = m;
        const int er = ozaki::scale_exponent(m);
        const int e[4] = {er, er, er, er};
        __nv_bfloat16 *dst = out + r * colsp;
#pragma unroll
        for (int i = 0; i < kRowGroups; ++i) {
            const int64_t g = lt + (int64_t)i * TPR;
            if (g >= groups) break;
            uint32_t pk[S][2];
            digits4<S>(x[i], e, pk);
#pragma unroll
            for (int q = 0; q < S; ++q)
                *reinterpret_cast<uint2 *>(dst + 4 * g + q * plane) = make_uint2(pk[q][0], pk[q][1]);
        }
    }
}

template <int TPR, int S>
void run_row_slices_t(const double *X, int64_t rows, int64_t cols, int64_t colsp, uint64_t *rmax, uint64_t *col_zero,
                      int64_t ncz, __nv_bfloat16 *out, cudaStream_t s) {
    constexpr int RPC = 256 / TPR;
    const int64_t ctas = (rows + RPC - 1) / RPC;
    const int64_t grid = ctas < 152 * 2 * 8 ? (ctas > 0 ? ctas : 1) : 152 * 2 * 8;
    row_slice_kernel<TPR, S><<<(unsigned)grid, 256, 0, s>>>(X, rows, cols, colsp, rmax, col_zero, ncz, out);
}

// The fused row pass where it applies (S of 6 or 7, rows that fit the
// registers, 16-byte rows); false leaves the two-pass form to the caller.
bool run_row_slices(const double *X, int64_t rows, int64_t cols, int64_t colsp, uint64_t *rmax, uint64_t *col_zero,
                    int64_t ncz, int S, __nv_bfloat16 *out, cudaStream_t s) {
    if ((S != 6 && S != 7) || cols % 4 != 0 || (uintptr_t)X % 16 != 0 || colsp > 32 * 256) return false;
    const int tpr = colsp <= 32 * 32 ? 32 : (colsp <= 32 * 64 ? 64 : (colsp <= 32 * 128 ? 128 : 256));
#define MOA_ROW_SLICES(T)                                                                                               \
    if (tpr == T) {                                                                                                     \
        if (S == 6) run_row_slices_t<T, 6>(X, rows, cols, colsp, rmax, col_zero, ncz, out, s);                          \
        else run_row_slices_t<T, 7>(X, rows, cols, colsp, rmax, col_zero, ncz, out, s);                                \
        return true;                                                                                                    \
    }
    MOA_ROW_SLICES(32)
    MOA_ROW_SLICES(64)
    MOA_ROW_SLICES(128)
    MOA_ROW_SLICES(256)
#undef MOA_ROW_SLICES
    return false;
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
    // A's row maxima and digit planes in one pass where the rows fit, else the maxima first
    const bool fused = run_row_slices(A, M, K, Kp, rmax, cmax, N, S, a, s);
    if (!fused) {
        int64_t warps = M < 152 * 32 ? M : 152 * 32;
        row_max_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(A, M, K, rmax, cmax, N);
    }
    // B's column maxima
    launch_col_max(B, K, N, cmax, s);
    // digit planes
    if ((!fused && !run_slices<true>(A, M, K, Kp, rmax, S, a, s)) || !run_slices<false>(B, K, N, Np, cmax, S, b, s))
        return MOA_ERR_INTERNAL;
    if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    // accumulator units 2^-lsb with lsb = (S + 1) beta: every kept pair weight 2^(lsb - (s+u+2) beta) >= 1
    const int lsb = (S + 1) * kBeta;
    const int chunk = ozaki_chunk(K);
    return tc_gemm_ozaki(a, Kp, b, Np, S, kBeta, lsb, chunk, ozaki_acc_pairs(chunk), rmax, cmax, D, N, M, N, K, rs, s);
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
    launch_col_max(B, K, N, cmax, s);
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
    if (!run_row_slices(A, M, K, Kp, rmax, nullptr, 0, S, a, s)) {
        const int64_t warps = M < 152 * 32 ? M : 152 * 32;
        row_max_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(A, M, K, rmax, nullptr, 0);
        if (!run_slices<true>(A, M, K, Kp, rmax, S, a, s)) return MOA_ERR_INTERNAL;
    }
    if (cudaGetLastError() != cudaSuccess) return MOA_ERR_CUDA;
    const int lsb = (S + 1) * kBeta;
    const int chunk = ozaki_chunk(K);
    return tc_gemm_ozaki(a, Kp, ob.planes, round8(N), S, kBeta, lsb, chunk, ozaki_acc_pairs(chunk), rmax, ob.cmax, D, N,
                         M, N, K, rs, s);
}

}  // namespace moa
