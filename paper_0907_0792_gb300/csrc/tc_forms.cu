// Precision forms of the (add, mul) inner product (Eq. 2, the matrix-
// multiply special case of Sec. I) built on the tcgen05 GEMM of tc_gemm.cu:
//   bf16 operands as given          -> one term, no pre-pass when aligned;
//   FP32 operands, MOA_FORM_BF16     -> round each operand to bf16 (RNE);
//   fp16 operands as given           -> the same kernels with fp16 operand
//       formats (one MMA takes one type for both operands);
//   FP32 operands, MOA_FORM_F16      -> round each operand to fp16 (RNE,
//       magnitudes beyond fp16's largest finite value 65504 held at it);
//   FP32 operands, MOA_FORM_BF16X3   -> split each operand exactly-ish into
//       x = hi + mid + lo (three bf16 values, each the RNE rounding of what
//       the previous ones left), then accumulate the six cross products of
//       total order <= 2 (hh, hm, mh, hl, lh, mm) in one FP32 accumulator
//       (Henry, Tang & Heinecke, "Leveraging the bfloat16 AI datatype for
//       higher-precision computations", ARITH 2019);
//   int32 operands (the integer (add, mul) of Sec. I) -> when every value
//       lies in [-128, 127], each is a bf16 exactly, every product and partial
//       sum is an integer of magnitude <= 2^14 K <= 2^24 for K <= 1024, so the
//       FP32 accumulation is exact in any order and the result equals the
//       int32 definition bit for bit (no sum reaches the wrap-around).
// The pre-pass is memory bound: one read of the FP32 operand, one write of
// each bf16 plane, rows padded to a multiple of 8 elements (16 bytes) so the
// planes meet the TMA stride rule.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "tc.h"

namespace moa {

moa_status tc_gemm_planes(const __nv_bfloat16 *A, int64_t lda, int planesA, const __nv_bfloat16 *B, int64_t ldb,
                          int planesB, int n_terms, const int *term_a, const int *term_b, float *D, int64_t ldd,
                          int64_t M, int64_t N, int64_t K, bool promote, cudaStream_t s, bool i32_out = false,
                          bool fp16 = false);

namespace {

template <typename Tin> MOA_DEV float to_f32(Tin x) { return (float)x; }
template <> MOA_DEV float to_f32<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

// X: rows x cols (row stride cols); out: NPL planes of rows x colsp, plane
// stride plane_elems; columns cols..colsp-1 are zero.  Eight consecutive
// columns per thread (colsp is a multiple of 8, so every plane row starts on
// a 16-byte boundary): two 16-byte loads when the rows allow it (VEC: float
// rows, cols % 4 == 0, 16-byte aligned; each 4-column half is then wholly
// inside the row or wholly in its padding) and one 16-byte store per plane.
template <typename Tin, int NPL, bool VEC>
__global__ void __launch_bounds__(256) split_planes(const Tin *__restrict__ X, int64_t rows, int64_t cols, int64_t colsp,
                                                     __nv_bfloat16 *__restrict__ out, int64_t plane_elems) {
    const int64_t groups = colsp / 8;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const Tin *src = X + r * cols;
        __nv_bfloat16 *dst = out + r * colsp;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c = 8 * g;
            float x[8];
            if constexpr (VEC) {
                const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float4 v0 = c < cols ? __ldg(reinterpret_cast<const float4 *>(src + c)) : z;
                const float4 v1 = c + 4 < cols ? __ldg(reinterpret_cast<const float4 *>(src + c + 4)) : z;
                x[0] = v0.x, x[1] = v0.y, x[2] = v0.z, x[3] = v0.w, x[4] = v1.x, x[5] = v1.y, x[6] = v1.z, x[7] = v1.w;
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) x[t] = c + t < cols ? to_f32(src[c + t]) : 0.0f;
            }
            __align__(16) __nv_bfloat16 pl[NPL][8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const __nv_bfloat16 hi = __float2bfloat16_rn(x[t]);
                pl[0][t] = hi;
                if constexpr (NPL > 1) {
                    const float r1 = __fsub_rn(x[t], __bfloat162float(hi));  // exact
                    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
                    pl[1][t] = mid;
                    if constexpr (NPL > 2) pl[2][t] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(mid)));
                }
            }
#pragma unroll
            for (int q = 0; q < NPL; ++q)
                *reinterpret_cast<uint4 *>(dst + q * plane_elems + c) = *reinterpret_cast<const uint4 *>(pl[q]);
        }
    }
}

int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// int32 X (rows x cols) -> bf16 rows x colsp, zero columns past cols; sets
// *out_of_range when a value lies outside [-128, 127].  V consecutive
// columns per thread (V = 4 needs cols % 4 == 0 and a 16-byte aligned X).
template <int V>
__global__ void __launch_bounds__(256) i8range_to_bf16(const int32_t *__restrict__ X, int64_t rows, int64_t cols,
                                                        int64_t colsp, __nv_bfloat16 *__restrict__ out,
                                                        uint32_t *out_of_range) {
    bool bad = false;
    const int64_t groups = colsp / V, total = rows * groups;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / groups, c = (idx - r * groups) * V;
        int32_t x[V];
        if constexpr (V == 4) {
            const int4 v = c < cols ? __ldg(reinterpret_cast<const int4 *>(X + r * cols + c)) : make_int4(0, 0, 0, 0);
            x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
        } else {
            x[0] = c < cols ? __ldg(X + r * cols + c) : 0;
        }
        __align__(8) __nv_bfloat16 y[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            bad |= (x[j] < -128) | (x[j] > 127);
            y[j] = __float2bfloat16_rn((float)x[j]);
        }
        if constexpr (V == 4)
            *reinterpret_cast<uint2 *>(out + r * colsp + c) = *reinterpret_cast<const uint2 *>(y);
        else
            out[r * colsp + c] = y[0];
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(out_of_range, 1u);
}

cudaError_t run_i8range(const int32_t *X, int64_t rows, int64_t cols, int64_t colsp, __nv_bfloat16 *out, uint32_t *flag,
                        cudaStream_t s) {
    const bool vec = cols % 4 == 0 && (uintptr_t)X % 16 == 0;  // colsp is a multiple of 8
    const int64_t total = rows * colsp / (vec ? 4 : 1);
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (vec)
        i8range_to_bf16<4><<<grid, 256, 0, s>>>(X, rows, cols, colsp, out, flag);
    else
        i8range_to_bf16<1><<<grid, 256, 0, s>>>(X, rows, cols, colsp, out, flag);
    return cudaGetLastError();
}

template <typename Tin, int NPL>
cudaError_t run_split(const Tin *X, int64_t rows, int64_t cols, int64_t colsp, __nv_bfloat16 *out, cudaStream_t s) {
    if (rows == 0 || colsp == 0) return cudaSuccess;
    const int64_t groups = colsp / 8;
    const int64_t gx = groups >= 256 * 4 ? 4 : (groups + 255) / 256;
    int64_t gy = rows < 2048 ? rows : 2048;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    bool vec = false;
    if constexpr (std::is_same<Tin, float>::value) {
        vec = cols % 4 == 0 && (uintptr_t)X % 16 == 0;
        if (vec) split_planes<Tin, NPL, true><<<grid, 256, 0, s>>>(X, rows, cols, colsp, out, rows * colsp);
    }
    if (!vec) split_planes<Tin, NPL, false><<<grid, 256, 0, s>>>(X, rows, cols, colsp, out, rows * colsp);
    return cudaGetLastError();
}

// X (rows x cols, float or fp16) -> fp16 rows x colsp (zero columns past
// cols): RNE rounding of FP32 values with the magnitude held at 65504, or a
// copy of fp16 values.  Eight consecutive columns per thread and one 16-byte
// store (colsp is a multiple of 8); two 16-byte loads when the float rows
// allow it (VEC: cols % 4 == 0, 16-byte aligned X).
template <typename Tin, bool VEC>
__global__ void __launch_bounds__(256) to_f16_rows(const Tin *__restrict__ X, int64_t rows, int64_t cols, int64_t colsp,
                                                    __half *__restrict__ out) {
    const int64_t groups = colsp / 8;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const Tin *src = X + r * cols;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c = 8 * g;
            __align__(16) __half y[8];
            if constexpr (VEC) {  // each 4-column half is all in or all out
                const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float4 v0 = c < cols ? __ldg(reinterpret_cast<const float4 *>(src + c)) : z;
                const float4 v1 = c + 4 < cols ? __ldg(reinterpret_cast<const float4 *>(src + c + 4)) : z;
                const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int t = 0; t < 8; ++t) y[t] = __float2half_rn(fminf(fmaxf(x[t], -65504.0f), 65504.0f));
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if constexpr (std::is_same<Tin, float>::value) {
                        const float x = c + t < cols ? src[c + t] : 0.0f;
                        y[t] = __float2half_rn(fminf(fmaxf(x, -65504.0f), 65504.0f));
                    } else {
                        y[t] = c + t < cols ? src[c + t] : __ushort_as_half((unsigned short)0);
                    }
                }
            }
            *reinterpret_cast<uint4 *>(out + r * colsp + c) = *reinterpret_cast<const uint4 *>(y);
        }
    }
}

template <typename Tin>
cudaError_t run_to_f16(const Tin *X, int64_t rows, int64_t cols, int64_t colsp, __half *out, cudaStream_t s) {
    if (rows == 0 || colsp == 0) return cudaSuccess;
    const int64_t groups = colsp / 8;
    const int64_t gx = groups >= 256 * 4 ? 4 : (groups + 255) / 256;
    const dim3 grid((unsigned)gx, (unsigned)(rows < 2048 ? rows : 2048));
    if (std::is_same<Tin, float>::value && cols % 4 == 0 && (uintptr_t)X % 16 == 0)
        to_f16_rows<Tin, std::is_same<Tin, float>::value><<<grid, 256, 0, s>>>(X, rows, cols, colsp, out);
    else
        to_f16_rows<Tin, false><<<grid, 256, 0, s>>>(X, rows, cols, colsp, out);
    return cudaGetLastError();
}

}  // namespace

moa_status tc_inner_f16(const __half *A, const __half *B, float *D, int64_t M, int64_t N, int64_t K, cudaStream_t s) {
    const int ta[1] = {0}, tb[1] = {0};
    auto bf = [](const __half *p) { return reinterpret_cast<const __nv_bfloat16 *>(p); };  // 2-byte planes, fp16 bits
    if ((uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0 && K % 8 == 0 && N % 8 == 0)
        return tc_gemm_planes(bf(A), K, 1, bf(B), N, 1, 1, ta, tb, D, N, M, N, K, false, s, false, true);
    // copy into 16-byte-aligned, padded rows first
    const int64_t Kp = round8(K), Np = round8(N);
    moa_status st;
    __half *ws = (__half *)workspace_get(s, (size_t)(M * Kp + K * Np) * 2, &st);
    if (st != MOA_OK) return st;
    __half *a = ws, *b = ws + M * Kp;
    if (run_to_f16(A, M, K, Kp, a, s) != cudaSuccess || run_to_f16(B, K, N, Np, b, s) != cudaSuccess) return MOA_ERR_CUDA;
    return tc_gemm_planes(bf(a), Kp, 1, bf(b), Np, 1, 1, ta, tb, D, N, M, N, K, false, s, false, true);
}

moa_status tc_inner_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *D, int64_t M, int64_t N, int64_t K,
                         cudaStream_t s) {
    const int ta[1] = {0}, tb[1] = {0};
    if ((uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0 && K % 8 == 0 && N % 8 == 0)
        return tc_gemm_planes(A, K, 1, B, N, 1, 1, ta, tb, D, N, M, N, K, false, s);
    // copy into 16-byte-aligned, padded rows first
    const int64_t Kp = round8(K), Np = round8(N);
    moa_status st;
    __nv_bfloat16 *ws = (__nv_bfloat16 *)workspace_get(s, (size_t)(M * Kp + K * Np) * 2, &st);
    if (st != MOA_OK) return st;
    __nv_bfloat16 *a = ws, *b = ws + M * Kp;
    if (run_split<__nv_bfloat16, 1>(A, M, K, Kp, a, s) != cudaSuccess) return MOA_ERR_CUDA;
    if (run_split<__nv_bfloat16, 1>(B, K, N, Np, b, s) != cudaSuccess) return MOA_ERR_CUDA;
    return tc_gemm_planes(a, Kp, 1, b, Np, 1, 1, ta, tb, D, N, M, N, K, false, s);
}

moa_status tc_inner_f32(moa_form form, const float *A, const float *B, float *D, int64_t M, int64_t N, int64_t K,
                        cudaStream_t s) {
    if (form == MOA_FORM_FP8_T128) return tc_inner_fp8(A, B, D, M, N, K, s);
    if (form == MOA_FORM_F16) {
        const int64_t Kp = round8(K), Np = round8(N);
        moa_status st;
        __half *ws = (__half *)workspace_get(s, (size_t)(M * Kp + K * Np) * 2, &st);
        if (st != MOA_OK) return st;
        __half *a = ws, *b = ws + M * Kp;
        if (run_to_f16(A, M, K, Kp, a, s) != cudaSuccess || run_to_f16(B, K, N, Np, b, s) != cudaSuccess)
            return MOA_ERR_CUDA;
        const int ta[1] = {0}, tb[1] = {0};
        return tc_gemm_planes(reinterpret_cast<const __nv_bfloat16 *>(a), Kp, 1, reinterpret_cast<const __nv_bfloat16 *>(b),
                              Np, 1, 1, ta, tb, D, N, M, N, K, false, s, false, true);
    }
    if (form != MOA_FORM_BF16 && form != MOA_FORM_BF16X3) return MOA_ERR_UNSUPPORTED;
    const int npl = form == MOA_FORM_BF16 ? 1 : 3;
    const int64_t Kp = round8(K), Np = round8(N);
    moa_status st;
    __nv_bfloat16 *ws = (__nv_bfloat16 *)workspace_get(s, (size_t)npl * (M * Kp + K * Np) * 2, &st);
    if (st != MOA_OK) return st;
    __nv_bfloat16 *a = ws, *b = ws + npl * M * Kp;
    cudaError_t e1, e2;
    if (npl == 1) {
        e1 = run_split<float, 1>(A, M, K, Kp, a, s);
        e2 = run_split<float, 1>(B, K, N, Np, b, s);
    } else {
        e1 = run_split<float, 3>(A, M, K, Kp, a, s);
        e2 = run_split<float, 3>(B, K, N, Np, b, s);
    }
    if (e1 != cudaSuccess || e2 != cudaSuccess) return MOA_ERR_CUDA;
    if (npl == 1) {
        const int ta[1] = {0}, tb[1] = {0};
        return tc_gemm_planes(a, Kp, 1, b, Np, 1, 1, ta, tb, D, N, M, N, K, false, s);
    }
    // planes 0 = hi, 1 = mid, 2 = lo; the small products go first in each
    // k-block so they accumulate at their own magnitude, hi*hi last
    const int ta[6] = {1, 0, 2, 0, 1, 0};
    const int tb[6] = {1, 2, 0, 1, 0, 0};
    return tc_gemm_planes(a, Kp, 3, b, Np, 3, 6, ta, tb, D, N, M, N, K, true, s);
}

size_t tc_bf16x3_scratch_bytes(int64_t M, int64_t N, int64_t K) {
    return (size_t)3 * (size_t)(M * round8(K) + K * round8(N)) * 2;
}

moa_status tc_inner_bf16x3_scratch(const float *A, const float *B, float *D, int64_t M, int64_t N, int64_t K,
                                   void *scratch, cudaStream_t s) {
    const int64_t Kp = round8(K), Np = round8(N);
    __nv_bfloat16 *a = (__nv_bfloat16 *)scratch, *b = a + 3 * M * Kp;
    if (run_split<float, 3>(A, M, K, Kp, a, s) != cudaSuccess) return MOA_ERR_CUDA;
    if (run_split<float, 3>(B, K, N, Np, b, s) != cudaSuccess) return MOA_ERR_CUDA;
    const int ta[6] = {1, 0, 2, 0, 1, 0};
    const int tb[6] = {1, 2, 0, 1, 0, 0};
    return tc_gemm_planes(a, Kp, 3, b, Np, 3, 6, ta, tb, D, N, M, N, K, true, s);
}

bool i32_tc_applies(int64_t M, int64_t N, int64_t K) {
    return M > 128 && N > 128 && K >= 1 && K <= 1024 && M < (1ll << 31) && N < (1ll << 31) && pair_mma_enabled();
}

size_t i32_tc_workspace_bytes(int64_t M, int64_t N, int64_t K) {
    return 16 + (size_t)(M * round8(K) + K * round8(N)) * 2;
}

// The range flag sits at the start of the workspace: the CUDA-core kernel
// launched after the GEMM recomputes D only when the flag is set.
moa_status tc_inner_i32(const int32_t *A, const int32_t *B, int32_t *D, int64_t M, int64_t N, int64_t K, void *ws,
                        cudaStream_t s) {
    const int64_t Kp = round8(K), Np = round8(N);
    uint32_t *flag = (uint32_t *)ws;
    __nv_bfloat16 *a = (__nv_bfloat16 *)((uint8_t *)ws + 16), *b = a + M * Kp;
    if (cudaMemsetAsync(flag, 0, sizeof(uint32_t), s) != cudaSuccess) return MOA_ERR_CUDA;
    if (run_i8range(A, M, K, Kp, a, flag, s) != cudaSuccess) return MOA_ERR_CUDA;
    if (run_i8range(B, K, N, Np, b, flag, s) != cudaSuccess) return MOA_ERR_CUDA;
    const int ta[1] = {0}, tb[1] = {0};
    const moa_status st = tc_gemm_planes(a, Kp, 1, b, Np, 1, 1, ta, tb, (float *)D, N, M, N, K, false, s, true);
    if (st != MOA_OK) return st;
    return launch_semiring(SR_I32_PLUS_TIMES, A, B, D, M, N, K, s, flag) == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
}

}  // namespace moa
