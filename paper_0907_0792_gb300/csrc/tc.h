// Host interface of the tensor-core (tcgen05) forms of the (add, mul) inner
// product, Eq. (2) with * = multiply: the matrix-multiply special case that
// Sec. I singles out.  All take the psi-flattened problem D (M x N) =
// A (M x K) . B (K x N), row-major, and enqueue on `stream`.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda.h>

#include "moa.h"

namespace moa {

// 3-D tensor map [planes][rows][inner] with the given byte strides, swizzled
// boxes of box_inner x box_rows x box_planes (TMA rules: base 16-byte
// aligned, strides multiples of 16 bytes).  False if encoding failed.
bool make_tmap(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint64_t planes, uint64_t row_bytes,
               uint64_t plane_bytes, uint32_t box_inner, uint32_t box_rows,
               CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
               CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B, uint32_t box_planes = 1);

// bf16 operands as given, FP32 out.
moa_status tc_inner_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *D, int64_t M, int64_t N, int64_t K,
                         cudaStream_t stream);
// fp16 operands as given, FP32 out (the same kernels with fp16 operand formats).
moa_status tc_inner_f16(const __half *A, const __half *B, float *D, int64_t M, int64_t N, int64_t K,
                        cudaStream_t stream);
// e4m3 operands as given, FP32 out: unit scales, or the caller's
// power-of-two scales scale_a [M][ceil(K/128)], scale_b [ceil(K/128)][ceil(N/128)].
moa_status tc_inner_e4m3(const uint8_t *A, const uint8_t *B, float *D, int64_t M, int64_t N, int64_t K,
                         cudaStream_t stream, const float *scale_a = nullptr, const float *scale_b = nullptr);
// FP32 operands, FP32 out: MOA_FORM_BF16, MOA_FORM_F16, MOA_FORM_BF16X3 or MOA_FORM_FP8_T128.
moa_status tc_inner_f32(moa_form form, const float *A, const float *B, float *D, int64_t M, int64_t N, int64_t K,
                        cudaStream_t stream);
// FP32 operands, FP32 out, e4m3 with per-128 power-of-two block scales.
moa_status tc_inner_fp8(const float *A, const float *B, float *D, int64_t M, int64_t N, int64_t K, cudaStream_t stream);
// ozaki_plan.cu — the Ozaki form's slices per operand for a contraction of
// length K, k-blocks of 64 per exact chunk, and slice pairs per accumulator.
int ozaki_slices(int64_t K);
int ozaki_chunk(int64_t K);
int ozaki_acc_pairs(int chunk);

// FP64 operands, FP64 out, Ozaki-sliced on bf16 tensor cores.
moa_status tc_inner_ozaki(const double *A, const double *B, double *D, int64_t M, int64_t N, int64_t K,
                          cudaStream_t stream);
// The Ozaki form in two steps (several blocks of result rows against one B):
// B's column maxima and digit planes into ws (ozaki_b_bytes), then per block
// of rows A's maxima, planes and the GEMM with scratch ws (ozaki_rows_bytes).
struct OzakiB {
    const __nv_bfloat16 *planes;
    const uint64_t *cmax;
    int S;
    int64_t K, N;
};
size_t ozaki_b_bytes(int64_t K, int64_t N);
size_t ozaki_rows_bytes(int64_t M, int64_t K);
moa_status ozaki_prepare_b(const double *B, int64_t K, int64_t N, void *ws, OzakiB *ob, cudaStream_t stream);
moa_status ozaki_rows(const double *A, int64_t M, const OzakiB &ob, double *D, void *ws, cudaStream_t stream);
// int32 operands, int32 out, on bf16 tensor cores when every operand value
// lies in [-128, 127] (else on CUDA cores): see tc_forms.cu.
bool i32_tc_applies(int64_t M, int64_t N, int64_t K);
size_t i32_tc_workspace_bytes(int64_t M, int64_t N, int64_t K);
moa_status tc_inner_i32(const int32_t *A, const int32_t *B, int32_t *D, int64_t M, int64_t N, int64_t K, void *ws,
                        cudaStream_t stream);
// Split-BF16x3 with caller-provided scratch of tc_bf16x3_scratch_bytes()
// bytes (16-byte aligned); allocates nothing.
size_t tc_bf16x3_scratch_bytes(int64_t M, int64_t N, int64_t K);
moa_status tc_inner_bf16x3_scratch(const float *A, const float *B, float *D, int64_t M, int64_t N, int64_t K,
                                   void *scratch, cudaStream_t stream);
// Pair-MMA GEMM (tc_gemm_pair.cu): 256 x 256 tiles on CTA pairs, the same
// tensor maps and term encoding as the single-CTA kernel (A boxes 64 x 128,
// B boxes 64 x 64); promote = FP32 register accumulation per k-block;
// i32_out = D is int32, each accumulator rounded to the nearest integer
// (store mode only).  MOA_PAIR_MMA=0 turns the pair path off.
bool pair_mma_enabled();
cudaError_t tc_gemm_pair_launch(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, int n_terms,
                                uint32_t term_a, uint32_t term_b, float *D, int64_t ldd, bool promote,
                                cudaStream_t stream, bool i32_out = false, bool fp16 = false);
// FP8 (e4m3) pair GEMM with block-scaled MMAs: A8 [M][lda] and B
// transposed, Bt8 [N][ldb] (both K-major, lda and ldb multiples of 16,
// 16-byte aligned).  Scale factors as UE8M0 bytes, each repeated in the four
// bytes of a word, in the TMEM-word order of the kernel (k-block kb = k / 128):
//   sfa [ceil(M/128)][kb][128]: word 4 l + c = row 128 rb + 32 c + l;
//   sfb [ceil(N/T)][kb][256] with T = pair_fp8_tile_n(): word 128 h + 4 l + c
//   = column T tn + 32 (4 h + c) + l (columns at or past T or N: any value).
int pair_fp8_tile_n();
// With `bits_out` (N a multiple of 32) the result is written as the packed
// bit stream of [D > 0] instead of D (the exact-count (or, and) form).
cudaError_t tc_gemm_pair_fp8_launch(const uint8_t *A8, int64_t lda, const uint8_t *Bt8, int64_t ldb, int M, int N,
                                    int K, const uint32_t *sfa, const uint32_t *sfb, float *D, int64_t ldd,
                                    cudaStream_t stream, uint32_t *bits_out = nullptr);
// Ozaki slice-pair pair GEMM (same tensor maps and arguments as the
// single-CTA tc_gemm_ozaki; 256 x 256 tiles on CTA pairs).
// `scratch`: pair_ozaki_scratch_bytes() of device memory for the running
// sums (16-byte aligned).
size_t pair_ozaki_scratch_bytes();
cudaError_t tc_gemm_pair_ozaki_launch(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, int S, int beta,
                                      int lsb, int chunk_kblocks, int acc_pairs, const uint64_t *row_max,
                                      const uint64_t *col_max, double *D, int64_t ldd, void *scratch,
                                      cudaStream_t stream);
cudaError_t pair_read_and_clear_status(uint32_t *flags);
// Launch the bounded-wait self-test (a wait that can only time out).
cudaError_t tc_wait_probe(uint64_t limit_ns, cudaStream_t stream);
// Read and clear the status word of the tensor-core kernels (bounded waits).
cudaError_t tc_read_and_clear_status(uint32_t *flags);

}  // namespace moa
