// Generalized outer product, Eq. (1) (Sec. I):
//   C_{i.., j..} = A_{i..} op B_{j..},  rho C = rho A ++ rho B.
// Flattened by psi to C[i, j] = A[i] op B[j] with i < M = |A|, j < N = |B|,
// C row-major M x N.  The kernel is bound by HBM writes (|C| elements written,
// |A| + |B| read), so the design is about the store stream:
//  - each thread owns one 16-byte column vector of C and keeps the matching
//    B values in registers for every row it writes;
//  - A[i] is one broadcast load per row;
//  - stores are 128-bit streaming stores (st.global.cs: C is written once
//    and not re-read, so it should not displace other lines in L2);
//  - the grid is a multiple of the SM count, each block striding over rows;
//  - bf16 / bf16 -> bf16 multiplies by the correctly rounded FP32 reciprocal
//    of each B element (taken once per column) instead of dividing.  The
//    result is the same bf16: an 8-bit significand over an 8-bit significand
//    is never an odd multiple of half a bf16 unit (the odd part of m * B_sig,
//    m >= 257 odd, exceeds any 8-bit odd part), so the exact quotient lies at
//    least 2^-17 (relative) from every bf16 rounding midpoint, while both
//    RN(a / b) and RN(a * RN(1 / b)) stay within 2^-22 of it.  Below 2^-126
//    a quotient is either at least 2^-143 from every midpoint (the two
//    roundings err by at most 2^-149) or exactly on one, a multiple of
//    2^-149 that both roundings return unchanged (the reciprocal's error
//    moves it by less than 2^-150).  Columns whose reciprocal is neither a
//    normal FP32 number nor exact (|b| < 2^-126 or 2^126 < |b| < inf)
//    divide.
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace moa {
namespace {

template <typename T> struct Compute { using type = T; };
template <> struct Compute<__nv_bfloat16> { using type = float; };

template <typename Tin> MOA_DEV typename Compute<Tin>::type widen(Tin x) { return x; }
template <> MOA_DEV float widen<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename Tout, typename Tc> MOA_DEV Tout narrow(Tc x) { return (Tout)x; }
template <> MOA_DEV __nv_bfloat16 narrow<__nv_bfloat16, float>(float x) { return __float2bfloat16_rn(x); }

template <int OP, typename Tc> MOA_DEV Tc apply(Tc a, Tc b) { return op_apply(OP, a, b); }

template <int OP, typename Tin, typename Tout>
constexpr bool kRcpDiv = OP == MOA_OP_DIV && std::is_same<Tin, __nv_bfloat16>::value &&
                         std::is_same<Tout, __nv_bfloat16>::value;

// 1 / b is a normal FP32 number, or b is 0, inf or NaN (exact specials).
MOA_DEV bool rcp_usable(float b) {
    const float m = fabsf(b);
    return !(m > 0.0f && m < 0x1p-126f) && !(m > 0x1p126f && m <= 3.4028234663852886e38f);
}

// One 16-byte vector of output elements.
template <typename Tout> struct alignas(16) Vec16 {
    static constexpr int n = 16 / sizeof(Tout);
    Tout v[n];
};

template <typename Tout> MOA_DEV void store_cs(Tout *dst, const Vec16<Tout> &x) {
    const uint4 u = *reinterpret_cast<const uint4 *>(&x);
    __stcs(reinterpret_cast<uint4 *>(dst), u);
}

constexpr int kThreads = 256;

// Row path: N % VEC == 0 and C 16-byte aligned, so every row starts on a
// vector boundary.  vpr = N / VEC vectors per row; tpr = threads per row.
template <int OP, typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads) outer_rows(const Tin *__restrict__ A, const Tin *__restrict__ B,
                                                       Tout *__restrict__ C, int64_t M, int64_t N, int64_t vpr,
                                                       int tpr, int rows_per_iter) {
    using Tc = typename Compute<Tin>::type;
    constexpr int VEC = Vec16<Tout>::n;
    const int t = threadIdx.x;
    const int64_t cv = (int64_t)blockIdx.x * tpr + (t % tpr);  // column vector owned by this thread
    const int ro = t / tpr;                                     // row offset inside one iteration
    if (ro >= rows_per_iter || cv >= vpr) return;
    Tc b[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) b[k] = widen(B[cv * VEC + k]);
    [[maybe_unused]] float rb[VEC];
    [[maybe_unused]] bool rcp_all = true;
    if constexpr (kRcpDiv<OP, Tin, Tout>) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            rb[k] = __frcp_rn(b[k]);
            rcp_all &= rcp_usable(b[k]);
        }
    }
    const int64_t step = (int64_t)gridDim.y * rows_per_iter;
    for (int64_t r = (int64_t)blockIdx.y * rows_per_iter + ro; r < M; r += step) {
        const Tc a = widen(__ldg(A + r));
        Vec16<Tout> o;
        if constexpr (kRcpDiv<OP, Tin, Tout>) {
            if (rcp_all) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) o.v[k] = narrow<Tout>(__fmul_rn(a, rb[k]));
            } else {
#pragma unroll
                for (int k = 0; k < VEC; ++k) o.v[k] = narrow<Tout>(apply<OP>(a, b[k]));
            }
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) o.v[k] = narrow<Tout>(apply<OP>(a, b[k]));
        }
        store_cs(C + r * N + cv * VEC, o);
    }
}

// General path: any N, any alignment; one element per iteration.
template <int OP, typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads) outer_flat(const Tin *__restrict__ A, const Tin *__restrict__ B,
                                                       Tout *__restrict__ C, int64_t M, int64_t N) {
    using Tc = typename Compute<Tin>::type;
    const int64_t total = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N;
        C[e] = narrow<Tout>(apply<OP>(widen(A[i]), widen(B[j])));
    }
}

int sm_count() {
    static const int n = [] {  // read once, thread-safe
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

template <int OP, typename Tin, typename Tout>
cudaError_t run(const void *A, const void *B, void *C, int64_t M, int64_t N, cudaStream_t s) {
    constexpr int VEC = Vec16<Tout>::n;
    const int sms = sm_count();
    const bool aligned = ((uintptr_t)C % 16 == 0) && (N % VEC == 0);
    if (aligned && N / VEC >= 1) {
        const int64_t vpr = N / VEC;
        const int tpr = (int)(vpr < kThreads ? vpr : kThreads);
        const int rows_per_iter = kThreads / tpr;
        const int64_t gx = (vpr + tpr - 1) / tpr;
        const int64_t row_iters = (M + rows_per_iter - 1) / rows_per_iter;
        int64_t gy = ((int64_t)sms * 8 + gx - 1) / gx;  // about 8 blocks per SM in total
        if (gy > row_iters) gy = row_iters;
        if (gy > 65535) gy = 65535;
        if (gx > 0x7fffffff) return cudaErrorInvalidValue;
        outer_rows<OP, Tin, Tout><<<dim3((unsigned)gx, (unsigned)gy), kThreads, 0, s>>>(
            (const Tin *)A, (const Tin *)B, (Tout *)C, M, N, vpr, tpr, rows_per_iter);
    } else {
        int64_t blocks = (M * N + kThreads - 1) / kThreads;
        if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
        outer_flat<OP, Tin, Tout><<<(unsigned)blocks, kThreads, 0, s>>>((const Tin *)A, (const Tin *)B, (Tout *)C, M, N);
    }
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t run_op(int op, const void *A, const void *B, void *C, int64_t M, int64_t N, cudaStream_t s) {
    switch (op) {
    case MOA_OP_ADD: return run<MOA_OP_ADD, Tin, Tout>(A, B, C, M, N, s);
    case MOA_OP_SUB: return run<MOA_OP_SUB, Tin, Tout>(A, B, C, M, N, s);
    case MOA_OP_MUL: return run<MOA_OP_MUL, Tin, Tout>(A, B, C, M, N, s);
    case MOA_OP_DIV: return run<MOA_OP_DIV, Tin, Tout>(A, B, C, M, N, s);
    case MOA_OP_MIN: return run<MOA_OP_MIN, Tin, Tout>(A, B, C, M, N, s);
    case MOA_OP_MAX: return run<MOA_OP_MAX, Tin, Tout>(A, B, C, M, N, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
__global__ void fill_kernel(T *p, T v, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) p[e] = v;
}

}  // namespace

cudaError_t launch_outer(int op, moa_dtype dtype, moa_dtype out_dtype, const void *A, const void *B, void *C,
                         int64_t M, int64_t N, cudaStream_t s) {
    if (dtype == MOA_F64 && out_dtype == MOA_F64) return run_op<double, double>(op, A, B, C, M, N, s);
    if (dtype == MOA_F32 && out_dtype == MOA_F32) return run_op<float, float>(op, A, B, C, M, N, s);
    if (dtype == MOA_BF16 && out_dtype == MOA_BF16) return run_op<__nv_bfloat16, __nv_bfloat16>(op, A, B, C, M, N, s);
    if (dtype == MOA_BF16 && out_dtype == MOA_F32) return run_op<__nv_bfloat16, float>(op, A, B, C, M, N, s);
    if (dtype == MOA_I32 && out_dtype == MOA_I32) {
        switch (op) {
        case MOA_OP_ADD: return run<MOA_OP_ADD, int32_t, int32_t>(A, B, C, M, N, s);
        case MOA_OP_SUB: return run<MOA_OP_SUB, int32_t, int32_t>(A, B, C, M, N, s);
        case MOA_OP_MUL: return run<MOA_OP_MUL, int32_t, int32_t>(A, B, C, M, N, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fill32(uint32_t *p, uint32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    fill_kernel<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(p, v, n);
    return cudaGetLastError();
}

cudaError_t launch_fill64(uint64_t *p, uint64_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    fill_kernel<uint64_t><<<(unsigned)blocks, 256, 0, s>>>(p, v, n);
    return cudaGetLastError();
}

}  // namespace moa
