// Skinny (add, mul) inner product, Eq. (2) with * = multiply, for a result
// of M <= 8 rows: D (M x N) = A (M x K) . B (K x N) on the psi-flattened
// operands, FP64 or FP32.  This is the shape of the method's own
// measurement in Sec. IV (an m x 128 array times a 128 x n array, m <= 4, n
// up to 2^26): every element of B is used M times, so the work is a stream
// over B -- HBM-bound in FP32, and bound by the FP64 pipe in FP64 (this
// part issues only a few DFMA per clock per SM).
//
// One thread owns CW consecutive columns of D (a 16-byte vector of B per k
// when N and the pointers allow it, one column otherwise) and keeps the
// M x CW sums in registers; A is staged in shared memory 128 k at a time
// and read as a broadcast.  Each k step issues the B loads of 8 k ahead of
// their FMAs so that enough bytes are in flight to cover HBM latency.
// Every output is the left fold over k of fma(A[i][k], B[k][j], acc) from
// zero, i.e. the plain definition's summation order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace moa {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 128;  // k per staged chunk of A
constexpr int kAhead = 8;    // k steps whose B loads are issued together

template <typename T, int CW> struct Vec;
template <> struct Vec<double, 2> {
    using V = double2;
    static MOA_DEV void get(const V &v, double (&o)[2]) { o[0] = v.x, o[1] = v.y; }
    static MOA_DEV V make(const double (&o)[2]) { return make_double2(o[0], o[1]); }
};
template <> struct Vec<float, 4> {
    using V = float4;
    static MOA_DEV void get(const V &v, float (&o)[4]) { o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w; }
    static MOA_DEV V make(const float (&o)[4]) { return make_float4(o[0], o[1], o[2], o[3]); }
};

MOA_DEV double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
MOA_DEV float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Streaming (read-once) load of B.
template <typename V> MOA_DEV V ld_stream(const V *p) { return __ldcs(p); }

// MR rows of D; CW columns per thread (CW > 1: vector loads and stores).
template <typename T, int MR, int CW>
__global__ void __launch_bounds__(kThreads) skinny_kernel(const T *__restrict__ A, const T *__restrict__ B,
                                                          T *__restrict__ D, int64_t N, int K) {
    __shared__ T sA[MR][kChunk];
    const int64_t col = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * CW;
    const bool active = col < N;
    T acc[MR][CW];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int c = 0; c < CW; ++c) acc[i][c] = T(0);

    for (int k0 = 0; k0 < K; k0 += kChunk) {
        const int kc = min(kChunk, K - k0);
        __syncthreads();  // the previous chunk is no longer read
        for (int e = threadIdx.x; e < MR * kChunk; e += kThreads) {
            const int i = e / kChunk, k = e - i * kChunk;
            sA[i][k] = k < kc ? A[(int64_t)i * K + k0 + k] : T(0);
        }
        __syncthreads();
        if (!active) continue;
        const T *bcol = B + (int64_t)k0 * N + col;
        int k = 0;
        for (; k + kAhead <= kc; k += kAhead) {
            T b[kAhead][CW];
#pragma unroll
            for (int u = 0; u < kAhead; ++u) {
                if constexpr (CW > 1)
                    Vec<T, CW>::get(ld_stream(reinterpret_cast<const typename Vec<T, CW>::V *>(bcol + (int64_t)(k + u) * N)),
                                    b[u]);
                else
                    b[u][0] = __ldcs(bcol + (int64_t)(k + u) * N);
            }
#pragma unroll
            for (int u = 0; u < kAhead; ++u)
#pragma unroll
                for (int i = 0; i < MR; ++i) {
                    const T a = sA[i][k + u];
#pragma unroll
                    for (int c = 0; c < CW; ++c) acc[i][c] = fma_rn(a, b[u][c], acc[i][c]);
                }
        }
        for (; k < kc; ++k) {
            T b[CW];
            if constexpr (CW > 1)
                Vec<T, CW>::get(ld_stream(reinterpret_cast<const typename Vec<T, CW>::V *>(bcol + (int64_t)k * N)), b);
            else
                b[0] = __ldcs(bcol + (int64_t)k * N);
#pragma unroll
            for (int i = 0; i < MR; ++i) {
                const T a = sA[i][k];
#pragma unroll
                for (int c = 0; c < CW; ++c) acc[i][c] = fma_rn(a, b[c], acc[i][c]);
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int i = 0; i < MR; ++i) {
        T *drow = D + (int64_t)i * N + col;
        if constexpr (CW > 1)
            __stcs(reinterpret_cast<typename Vec<T, CW>::V *>(drow), Vec<T, CW>::make(acc[i]));
        else
            __stcs(drow, acc[i][0]);
    }
}

template <typename T, int MR>
cudaError_t launch_mr(const T *A, const T *B, T *D, int64_t N, int K, cudaStream_t s) {
    constexpr int CWV = 16 / sizeof(T);
    const bool vec = N % CWV == 0 && (uintptr_t)B % 16 == 0 && (uintptr_t)D % 16 == 0;
    if (vec) {
        const int64_t blocks = (N / CWV + kThreads - 1) / kThreads;
        skinny_kernel<T, MR, CWV><<<(unsigned)blocks, kThreads, 0, s>>>(A, B, D, N, K);
    } else {
        const int64_t blocks = (N + kThreads - 1) / kThreads;
        skinny_kernel<T, MR, 1><<<(unsigned)blocks, kThreads, 0, s>>>(A, B, D, N, K);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_skinny_t(const T *A, const T *B, T *D, int64_t M, int64_t N, int64_t K, cudaStream_t s) {
    const int k = (int)K;
    switch (M) {
    case 1: return launch_mr<T, 1>(A, B, D, N, k, s);
    case 2: return launch_mr<T, 2>(A, B, D, N, k, s);
    case 3: return launch_mr<T, 3>(A, B, D, N, k, s);
    case 4: return launch_mr<T, 4>(A, B, D, N, k, s);
    case 5: return launch_mr<T, 5>(A, B, D, N, k, s);
    case 6: return launch_mr<T, 6>(A, B, D, N, k, s);
    case 7: return launch_mr<T, 7>(A, B, D, N, k, s);
    case 8: return launch_mr<T, 8>(A, B, D, N, k, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool skinny_applies(int64_t M, int64_t N, int64_t K) {
    // one thread walks all of K for its columns: keep that walk short, or
    // have enough columns to fill the machine (grid.x < 2^31, K an int)
    return M >= 1 && M <= kSkinnyMaxM && (K <= 1024 || N >= (1 << 16)) && K < (1ll << 30) &&
           N / kThreads < (1ll << 31) - 1;
}

cudaError_t launch_skinny(bool f64, const void *A, const void *B, void *D, int64_t M, int64_t N, int64_t K,
                          cudaStream_t s) {
    if (f64) return launch_skinny_t((const double *)A, (const double *)B, (double *)D, M, N, K, s);
    return launch_skinny_t((const float *)A, (const float *)B, (float *)D, M, N, K, s);
}

}  // namespace moa
