// Generalized inner product on CUDA cores, Eq. (2) with a general
// (reduce, combine) pair (Sec. I lets the operation be any binary one):
//   D[i, j] = reduce_{p < K} ( A[i, p] combine B[p, j] ),
// on the psi-flattened problem (A: M x K, B: K x N, D: M x N, row-major).
//
// The paper computes one result row at a time, accumulating rows of B scaled
// by elements of A (Fig. 1 and the appendix).  On the GPU the same reuse is
// organised as a two-level tile: a 128 x 128 block of D per CTA, with A and B
// panels of depth BK staged in shared memory (double-buffered through
// registers), and an 8 x 8 register micro-tile per thread.  Every element of
// an A panel is reused 128 times from shared memory and every loaded value 8
// times from registers.  A thread's 8 rows (and 8 columns) are two groups of
// 4 that lie half a tile apart, so the 16-byte shared-memory reads of a
// half-warp cover one contiguous 256-byte row segment (no bank conflicts).
//
// Exactness: min / max / integer results do not depend on the order of the
// reduction, and each combine is one correctly rounded operation, so the
// result is bit-identical to the definition.  The contraction tail (K not a
// multiple of BK) runs a shortened loop instead of padding with values: a
// padded +inf/-inf could meet a real -inf/+inf and make NaN.
#include "common.cuh"
#include "internal.h"
#include "semiring_ops.cuh"

namespace moa {
namespace {

// --------------------------------------------------------------- kernel
template <int BM, int BN, int BK, int TM, int TN> struct Tile {
    static constexpr int NT = (BM / TM) * (BN / TN);  // threads
    static constexpr int PAD = 4;                      // keeps float4 alignment, spreads banks
    static constexpr int LA = BM * BK / NT;            // A elements loaded per thread per panel
    static constexpr int LB = BK * BN / NT;
    static_assert(BM * BK % NT == 0 && BK * BN % NT == 0, "panel must split evenly over threads");
    static_assert(NT % BK == 0 && NT % BN == 0, "load mapping");
};

template <class Op, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(Tile<BM, BN, BK, TM, TN>::NT, 2)  // two CTAs (16 warps) per SM
    semiring_gemm(const typename Op::T *__restrict__ A, const typename Op::T *__restrict__ B,
                  typename Op::T *__restrict__ D, int64_t M, int64_t N, int64_t K, const uint32_t *run_if) {
    if (run_if && __ldg(run_if) == 0u) return;  // uniform over the grid
    using T = typename Op::T;
    using TL = Tile<BM, BN, BK, TM, TN>;
    constexpr int NT = TL::NT;
    __shared__ __align__(16) T As[2][BK][BM + TL::PAD];  // A panel stored k-major
    __shared__ __align__(16) T Bs[2][BK][BN + TL::PAD];

    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;

    // load mapping: A panel rows of BK consecutive k (coalesced along k),
    // B panel rows of BN consecutive n (coalesced along n).
    const int a_k = tid % BK, a_m = tid / BK;
    constexpr int A_MSTEP = NT / BK;
    const int b_n = tid % BN, b_k = tid / BN;
    constexpr int B_KSTEP = NT / BN;

    T ra[TL::LA], rb[TL::LB];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < TL::LA; ++r) {
            const int64_t m = m0 + a_m + r * A_MSTEP, k = k0 + a_k;
            ra[r] = (m < M && k < K) ? __ldg(A + m * K + k) : Op::identity();
        }
#pragma unroll
        for (int r = 0; r < TL::LB; ++r) {
            const int64_t k = k0 + b_k + r * B_KSTEP, n = n0 + b_n;
            rb[r] = (k < K && n < N) ? __ldg(B + k * N + n) : Op::identity();
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int r = 0; r < TL::LA; ++r) As[buf][a_k][a_m + r * A_MSTEP] = ra[r];
#pragma unroll
        for (int r = 0; r < TL::LB; ++r) Bs[buf][b_k + r * B_KSTEP][b_n] = rb[r];
    };

    constexpr int HM = TM / 2, HN = TN / 2;  // each half of the micro-tile
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = Op::identity();

    const int64_t full_panels = K / BK;
    const int tail = (int)(K - full_panels * BK);
    const int64_t panels = full_panels + (tail ? 1 : 0);
    if (panels > 0) {
        load(0);
        stash(0);
    }
    __syncthreads();
    for (int64_t p = 0; p < panels; ++p) {
        const int buf = (int)(p & 1);
        if (p + 1 < panels) load((p + 1) * BK);  // next panel in flight during compute
        const T *as = &As[buf][0][ty * HM];
        const T *bs = &Bs[buf][0][tx * HN];
        if (p < full_panels) {
#pragma unroll
            for (int kk = 0; kk < BK; kk += 2) {
                T a0[TM], b0[TN], a1[TM], b1[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) {
                    const int r = (i % HM) + (i / HM) * (BM / 2);
                    a0[i] = as[kk * (BM + TL::PAD) + r];
                    a1[i] = as[(kk + 1) * (BM + TL::PAD) + r];
                }
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const int c = (j % HN) + (j / HN) * (BN / 2);
                    b0[j] = bs[kk * (BN + TL::PAD) + c];
                    b1[j] = bs[(kk + 1) * (BN + TL::PAD) + c];
                }
#pragma unroll
                for (int i = 0; i < TM; ++i) {
                    if constexpr (Op::kPacked) {  // two adjacent columns per packed FP32 instruction
#pragma unroll
                        for (int j = 0; j < TN; j += 2)
                            Op::step2x2(acc[i][j], acc[i][j + 1], a0[i], b0[j], b0[j + 1], a1[i], b1[j], b1[j + 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] = Op::step2(acc[i][j], a0[i], b0[j], a1[i], b1[j]);
                    }
                }
            }
        } else {
            for (int kk = 0; kk < tail; ++kk) {  // contraction tail: shortened loop, no padding values
                T a0[TM], b0[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a0[i] = as[kk * (BM + TL::PAD) + (i % HM) + (i / HM) * (BM / 2)];
#pragma unroll
                for (int j = 0; j < TN; ++j) b0[j] = bs[kk * (BN + TL::PAD) + (j % HN) + (j / HN) * (BN / 2)];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = Op::step(acc[i][j], a0[i], b0[j]);
            }
        }
        if (p + 1 < panels) {
            stash(buf ^ 1);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t m = m0 + ty * HM + (i % HM) + (i / HM) * (BM / 2);
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t n = n0 + tx * HN + (j % HN) + (j / HN) * (BN / 2);
            if (n < N) D[m * N + n] = acc[i][j];
        }
    }
}

template <class Op, int BM, int BN, int BK, int TM, int TN>
cudaError_t run(const void *A, const void *B, void *D, int64_t M, int64_t N, int64_t K, cudaStream_t s,
              const uint32_t *run_if) {
    const int64_t gx = (N + BN - 1) / BN, gy = (M + BM - 1) / BM;
    if (gy > 65535 || gx > 0x7fffffff) return cudaErrorInvalidConfiguration;
    semiring_gemm<Op, BM, BN, BK, TM, TN><<<dim3((unsigned)gx, (unsigned)gy), Tile<BM, BN, BK, TM, TN>::NT, 0, s>>>(
        (const typename Op::T *)A, (const typename Op::T *)B, (typename Op::T *)D, M, N, K, run_if);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_semiring(SemiringKind kind, const void *A, const void *B, void *D, int64_t M, int64_t N, int64_t K,
                            cudaStream_t s, const uint32_t *run_if) {
    switch (kind) {
    case SR_F64_PLUS_TIMES: return run<sr::F64PlusTimes, 64, 64, 8, 4, 4>(A, B, D, M, N, K, s, run_if);
    case SR_F32_PLUS_TIMES: return run<sr::F32PlusTimes, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MIN_PLUS: return run<sr::F32MinPlus, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MAX_PLUS: return run<sr::F32MaxPlus, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MIN_TIMES: return run<sr::F32MinTimes, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MAX_TIMES: return run<sr::F32MaxTimes, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_I32_PLUS_TIMES: return run<sr::I32PlusTimes, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MIN_MINUS: return run<sr::F32MinMax<false, sr::C_SUB>, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MAX_MINUS: return run<sr::F32MinMax<true, sr::C_SUB>, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MAX_MIN: return run<sr::F32MinMax<true, sr::C_MIN>, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MIN_MAX: return run<sr::F32MinMax<false, sr::C_MAX>, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MIN_MIN: return run<sr::F32MinMax<false, sr::C_MIN>, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    case SR_F32_MAX_MAX: return run<sr::F32MinMax<true, sr::C_MAX>, 128, 128, 16, 8, 8>(A, B, D, M, N, K, s, run_if);
    }
    return cudaErrorInvalidValue;
}

}  // namespace moa
