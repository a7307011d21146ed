// Tensor-core forms of the (add, mul) inner product, Eq. (2) with * =
// multiply — the matrix-multiply special case of Sec. I — on the psi-
// flattened problem D (M x N, FP32) = A (M x K) . B (K x N).
//
// Kernel: persistent, warp-specialised tcgen05 GEMM for sm_103a.
//   warp 0      TMA producer: 128 x 64 tile of A (K-major, 128-B swizzle)
//               and 64 x BN tile of B (row-major = MN-major, 128-B swizzle,
//               BN/64 boxes) per pipeline stage, completion on an mbarrier.
//   warp 1      allocates TMEM and issues tcgen05.mma (128 x BN x 16, bf16 in,
//               FP32 accumulate in TMEM); tcgen05.commit frees each stage and
//               publishes each finished accumulator.
//   warps 2-9   epilogue: tcgen05.ld of the accumulator (warp w may read
//               the 32-lane quarter w % 4 of TMEM; two warps per quarter,
//               each taking half of the BN columns), stores of FP32 rows.
// Two TMEM accumulators (2 x BN columns) let the epilogue of tile t overlap
// the main loop of tile t+1.  Tiles are walked in groups of 16 row-tiles so
// the A and B panels in flight stay resident in L2.
//
// Promoted accumulation (PROMOTE): the tensor core's FP32 accumulation is
// not round-to-nearest (its error grows with the number of MMAs folded into
// one accumulator), so for the split-BF16x3 form every 64-deep k-block is
// accumulated in a fresh TMEM accumulator and then added into FP32
// registers by the epilogue with IEEE adds; the two TMEM buffers then
// alternate per k-block instead of per tile.
//
// One launch accumulates a list of "terms": pairs (plane of A, plane of B)
// of 3-D bf16 tensors [plane][rows][cols].  One term is the plain bf16
// product; six terms give the split-BF16x3 form (hi/mid/lo planes, products
// of total order <= 2), all into the same FP32 accumulator.
//
// FP8 mode (MODE_FP8): e4m3 operands (1-byte elements, 128-deep k-blocks,
// kind::f8f6f4 MMAs of depth 32) with a power-of-two scale per 1 x 128 block
// of A (row, k-block) and per 128 x 128 tile of B (k-block, column block).
// Every k-block is accumulated in a fresh TMEM accumulator and the epilogue
// adds it into FP32 registers times sA * sB (exact: both are powers of two).
//
// Ozaki mode (MODE_OZAKI): the planes hold fixed-point digit slices (small
// integers, exact in bf16) and the terms are the slice pairs (s, u) with
// s + u < S, grouped by weight class g = s + u.  The contraction is cut into
// chunks short enough that the FP32 accumulator holds the exact integer sum
// of one pair; a class runs chunk by chunk over all of its pairs (ozaki::Iter),
// the epilogue adds every (chunk, pair) accumulator of the class exactly in
// int32 registers, and at the end of the class folds that integer, scaled
// by the class's power-of-two weight, into a double-float running sum
// (hi + lo FP32 pair, TwoSum; ~48 bits relative to the running sum) kept in
// the output buffer itself (each FP64 slot holds the FP32 pair until the
// tile is finished).  FP64 arithmetic (scarce on this part) is used once
// per output: hi + lo in FP64 and the power-of-two scaling by the row /
// column exponents.
//
// Every mbarrier wait is bounded; a wait that gives up sets the CTA's abort
// flag and the device status word, lets in-flight copies and MMAs land, frees
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tc.h"
#include "ozaki_epi.cuh"
#include "tc_ptx.cuh"

namespace moa {

__device__ uint32_t g_tc_status;

namespace {

constexpr int BM = 128;
constexpr int BK = 64;  // bf16 elements per k-block: 64 x 2 B = 128 B = one swizzle row
constexpr int kMaxTerms = 8;
// Warps: 1 producer, 1 MMA, and 8 epilogue warps (2 per TMEM lane quarter),
// or 16 (4 per quarter) for the FP8 mode, whose epilogue scales and adds
// every accumulator once per k-block, so each thread holds fewer columns.
__host__ __device__ constexpr int epi_warps(int mode) { return mode == 3 ? 16 : 8; }
__host__ __device__ constexpr int cta_threads(int mode) { return 64 + 32 * epi_warps(mode); }

enum Mode { MODE_STORE = 0, MODE_PROMOTE = 1, MODE_OZAKI = 2, MODE_FP8 = 3 };

struct GemmParams {
    int M, N, K;
    int tiles_m, tiles_n;
    int kblocks;  // ceil(K / BK) per term
    int n_terms;
    uint32_t term_a, term_b;  // plane of A / B for term i in bits 4i..4i+3 (store / promote modes)
    float *D;
    int64_t ldd;
    int vec_store;  // D rows 16-byte aligned and ldd % 4 == 0
    uint32_t ab_fmt;  // kind::f16 operand format bits (bf16 or fp16 planes)
    // Ozaki mode
    int slices;      // S: digit planes per operand
    int beta;        // bits per digit
    int lsb;         // the accumulator counts units of 2^-lsb of 2^(e_row + e_col)
    int chunk;       // k-blocks per chunk of the contraction
    int acc_pairs;   // slice pairs of a (class, chunk) per exact FP32 accumulator
    double *D64;
    const uint64_t *row_max;  // |A| row maxima as FP64 bit patterns
    const uint64_t *col_max;  // |B| column maxima as FP64 bit patterns
    // FP8 mode
    const float *scale_a;  // [M][kblocks]: power-of-two scale of A's 1 x 128 blocks
    const float *scale_b;  // [kblocks][ceil(N / 128)]: scale of B's 128 x 128 tiles
    int nblk_b;            // ceil(N / 128)
};

template <int BN, int STAGES, int MODE = 0> struct Cfg {
    static constexpr int ESZ = MODE == 3 ? 1 : 2;  // element bytes (e4m3 / bf16)
    static constexpr int BKE = 128 / ESZ;          // elements per k-block (one 128-B swizzle row)
    static constexpr int UK = 32 / ESZ;            // contraction depth of one MMA
    static constexpr int BOXN = 128 / ESZ;         // N elements per B box
    static constexpr int BOX_BYTES = BKE * 128;    // one B box: BKE rows of 128 B
    static constexpr int A_BYTES = BM * 128;
    static constexpr int B_BYTES = BKE * BN * ESZ;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int NBARS = 2 * STAGES + 5;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 1024;  // + barriers, + alignment slack
    // TMEM is allocated in powers of two (>= 32 columns): two BN-wide
    // accumulators, the second starting at a power-of-two column
    static constexpr int ACC_STRIDE = BN <= 128 ? 128 : 256;
    static constexpr int TMEM_COLS = 2 * ACC_STRIDE;
    static constexpr uint32_t IDESC = MODE == 3 ? ptx::idesc_e4m3_f32(BM, BN, 1) : ptx::idesc_bf16_f32(BM, BN, 1);
    static_assert(NBARS * 8 + 16 <= 1024, "barrier area");
    static_assert(TMEM_COLS <= 512, "TMEM has 512 columns");
};

MOA_DEV void tile_of(int t, int tiles_m, int tiles_n, int &tm, int &tn) {
    constexpr int GM = 16;
    const int group = t / (GM * tiles_n);
    const int first = group * GM;
    const int gsz = min(tiles_m - first, GM);
    const int local = t - group * GM * tiles_n;
    tm = first + local % gsz;
    tn = local / gsz;
}

// Wait used only while shutting down after an abort: ignores the abort flag.
MOA_DEV bool drain_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

template <int BN, int STAGES, int MODE>
__global__ void __launch_bounds__(cta_threads(MODE), 1)
    tc_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmParams p) {
    using C = Cfg<BN, STAGES, MODE>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + STAGES * C::STAGE_BYTES);
    uint32_t *tmem_slot = (uint32_t *)(bars + C::NBARS);
    volatile uint32_t *abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tiles0 = ptx::smem_u32(smem);
    const uint32_t bar0 = ptx::smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto tfull = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto tempty = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
    const uint32_t drain = bar0 + 8u * (2 * STAGES + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(full(s), 1);
            ptx::mbar_init(empty(s), 1);  // released by this CTA's MMA warp
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(tfull(b), 1);
            ptx::mbar_init(tempty(b), epi_warps(MODE));  // one arrival per epilogue warp
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0u;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async_smem();
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(tmem_slot), C::TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // persistent CTAs walk the tiles with a stride of the grid
    const int cfirst = (int)blockIdx.x;
    const int cstride = (int)gridDim.x;
    const int num_tiles = p.tiles_m * p.tiles_n;
    const int kiters = p.kblocks * p.n_terms;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t phase = 0, issued = 0, last_par = 0;
        bool ok = true;
        for (int t = cfirst; t < num_tiles && ok; t += cstride) {
            int tm, tn;
            tile_of(t, p.tiles_m, p.tiles_n, tm, tn);
            ozaki::Iter oz;
            oz.start(p.slices, p.chunk, p.kblocks, p.acc_pairs);
            for (int it = 0; it < kiters; ++it) {
                int kb, pa, pb;
                if constexpr (MODE == MODE_OZAKI) {  // class, chunk, pair, k-block (ozaki::Iter)
                    kb = oz.kb(p.chunk);
                    pa = oz.s;
                    pb = oz.g - oz.s;
                    oz.next(p.chunk, p.kblocks);
                } else {  // k-block-major: every term of one k-block
                    kb = it / p.n_terms;
                    const int term = it - kb * p.n_terms;
                    pa = (int)((p.term_a >> (4 * term)) & 15u);
                    pb = (int)((p.term_b >> (4 * term)) & 15u);
                }
                if (!ptx::mbar_wait(empty(stage), phase ^ 1u, abort_flag, &g_tc_status)) {
                    ok = false;
                    break;
                }
                const uint32_t sa = tiles0 + stage * C::STAGE_BYTES, sb = sa + C::A_BYTES;
                ptx::mbar_arrive_expect_tx(full(stage), C::STAGE_BYTES);
                ptx::tma_load_3d(sa, &tmA, full(stage), kb * C::BKE, tm * BM, pa);
#pragma unroll
                for (int j = 0; j < BN / C::BOXN; ++j)
                    ptx::tma_load_3d(sb + j * C::BOX_BYTES, &tmB, full(stage), tn * BN + j * C::BOXN, kb * C::BKE, pb);
                issued |= 1u << stage;
                last_par = (last_par & ~(1u << stage)) | (phase << stage);
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        if (!ok) {  // let every copy already issued land before the CTA exits
            for (int s = 0; s < STAGES; ++s)
                if (issued & (1u << s)) drain_wait(full(s), (last_par >> s) & 1u);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        const uint32_t idesc = (C::IDESC & ~ptx::kIdescAbMask) | p.ab_fmt;  // kind::f16: bf16 or fp16 planes
        int stage = 0, abuf = 0;
        uint32_t phase = 0, aphase = 0;
        bool ok = true;
        // an accumulator is handed to the epilogue once per tile (store),
        // once per k-block with all its terms (promote), or once per chunk of
        // a slice pair (Ozaki)
        for (int t = cfirst; t < num_tiles && ok; t += cstride) {
            ozaki::Iter oz;
            oz.start(p.slices, p.chunk, p.kblocks, p.acc_pairs);
            for (int it = 0; it < kiters; ++it) {
                int j, last;  // position inside the current accumulator; whether it is its last step
                if constexpr (MODE == MODE_STORE) {
                    j = it;
                    last = it == kiters - 1;
                } else if constexpr (MODE == MODE_PROMOTE || MODE == MODE_FP8) {
                    j = it % p.n_terms;
                    last = j == p.n_terms - 1;
                } else {  // one accumulator per (class, chunk, pair)
                    j = oz.acc_pos();
                    last = oz.acc_last();
                    oz.next(p.chunk, p.kblocks);
                }
                if (j == 0) {
                    if (!ptx::mbar_wait(tempty(abuf), aphase ^ 1u, abort_flag, &g_tc_status)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                }
                const uint32_t dacc = tmem + (uint32_t)(abuf * C::ACC_STRIDE);
                if (!ptx::mbar_wait(full(stage), phase, abort_flag, &g_tc_status)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t sa = tiles0 + stage * C::STAGE_BYTES, sb = sa + C::A_BYTES;
#pragma unroll
                for (int k = 0; k < C::BKE / C::UK; ++k) {
                    // A: +32 B along the swizzled K row; B: +UK rows of 128 B
                    const uint64_t ad = ptx::smem_desc_sw128(sa + k * 32, 16, 1024);
                    const uint64_t bd = ptx::smem_desc_sw128(sb + k * C::UK * 128, C::BOX_BYTES, 1024);
                    if constexpr (MODE == MODE_FP8)
                        ptx::mma_e4m3(dacc, ad, bd, C::IDESC, (j > 0 || k > 0) ? 1u : 0u);
                    else
                        ptx::mma_bf16(dacc, ad, bd, idesc, (j > 0 || k > 0) ? 1u : 0u);
                }
                ptx::mma_commit(empty(stage));
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
                if (last) {
                    ptx::mma_commit(tfull(abuf));
                    abuf ^= 1;
                    if (!abuf) aphase ^= 1u;
                }
            }
        }
        if (!ok) {  // MMAs already issued must finish before TMEM is freed
            ptx::mma_commit(drain);
            drain_wait(drain, 0);
        }
    } else if (warp >= 2) {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;                  // TMEM lane quarter this warp may access
        const int half = (warp - 2) / 4;                 // which part of the BN columns
        constexpr int HC = BN / (epi_warps(MODE) / 4);   // columns per epilogue warp
        int abuf = 0;
        uint32_t aphase = 0;
        auto wait_acc = [&]() -> bool {
            int okw = 1;
            if (lane == 0) okw = ptx::mbar_wait(tfull(abuf), aphase, abort_flag, &g_tc_status) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (okw) ptx::tc_fence_after();
            return okw != 0;
        };
        auto release_acc = [&]() {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(tempty(abuf));
            abuf ^= 1;
            if (!abuf) aphase ^= 1u;
        };
        // 32 consecutive columns of one row (registers indexed at compile time only)
        auto store32 = [&](int64_t row, int64_t col0, const uint32_t (&v)[32]) {
            if (row >= p.M || col0 >= p.N) return;
            float *dst = p.D + row * p.ldd + col0;
            if (p.vec_store && col0 + 32 <= p.N) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4 *>(dst + j) = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                                       __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (col0 + j < p.N) dst[j] = __uint_as_float(v[j]);
            }
        };
        bool ok = true;
        for (int t = cfirst; t < num_tiles && ok; t += cstride) {
            int tm, tn;
            tile_of(t, p.tiles_m, p.tiles_n, tm, tn);
            const int64_t row = (int64_t)tm * BM + q * 32 + lane;
            const int64_t colh = (int64_t)tn * BN + half * HC;
            if constexpr (MODE == MODE_OZAKI) {
                const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
                const bool row_ok = row < p.M;
                double *drow = p.D64 + row * p.ldd;
                bool first = true;  // no running sum stored yet for this tile
                int qacc[HC];
#pragma unroll
                for (int j = 0; j < HC; ++j) qacc[j] = 0;
                const int chunks = (p.kblocks + p.chunk - 1) / p.chunk;
                for (int cls = p.slices - 1; cls >= 0 && ok; --cls) {
                    const bool class_ends = true;  // the loops below consume the whole class
                    // the class's power-of-two weight in accumulator units, exact in FP32
                    const float w = ozaki::class_weight(cls, p.lsb, p.beta);
                    for (int c = 0; c < ozaki::accs_in_class(cls, chunks, p.acc_pairs); ++c) {  // the class's accumulators
                        if (!wait_acc()) {
                            ok = false;
                            break;
                        }
                        const uint32_t tb = lane_base + (uint32_t)(abuf * C::ACC_STRIDE + half * HC);
#pragma unroll
                        for (int c0 = 0; c0 < HC; c0 += 16) {
                            uint32_t r[16];
                            ptx::tmem_ld16(tb + c0, r);
                            ptx::tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 16; ++j)  // exact: chunk sums are integers below 2^24
                                qacc[c0 + j] += __float2int_rz(__uint_as_float(r[j]));
                        }
                        release_acc();  // the accumulator is consumed; the MMA may refill it during the fold
                    }
                    if (!ok) break;
                    if (class_ends && row_ok) ozaki::fold<HC>(qacc, w, drow, colh, p.N, first);
                    if (!ok) break;
                    if (class_ends) {
#pragma unroll
                        for (int j = 0; j < HC; ++j) qacc[j] = 0;
                        first = false;
                    }
                }
                if (!ok) break;
                if (row_ok) ozaki::finish<HC>(drow, colh, p.N, p.row_max[row], p.col_max, p.lsb);
            } else if constexpr (MODE == MODE_FP8) {
                float acc[HC];
#pragma unroll
                for (int j = 0; j < HC; ++j) acc[j] = 0.0f;
                const int colblk = (int)(colh / 128);  // HC <= 128 columns, all in one B scale block
                const bool row_ok = row < p.M, col_ok = colh < p.N;
                // scales of the next k-block are loaded while this one is added
                float sa_next = row_ok ? p.scale_a[row * p.kblocks] : 0.0f;
                float sb_next = col_ok ? p.scale_b[colblk] : 0.0f;
                for (int kb = 0; kb < p.kblocks; ++kb) {
                    const float sa = sa_next, sb = sb_next;
                    if (kb + 1 < p.kblocks) {
                        sa_next = row_ok ? p.scale_a[row * p.kblocks + kb + 1] : 0.0f;
                        sb_next = col_ok ? p.scale_b[(int64_t)(kb + 1) * p.nblk_b + colblk] : 0.0f;
                    }
                    if (!wait_acc()) {
                        ok = false;
                        break;
                    }
                    const float f = __fmul_rn(sa, sb);
                    const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * C::ACC_STRIDE + half * HC);
#pragma unroll
                    for (int c = 0; c < HC; c += 16) {
                        uint32_t r[16];
                        ptx::tmem_ld16(tb + c, r);
                        ptx::tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) acc[c + j] = fmaf(__uint_as_float(r[j]), f, acc[c + j]);
                    }
                    release_acc();
                }
                if (!ok) break;
#pragma unroll
                for (int c = 0; c < HC; c += 32) {
                    uint32_t r[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(acc[c + j]);
                    store32(row, colh + c, r);
                }
            } else if constexpr (MODE == MODE_PROMOTE) {
                float acc[HC];
#pragma unroll
                for (int j = 0; j < HC; ++j) acc[j] = 0.0f;
                for (int kb = 0; kb < p.kblocks; ++kb) {
                    if (!wait_acc()) {
                        ok = false;
                        break;
                    }
                    const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * C::ACC_STRIDE + half * HC);
#pragma unroll
                    for (int c = 0; c < HC; c += 32) {
                        uint32_t r[32];
                        ptx::tmem_ld32(tb + c, r);
                        ptx::tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[c + j] = __fadd_rn(acc[c + j], __uint_as_float(r[j]));
                    }
                    release_acc();
                }
                if (!ok) break;
#pragma unroll
                for (int c = 0; c < HC; c += 32) {
                    uint32_t r[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(acc[c + j]);
                    store32(row, colh + c, r);
                }
            } else {
                if (!wait_acc()) break;
                const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * C::ACC_STRIDE + half * HC);
#pragma unroll 1
                for (int c = 0; c < HC; c += 32) {
                    uint32_t r[32];
                    ptx::tmem_ld32(tb + c, r);
                    ptx::tmem_ld_wait();
                    store32(row, colh + c, r);
                }
                release_acc();
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// ------------------------------------------------------------------ host
int num_sms() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

template <int BN, int STAGES, int MODE>
cudaError_t launch_tc(const CUtensorMap &ta, const CUtensorMap &tb, GemmParams &p, cudaStream_t s) {
    using C = Cfg<BN, STAGES, MODE>;
    auto kern = tc_gemm_bf16<BN, STAGES, MODE>;
    // shared-memory attribute, set up once per process (under a lock, so
    // concurrent first calls agree; a failure is retried)
    static std::mutex mu;
    static bool ready = false;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!ready) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
            if (e != cudaSuccess) return e;
            ready = true;
        }
    }
    p.tiles_m = (p.M + BM - 1) / BM;
    p.tiles_n = (p.N + BN - 1) / BN;
    const int tiles = p.tiles_m * p.tiles_n;
    const int ctas = tiles < num_sms() ? tiles : num_sms();
    GemmTimer timer(s);
    kern<<<ctas, cta_threads(MODE), C::SMEM, s>>>(ta, tb, p);
    const cudaError_t e = cudaGetLastError();
    timer.done();
    return e;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return fn;
}

// 3-D tensor [planes][rows][inner] of `dt` with the given strides (bytes),
// boxes of box_inner x box_rows (128-B swizzled unless `swizzle` says otherwise).
bool make_tmap(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint64_t planes, uint64_t row_bytes,
               uint64_t plane_bytes, uint32_t box_inner, uint32_t box_rows, CUtensorMapDataType dt,
               CUtensorMapSwizzle swizzle, uint32_t box_planes) {
    auto enc = tmap_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {inner, rows, planes};
    cuuint64_t strides[2] = {row_bytes, plane_bytes};
    cuuint32_t box[3] = {box_inner, box_rows, box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Planes of A are [planes][M][lda] bf16, of B [planes][K][ldb] bf16;
// lda, ldb multiples of 8 and the bases 16-byte aligned (TMA rules).
moa_status tc_gemm_planes(const __nv_bfloat16 *A, int64_t lda, int planesA, const __nv_bfloat16 *B, int64_t ldb,
                          int planesB, int n_terms, const int *term_a, const int *term_b, float *D, int64_t ldd,
                          int64_t M, int64_t N, int64_t K, bool promote, cudaStream_t s, bool i32_out, bool fp16) {
    if (M >= (1ll << 31) || N >= (1ll << 31) || K >= (1ll << 31)) return MOA_ERR_OVERFLOW;
    if (n_terms < 1 || n_terms > kMaxTerms) return MOA_ERR_INTERNAL;
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16 || lda % 8 || ldb % 8) return MOA_ERR_INTERNAL;
    const int BN = (N <= 128) ? 128 : 256;
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, A, (uint64_t)K, (uint64_t)M, (uint64_t)planesA, (uint64_t)lda * 2, (uint64_t)(lda * M * 2), BK, BM))
        return MOA_ERR_CUDA;
    if (!make_tmap(&tb, B, (uint64_t)N, (uint64_t)K, (uint64_t)planesB, (uint64_t)ldb * 2, (uint64_t)(ldb * K * 2), 64, BK))
        return MOA_ERR_CUDA;
    GemmParams p{};
    p.M = (int)M, p.N = (int)N, p.K = (int)K;
    p.kblocks = (int)((K + BK - 1) / BK);
    p.n_terms = n_terms;
    for (int i = 0; i < n_terms; ++i) {
        if (term_a[i] < 0 || term_a[i] >= planesA || term_b[i] < 0 || term_b[i] >= planesB) return MOA_ERR_INTERNAL;
        p.term_a |= (uint32_t)term_a[i] << (4 * i);
        p.term_b |= (uint32_t)term_b[i] << (4 * i);
    }
    p.D = D;
    p.ldd = ldd;
    p.vec_store = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0);
    p.ab_fmt = ptx::idesc_ab_f16(fp16);
    cudaError_t e;
    if (BN == 256 && M > BM && pair_mma_enabled()) {
        e = tc_gemm_pair_launch(ta, tb, p.M, p.N, p.K, n_terms, p.term_a, p.term_b, D, ldd, promote, s, i32_out, fp16);
        return e == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
    }
    if (i32_out) return MOA_ERR_INTERNAL;  // int32 results only from the pair kernel
    if (promote)
        e = BN == 128 ? launch_tc<128, 6, MODE_PROMOTE>(ta, tb, p, s) : launch_tc<256, 4, MODE_PROMOTE>(ta, tb, p, s);
    else
        e = BN == 128 ? launch_tc<128, 6, MODE_STORE>(ta, tb, p, s) : launch_tc<256, 4, MODE_STORE>(ta, tb, p, s);
    return e == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
}

// FP8 GEMM: A8 [M][lda] and B8 [K][ldb] e4m3 bytes (lda, ldb multiples of 16),
// scale_a [M][ceil(K/128)], scale_b [ceil(K/128)][ceil(N/128)] powers of two;
// D (M x N, FP32, row stride ldd) = sum over k-blocks of sA * sB * (A8 . B8).
moa_status tc_gemm_fp8(const uint8_t *A, int64_t lda, const uint8_t *B, int64_t ldb, const float *scale_a,
                       const float *scale_b, float *D, int64_t ldd, int64_t M, int64_t N, int64_t K, cudaStream_t s) {
    if (M >= (1ll << 31) || N >= (1ll << 31) || K >= (1ll << 31)) return MOA_ERR_OVERFLOW;
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16 || lda % 16 || ldb % 16) return MOA_ERR_INTERNAL;
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, A, (uint64_t)K, (uint64_t)M, 1, (uint64_t)lda, (uint64_t)(lda * M), 128, BM,
                   CU_TENSOR_MAP_DATA_TYPE_UINT8))
        return MOA_ERR_CUDA;
    if (!make_tmap(&tb, B, (uint64_t)N, (uint64_t)K, 1, (uint64_t)ldb, (uint64_t)(ldb * K), 128, 128,
                   CU_TENSOR_MAP_DATA_TYPE_UINT8))
        return MOA_ERR_CUDA;
    GemmParams p{};
    p.M = (int)M, p.N = (int)N, p.K = (int)K;
    p.kblocks = (int)((K + 127) / 128);
    p.n_terms = 1;
    p.D = D, p.ldd = ldd;
    p.vec_store = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0);
    p.scale_a = scale_a, p.scale_b = scale_b, p.nblk_b = (int)((N + 127) / 128);
    const cudaError_t e = launch_tc<256, 4, MODE_FP8>(ta, tb, p, s);
    return e == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
}

// Ozaki slice-pair GEMM: planes [S][M][lda] and [S][K][ldb] of bf16 digits,
// D64 (M x N, FP64, row stride ldd) = sum over pairs s + u < S of
// 2^(e_row + e_col - (s + u + 2) * beta) * (A_s . B_u); lsb is chosen so
// every pair weight 2^(lsb - (s + u + 2) beta) is within FP32's range.
moa_status tc_gemm_ozaki(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb, int S, int beta,
                         int lsb, int chunk_kblocks, int acc_pairs, const uint64_t *row_max, const uint64_t *col_max,
                         double *D, int64_t ldd, int64_t M, int64_t N, int64_t K, void *scratch, cudaStream_t s) {
    if (M >= (1ll << 31) || N >= (1ll << 31) || K >= (1ll << 31)) return MOA_ERR_OVERFLOW;
    // weights 2^(lsb - (g+2) beta) must be exact FP32 powers of two >= 1, and a
    // class sum (g+1 <= S pairs of K balanced digit products, each at most
    // 2^(2 beta - 2) in magnitude) must stay below 2^31
    // an accumulator (acc_pairs pairs of a chunk of chunk_kblocks k-blocks of 64 products of at most
    // 2^(2 beta - 2)) must stay at or below 2^24 to be exact in FP32
    if (acc_pairs < 1 || (double)acc_pairs * chunk_kblocks * 64.0 * (double)(1 << (2 * beta - 2)) > 16777216.0)
        return MOA_ERR_INTERNAL;
    if (S < 1 || S > 10 || chunk_kblocks < 1 || lsb - 2 * beta > 100 || lsb - (S + 1) * beta < 0 ||
        (double)S * (double)K * (double)(1 << (2 * beta - 2)) >= 2147483648.0)
        return MOA_ERR_INTERNAL;
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16 || lda % 8 || ldb % 8) return MOA_ERR_INTERNAL;
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, A, (uint64_t)K, (uint64_t)M, (uint64_t)S, (uint64_t)lda * 2, (uint64_t)(lda * M * 2), BK, BM))
        return MOA_ERR_CUDA;
    if (!make_tmap(&tb, B, (uint64_t)N, (uint64_t)K, (uint64_t)S, (uint64_t)ldb * 2, (uint64_t)(ldb * K * 2), 64, BK))
        return MOA_ERR_CUDA;
    GemmParams p{};
    p.M = (int)M, p.N = (int)N, p.K = (int)K;
    p.kblocks = (int)((K + BK - 1) / BK);
    p.n_terms = S * (S + 1) / 2;
    p.slices = S, p.beta = beta, p.lsb = lsb, p.chunk = chunk_kblocks, p.acc_pairs = acc_pairs;
    p.D64 = D, p.ldd = ldd, p.row_max = row_max, p.col_max = col_max;
    p.ab_fmt = ptx::idesc_ab_f16(false);
    if (M > BM && N > 128 && pair_mma_enabled() && scratch) {  // 256 x 256 tiles on CTA pairs
        const cudaError_t e = tc_gemm_pair_ozaki_launch(ta, tb, p.M, p.N, p.K, S, beta, lsb, chunk_kblocks, acc_pairs,
                                                        row_max, col_max, D, ldd, scratch, s);
        return e == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
    }
    // 192-wide tiles: two accumulators fit TMEM and the int32 class sums of a
    // thread's 96 columns fit its registers
    const cudaError_t e = launch_tc<192, 5, MODE_OZAKI>(ta, tb, p, s);
    return e == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
}

// Self-test of the bounded waits: one CTA waits on an mbarrier that nothing
// ever arrives on, gives up after limit_ns and records kStatusTimeout.
__global__ void wait_probe_kernel(uint64_t limit_ns) {
    __shared__ uint64_t bar;
    const uint32_t b = ptx::smem_u32(&bar);
    if (threadIdx.x == 0) {
        ptx::mbar_init(b, 1);
        ptx::fence_mbar_init();
        const uint64_t t0 = globaltimer();
        while (!ptx::mbar_try_wait(b, 0)) {
            if (globaltimer() - t0 > limit_ns) {
                atomicOr(&g_tc_status, kStatusTimeout);
                break;
            }
        }
    }
}

cudaError_t tc_wait_probe(uint64_t limit_ns, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(limit_ns);
    return cudaGetLastError();
}

cudaError_t tc_read_and_clear_status(uint32_t *flags) {
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_tc_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    const uint32_t zero = 0;
    return cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(uint32_t));
}

}  // namespace moa
