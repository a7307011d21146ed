// Batched execution of many generalized inner / outer products of uneven
// ranks and shapes (Eq. 1 and Eq. 2 per problem) in one grouped launch.
//
// Plan (host, moa_batch_plan_create): every problem is validated as its
// single call would be and psi-flattened; its work is cut into items —
//   TC   one 128 x 128 tile of a split-BF16x3 (+,*) problem (tensor cores),
//   GEMV rows or columns of a split-BF16x3 problem with M = 1 or N = 1, on the
//        CUDA cores straight from the FP32 operands (a compensated dot
//        product, more accurate than the split form),
//   CC   one 128 x 128 tile of a CUDA-core semiring problem ((min|max|+),
//        (+|*)) — 8 x 8 register micro-tiles, shared-memory panels,
//   OUT  a block of rows of an outer product,
//   FILL the reduce identity for an inner product with an empty contraction.
// Items are ordered by an estimated cost (the ordering policy is picked by
// the autotuner), and per-problem descriptors, the TMA tensor maps of the
// split planes and the item list are uploaded once.
//
// Execute (moa_batch_execute): a CUDA graph, captured on the first execute
// and replayed after.  It holds (1) persistent CUDA-core kernels, one per
// (operator, occupied tile halves) present, two 256-thread CTAs per SM, each
// pulling its CC items from its own queue counter; (2) the grouped split
// pre-pass (FP32 -> three bf16 planes for every BF16x3 problem); (3) one
// persistent grouped kernel (one CTA per SM) for the TC / OUT / FILL items.
// In that kernel a scheduler warp pulls item indices from a device-side
// queue (one atomic counter), copies each item and its problem descriptor
// into an 8-slot shared-memory ring guarded by mbarriers (prefetching the
// tensor maps of tensor-core items), and the TMA warp, the MMA warp and the
// 16 epilogue warps take their work from that ring.
// TC items run the tcgen05 pipeline of tc_gemm.cu in its promoted form
// (per-k-block FP32 promotion) with four TMEM accumulators in turn; OUT /
// FILL items are computed by the epilogue warps.  The two schedules differ
// in the grouped queue's order (longest first over all items, or tensor-core
// tiles first); the autotuner times them on the first execute.  Every wait
// is bounded and reports through the batch status word.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <sys/stat.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "semiring_ops.cuh"
#include "tc.h"
#include "tc_ptx.cuh"

namespace moa {

__device__ uint32_t g_batch_status;

namespace {

enum ItemType { IT_TC = 0, IT_CC = 1, IT_OUT = 2, IT_FILL = 3, IT_GEMV = 4 };
// IT_GEMV: a split-BF16x3 (+,*) or CUDA-core semiring problem with M = 1 or N = 1, on the CUDA cores
// (shape GV_ROWS: rows [a, a + b) of an N = 1 product, one warp per row;
// GV_COLS: columns [a, a + b) of an M = 1 product, one thread per column)
constexpr int GV_ROWS = 1, GV_COLS = 2;
enum CcOp { CC_MIN_PLUS = 0, CC_MAX_PLUS = 1, CC_MIN_TIMES = 2, CC_MAX_TIMES = 3, CC_PLUS_TIMES = 4 };
constexpr int kCcOps = 5, kCcGroups = 4 * kCcOps;  // CUDA-core kernels: operator x occupied tile halves

struct alignas(16) BInst {
    int32_t type;  // IT_*
    int32_t op;    // CcOp (CC), moa_op (OUT), fill bit pattern (FILL)
    int32_t M, N, K, kblocks;
    const float *A;
    const float *B;
    float *D;
    int32_t tmap;  // TC: index of A's tensor map; B's follows it
    int32_t vec;   // D 16-byte aligned and N % 4 == 0
};

struct alignas(16) BItem {
    int32_t inst, type, a, b;  // TC / CC: tile (a = row tile, b = column tile); OUT / FILL: rows [a, a + b)
    // TC tile shape: bit 0 a 128 x 64 tile (b counts 64-column tiles; one B half,
    // N = 64 MMAs), bit 1 a 64-row A box (problems with M <= 64; the MMA rows
    // 64..127 read stale planes and are never stored)
    int32_t shape, pad0, pad1, pad2;
};
constexpr int SH_NARROW = 1, SH_SHORT = 2;

// One slot of the grouped kernel's item ring: the scheduler copies the item
// and its problem descriptor here ahead of use, so the other roles read them
// from shared memory.
struct alignas(16) RingSlot {
    BItem it;
    BInst in;
    int32_t item, pad[3];
};

struct SplitJob {
    const float *src;
    __nv_bfloat16 *dst;
    int64_t cols, colsp, plane, r0, r1;
};

// A stage is one 32-deep slice of K holding all three bf16 planes of the A
// tile and of the B tile (one 3-plane TMA box each), so each plane tile is
// loaded once for the six products it takes part in; the FP32 promotion is
// per 64-deep block (two stages).
constexpr int BM = 128, BN = 128, BK = 32, KB = 64, STAGES = 3, RING = 8, TERMS = 6, PLANES = 3;
// warp 0 the scheduler, warp 1 the TMA producer, warp 2 the MMA issuer, then
// 16 epilogue warps (four per TMEM lane quarter, 32 columns each) and four
// TMEM accumulators, so the promotion and stores of short tiles keep up with
// the MMA warp
constexpr int kCtlWarps = 3, kEpiWarps = 16, kThreads = 32 * (kCtlWarps + kEpiWarps), kEpiThreads = 32 * kEpiWarps,
              NACC = 4;
constexpr int A_PLANE = BM * BK * 2;        // 128 rows x 64 B, 64-B swizzle
constexpr int B_PLANE = BK * 64 * 2;        // one 64-column half: 32 rows x 128 B, 128-B swizzle
constexpr int B_HALF = PLANES * B_PLANE;    // a half's three planes
constexpr int A_BYTES = PLANES * A_PLANE, B_BYTES = 2 * B_HALF, STAGE_BYTES = A_BYTES + B_BYTES;
static_assert(STAGE_BYTES % 1024 == 0 && A_PLANE % 1024 == 0 && B_PLANE % 1024 == 0, "swizzle atoms stay aligned");
// CUDA-core tiles: panels of 16 k, four stages in flight (cp.async)
constexpr int CC_BK = 16, CC_PAD = 4, CC_LD = 128 + CC_PAD, CC_STAGES = 4;
constexpr int CC_PANEL = CC_BK * CC_LD;                 // floats of one operand's panel
constexpr int CC_BYTES = CC_STAGES * 2 * CC_PANEL * 4;  // As[4][16][132] + Bs[4][16][132]
constexpr int NBARS = 2 * STAGES + 2 * NACC + 1 + 2 * RING;
constexpr int TC_STG_FLOATS = 32 * 33;                  // an epilogue warp's 32 x 32 staging slice (padded rows)
constexpr int TC_STG_BYTES = kEpiWarps * TC_STG_FLOATS * 4;
constexpr int RING_BYTES = RING * (int)sizeof(RingSlot);
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + TC_STG_BYTES + RING_BYTES + 1024;
constexpr int TMEM_COLS = NACC * BN;
static_assert(TMEM_COLS <= 512 && NBARS * 8 + 16 <= 1024 && SMEM <= 227 * 1024, "grouped kernel resources");
constexpr uint32_t IDESC = ptx::idesc_bf16_f32(BM, BN, 1);
constexpr uint32_t IDESC_N64 = ptx::idesc_bf16_f32(BM, 64, 1);
// split-BF16x3 terms (plane of A, plane of B): small products first, hi*hi last
MOA_DEV constexpr int term_a(int t) { return t == 0 ? 1 : t == 2 ? 2 : t == 4 ? 1 : 0; }  // 1, 0, 2, 0, 1, 0
MOA_DEV constexpr int term_b(int t) { return t == 0 ? 1 : t == 1 ? 2 : t == 3 ? 1 : 0; }  // 1, 2, 0, 1, 0, 0

struct BatchParams {
    const BInst *inst;
    const BItem *items;
    int n_items;
    int *queue;
    const CUtensorMap *tmaps;
};

MOA_DEV void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Compensated dot product in FP32 (Ogita, Rump and Oishi's Dot2): the product
// split exactly into p + e by an FMA, p added to the running sum by TwoSum,
// both error terms collected in `cmp`; sum + cmp is as accurate as a dot
// product computed in twice the working precision and then rounded.  Every
// step is an explicitly rounded operation, so no contraction changes it.
MOA_DEV void dot2_step(float &sum, float &cmp, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(sum, p);
    const float z = __fsub_rn(t, sum);
    const float err = __fadd_rn(__fsub_rn(sum, __fsub_rn(t, z)), __fsub_rn(p, z));
    sum = t;
    cmp = __fadd_rn(cmp, __fadd_rn(err, e));
}
// (sum, cmp) += (sum2, cmp2), the two sums added by TwoSum.
MOA_DEV void dot2_merge(float &sum, float &cmp, float sum2, float cmp2) {
    const float t = __fadd_rn(sum, sum2);
    const float z = __fsub_rn(t, sum);
    const float err = __fadd_rn(__fsub_rn(sum, __fsub_rn(t, z)), __fsub_rn(sum2, z));
    sum = t;
    cmp = __fadd_rn(__fadd_rn(cmp, cmp2), err);
}

// Rows [a, a + b) of an outer product's row-major result, D[r, c] = A[r] op
// B[c], walked as one flat range by `nthreads` threads from `tid`; each
// thread divides once and then steps its row and column by the stride, so no
// element pays an integer division.  An item holds fewer than 2^31 elements
// (rows of about 128K elements, or a single row).
MOA_DEV void outer_rows(const BInst &in, const BItem &it, int tid, int nthreads) {
    const int N = in.N, count = it.b * N;
    if (tid >= count) return;
    float *D = in.D + (int64_t)it.a * N;
    const float *A = in.A + it.a;
    int r = tid / N, c = tid - r * N;
    const int dr = nthreads / N, dc = nthreads - dr * N;
    for (int t = tid; t < count; t += nthreads) {
        D[t] = op_apply(in.op, __ldg(A + r), __ldg(in.B + c));
        r += dr;
        c += dc;
        if (c >= N) c -= N, ++r;
    }
}

// One 128 x 128 CUDA-core tile of D = reduce_p(A combine B), 256 threads.
// The panels of A (transposed to [k][m]) and B ([k][n]) stream through four
// shared-memory stages by 4-byte cp.async copies, three panels ahead of the
// one being reduced, so short contractions wait for one load latency rather
// than one per panel.  Elements outside the problem are zero-filled: rows and
// columns past M / N give results that are never stored, and k past K is
// never read (the last panel is reduced over its K % 16 valid k only).
// RH / CH: whether the tile's second 64 rows / columns hold any output; the
// halves a thread would compute outside the problem are skipped (the flags
// are the same for every thread of the tile, so no warp diverges).
template <class Op, bool RH, bool CH>
__device__ __forceinline__ void cc_tile_body(const BInst &in, int tm, int tn, float *As, float *Bs, int tid) {
    const int64_t M = in.M, N = in.N, K = in.K;
    const float *A = in.A, *B = in.B;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)tm * 128, n0 = (int64_t)tn * 128;
    const int a_k = tid % CC_BK, a_m = tid / CC_BK;  // 16 rows per pass
    const int b_n = tid % 128, b_k = tid / 128;      // 2 rows per pass
    const int64_t full = K / CC_BK;
    const int tail = (int)(K - full * CC_BK);
    const int64_t panels = full + (tail ? 1 : 0);
    auto issue = [&](int64_t p) {
        float *as = As + (int)(p & (CC_STAGES - 1)) * CC_PANEL, *bs = Bs + (int)(p & (CC_STAGES - 1)) * CC_PANEL;
        const int64_t k0 = p * CC_BK;
#pragma unroll
        for (int r = 0; r < (RH ? 8 : 4); ++r) {
            const int64_t m = m0 + a_m + r * 16, k = k0 + a_k;
            const bool ok = m < M && k < K;
            ptx::cp_async4_zfill(as + a_k * CC_LD + a_m + r * 16, ok ? A + m * K + k : A, ok);
        }
        if (CH || b_n < 64) {  // warp-uniform: a warp's 32 columns lie in one half
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int64_t k = k0 + b_k + r * 2, n = n0 + b_n;
                const bool ok = k < K && n < N;
                ptx::cp_async4_zfill(bs + (b_k + r * 2) * CC_LD + b_n, ok ? B + k * N + n : B, ok);
            }
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = Op::identity();
#pragma unroll
    for (int s = 0; s < CC_STAGES - 1; ++s) {
        if (s < panels) issue(s);
        ptx::cp_async_commit();  // empty groups keep the count of groups per panel fixed
    }
    for (int64_t p = 0; p < panels; ++p) {
        ptx::cp_async_wait<CC_STAGES - 2>();  // this thread's copies of panel p have landed
        epi_bar();  // everyone's copies of panel p are visible; panel p - 1's stage is free again
        if (p + CC_STAGES - 1 < panels) issue(p + CC_STAGES - 1);
        ptx::cp_async_commit();
        const int buf = (int)(p & (CC_STAGES - 1));
        // two groups of 4 rows / columns half a tile apart: conflict-free 16-byte reads
        const float *as = As + buf * CC_PANEL + ty * 4, *bs = Bs + buf * CC_PANEL + tx * 4;
        if (p < full) {
#pragma unroll
            for (int kk = 0; kk < CC_BK; kk += 2) {
                float a0[8], b0[8], a1[8], b1[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = (i & 3) + (i >> 2) * 64;
                    a0[i] = as[kk * CC_LD + r], a1[i] = as[(kk + 1) * CC_LD + r];
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = (j & 3) + (j >> 2) * 64;
                    b0[j] = bs[kk * CC_LD + c], b1[j] = bs[(kk + 1) * CC_LD + c];
                }
#pragma unroll
                for (int i = 0; i < (RH ? 8 : 4); ++i) {
                    if constexpr (Op::kPacked) {  // two adjacent columns per packed FP32 instruction
#pragma unroll
                        for (int j = 0; j < (CH ? 8 : 4); j += 2)
                            Op::step2x2(acc[i][j], acc[i][j + 1], a0[i], b0[j], b0[j + 1], a1[i], b1[j], b1[j + 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < (CH ? 8 : 4); ++j) acc[i][j] = Op::step2(acc[i][j], a0[i], b0[j], a1[i], b1[j]);
                    }
                }
            }
        } else {
            for (int kk = 0; kk < tail; ++kk) {
                float a0[8], b0[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) a0[i] = as[kk * CC_LD + (i & 3) + (i >> 2) * 64];
#pragma unroll
                for (int j = 0; j < 8; ++j) b0[j] = bs[kk * CC_LD + (j & 3) + (j >> 2) * 64];
#pragma unroll
                for (int i = 0; i < (RH ? 8 : 4); ++i)
#pragma unroll
                    for (int j = 0; j < (CH ? 8 : 4); ++j) acc[i][j] = Op::step(acc[i][j], a0[i], b0[j]);
            }
        }
    }
    ptx::cp_async_wait<0>();  // no copy of this tile outlives it (the last groups are empty)
    // four consecutive columns per store where the rows allow 16-byte stores
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
        if (m >= M) continue;
        float *row = in.D + m * N;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t n = n0 + tx * 4 + h * 64;
            if (in.vec && n + 3 < N) {
                *reinterpret_cast<float4 *>(row + n) = make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2],
                                                                   acc[i][4 * h + 3]);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (n + t < N) row[n + t] = acc[i][4 * h + t];
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    batch_grouped_kernel(const __grid_constant__ BatchParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    float *tcstg = (float *)(smem + STAGES * STAGE_BYTES + 1024);  // TC epilogue staging, per warp
    RingSlot *rs = (RingSlot *)(smem + STAGES * STAGE_BYTES + 1024 + TC_STG_BYTES);
    uint32_t *tmem_slot = (uint32_t *)(bars + NBARS);
    volatile uint32_t *abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t tiles0 = ptx::smem_u32(smem);
    const uint32_t bar0 = ptx::smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto tfull = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto tempty = [&](int b) { return bar0 + 8u * (2 * STAGES + NACC + b); };
    const uint32_t drain = bar0 + 8u * (2 * STAGES + 2 * NACC);
    auto rfull = [&](int s) { return bar0 + 8u * (2 * STAGES + 2 * NACC + 1 + s); };
    auto rempty = [&](int s) { return bar0 + 8u * (2 * STAGES + 2 * NACC + 1 + RING + s); };
    uint32_t *status = &g_batch_status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) ptx::mbar_init(full(s), 1), ptx::mbar_init(empty(s), 1);
        for (int b = 0; b < NACC; ++b) ptx::mbar_init(tfull(b), 1), ptx::mbar_init(tempty(b), kEpiWarps);
        ptx::mbar_init(drain, 1);
        // a slot is released by the producer, the MMA issuer and every epilogue warp
        for (int s = 0; s < RING; ++s) ptx::mbar_init(rfull(s), 1), ptx::mbar_init(rempty(s), 2 + kEpiWarps);
        *abort_flag = 0u;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async_smem();
    }
    if (warp == 2) {
        ptx::tmem_alloc(ptx::smem_u32(tmem_slot), TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ scheduler: queue -> ring
        // Items are claimed and their descriptors copied up to RING slots ahead of
        // the roles that run them; the tensor maps of tensor-core items are
        // prefetched so the producer's first copy of a tile does not wait on them.
        int slot = 0;
        uint32_t rphase = 0;
        for (;;) {
            int item = atomicAdd(p.queue, 1);
            if (item >= p.n_items) item = -1;
            BItem it{};
            BInst in{};
            if (item >= 0) {
                it = p.items[item];
                in = p.inst[it.inst];
                if (it.type == IT_TC) {
                    ptx::prefetch_tmap(p.tmaps + in.tmap + ((it.shape & SH_SHORT) ? 2 : 0));
                    ptx::prefetch_tmap(p.tmaps + in.tmap + 1);
                }
            }
            if (!ptx::mbar_wait(rempty(slot), rphase ^ 1u, abort_flag, status)) break;
            rs[slot].it = it;
            rs[slot].in = in;
            rs[slot].item = item;
            ptx::mbar_arrive(rfull(slot));  // release: the slot's contents before the arrival
            if (++slot == RING) slot = 0, rphase ^= 1u;
            if (item < 0) break;
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------ TMA producer
        int stage = 0, slot = 0;
        uint32_t phase = 0, rphase = 0, issued = 0, last_par = 0;
        bool ok = true;
        for (;;) {
            if (!ptx::mbar_wait(rfull(slot), rphase, abort_flag, status)) {
                ok = false;
                break;
            }
            const int item = rs[slot].item;
            const BItem it = rs[slot].it;
            const int tmap = rs[slot].in.tmap, kslices = (rs[slot].in.K + BK - 1) / BK;
            ptx::mbar_arrive(rempty(slot));
            if (++slot == RING) slot = 0, rphase ^= 1u;
            if (item < 0) break;
            if (it.type != IT_TC) continue;
            const bool narrow = it.shape & SH_NARROW, short_a = it.shape & SH_SHORT;
            // A's maps: [tmap] 128-row boxes, [tmap + 2] 64-row boxes; B's at [tmap + 1]
            const CUtensorMap *ta = p.tmaps + tmap + (short_a ? 2 : 0), *tb = p.tmaps + tmap + 1;
            const uint32_t bytes = (short_a ? A_BYTES / 2 : A_BYTES) + (narrow ? B_HALF : 2 * B_HALF);
            const int b_col = narrow ? it.b * 64 : it.b * BN;
            ptx::fence_tensormap(ta);
            ptx::fence_tensormap(tb);
            for (int i = 0; i < kslices; ++i) {
                if (!ptx::mbar_wait(empty(stage), phase ^ 1u, abort_flag, status)) {
                    ok = false;
                    break;
                }
                const uint32_t sa = tiles0 + stage * STAGE_BYTES, sb = sa + A_BYTES;
                ptx::mbar_arrive_expect_tx(full(stage), bytes);
                ptx::tma_load_3d(sa, ta, full(stage), i * BK, it.a * BM, 0);  // three planes in one box
                for (int j = 0; j < (narrow ? 1 : BN / 64); ++j)
                    ptx::tma_load_3d(sb + j * B_HALF, tb, full(stage), b_col + j * 64, i * BK, 0);
                issued |= 1u << stage;
                last_par = (last_par & ~(1u << stage)) | (phase << stage);
                if (++stage == STAGES) stage = 0, phase ^= 1u;
            }
            if (!ok) break;
        }
        if (!ok) {
            for (int s = 0; s < STAGES; ++s)
                if (issued & (1u << s)) {
                    const uint64_t t0 = globaltimer();
                    while (!ptx::mbar_try_wait(full(s), (last_par >> s) & 1u) && globaltimer() - t0 < kWaitLimitNs) {
                    }
                }
        }
    } else if (warp == 2 && lane == 0) {
        // ------------------------------------------------ MMA issuer
        int stage = 0, abuf = 0, slot = 0;
        uint32_t phase = 0, aphase = 0, rphase = 0;
        bool ok = true;
        for (;;) {
            if (!ptx::mbar_wait(rfull(slot), rphase, abort_flag, status)) {
                ok = false;
                break;
            }
            const int item = rs[slot].item, type = rs[slot].it.type, kslices = (rs[slot].in.K + BK - 1) / BK;
            const int shape = rs[slot].it.shape;
            ptx::mbar_arrive(rempty(slot));
            if (++slot == RING) slot = 0, rphase ^= 1u;
            if (item < 0) break;
            if (type != IT_TC) continue;
            constexpr int SPB = KB / BK;  // stages per promotion block
            const uint32_t idesc = (shape & SH_NARROW) ? IDESC_N64 : IDESC;
            const int a_plane = (shape & SH_SHORT) ? A_PLANE / 2 : A_PLANE;  // a 64-row box packs its planes
            for (int i = 0; i < kslices; ++i) {
                const int j = i % SPB;
                if (j == 0) {
                    if (!ptx::mbar_wait(tempty(abuf), aphase ^ 1u, abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                }
                if (!ptx::mbar_wait(full(stage), phase, abort_flag, status)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t sa = tiles0 + stage * STAGE_BYTES, sb = sa + A_BYTES;
                const uint32_t dacc = tmem + (uint32_t)(abuf * BN);
#pragma unroll
                for (int t = 0; t < TERMS; ++t) {
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        // A: K-major rows of 64 B (8-row atoms 512 B apart), 32 B per k-step;
                        // B: the two 64-column halves B_HALF apart, 16 rows of 128 B per k-step
                        const uint64_t ad = ptx::smem_desc_sw64(sa + term_a(t) * a_plane + k * 32, 512);
                        const uint64_t bd = ptx::smem_desc_sw128(sb + term_b(t) * B_PLANE + k * 2048, B_HALF, 1024);
                        ptx::mma_bf16(dacc, ad, bd, idesc, (j > 0 || t > 0 || k > 0) ? 1u : 0u);
                    }
                }
                ptx::mma_commit(empty(stage));
                if (++stage == STAGES) stage = 0, phase ^= 1u;
                if (j == SPB - 1 || i == kslices - 1) {
                    ptx::mma_commit(tfull(abuf));
                    if (++abuf == NACC) abuf = 0, aphase ^= 1u;
                }
            }
            if (!ok) break;
        }
        if (!ok) {
            ptx::mma_commit(drain);
            const uint64_t t0 = globaltimer();
            while (!ptx::mbar_try_wait(drain, 0) && globaltimer() - t0 < kWaitLimitNs) {
            }
        }
    } else if (warp >= kCtlWarps) {
        // ------------------------------------------------ epilogue warps
        // warp % 4 is the TMEM lane quarter the warp may read; `part` picks its 32 columns
        const int ew = warp - kCtlWarps, q = warp & 3, part = ew / 4, etid = threadIdx.x - 32 * kCtlWarps;
        constexpr int HC = BN / (kEpiWarps / 4);  // columns of the tile per epilogue warp
        int abuf = 0, slot = 0;
        uint32_t aphase = 0, rphase = 0;
        bool ok = true;
        for (;;) {
            int okw = 1;
            if (lane == 0) okw = ptx::mbar_wait(rfull(slot), rphase, abort_flag, status) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) break;
            __syncwarp();  // lane 0's acquire of the slot orders the other lanes' reads too
            const int item = rs[slot].item;
            const BItem it = rs[slot].it;
            const BInst in = rs[slot].in;
            __syncwarp();  // every lane has read the slot before it is released
            if (lane == 0) ptx::mbar_arrive(rempty(slot));
            if (++slot == RING) slot = 0, rphase ^= 1u;
            if (item < 0) break;
            if (it.type == IT_TC) {
                const bool narrow = it.shape & SH_NARROW;
                const bool active = !narrow || part * HC < 64;  // a 128 x 64 tile leaves columns 64..127 unwritten
                float acc[HC];
#pragma unroll
                for (int j = 0; j < HC; ++j) acc[j] = 0.0f;
                for (int kb = 0; kb < in.kblocks; ++kb) {
                    int w = 1;
                    if (lane == 0) w = ptx::mbar_wait(tfull(abuf), aphase, abort_flag, status) ? 1 : 0;
                    w = __shfl_sync(0xffffffffu, w, 0);
                    if (!w) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * BN + part * HC);
                    if (active) {
#pragma unroll
                        for (int c = 0; c < HC; c += 32) {
                            uint32_t r[32];
                            ptx::tmem_ld32(tb + c, r);
                            ptx::tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 32; ++j) acc[c + j] = __fadd_rn(acc[c + j], __uint_as_float(r[j]));
                        }
                    }
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(tempty(abuf));
                    if (++abuf == NACC) abuf = 0, aphase ^= 1u;
                }
                if (!ok) break;
                // the warp's 32 rows x HC columns leave through its own shared-memory
                // slice, 32 columns at a time, so that every store instruction writes
                // 32 consecutive columns of one row (128 contiguous bytes)
                const int64_t row0 = (int64_t)it.a * BM + q * 32;
                const int64_t col0 = (narrow ? (int64_t)it.b * 64 : (int64_t)it.b * BN) + part * HC;
                const int rows_here = (int)min((int64_t)32, in.M - row0);
                float *sl = tcstg + ew * TC_STG_FLOATS;
                if (active && rows_here > 0) {
#pragma unroll
                    for (int c = 0; c < HC; c += 32) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) sl[lane * 33 + j] = acc[c + j];
                        __syncwarp();
                        const int64_t gcol = col0 + c + lane;
                        if (gcol < in.N) {
                            float *dst = in.D + row0 * in.N + gcol;
                            for (int r = 0; r < rows_here; ++r) dst[r * in.N] = sl[r * 33 + lane];
                        }
                        __syncwarp();
                    }
                }
            } else if (it.type == IT_OUT) {
                outer_rows(in, it, etid, kEpiThreads);
            } else {  // IT_FILL
                const int64_t e0 = (int64_t)it.a * in.N, e1 = (int64_t)(it.a + it.b) * in.N;
                const float v = __int_as_float(in.op);
                for (int64_t e = e0 + etid; e < e1; e += kEpiThreads) in.D[e] = v;
            }
        }
        (void)ok;
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// Accumulators of the matrix-vector items: a compensated FP32 dot product
// (Dot2) for split-BF16x3 problems, a semiring reduction for CUDA-core ones.
// Partial accumulators of one output are merged in a fixed order, so a graph
// replay gives the same bits.
struct Dot2Acc {
    float s = 0.0f, c = 0.0f;
    MOA_DEV void step(float a, float b) { dot2_step(s, c, a, b); }
    MOA_DEV void merge(const Dot2Acc &o) { dot2_merge(s, c, o.s, o.c); }
    MOA_DEV Dot2Acc shfl_xor(int o) const {
        Dot2Acc r;
        r.s = __shfl_xor_sync(0xffffffffu, s, o);
        r.c = __shfl_xor_sync(0xffffffffu, c, o);
        return r;
    }
    MOA_DEV float result() const { return __fadd_rn(s, c); }
    MOA_DEV void put(float2 *slot) const { *slot = make_float2(s, c); }
    MOA_DEV static Dot2Acc get(const float2 *slot) {
        Dot2Acc r;
        r.s = slot->x, r.c = slot->y;
        return r;
    }
};
template <class Op> struct SemiringAcc {
    float v = Op::identity();
    MOA_DEV void step(float a, float b) { v = Op::step(v, a, b); }
    MOA_DEV void merge(const SemiringAcc &o) { v = Op::red(v, o.v); }
    MOA_DEV SemiringAcc shfl_xor(int o) const {
        SemiringAcc r;
        r.v = __shfl_xor_sync(0xffffffffu, v, o);
        return r;
    }
    MOA_DEV float result() const { return v; }
    MOA_DEV void put(float2 *slot) const { slot->x = v; }
    MOA_DEV static SemiringAcc get(const float2 *slot) {
        SemiringAcc r;
        r.v = slot->x;
        return r;
    }
};

// Columns of one matrix-vector item at most (M = 1 items); the CTA's other
// threads split the contraction.
constexpr int kGvCols = 128;

// Rows [a, a + b) of an N = 1 product, D[r] = A[r, :] . B[:, 0]: W lanes per
// row (a power of two, about K / 8, at most 32) striding along the
// contraction, four loads of each in flight, so a warp takes 32 / W rows at
// once and short contractions still keep every lane busy; the W partial
// accumulators of a row are merged by shuffles.
template <class Acc>
MOA_DEV void gemv_rows(const BInst &in, const BItem &it) {
    const int64_t K = in.K;
    int W = 1;
    while (W < 32 && 8 * (int64_t)(2 * W) <= K) W *= 2;
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, li = lane % W, G = 32 / W;
    const int r_end = it.a + it.b;
    for (int r0 = it.a + warp * G; r0 < r_end; r0 += 8 * G) {  // uniform over the warp
        const int r = r0 + lane / W;
        Acc acc;
        if (r < r_end) {
            const float *arow = in.A + (int64_t)r * K;
            int64_t k = li;
            for (; k + 3 * W < K; k += 4 * W) {
                float a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = __ldg(arow + k + u * W), b[u] = __ldg(in.B + k + u * W);
#pragma unroll
                for (int u = 0; u < 4; ++u) acc.step(a[u], b[u]);
            }
            for (; k < K; k += W) acc.step(__ldg(arow + k), __ldg(in.B + k));
        }
        for (int o = W / 2; o > 0; o >>= 1) acc.merge(acc.shfl_xor(o));
        if (r < r_end && li == 0) in.D[r] = acc.result();
    }
}

// Columns [a, a + b) (b <= kGvCols) of an M = 1 product, D[n] = A[0, :] .
// B[:, n]: Cw threads across the columns (a power of two >= b) and 256 / Cw
// slices of the contraction, four loads in flight each; the slices' partial
// accumulators are merged by shuffles within a warp and then, in warp order,
// through shared memory.
template <class Acc>
MOA_DEV void gemv_cols(const BInst &in, const BItem &it, float2 *stash) {
    const int64_t K = in.K, N = in.N;
    int Cw = 1;
    while (Cw < it.b) Cw *= 2;
    const int KS = 256 / Cw, cc = threadIdx.x % Cw, kk = threadIdx.x / Cw;
    const int64_t n = it.a + cc;
    Acc acc;
    if (cc < it.b) {
        int64_t k = kk;
        for (; k + 3 * KS < K; k += 4 * KS) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = __ldg(in.A + k + u * KS), b[u] = __ldg(in.B + (k + u * KS) * N + n);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc.step(a[u], b[u]);
        }
        for (; k < K; k += KS) acc.step(__ldg(in.A + k), __ldg(in.B + k * N + n));
    }
    for (int o = 16; o >= Cw; o >>= 1) acc.merge(acc.shfl_xor(o));  // the warp's slices of column cc
    acc.put(stash + threadIdx.x);
    __syncthreads();
    if ((int)threadIdx.x < Cw && cc < it.b) {  // kk == 0
        const int parts = Cw < 32 ? 8 : KS, stride = Cw < 32 ? 32 : Cw;
        for (int q = 1; q < parts; ++q) acc.merge(Acc::get(stash + q * stride + cc));
        in.D[n] = acc.result();
    }
    __syncthreads();
}

template <class Acc>
MOA_DEV void gemv_item(const BInst &in, const BItem &it, float2 *stash) {
    if (it.shape == GV_ROWS) gemv_rows<Acc>(in, it);
    else gemv_cols<Acc>(in, it, stash);
}

// The thin items on their own: matrix-vector items (split-BF16x3 or CUDA-core
// semiring problems with M = 1 or N = 1) and, under schedule bit 3,
// outer-product rows and fills.  A persistent kernel of two CTAs per SM (256
// threads, at most 40 registers, 2 KB of shared memory) on the side stream:
// it needs nothing from the split planes, so its CTAs take SMs while the
// CUDA-core kernels and the split pass run and as the grouped kernel's CTAs
// leave (a grouped CTA, 608 threads of 96 registers, leaves too few registers
// for one of these beside it), all of them pulling work from queues.
__global__ void __launch_bounds__(256, 6)
    batch_gemv_kernel(const BInst *__restrict__ inst, const BItem *__restrict__ items, int n_items, int *queue) {
    __shared__ int s_next;
    __shared__ float2 stash[256];
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int i = s_next;
        __syncthreads();
        if (i >= n_items) break;
        const BItem it = items[i];
        const BInst in = inst[it.inst];
        if (it.type == IT_OUT) {
            outer_rows(in, it, threadIdx.x, blockDim.x);
        } else if (it.type == IT_FILL) {  // rows [a, a + b) of an empty contraction
            const int64_t e0 = (int64_t)it.a * in.N, e1 = (int64_t)(it.a + it.b) * in.N;
            const float v = __int_as_float(in.op);
            for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) in.D[e] = v;
        } else {
            switch (in.op) {
            case -1: gemv_item<Dot2Acc>(in, it, stash); break;  // split-BF16x3 (+,*)
            case CC_MIN_PLUS: gemv_item<SemiringAcc<sr::F32MinPlus>>(in, it, stash); break;
            case CC_MAX_PLUS: gemv_item<SemiringAcc<sr::F32MaxPlus>>(in, it, stash); break;
            case CC_MIN_TIMES: gemv_item<SemiringAcc<sr::F32MinTimes>>(in, it, stash); break;
            case CC_MAX_TIMES: gemv_item<SemiringAcc<sr::F32MaxTimes>>(in, it, stash); break;
            default: gemv_item<SemiringAcc<sr::F32PlusTimes>>(in, it, stash); break;
            }
        }
    }
}

// Grouped split pre-pass: each job is a block of rows of one operand; the
// threads of a CTA walk the job's rows as one flat range of 8-column groups
// (padded rows are a multiple of 8 columns), so short rows still keep every
// thread busy.  A group is two 16-byte loads where the source row allows it
// (cols % 4 == 0: each 4-column half lies wholly inside the row or wholly in
// its padding) and one 16-byte store per plane (plane rows start on 16-byte
// boundaries); each thread has two groups' loads in flight before it stores.
__global__ void __launch_bounds__(256) batch_split_kernel(const SplitJob *__restrict__ jobs, int n_jobs) {
    for (int j = blockIdx.x; j < n_jobs; j += gridDim.x) {
        const SplitJob jb = jobs[j];
        const int gpr = (int)(jb.colsp / 8);  // colsp < 2^31 (checked at plan creation)
        const int count = (int)((jb.r1 - jb.r0) * gpr);  // <= ~8K + one row
        const bool vec = (jb.cols & 3) == 0 && ((uintptr_t)jb.src & 15) == 0;
        auto load = [&](int e, float (&x)[8]) {
            const int rr = e / gpr, c = (e - rr * gpr) * 8;
            const float *src = jb.src + (jb.r0 + rr) * jb.cols + c;
            if (vec) {
                const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float4 v0 = c < jb.cols ? __ldg(reinterpret_cast<const float4 *>(src)) : z;
                const float4 v1 = c + 4 < jb.cols ? __ldg(reinterpret_cast<const float4 *>(src + 4)) : z;
                x[0] = v0.x, x[1] = v0.y, x[2] = v0.z, x[3] = v0.w, x[4] = v1.x, x[5] = v1.y, x[6] = v1.z, x[7] = v1.w;
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) x[t] = c + t < jb.cols ? __ldg(src + t) : 0.0f;
            }
        };
        auto split_store = [&](int e, const float (&x)[8]) {
            const int rr = e / gpr, c = (e - rr * gpr) * 8;
            __align__(16) __nv_bfloat16 hi[8], mid[8], lo[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                hi[t] = __float2bfloat16_rn(x[t]);
                const float r1 = __fsub_rn(x[t], __bfloat162float(hi[t]));
                mid[t] = __float2bfloat16_rn(r1);
                lo[t] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(mid[t])));
            }
            __nv_bfloat16 *dst = jb.dst + (jb.r0 + rr) * jb.colsp + c;
            *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(hi);
            *reinterpret_cast<uint4 *>(dst + jb.plane) = *reinterpret_cast<const uint4 *>(mid);
            *reinterpret_cast<uint4 *>(dst + 2 * jb.plane) = *reinterpret_cast<const uint4 *>(lo);
        };
        for (int e = threadIdx.x; e < count; e += 2 * blockDim.x) {
            const int e1 = e + blockDim.x;
            float x0[8], x1[8];
            load(e, x0);
            if (e1 < count) load(e1, x1);
            split_store(e, x0);
            if (e1 < count) split_store(e1, x1);
        }
    }
}

// CUDA-core items on their own: a persistent kernel of two 256-thread CTAs
// per SM (16 warps, against the grouped kernel's 8 epilogue warps per SM)
// pulling CC items from a second queue counter.
template <class Op, bool RH, bool CH>
__global__ void __launch_bounds__(256, 2)
    batch_cc_kernel(const BInst *__restrict__ inst, const BItem *__restrict__ items, int n_items, int *queue) {
    extern __shared__ __align__(16) float cc_smem[];  // CC_BYTES
    __shared__ int s_next;
    float *ccA = cc_smem, *ccB = cc_smem + CC_STAGES * CC_PANEL;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int i = s_next;
        __syncthreads();  // every thread has read s_next before it is overwritten
        if (i >= n_items) break;
        const BItem it = items[i];
        cc_tile_body<Op, RH, CH>(inst[it.inst], it.a, it.b, ccA, ccB, (int)threadIdx.x);
    }
}

int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

int sm_count_dev() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

struct Problem {
    int type, op;
    int64_t M, N, K;
    const float *A, *B;
    float *D;
};

moa_status count_elems(int rank, const int64_t *shape, int64_t *n) {
    int64_t c = 1;
    for (int k = 0; k < rank; ++k) {
        if (shape[k] < 0) return MOA_ERR_OVERFLOW;
        if (shape[k] != 0 && c > INT64_MAX / shape[k]) return MOA_ERR_OVERFLOW;
        c *= shape[k];
    }
    *n = c;
    return MOA_OK;
}

// Which halves of a CUDA-core tile hold output: bit 1 rows 64..127, bit 0
// columns 64..127 (the kernel variant that runs the item).
int cc_quadrants(const Problem &p, const BItem &it) {
    return ((int64_t)it.a * 128 + 64 < p.M ? 2 : 0) | ((int64_t)it.b * 128 + 64 < p.N ? 1 : 0);
}

template <class Op, bool RH, bool CH>
cudaError_t launch_cc(int grid, const BInst *inst, const BItem *items, int cnt, int *queue, cudaStream_t s) {
    static std::once_flag once;  // the dynamic shared-memory limit of this instance, raised once
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(batch_cc_kernel<Op, RH, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, CC_BYTES);
    });
    if (attr != cudaSuccess) return attr;
    batch_cc_kernel<Op, RH, CH><<<grid, 256, CC_BYTES, s>>>(inst, items, cnt, queue);
    return cudaSuccess;
}

template <class Op>
cudaError_t launch_cc_quad(int q, int grid, const BInst *inst, const BItem *items, int cnt, int *queue,
                           cudaStream_t s) {
    switch (q) {
    case 3: return launch_cc<Op, true, true>(grid, inst, items, cnt, queue, s);
    case 2: return launch_cc<Op, true, false>(grid, inst, items, cnt, queue, s);
    case 1: return launch_cc<Op, false, true>(grid, inst, items, cnt, queue, s);
    default: return launch_cc<Op, false, false>(grid, inst, items, cnt, queue, s);
    }
}

// Validate one problem like its single call and reduce it to (type, op, M, N, K).
moa_status classify(const moa_problem &q, Problem *out) {
    if (!q.shapeA && q.rankA > 0) return MOA_ERR_NULL;
    if (!q.shapeB && q.rankB > 0) return MOA_ERR_NULL;
    if (q.rankA < 0 || q.rankB < 0 || q.rankA > 8 || q.rankB > 8) return MOA_ERR_RANK;
    if (q.dtype != MOA_F32 || q.out_dtype != MOA_F32) return MOA_ERR_UNSUPPORTED;
    Problem p{};
    p.A = (const float *)q.A, p.B = (const float *)q.B, p.D = (float *)q.out;
    moa_status st;
    if (q.kind == 1) {  // outer, Eq. (1)
        if (q.combine < MOA_OP_ADD || q.combine > MOA_OP_MAX) return MOA_ERR_UNSUPPORTED;
        if ((st = count_elems(q.rankA, q.shapeA, &p.M)) != MOA_OK) return st;
        if ((st = count_elems(q.rankB, q.shapeB, &p.N)) != MOA_OK) return st;
        p.type = IT_OUT, p.op = q.combine, p.K = 0;
    } else if (q.kind == 0) {  // inner, Eq. (2)
        if (q.rankA < 1 || q.rankB < 1) return MOA_ERR_RANK;
        int64_t nA, nB;
        if ((st = count_elems(q.rankA, q.shapeA, &nA)) != MOA_OK) return st;
        if ((st = count_elems(q.rankB, q.shapeB, &nB)) != MOA_OK) return st;
        if (q.shapeA[q.rankA - 1] != q.shapeB[0]) return MOA_ERR_SHAPE_MISMATCH;
        if ((st = count_elems(q.rankA - 1, q.shapeA, &p.M)) != MOA_OK) return st;
        if ((st = count_elems(q.rankB - 1, q.shapeB + 1, &p.N)) != MOA_OK) return st;
        p.K = q.shapeA[q.rankA - 1];
        if (q.reduce == MOA_OP_ADD && q.combine == MOA_OP_MUL && q.form == MOA_FORM_BF16X3) {
            p.type = IT_TC;
        } else if (q.form != MOA_FORM_NATIVE) {
            return MOA_ERR_UNSUPPORTED;
        } else if (q.reduce == MOA_OP_ADD && q.combine == MOA_OP_MUL) {
            p.type = IT_CC, p.op = CC_PLUS_TIMES;
        } else if ((q.reduce == MOA_OP_MIN || q.reduce == MOA_OP_MAX) &&
                   (q.combine == MOA_OP_ADD || q.combine == MOA_OP_MUL)) {
            p.type = IT_CC;
            p.op = q.reduce == MOA_OP_MIN ? (q.combine == MOA_OP_ADD ? CC_MIN_PLUS : CC_MIN_TIMES)
                                          : (q.combine == MOA_OP_ADD ? CC_MAX_PLUS : CC_MAX_TIMES);
        } else {
            return MOA_ERR_UNSUPPORTED;
        }
        if (p.K == 0) {  // empty contraction: the reduce identity
            p.type = IT_FILL;
            const float v = q.reduce == MOA_OP_MIN ? INFINITY : (q.reduce == MOA_OP_MAX ? -INFINITY : 0.0f);
            std::memcpy(&p.op, &v, 4);
        }
    } else {
        return MOA_ERR_INVALID;
    }
    if (p.M != 0 && p.N > INT64_MAX / p.M) return MOA_ERR_OVERFLOW;
    if (p.M >= (1ll << 31) || p.N >= (1ll << 31) || p.K >= (1ll << 31)) return MOA_ERR_OVERFLOW;
    if (p.M * p.N > 0) {
        if (!p.D) return MOA_ERR_NULL;
        if (p.type != IT_FILL && (!p.A || !p.B)) return MOA_ERR_NULL;
    }
    if ((uintptr_t)p.A % 4 || (uintptr_t)p.B % 4 || (uintptr_t)p.D % 4) return MOA_ERR_ALIGNMENT;
    *out = p;
    return MOA_OK;
}

// estimated microseconds of one item on one SM (orders the queue)
double item_cost(const Problem &p, const BItem &it) {
    switch (it.type) {
    case IT_TC: {  // by the bytes a stage loads: A's share and B's share
        const double f = (((it.shape & SH_SHORT) ? 0.5 : 1.0) + ((it.shape & SH_NARROW) ? 0.5 : 1.0)) / 2.0;
        return 1.0 + 0.26 * (double)((p.K + KB - 1) / KB) * TERMS * f;
    }
    case IT_CC: return 1.0 + 128.0 * 128.0 * (double)p.K / 79000.0;
    case IT_GEMV: return 0.5 + (double)it.b * (double)p.K / 40000.0;
    default: return 0.5 + (double)it.b * (double)p.N * 4.0 / 43000.0;
    }
}

std::string gpu_signature() {
    int dev = 0, drv = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    cudaDriverGetVersion(&drv);
    std::ostringstream o;
    o << prop.name << "|sm" << prop.multiProcessorCount << "|drv" << drv;
    std::string s = o.str();
    for (auto &c : s)
        if (c == ' ') c = '_';
    return s;
}

std::string tune_cache_path() {
    const char *e = std::getenv("MOA_TUNE_CACHE");
    if (e && *e) return e;
    const char *h = std::getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/moa_autotune.txt";
}

int tune_mode() {  // 0 off, 1 cached, 2 force
    const char *e = std::getenv("MOA_AUTOTUNE");
    if (!e) return 1;
    if (!std::strcmp(e, "off")) return 0;
    if (!std::strcmp(e, "force")) return 2;
    return 1;
}

// Schedules the autotuner picks from, three bits: bit 0 the grouped queue's
// order (0 longest first over all its items, 1 tensor-core tiles first);
// bit 1 the tensor-core tile shapes (0 every tile 128 x 128; 1 a 64-row A
// box for problems with M <= 64 and a 128 x 64 last column tile where at most
// 64 columns remain); bit 2 the CUDA-core kernels one after another on the
// caller's stream (0) or side by side on streams of their own, the largest
// first, so one kernel's tail overlaps the next (1); bit 3 the outer-product
// and fill items on the grouped kernel's epilogue warps (0) or in the
// thin-item kernel beside it (1), away from the tensor-core tile epilogues.
// Schedules with bit 1 exist only for plans where a tile changes shape, with
// bit 2 only for plans with more than one CUDA-core kernel, with bit 3 only
// for plans with outer-product or fill items.
constexpr int kPolicies = 16;

}  // namespace
}  // namespace moa

using namespace moa;

struct moa_batch_plan {
    int device = 0;
    int count = 0;
    std::vector<Problem> probs;
    std::vector<BItem> items;      // unordered, tensor-core tiles 128 x 128
    std::vector<BItem> tc_shaped;  // the tensor-core tiles of the shaped schedules
    bool shapes_differ = false;    // some tile of tc_shaped is not 128 x 128
    int n_items = 0, n_jobs = 0;
    int n_grouped = 0, n_cc = 0;  // items in the grouped kernel / the CUDA-core kernels (set by the policy)
    int n_gv = 0;                 // matrix-vector items (after the CUDA-core items in d_cc_items)
    int cc_off[kCcGroups] = {}, cc_cnt[kCcGroups] = {};  // CUDA-core items of each kernel in d_cc_items
    double work = 0.0;
    std::string signature;
    int policy = -1;
    // device memory owned by the plan
    BInst *d_inst = nullptr;
    BItem *d_items = nullptr;
    BItem *d_cc_items = nullptr;
    CUtensorMap *d_tmaps = nullptr;
    SplitJob *d_jobs = nullptr;
    int *d_queue = nullptr;
    void *d_ws = nullptr;
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side = nullptr;  // the split pre-pass runs here, beside the CUDA-core kernels, then
                                  // the thin-item kernel, sharing the SMs with the others
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_gv = nullptr;
    // under the schedules that run the CUDA-core kernels side by side: their streams and join events
    cudaStream_t cc_streams[kCcGroups] = {};
    cudaEvent_t cc_join[kCcGroups] = {};
    int policy_now = 0;  // the schedule whose order is uploaded (what enqueue launches)
    cudaGraphExec_t exec = nullptr;
    std::mutex mu;
};

namespace moa {
namespace {

int cc_group(const moa_batch_plan &pl, const BItem &it) {
    const Problem &p = pl.probs[it.inst];
    return 4 * p.op + cc_quadrants(p, it);
}

// The grouped kernel's queue and the CUDA-core kernels' queues for a policy.
void order_items(const moa_batch_plan &pl, int policy, std::vector<BItem> &grouped, std::vector<BItem> &cc,
                 std::vector<BItem> &gv) {
    const bool shaped = (policy & 2) != 0;
    std::vector<BItem> all;
    all.reserve(pl.items.size());
    for (const BItem &it : pl.items)
        if (!(shaped && it.type == IT_TC)) all.push_back(it);
    if (shaped) all.insert(all.end(), pl.tc_shaped.begin(), pl.tc_shaped.end());
    std::vector<double> cost(all.size());
    for (size_t i = 0; i < all.size(); ++i) cost[i] = item_cost(pl.probs[all[i].inst], all[i]);
    std::vector<int> idx(all.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    grouped.clear();
    cc.clear();
    gv.clear();
    std::vector<int> tc, ccs, other;
    const bool thin_out = (policy & 8) != 0;  // outer-product and fill items in the thin-item kernel
    auto to_thin = [&](const BItem &it) {
        return it.type == IT_GEMV || (thin_out && (it.type == IT_OUT || it.type == IT_FILL));
    };
    for (int i : idx) {
        if (to_thin(all[i]))
            gv.push_back(all[i]);  // the thin-item kernel's queue, longest first
        else
            (all[i].type == IT_TC ? tc : all[i].type == IT_CC ? ccs : other).push_back(i);
    }
    if ((policy & 1) == 0) {
        for (int i : idx)
            if (all[i].type != IT_CC && !to_thin(all[i])) grouped.push_back(all[i]);
    } else {
        for (int i : tc) grouped.push_back(all[i]);
        for (int i : other) grouped.push_back(all[i]);
    }
    for (int g = 0; g < kCcGroups; ++g)  // by kernel (operator, tile halves), longest first within each
        for (int i : ccs)
            if (cc_group(pl, all[i]) == g) cc.push_back(all[i]);
}

moa_status upload_order(moa_batch_plan *pl, int policy, cudaStream_t s) {
    std::vector<BItem> grouped, cc, gv;
    order_items(*pl, policy, grouped, cc, gv);
    pl->policy_now = policy;
    pl->n_grouped = (int)grouped.size();
    pl->n_cc = (int)cc.size();
    pl->n_gv = (int)gv.size();
    for (int g = 0; g < kCcGroups; ++g) pl->cc_cnt[g] = 0;
    for (const BItem &it : cc) ++pl->cc_cnt[cc_group(*pl, it)];
    cc.insert(cc.end(), gv.begin(), gv.end());  // the matrix-vector items follow the CUDA-core tiles
    for (int g = 0, off = 0; g < kCcGroups; ++g) pl->cc_off[g] = off, off += pl->cc_cnt[g];
    if (!grouped.empty() && cudaMemcpyAsync(pl->d_items, grouped.data(), grouped.size() * sizeof(BItem),
                                            cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MOA_ERR_CUDA;
    if (!cc.empty() &&
        cudaMemcpyAsync(pl->d_cc_items, cc.data(), cc.size() * sizeof(BItem), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MOA_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
}

// The work of one execute, enqueued on s (also what the graph captures).
cudaError_t enqueue(moa_batch_plan *pl, cudaStream_t s) {
    static std::mutex attr_mu;  // the grouped kernel's shared-memory attribute, set once (retried on failure)
    static bool attr = false;
    {
        std::lock_guard<std::mutex> lk(attr_mu);
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(batch_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
            if (e != cudaSuccess) return e;
            attr = true;
        }
    }
    if (pl->n_grouped > 0 || pl->n_cc > 0 || pl->n_gv > 0) {
        cudaError_t e = cudaMemsetAsync(pl->d_queue, 0, (2 + kCcGroups) * sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    // the split pre-pass (memory bound) on the plan's side stream, beside the
    // CUDA-core kernels (ALU bound); the grouped kernel waits for both
    const bool fork = pl->n_jobs > 0 && pl->n_cc > 0;
    const bool cc_side_by_side = (pl->policy_now & 4) != 0;
    if (fork || cc_side_by_side || pl->n_gv > 0) {
        const cudaError_t e = cudaEventRecord(pl->ev_fork, s);
        if (e != cudaSuccess) return e;
    }
    if (fork) {
        cudaError_t e = cudaStreamWaitEvent(pl->side, pl->ev_fork, 0);
        if (e != cudaSuccess) return e;
        const int blocks = std::min(pl->n_jobs, sm_count_dev() * 8);
        batch_split_kernel<<<blocks, 256, 0, pl->side>>>(pl->d_jobs, pl->n_jobs);
        e = cudaEventRecord(pl->ev_join, pl->side);
        if (e != cudaSuccess) return e;
    }
    // the thin items need nothing from the other kernels: on the side stream
    // (after the split pass when it runs there), beside the others
    if (pl->n_gv > 0) {
        cudaError_t e = fork ? cudaSuccess : cudaStreamWaitEvent(pl->side, pl->ev_fork, 0);
        if (e != cudaSuccess) return e;
        const int grid = std::min(2 * sm_count_dev(), pl->n_gv);
        batch_gemv_kernel<<<grid, 256, 0, pl->side>>>(pl->d_inst, pl->d_cc_items + pl->n_cc, pl->n_gv,
                                                      pl->d_queue + 1 + kCcGroups);
        e = cudaEventRecord(pl->ev_gv, pl->side);
        if (e != cudaSuccess) return e;
    }
    // one persistent kernel per (operator, occupied tile halves) present, each with its own queue;
    // side by side: each on a stream of its own, the kernel with the most items launched first
    int order[kCcGroups], n_used = 0;
    for (int g = 0; g < kCcGroups; ++g)
        if (pl->cc_cnt[g] > 0) order[n_used++] = g;
    if (cc_side_by_side)
        std::stable_sort(order, order + n_used, [&](int a, int b) { return pl->cc_cnt[a] > pl->cc_cnt[b]; });
    for (int k = 0; k < n_used; ++k) {
        const int g = order[k], cnt = pl->cc_cnt[g];
        const int grid = std::min(2 * sm_count_dev(), cnt);
        const BItem *items = pl->d_cc_items + pl->cc_off[g];
        int *queue = pl->d_queue + 1 + g;
        const int q = g % 4;
        cudaStream_t cs = s;
        if (cc_side_by_side) {
            cs = pl->cc_streams[k];
            const cudaError_t e = cudaStreamWaitEvent(cs, pl->ev_fork, 0);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e;
        switch (g / 4) {
        case CC_MIN_PLUS: e = launch_cc_quad<sr::F32MinPlus>(q, grid, pl->d_inst, items, cnt, queue, cs); break;
        case CC_MAX_PLUS: e = launch_cc_quad<sr::F32MaxPlus>(q, grid, pl->d_inst, items, cnt, queue, cs); break;
        case CC_MIN_TIMES: e = launch_cc_quad<sr::F32MinTimes>(q, grid, pl->d_inst, items, cnt, queue, cs); break;
        case CC_MAX_TIMES: e = launch_cc_quad<sr::F32MaxTimes>(q, grid, pl->d_inst, items, cnt, queue, cs); break;
        default: e = launch_cc_quad<sr::F32PlusTimes>(q, grid, pl->d_inst, items, cnt, queue, cs); break;
        }
        if (e != cudaSuccess) return e;
        if (cc_side_by_side) {
            e = cudaEventRecord(pl->cc_join[k], cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pl->cc_join[k], 0);
            if (e != cudaSuccess) return e;
        }
    }
    if (fork) {
        const cudaError_t e = cudaStreamWaitEvent(s, pl->ev_join, 0);
        if (e != cudaSuccess) return e;
    } else if (pl->n_jobs > 0) {
        const int blocks = std::min(pl->n_jobs, sm_count_dev() * 8);
        batch_split_kernel<<<blocks, 256, 0, s>>>(pl->d_jobs, pl->n_jobs);
    }
    if (pl->n_grouped > 0) {
        BatchParams bp{pl->d_inst, pl->d_items, pl->n_grouped, pl->d_queue, pl->d_tmaps};
        const int grid = std::min(sm_count_dev(), std::max(1, pl->n_grouped));
        batch_grouped_kernel<<<grid, kThreads, SMEM, s>>>(bp);
    }
    if (pl->n_gv > 0) {
        const cudaError_t e = cudaStreamWaitEvent(s, pl->ev_gv, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

moa_status autotune(moa_batch_plan *pl, cudaStream_t s) {
    const char *force = std::getenv("MOA_BATCH_SCHEDULE");  // a fixed schedule (0..kPolicies-1), no timing
    const int forced = force && force[0] >= '0' && force[0] <= '9' ? std::atoi(force) : -1;
    if (forced >= 0 && forced < kPolicies) {
        pl->policy = forced;
        return upload_order(pl, pl->policy, s);
    }
    const int mode = tune_mode();
    const std::string key = gpu_signature() + "|s7|" + pl->signature;  // s7: the schedules listed at kPolicies
    if (mode == 0) {
        pl->policy = 0;
        return upload_order(pl, 0, s);
    }
    if (mode == 1) {  // cached choice for this GPU and plan signature
        std::ifstream f(tune_cache_path());
        std::string k;
        int pol;
        double t;
        while (f >> k >> pol >> t)
            if (k == key && pol >= 0 && pol < kPolicies) {
                pl->policy = pol;
                return upload_order(pl, pol, s);
            }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MOA_ERR_CUDA;
    double best = 1e30;
    int best_pol = 0;
    int n_cc_kernels = 0;
    bool has_out = false;
    for (const BItem &it : pl->items) has_out |= it.type == IT_OUT || it.type == IT_FILL;
    {
        bool used[kCcGroups] = {};
        for (const BItem &it : pl->items)
            if (it.type == IT_CC) used[cc_group(*pl, it)] = true;
        for (bool u : used) n_cc_kernels += u;
    }
    for (int pol = 0; pol < kPolicies; ++pol) {
        if ((pol & 2) && !pl->shapes_differ) continue;  // the same tiles as pol & ~2
        if ((pol & 4) && n_cc_kernels < 2) continue;     // nothing to run side by side
        if ((pol & 8) && !has_out) continue;             // no outer-product or fill item to move
        moa_status st = upload_order(pl, pol, s);
        if (st != MOA_OK) return st;
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            if (enqueue(pl, s) != cudaSuccess) return MOA_ERR_CUDA;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return MOA_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best_ms = std::min(best_ms, ms);
        }
        if (best_ms < best) best = best_ms, best_pol = pol;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->policy = best_pol;
    {
        const std::string path = tune_cache_path();
        const size_t slash = path.find_last_of('/');
        if (slash != std::string::npos && slash > 0)  // the cache directory, if missing (best effort)
            mkdir(path.substr(0, slash).c_str(), 0755);
        std::ofstream f(path, std::ios::app);
        if (f) f << key << " " << best_pol << " " << best * 1000.0 << "\n";
    }
    return upload_order(pl, best_pol, s);
}

// The streams and join events of the side-by-side CUDA-core kernels (one per kernel present).
bool make_cc_streams(moa_batch_plan *pl) {
    bool used[kCcGroups] = {};
    for (const BItem &it : pl->items)
        if (it.type == IT_CC) used[cc_group(*pl, it)] = true;
    int k = 0;
    for (int g = 0; g < kCcGroups; ++g)
        if (used[g]) {
            if (cudaStreamCreateWithFlags(&pl->cc_streams[k], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&pl->cc_join[k], cudaEventDisableTiming) != cudaSuccess)
                return false;
            ++k;
        }
    return true;
}

void plan_free(moa_batch_plan *pl) {
    if (!pl) return;
    cudaDeviceSynchronize();
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    if (pl->side) cudaStreamDestroy(pl->side);
    for (int g = 0; g < kCcGroups; ++g) {
        if (pl->cc_streams[g]) cudaStreamDestroy(pl->cc_streams[g]);
        if (pl->cc_join[g]) cudaEventDestroy(pl->cc_join[g]);
    }
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    if (pl->ev_gv) cudaEventDestroy(pl->ev_gv);
    cudaFree(pl->d_inst);
    cudaFree(pl->d_items);
    cudaFree(pl->d_cc_items);
    cudaFree(pl->d_tmaps);
    cudaFree(pl->d_jobs);
    cudaFree(pl->d_queue);
    cudaFree(pl->d_ws);
    delete pl;
}

}  // namespace
}  // namespace moa

extern "C" {

moa_status moa_batch_plan_create(int count, const moa_problem *problems, moa_batch_plan **plan, int *bad_index) {
    if (bad_index) *bad_index = -1;
    if (!plan) return MOA_ERR_NULL;
    *plan = nullptr;
    if (count < 0 || (count > 0 && !problems)) return count < 0 ? MOA_ERR_INVALID : MOA_ERR_NULL;
    moa_batch_plan *pl = new moa_batch_plan();
    cudaGetDevice(&pl->device);
    pl->count = count;
    pl->probs.resize(count);
    for (int i = 0; i < count; ++i) {
        moa_status st = classify(problems[i], &pl->probs[i]);
        if (st != MOA_OK) {
            if (bad_index) *bad_index = i;
            delete pl;
            return st;
        }
        // a matrix-vector product: a tile would be at most 1/64 (tensor cores) or 1/128 (CUDA cores)
        // full, so the thin-item kernel takes it straight from the FP32 operands (no split planes);
        // op -1 marks the split-BF16x3 (+,*) form, otherwise the CUDA-core operator
        Problem &q = pl->probs[i];
        if ((q.type == IT_TC || q.type == IT_CC) && (q.M == 1 || q.N == 1)) {
            if (q.type == IT_TC) q.op = -1;
            q.type = IT_GEMV;
        }
    }
    // every problem well formed: then its operands and result must be memory of this device
    for (int i = 0; i < count; ++i) {
        const Problem &p = pl->probs[i];
        if (p.M * p.N == 0) continue;
        const void *used[3] = {p.type != IT_FILL ? p.A : nullptr, p.type != IT_FILL ? p.B : nullptr, p.D};
        const moa_status st = check_device_ptrs(used, 3);
        if (st != MOA_OK) {
            if (bad_index) *bad_index = i;
            delete pl;
            return st;
        }
    }
    // descriptors, split planes, tensor maps, items
    std::vector<BInst> inst(count);
    std::vector<SplitJob> jobs;
    std::vector<size_t> ws_off(count, 0);
    size_t ws_bytes = 0;
    int n_tc = 0;
    for (int i = 0; i < count; ++i) {
        const Problem &p = pl->probs[i];
        if (p.type == IT_TC && p.M * p.N > 0) {
            const size_t bytes = (size_t)3 * (size_t)(p.M * round8(p.K) + p.K * round8(p.N)) * 2;
            ws_off[i] = ws_bytes;
            ws_bytes += (bytes + 255) / 256 * 256;
            ++n_tc;
        }
    }
    std::vector<CUtensorMap> tmaps((size_t)3 * n_tc);  // per problem: A (128-row boxes), B, A (64-row boxes)
    if (ws_bytes && cudaMalloc(&pl->d_ws, ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        plan_free(pl);
        return MOA_ERR_WORKSPACE;
    }
    int t = 0;
    uint64_t sig_tc = 0, sig_cc = 0, sig_out = 0;
    for (int i = 0; i < count; ++i) {
        const Problem &p = pl->probs[i];
        BInst &b = inst[i];
        b.type = p.type, b.op = p.op, b.M = (int)p.M, b.N = (int)p.N, b.K = (int)p.K;
        b.kblocks = (int)((p.K + KB - 1) / KB);  // promotion blocks
        b.A = p.A, b.B = p.B, b.D = p.D, b.tmap = -1;
        b.vec = ((uintptr_t)p.D % 16 == 0) && (p.N % 4 == 0);
        if (p.M * p.N == 0) continue;
        if (p.type == IT_TC) {
            const int64_t Kp = round8(p.K), Np = round8(p.N);
            __nv_bfloat16 *pa = (__nv_bfloat16 *)((uint8_t *)pl->d_ws + ws_off[i]);
            __nv_bfloat16 *pb = pa + 3 * p.M * Kp;
            if (!make_tmap(&tmaps[3 * t], pa, (uint64_t)p.K, (uint64_t)p.M, 3, (uint64_t)Kp * 2, (uint64_t)(Kp * p.M * 2),
                           BK, BM, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, CU_TENSOR_MAP_SWIZZLE_64B, PLANES) ||
                !make_tmap(&tmaps[3 * t + 1], pb, (uint64_t)p.N, (uint64_t)p.K, 3, (uint64_t)Np * 2,
                           (uint64_t)(Np * p.K * 2), 64, BK, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, CU_TENSOR_MAP_SWIZZLE_128B,
                           PLANES) ||
                !make_tmap(&tmaps[3 * t + 2], pa, (uint64_t)p.K, (uint64_t)p.M, 3, (uint64_t)Kp * 2,
                           (uint64_t)(Kp * p.M * 2), BK, BM / 2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           CU_TENSOR_MAP_SWIZZLE_64B, PLANES)) {
                if (bad_index) *bad_index = i;
                plan_free(pl);
                return MOA_ERR_CUDA;
            }
            b.tmap = 3 * t++;
            // split jobs: blocks of rows of about 64K elements
            const int64_t ra = std::max<int64_t>(1, 65536 / Kp), rb = std::max<int64_t>(1, 65536 / Np);
            for (int64_t r = 0; r < p.M; r += ra)
                jobs.push_back(SplitJob{p.A, pa, p.K, Kp, p.M * Kp, r, std::min(p.M, r + ra)});
            for (int64_t r = 0; r < p.K; r += rb)
                jobs.push_back(SplitJob{p.B, pb, p.N, Np, p.K * Np, r, std::min(p.K, r + rb)});
            const int nt = (int)((p.N + BN - 1) / BN);
            const bool short_a = p.M <= BM / 2, narrow_last = p.N - (int64_t)(nt - 1) * BN <= 64;
            for (int tm = 0; tm < (p.M + BM - 1) / BM; ++tm)
                for (int tn = 0; tn < nt; ++tn) {
                    pl->items.push_back(BItem{i, IT_TC, tm, tn});
                    const bool narrow = narrow_last && tn == nt - 1;  // the last tile: a 64-column tile
                    const int shape = (narrow ? SH_NARROW : 0) | (short_a ? SH_SHORT : 0);
                    pl->tc_shaped.push_back(BItem{i, IT_TC, tm, narrow ? 2 * tn : tn, shape});
                    pl->shapes_differ |= shape != 0;
                }
            pl->work += 2.0 * p.M * p.N * p.K;
            sig_tc += (uint64_t)p.M * p.N * p.K;
        } else if (p.type == IT_GEMV) {  // about 64K products per item
            if (p.N == 1) {
                const int64_t rows = std::max<int64_t>(1, 65536 / p.K);
                for (int64_t r = 0; r < p.M; r += rows)
                    pl->items.push_back(BItem{i, IT_GEMV, (int)r, (int)std::min(rows, p.M - r), GV_ROWS});
            } else {
                for (int64_t c = 0; c < p.N; c += kGvCols)
                    pl->items.push_back(BItem{i, IT_GEMV, (int)c, (int)std::min<int64_t>(kGvCols, p.N - c), GV_COLS});
            }
            pl->work += 2.0 * p.M * p.N * p.K;
            sig_tc += (uint64_t)p.M * p.N * p.K;
        } else if (p.type == IT_CC) {
            for (int tm = 0; tm < (p.M + 127) / 128; ++tm)
                for (int tn = 0; tn < (p.N + 127) / 128; ++tn) pl->items.push_back(BItem{i, IT_CC, tm, tn});
            pl->work += 2.0 * p.M * p.N * p.K;
            sig_cc += (uint64_t)p.M * p.N * p.K;
        } else {  // OUT and FILL: blocks of rows of about 128K elements
            const int64_t rows = std::max<int64_t>(1, 131072 / std::max<int64_t>(1, p.N));
            for (int64_t r = 0; r < p.M; r += rows)
                pl->items.push_back(BItem{i, p.type, (int)r, (int)std::min(rows, p.M - r)});
            pl->work += (double)p.M * p.N;
            sig_out += (uint64_t)p.M * p.N;
        }
    }
    pl->n_items = (int)pl->items.size();
    pl->n_jobs = (int)jobs.size();
    {
        std::ostringstream o;  // plan signature: counts and work, bucketed to two significant digits
        auto b2 = [](uint64_t v) {
            int e = 0;
            while (v >= 100) v /= 10, ++e;
            return std::to_string(v) + "e" + std::to_string(e);
        };
        o << "n" << count << "_i" << b2(pl->n_items) << "_tc" << b2(sig_tc) << "_cc" << b2(sig_cc) << "_o" << b2(sig_out);
        pl->signature = o.str();
    }
    bool ok = cudaMalloc(&pl->d_inst, std::max<size_t>(1, inst.size()) * sizeof(BInst)) == cudaSuccess &&
              cudaMalloc(&pl->d_items, std::max<size_t>(1, pl->items.size()) * sizeof(BItem)) == cudaSuccess &&
              cudaMalloc(&pl->d_cc_items, std::max<size_t>(1, pl->items.size()) * sizeof(BItem)) == cudaSuccess &&
              cudaMalloc(&pl->d_tmaps, std::max<size_t>(1, tmaps.size()) * sizeof(CUtensorMap)) == cudaSuccess &&
              cudaMalloc(&pl->d_jobs, std::max<size_t>(1, jobs.size()) * sizeof(SplitJob)) == cudaSuccess &&
              cudaMalloc(&pl->d_queue, (2 + kCcGroups) * sizeof(int)) == cudaSuccess;  // grouped, CUDA-core, matrix-vector
    if (!ok) {
        cudaGetLastError();
        plan_free(pl);
        return MOA_ERR_WORKSPACE;
    }
    ok = (inst.empty() || cudaMemcpy(pl->d_inst, inst.data(), inst.size() * sizeof(BInst), cudaMemcpyHostToDevice) == cudaSuccess) &&
         (tmaps.empty() || cudaMemcpy(pl->d_tmaps, tmaps.data(), tmaps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) == cudaSuccess) &&
         (jobs.empty() || cudaMemcpy(pl->d_jobs, jobs.data(), jobs.size() * sizeof(SplitJob), cudaMemcpyHostToDevice) == cudaSuccess);
    if (!ok || cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_gv, cudaEventDisableTiming) != cudaSuccess || !make_cc_streams(pl)) {
        plan_free(pl);
        return MOA_ERR_CUDA;
    }
    *plan = pl;
    return MOA_OK;
}

// A failed CUDA call of an execute; with MOA_DEBUG set its error is printed.
static moa_status batch_cuda_failed(cudaError_t e, const char *where) {
    if (std::getenv("MOA_DEBUG")) std::fprintf(stderr, "moa batch: %s: %s\n", where, cudaGetErrorString(e));
    return MOA_ERR_CUDA;
}

moa_status moa_batch_execute(moa_batch_plan *plan, moa_stream stream) {
    if (!plan) return MOA_ERR_NULL;
    std::lock_guard<std::mutex> lk(plan->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->policy < 0) {  // first execute: pick the item order (autotuner), then capture
        moa_status st = autotune(plan, s);
        if (st != MOA_OK) return st;
    }
    if (!plan->exec) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MOA_ERR_CUDA;
        cudaError_t e = enqueue(plan, plan->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(plan->cap_stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return batch_cuda_failed(e != cudaSuccess ? e : e2, "capture");
        }
        e = cudaGraphInstantiate(&plan->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            plan->exec = nullptr;
            return batch_cuda_failed(e, "instantiate");
        }
    }
    const cudaError_t e = cudaGraphLaunch(plan->exec, s);
    return e == cudaSuccess ? MOA_OK : batch_cuda_failed(e, "launch");
}

moa_status moa_batch_plan_info(const moa_batch_plan *plan, int64_t *n_problems, int64_t *n_launches, int64_t *n_tiles,
                               double *work_flops) {
    if (!plan) return MOA_ERR_NULL;
    if (n_problems) *n_problems = plan->count;
    if (n_launches) {  // before the first execute: the default schedule (CUDA-core items in their own kernel)
        int64_t cc = 0, gv = 0;
        for (const BItem &it : plan->items) cc += it.type == IT_CC, gv += it.type == IT_GEMV;
        const int64_t grouped = plan->n_items - cc - gv;
        bool used[kCcGroups] = {};  // one CUDA-core kernel per (operator, tile halves) present
        for (const BItem &it : plan->items)
            if (it.type == IT_CC) used[cc_group(*plan, it)] = true;
        int ops = 0;
        for (bool u : used) ops += u;
        *n_launches = (plan->n_jobs > 0 ? 1 : 0) + (grouped > 0 ? 1 : 0) + (gv > 0 ? 1 : 0) + ops;
    }
    if (n_tiles) *n_tiles = plan->n_items;
    if (work_flops) *work_flops = plan->work;
    return MOA_OK;
}

void moa_batch_plan_destroy(moa_batch_plan *plan) { plan_free(plan); }

}  // extern "C"

namespace moa {
cudaError_t batch_read_and_clear_status(uint32_t *flags) {
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_batch_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    const uint32_t zero = 0;
    return cudaMemcpyToSymbol(g_batch_status, &zero, sizeof(uint32_t));
}
}  // namespace moa
