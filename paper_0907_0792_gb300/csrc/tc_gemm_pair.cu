// Pair-MMA form of the tensor-core (add, mul) inner product, Eq. (2) with
// * = multiply, on the psi-flattened problem D (M x N, FP32) = A (M x K) .
// B (K x N): the same contraction as tc_gemm.cu, with each 256 x 256 output
// tile computed by a cluster of two CTAs that drive one tcgen05 MMA
// together (cta_group::2).
//
// Why: with a 128 x 256 tile on one SM every 128 x 256 x 16 MMA reads
// 4 KB of A and 8 KB of B from that SM's shared memory.  In the pair, each
// SM holds its 128 rows of A and its 128 of the 256 columns of B; the MMA
// of the pair reads both halves of B, so each SM feeds 4 KB + 4 KB per
// 128 x 256 x 16 of its own output, and its shared-memory stage shrinks
// from 48 KB to 32 KB (six stages in flight).  Each k-block's MMAs are
// issued by one elected lane of a converged warp.
//
// The tiles that would make up a last, at most half-full wave run as two
// units of half their columns each (an MMA of N = 128 on each half), so that
// wave takes half as long.
//
// Roles (both CTAs run the same code; rank 0 of the cluster leads):
//   warp 0     TMA producer in both CTAs: this CTA's 128 x 64 slice of A
//              and its 64 x 128 slice of B per stage, into its own shared
//              memory, with the bytes counted on the LEADER's full barrier
//              (.cta_group::2 lets the copy signal the peer's barrier).
//              The leader arms that barrier for both CTAs' bytes.
//   warp 1     both CTAs: collective TMEM allocation (512 columns each).
//              Leader only: issues the 256 x 256 x 16 MMAs and commits to
//              the stage barriers and accumulator barriers of both CTAs.
//   warps 2-   epilogue in both CTAs (4 warps, or 8 for MODE_PROMOTE): its
//              own 128 TMEM lanes = its 128 rows of the tile, written out
//              32 x 32 at a time through a swizzled staging tile and a TMA
//              store (whole 128-B lines instead of 16-B pieces of 32 rows);
//              tells the leader when an accumulator is free (one arrival
//              per epilogue warp of each CTA).
// Two 256-column TMEM accumulators let the epilogue of tile t overlap the
// main loop of tile t+1.  MODE_PROMOTE accumulates every 64-deep k-block in
// a fresh accumulator and adds it into FP32 registers (IEEE adds), as the
// single-CTA kernel does for the split-BF16x3 form.
//
// Every mbarrier wait is bounded; a wait that gives up sets the CTA's abort
// flag and the device status word, and the CTA winds down (in-flight MMAs
// are drained before TMEM is freed).
#include <cuda.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tc.h"
#include "ozaki_epi.cuh"
#include "tc_ptx.cuh"

namespace moa {

__device__ uint32_t g_pair_status;

namespace {

constexpr int BM = 128;                // rows per CTA; the pair covers 2 * BM
constexpr int STAGES = 6;
constexpr int MODE_STORE = 0, MODE_PROMOTE = 1, MODE_FP8 = 2, MODE_OZAKI = 3;
// Columns per pair tile; each CTA holds bn / 2 of B.  The FP8 mode leaves
// TMEM room for its scale factors: 2 x 224 accumulator columns + 4 x 16.
__host__ __device__ constexpr int bn(int mode) { return mode == MODE_FP8 ? 224 : 256; }
// Per mode: element bytes (bf16 2, e4m3 1); a k-block is one 128-B swizzle
// row of A (bk elements), an MMA contracts 32 bytes' worth (uk elements).
__host__ __device__ constexpr int esz(int mode) { return mode == MODE_FP8 ? 1 : 2; }
__host__ __device__ constexpr int bk(int mode) { return 128 / esz(mode); }
__host__ __device__ constexpr int uk(int mode) { return 32 / esz(mode); }
// bf16 modes: B is MN-major (rows of B as given); its boxes are 128 B wide
// (boxn elements) and bk k-rows high, and a CTA's bn / 2 columns take
// (bn / 2) / boxn of them.  FP8 mode: B is K-major (B transposed by the
// quantisation pre-pass), one box of bn / 2 rows of 128 B.
__host__ __device__ constexpr int boxn(int mode) { return 128 / esz(mode); }
__host__ __device__ constexpr int nbox(int mode) { return mode == MODE_FP8 ? 1 : (bn(mode) / 2) / boxn(mode); }
__host__ __device__ constexpr int box_bytes(int mode) { return mode == MODE_FP8 ? (bn(mode) / 2) * 128 : bk(mode) * 128; }
// Warps: producer, MMA, and epilogue warps: one per TMEM lane quarter when
// the accumulator is stored as it is, two per quarter when every k-block is
// added into registers (each thread then holds 128 running sums).
// The Ozaki mode keeps a 64-column slice of int32 class sums per thread: 16
// epilogue warps (four per quarter).
__host__ __device__ constexpr int epi_warps(int mode) { return mode == MODE_PROMOTE ? 8 : mode == MODE_OZAKI ? 16 : 4; }
__host__ __device__ constexpr int threads(int mode) { return 64 + 32 * epi_warps(mode); }
constexpr int A_BYTES = BM * 128;            // 16 KB: 128 rows of one 128-B k-block
__host__ __device__ constexpr int b_bytes(int mode) { return (bn(mode) / 2) * 128; }  // this CTA's part of B
// FP8 scale factors ride in each stage after A and B: A's 128 row scales
// (512 B) and B's scales of the tile's bn columns (two 512-B blocks), laid
// out as the TMEM words they are copied to (see tmem_cp_32x128b_pair).
constexpr int SFA_BYTES = 512, SFB_BYTES = 1024;
__host__ __device__ constexpr int sf_off(int mode) { return A_BYTES + b_bytes(mode); }
__host__ __device__ constexpr int stage_bytes(int mode) {
    return mode == MODE_FP8 ? (A_BYTES + b_bytes(mode) + SFA_BYTES + SFB_BYTES + 1023) / 1024 * 1024
                            : A_BYTES + b_bytes(mode);
}
__host__ __device__ constexpr int stage_tx(int mode) {  // bytes the TMA delivers per stage and CTA
    return A_BYTES + b_bytes(mode) + (mode == MODE_FP8 ? SFA_BYTES + SFB_BYTES : 0);
}
constexpr int STG_BYTES = 32 * 32 * 4;  // an epilogue warp's staging tile: 32 rows x 32 FP32
constexpr int SF_BUFS = 4;              // scale-factor buffers in TMEM (FP8), used in turn
constexpr int SF_COL0 = 448;            // first scale-factor column; buffer s at SF_COL0 + 16 s
constexpr int NBARS = 2 * STAGES + 5;
// Shared memory: the stages, the epilogue staging tiles (room for 8 warps),
// then the barriers.
__host__ __device__ constexpr int bar_offset(int mode) { return STAGES * stage_bytes(mode) + 8 * STG_BYTES; }
__host__ __device__ constexpr int smem_bytes(int mode) { return bar_offset(mode) + 1024 + 1024; }
constexpr int TMEM_COLS = 512;
__host__ __device__ constexpr uint32_t idesc(int mode) {
    // FP8: kind::mxf8f6f4 with UE8M0 block scales (bit 23), both operands K-major
    return mode == MODE_FP8
               ? (1u << 23) | ((uint32_t)(bn(mode) >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24)
               : ptx::idesc_bf16_f32(2 * BM, bn(mode), 1);
}
constexpr uint16_t kPair = 3;          // multicast mask: both CTAs
static_assert(box_bytes(MODE_STORE) * nbox(MODE_STORE) == b_bytes(MODE_STORE), "B slice bytes");
static_assert(stage_bytes(MODE_FP8) % 1024 == 0 && stage_bytes(MODE_STORE) % 1024 == 0, "1024-B aligned stages");
static_assert(NBARS * 8 + 16 <= 1024, "barrier area");
static_assert(2 * bn(MODE_STORE) <= TMEM_COLS && SF_COL0 >= 2 * bn(MODE_FP8) && SF_COL0 + 16 * SF_BUFS <= TMEM_COLS,
              "TMEM columns");
static_assert(smem_bytes(MODE_STORE) <= 227 * 1024 && smem_bytes(MODE_FP8) <= 227 * 1024, "shared memory per CTA");

struct PairParams {
    int M, N, K;
    int tiles_m, tiles_n;  // pair tiles: ceil(M / 256) x ceil(N / 256)
    int group_m;           // row tiles per raster group
    int full_units;        // tiles run whole; each later tile runs as two halves of its columns
    int kblocks, n_terms;
    uint32_t term_a, term_b;  // plane of A / B for term i in bits 4i..4i+3
    float *D;
    int64_t ldd;
    int vec_store;
    uint32_t ab_fmt;  // kind::f16 operand format bits (bf16 or fp16 planes)
    int tma_store;  // D written through per-warp staging tiles and TMA stores
    int d_evict_first;  // those stores under an evict-first L2 policy (D is not re-read)
    uint32_t *bits_out;  // store mode: write [D > 0] as the packed bit stream (N % 32 == 0) instead of D
    int i32_out;  // store mode: D holds int32 (every accumulator an exact integer, |x| <= 2^24)
    // Ozaki mode (ozaki_epi.cuh)
    int slices, beta, lsb, chunk;  // S, bits per digit, accumulator LSB, k-blocks per exact chunk
    int acc_pairs;                 // slice pairs of a (class, chunk) per accumulator
    double *D64;
    const uint64_t *row_max, *col_max;  // |A| row / |B| column maxima as FP64 bit patterns
    float2 *rs;  // running-sum scratch: per CTA, per epilogue warp, 64 columns x 32 lanes
};

// Groups of GM row tiles, column tiles within a group: the A and B panels
// in flight stay resident in L2.
MOA_DEV void pair_tile_of(int t, int tiles_m, int tiles_n, int GM, int &tm, int &tn) {
    const int group = t / (GM * tiles_n);
    const int first = group * GM;
    const int gsz = min(tiles_m - first, GM);
    const int local = t - group * GM * tiles_n;
    tm = first + local % gsz;
    tn = local / gsz;
}

MOA_DEV bool drain_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(threads(MODE), 1)
    tc_gemm_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmD, const __grid_constant__ CUtensorMap tmSA,
                 const __grid_constant__ CUtensorMap tmSB, const PairParams p) {
    constexpr int BN = bn(MODE), STAGE_BYTES = stage_bytes(MODE), ACC_STRIDE = BN;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + bar_offset(MODE));
    uint32_t *tmem_slot = (uint32_t *)(bars + NBARS);
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
            ptx::mbar_init(full(s), 1);   // leader's: armed once per phase by the leader's producer
            ptx::mbar_init(empty(s), 1);  // one commit of the leader's MMA per phase
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(tfull(b), 1);
            ptx::mbar_init(tempty(b), 2 * epi_warps(MODE));  // leader's: every epilogue warp of both CTAs
        }
        ptx::mbar_init(drain, 1);
        *abort_flag = 0u;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async_smem();
        ptx::prefetch_tmap(&tmA);
        ptx::prefetch_tmap(&tmB);
        if (p.tma_store) ptx::prefetch_tmap(&tmD);
        if constexpr (MODE == MODE_FP8) {
            ptx::prefetch_tmap(&tmSA);
            ptx::prefetch_tmap(&tmSB);
        }
    }
    if (warp == 1) {
        ptx::tmem_alloc_pair(ptx::smem_u32(tmem_slot), TMEM_COLS);
        ptx::tmem_relinquish_pair();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::cluster_sync();  // the peer's barriers exist before any remote arrive or copy
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int crank = (int)(ptx::cluster_ctarank() & 1u);
    const bool leader = crank == 0;
    const int cfirst = (int)ptx::cluster_id_x();
    const int cstride = (int)ptx::nclusters_x();
    // Work units: tiles [0, full_units) whole, then each remaining tile as two
    // units of half its columns (coff = 0 or BN / 2), so the last, partly
    // filled wave of whole tiles becomes half as long.
    const int num_tiles = p.tiles_m * p.tiles_n;
    const int num_units = p.full_units + 2 * (num_tiles - p.full_units);
    auto unit_of = [&](int u, int &t, int &coff, int &ncols) {
        if (u < p.full_units) {
            t = u, coff = 0, ncols = BN;
        } else {
            const int v = u - p.full_units;
            t = p.full_units + (v >> 1), coff = (v & 1) * (BN / 2), ncols = BN / 2;
        }
    };
    const int kiters = p.kblocks * p.n_terms;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs; one elected lane issues)
        int stage = 0;
        uint32_t phase = 0, issued = 0, last_par = 0;
        bool ok = true;
        for (int u = cfirst; u < num_units && ok; u += cstride) {
            int t, coff, ncols, tm, tn;
            unit_of(u, t, coff, ncols);
            pair_tile_of(t, p.tiles_m, p.tiles_n, p.group_m, tm, tn);
            const int row0 = tm * 2 * BM + crank * BM;
            const int col0 = tn * BN + coff + crank * (ncols / 2);
            const int boxes = (ncols / 2) / boxn(MODE);  // B boxes this CTA loads per stage (bf16 modes)
            ozaki::Iter oz;
            oz.start(p.slices, p.chunk, p.kblocks, p.acc_pairs);
            for (int it = 0; it < kiters; ++it) {
                int kb, pa, pb;
                if constexpr (MODE == MODE_OZAKI) {  // class, chunk, pair, k-block
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
                if (!ptx::mbar_wait_warp(empty(stage), phase ^ 1u, abort_flag, &g_pair_status)) {
                    ok = false;
                    break;
                }
                if (ptx::elect_one()) {
                    const uint32_t sa = tiles0 + stage * STAGE_BYTES, sb = sa + A_BYTES;
                    const uint32_t fbar = ptx::mapa(full(stage), 0);
                    if (leader)
                        ptx::mbar_arrive_expect_tx(
                            full(stage), MODE == MODE_FP8 ? 2 * stage_tx(MODE) : 2 * (A_BYTES + boxes * box_bytes(MODE)));
                    ptx::tma_load_3d_pair(sa, &tmA, fbar, kb * bk(MODE), row0, pa);
                    if constexpr (MODE == MODE_FP8) {  // K-major B: rows = columns of B; then the scale blocks
                        ptx::tma_load_3d_pair(sb, &tmB, fbar, kb * bk(MODE), col0, pb);
                        const uint32_t ssf = sa + sf_off(MODE);
                        ptx::tma_load_3d_pair(ssf, &tmSA, fbar, 0, (tm * 2 + crank) * p.kblocks + kb, 0);
                        ptx::tma_load_3d_pair(ssf + SFA_BYTES, &tmSB, fbar, 0, tn * p.kblocks + kb, 0);
                    } else {
#pragma unroll
                        for (int j = 0; j < nbox(MODE); ++j)
                            if (j < boxes)
                                ptx::tma_load_3d_pair(sb + j * box_bytes(MODE), &tmB, fbar, col0 + j * boxn(MODE),
                                                      kb * bk(MODE), pb);
                    }
                }
                __syncwarp();
                issued |= 1u << stage;
                last_par = (last_par & ~(1u << stage)) | (phase << stage);
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        if (!ok && leader && lane == 0) {  // let every copy counted on this CTA's barriers land before it exits
            for (int s = 0; s < STAGES; ++s)
                if (issued & (1u << s)) drain_wait(full(s), (last_par >> s) & 1u);
        }
    } else if (warp == 1 && leader) {
        // ------------------------------------------------ MMA issuer (leader; one elected lane issues)
        int stage = 0, abuf = 0, sfb = 0;
        uint32_t phase = 0, aphase = 0;
        bool ok = true, any = false;
        const uint32_t id16 = (idesc(MODE) & ~ptx::kIdescAbMask) | p.ab_fmt;  // kind::f16: bf16 or fp16 planes
        // descriptors of stage 0, k-step 0; A steps +32 B along the swizzled
        // K row, B (MN-major) +uk rows of 128 B or (K-major, FP8) +32 B, a
        // stage +STAGE_BYTES (offsets >> 4)
        constexpr uint32_t B_KSTEP = MODE == MODE_FP8 ? (32 >> 4) : (uk(MODE) * 128 >> 4);
        const ptx::DescHalves a0 = ptx::desc_halves(ptx::smem_desc_sw128(tiles0, 16, 1024));
        const ptx::DescHalves b0 = ptx::desc_halves(
            MODE == MODE_FP8 ? ptx::smem_desc_sw128(tiles0 + A_BYTES, 16, 1024)
                             : ptx::smem_desc_sw128(tiles0 + A_BYTES, box_bytes(MODE), 1024));
        // FP8: the stage's scale blocks, rows of 16 B in 8-row groups (no swizzle)
        const ptx::DescHalves s0 = ptx::desc_halves(ptx::smem_desc_plain(tiles0 + sf_off(MODE), 128));
        for (int u = cfirst; u < num_units && ok; u += cstride) {
            int t, coff, ncols;
            unit_of(u, t, coff, ncols);
            // the MMA's N: the whole tile or half of its columns (instruction descriptor bits 17-22: N / 8)
            const uint32_t id_u = (id16 & ~(0x3Fu << 17)) | ((uint32_t)(ncols >> 3) << 17);
            ozaki::Iter oz;
            oz.start(p.slices, p.chunk, p.kblocks, p.acc_pairs);
            for (int it = 0; it < kiters; ++it) {
                int j, last;  // position inside the current accumulator; whether it is its last step
                if constexpr (MODE == MODE_STORE || MODE == MODE_FP8) {
                    j = it;
                    last = it == kiters - 1;
                } else if constexpr (MODE == MODE_OZAKI) {  // one accumulator per (class, chunk, pair)
                    j = oz.acc_pos();
                    last = oz.acc_last();
                    oz.next(p.chunk, p.kblocks);
                } else {  // a fresh accumulator per k-block (all its terms)
                    j = it % p.n_terms;
                    last = j == p.n_terms - 1;
                }
                if (j == 0) {
                    if (!ptx::mbar_wait_warp(tempty(abuf), aphase ^ 1u, abort_flag, &g_pair_status)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                }
                const uint32_t dacc = tmem + (uint32_t)(abuf * ACC_STRIDE);
                if (!ptx::mbar_wait_warp(full(stage), phase, abort_flag, &g_pair_status)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t so = (uint32_t)stage * (STAGE_BYTES >> 4);
                if (ptx::elect_one()) {  // the same lane issues every MMA and commit
                    if constexpr (MODE == MODE_FP8) {
                        // this k-block's scale blocks: shared memory -> TMEM buffer sfb of both CTAs,
                        // ordered before the MMAs below in the tensor pipe
                        const uint32_t sfa = tmem + (uint32_t)(SF_COL0 + 16 * sfb);
                        const uint32_t slo = s0.lo + so;
                        ptx::tmem_cp_32x128b_pair(sfa, slo, s0.hi);
                        ptx::tmem_cp_32x128b_pair(sfa + 4, slo + (SFA_BYTES >> 4), s0.hi);
                        ptx::tmem_cp_32x128b_pair(sfa + 8, slo + ((SFA_BYTES + 512) >> 4), s0.hi);
                    }
#pragma unroll
                    for (int k = 0; k < bk(MODE) / uk(MODE); ++k) {
                        const uint32_t alo = a0.lo + so + k * (32 >> 4), blo = b0.lo + so + k * B_KSTEP;
                        if constexpr (MODE == MODE_FP8) {
                            // k-step k uses byte k of each scale word (all four hold the block's scale)
                            const uint32_t sfa = tmem + (uint32_t)(SF_COL0 + 16 * sfb);
                            ptx::mma_mxf8_pair_h(dacc, alo, a0.hi, blo, b0.hi, idesc(MODE) | ((uint32_t)k << 4) | ((uint32_t)k << 29),
                                                 sfa, sfa + 4, (j > 0 || k > 0) ? 1u : 0u);
                        } else {
                            ptx::mma_bf16_pair_h(dacc, alo, a0.hi, blo, b0.hi, id_u, (j > 0 || k > 0) ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit_pair_mc(empty(stage), kPair);
                    if (last) ptx::mma_commit_pair_mc(tfull(abuf), kPair);
                }
                __syncwarp();
                any = true;
                if constexpr (MODE == MODE_FP8) sfb = (sfb + 1) % SF_BUFS;
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
                if (last) {
                    abuf ^= 1;
                    if (!abuf) aphase ^= 1u;
                }
            }
        }
        if (!ok && any && ptx::elect_one()) {  // MMAs already issued must finish before TMEM is freed
            ptx::mma_commit_pair_mc(drain, 1);
            drain_wait(drain, 0);
        }
    } else if (warp >= 2 && warp < 2 + epi_warps(MODE)) {
        // ------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;          // TMEM lane quarter this warp may access
        const int half = (warp - 2) / 4;                 // which part of the 256 columns
        constexpr int HC = BN / (epi_warps(MODE) / 4);  // columns per epilogue warp
        const uint32_t tempty_leader0 = ptx::mapa(tempty(0), 0), tempty_leader1 = ptx::mapa(tempty(1), 0);
        int abuf = 0;
        uint32_t aphase = 0;
        auto wait_acc = [&]() -> bool {
            int okw = 1;
            if (lane == 0) okw = ptx::mbar_wait(tfull(abuf), aphase, abort_flag, &g_pair_status) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (okw) ptx::tc_fence_after();
            return okw != 0;
        };
        auto release_acc = [&]() {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive_cluster(abuf ? tempty_leader1 : tempty_leader0);
            abuf ^= 1;
            if (!abuf) aphase ^= 1u;
        };
        // 32 columns x the warp's 32 rows: through the warp's staging tile
        // (128-B swizzled rows, the layout of the store's tensor map) and one
        // TMA store, or with direct stores when D's layout rules TMA out
        const uint32_t stg = tiles0 + STAGES * STAGE_BYTES + (warp - 2) * STG_BYTES;
        auto store32 = [&](int64_t row, int64_t col0, const uint32_t (&v)[32]) {
            if (p.tma_store) {
                if (col0 >= p.N || row - lane >= p.M) return;  // warp-uniform
                if (lane == 0) ptx::bulk_wait_read0();  // the previous store has left the staging tile
                __syncwarp();
                const uint32_t rowa = stg + (uint32_t)lane * 128u;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    ptx::st_shared_v4(rowa + ((uint32_t)(j ^ (lane & 7)) << 4), v[4 * j], v[4 * j + 1], v[4 * j + 2],
                                      v[4 * j + 3]);
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if (p.d_evict_first)
                        ptx::tma_store_3d_hint(&tmD, stg, (int)col0, (int)(row - lane), 0, ptx::policy_evict_first());
                    else
                        ptx::tma_store_3d(&tmD, stg, (int)col0, (int)(row - lane), 0);
                    ptx::bulk_commit();
                }
                return;
            }
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
        for (int u = cfirst; u < num_units && ok; u += cstride) {
            int t, coff, ncols, tm, tn;
            unit_of(u, t, coff, ncols);
            pair_tile_of(t, p.tiles_m, p.tiles_n, p.group_m, tm, tn);
            const int64_t row = (int64_t)tm * 2 * BM + crank * BM + q * 32 + lane;
            const int64_t colh = (int64_t)tn * BN + coff + half * HC;
            // a warp whose columns lie past a half tile's only keeps the barrier
            // protocol (it waits for and releases every accumulator)
            const bool active = half * HC < ncols;
            const uint32_t lanes = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * HC);
            if constexpr (MODE == MODE_OZAKI) {
                // every (class, chunk, pair) accumulator of a class added exactly into int32, the class
                // folded into the double-float running sum kept in D's FP64 slots, FP64 at the end
                const bool row_ok = row < p.M;
                double *drow = p.D64 + row * p.ldd;
                float2 *rs = p.rs + ((int64_t)blockIdx.x * epi_warps(MODE) + (warp - 2)) * (HC * 32) + lane;
                bool first = true;
                int qacc[HC];
#pragma unroll
                for (int j = 0; j < HC; ++j) qacc[j] = 0;
                const int chunks = (p.kblocks + p.chunk - 1) / p.chunk;
                for (int cls = p.slices - 1; cls >= 0 && ok; --cls) {
                    for (int a = 0; a < ozaki::accs_in_class(cls, chunks, p.acc_pairs); ++a) {
                        if (!wait_acc()) {
                            ok = false;
                            break;
                        }
                        const uint32_t tb = lanes + (uint32_t)(abuf * ACC_STRIDE);
                        if (active) {
#pragma unroll
                            for (int c0 = 0; c0 < HC; c0 += 8) {  // 8 columns a load: the 64 class sums leave few registers
                                uint32_t r[8];
                                ptx::tmem_ld8(tb + c0, r);
                                ptx::tmem_ld_wait();
#pragma unroll
                                for (int j = 0; j < 8; ++j)  // exact: accumulator sums are integers of at most 2^24
                                    qacc[c0 + j] += __float2int_rz(__uint_as_float(r[j]));
                            }
                        }
                        release_acc();  // the MMA may refill the accumulator during the fold
                    }
                    if (!ok) break;
                    if (active) ozaki::fold_rs<HC>(qacc, ozaki::class_weight(cls, p.lsb, p.beta), rs, first);
#pragma unroll
                    for (int j = 0; j < HC; ++j) qacc[j] = 0;
                    first = false;
                }
                if (!ok) break;
                if (row_ok && active) ozaki::finish_rs<HC>(rs, drow, colh, p.N, p.row_max[row], p.col_max, p.lsb);
            } else if constexpr (MODE == MODE_PROMOTE) {
                float acc[HC];
#pragma unroll
                for (int j = 0; j < HC; ++j) acc[j] = 0.0f;
                for (int kb = 0; kb < p.kblocks; ++kb) {
                    if (!wait_acc()) {
                        ok = false;
                        break;
                    }
                    const uint32_t tb = lanes + (uint32_t)(abuf * ACC_STRIDE);
                    if (active) {
#pragma unroll
                        for (int c = 0; c < HC; c += 16) {
                            uint32_t r[16];
                            ptx::tmem_ld16(tb + c, r);
                            ptx::tmem_ld_wait();
#pragma unroll
                            for (int j = 0; j < 16; ++j) acc[c + j] = __fadd_rn(acc[c + j], __uint_as_float(r[j]));
                        }
                    }
                    release_acc();
                }
                if (!ok) break;
                if (!active) continue;
#pragma unroll
                for (int c = 0; c < HC; c += 32) {
                    uint32_t r[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(acc[c + j]);
                    store32(row, colh + c, r);
                }
            } else {
                if (!wait_acc()) break;
                const uint32_t tb = lanes + (uint32_t)(abuf * ACC_STRIDE);
#pragma unroll 1
                for (int c = 0; c < HC && c < ncols; c += 32) {
                    uint32_t r[32];
                    ptx::tmem_ld32(tb + c, r);
                    ptx::tmem_ld_wait();
                    if (p.bits_out) {  // 32 columns of one row -> one word of the bit stream
                        const int64_t col0 = colh + c;
                        uint32_t word = 0u;
#pragma unroll
                        for (int j = 0; j < 32; ++j) word |= (__uint_as_float(r[j]) > 0.0f ? 1u : 0u) << j;
                        if (row < p.M && col0 < p.N) p.bits_out[(row * p.N + col0) >> 5] = word;
                    } else {
                        if (p.i32_out) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) r[j] = (uint32_t)__float2int_rn(__uint_as_float(r[j]));
                        }
                        store32(row, colh + c, r);
                    }
                }
                release_acc();
            }
        }
        if (p.tma_store && lane == 0) ptx::bulk_wait0();  // every store done before the CTA exits
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::cluster_sync();  // no CTA leaves or frees TMEM while its peer may still use it
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc_pair(tmem, TMEM_COLS);
    }
}

// Row tiles per raster group: 16, and 8 in the Ozaki slice-pair mode
// (MOA_PAIR_GROUP_M overrides for all modes, MOA_OZAKI_GROUP_M for the Ozaki
// mode alone; 1..64).  Measured at 8192^3 with 6 slices (40 steps, power
// capped): group 2 / 4 / 6 / 8 / 12 / 16: 66.3 / 68.6 / 69.2 / 71.5 / 70.8 /
// 69.1 effective FP64 TFLOP/s.
int group_env(const char *name) {
    const char *e = std::getenv(name);
    const int v = e ? std::atoi(e) : 0;
    return (v >= 1 && v <= 64) ? v : 0;
}
int pair_group_m(int mode) {
    static const int all = group_env("MOA_PAIR_GROUP_M"), oz = group_env("MOA_OZAKI_GROUP_M");
    if (mode == MODE_OZAKI) return oz ? oz : (all ? all : 8);
    return all ? all : 16;
}

// MOA_PAIR_HALF_TILES=0 keeps every tile whole.
bool half_tiles_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("MOA_PAIR_HALF_TILES");
        return !(e && e[0] == '0');
    }();
    return on;
}

int pair_sms() {
    static const int n = [] {  // read once, thread-safe
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 2;
    }();
    return n;
}

template <int MODE>
cudaError_t launch_pair(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &td, const CUtensorMap &tsa,
                        const CUtensorMap &tsb, PairParams &p, cudaStream_t s) {
    auto kern = tc_gemm_pair<MODE>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2, at[0].val.clusterDim.y = 1, at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(threads(MODE)), cfg.dynamicSmemBytes = smem_bytes(MODE);
    cfg.attrs = at, cfg.numAttrs = 1;
    // shared-memory attribute and resident clusters, set up once per process
    // (under a lock, so concurrent first calls agree; a failure is retried)
    static std::mutex mu;
    static int cached = 0;
    int max_clusters;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!cached) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(MODE));
            if (e != cudaSuccess) return e;
            int mc = pair_sms() / 2;
            cfg.gridDim = dim3(2 * mc);
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0 && n < mc) mc = n;
            cudaGetLastError();
            cached = mc;
        }
        max_clusters = cached;
    }
    p.tiles_m = (p.M + 2 * BM - 1) / (2 * BM);
    p.tiles_n = (p.N + bn(MODE) - 1) / bn(MODE);
    p.group_m = pair_group_m(MODE);
    const int tiles = p.tiles_m * p.tiles_n;
    // the tiles of a last wave that would fill at most half of the resident
    // clusters run as column halves (twice the units, half as long) when the
    // launch has at most 8 waves; the FP8 mode's B box and scale blocks cover
    // whole tiles, so it keeps them whole.  Measured (same box, A/B): n = 4096
    // (3.4 waves) +2..4 % for the bf16, fp16, BF16x3 and Ozaki forms; n = 8192
    // (13.5 waves) no gain, so longer launches keep whole tiles.
    const int tail = tiles % max_clusters;
    p.full_units = (MODE != MODE_FP8 && tiles > max_clusters && tiles <= 8 * max_clusters && 2 * tail <= max_clusters &&
                    half_tiles_enabled())
                       ? tiles - tail
                       : tiles;
    const int units = p.full_units + 2 * (tiles - p.full_units);
    const int clusters = units < max_clusters ? units : max_clusters;
    cfg.gridDim = dim3(2 * clusters);
    cfg.stream = s;
    GemmTimer timer(s);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ta, tb, td, tsa, tsb, p);
    timer.done();
    return e;
}

}  // namespace

// MOA_TMA_STORE=0 makes the epilogue store D directly from registers.
static bool tma_store_enabled() {
    static const bool on = [] {  // read once, thread-safe
        const char *e = std::getenv("MOA_TMA_STORE");
        return !(e && e[0] == '0');
    }();
    return on;
}

// D goes out through the TMA stores under an evict-first L2 policy, so the
// stream of results does not push the A and B panels out of L2 (measured:
// bf16 8192 x 256 x 16384 +11 %, 8192 x 512 x 8192 +6 %, 8192^3 unchanged);
// MOA_D_EVICT_FIRST=0 stores with the default policy.
static int d_evict_first() {
    static const int on = [] {
        const char *e = std::getenv("MOA_D_EVICT_FIRST");
        return (e && e[0] == '0') ? 0 : 1;
    }();
    return on;
}

bool pair_mma_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("MOA_PAIR_MMA");
        return !(e && e[0] == '0');
    }();
    return on;
}

// D's tensor map for TMA stores (16-byte aligned base and row stride); false
// when D's layout rules TMA out and the epilogue stores directly.
static bool d_tmap(CUtensorMap *td, float *D, int64_t ldd, int M, int N) {
    std::memset(td, 0, sizeof(*td));
    return ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0) && tma_store_enabled() &&
           make_tmap(td, D, (uint64_t)N, (uint64_t)M, 1, (uint64_t)ldd * 4, (uint64_t)ldd * 4 * (uint64_t)M, 32, 32,
                     CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
}

int pair_fp8_tile_n() { return bn(MODE_FP8); }

cudaError_t tc_gemm_pair_fp8_launch(const uint8_t *A8, int64_t lda, const uint8_t *Bt8, int64_t ldb, int M, int N, int K,
                                    const uint32_t *sfa, const uint32_t *sfb, float *D, int64_t ldd, cudaStream_t s,
                                    uint32_t *bits_out) {
    const int64_t kb = (K + bk(MODE_FP8) - 1) / bk(MODE_FP8);
    const int64_t mb = (M + BM - 1) / BM, tn = (N + bn(MODE_FP8) - 1) / bn(MODE_FP8);
    CUtensorMap ta, tb, tsa, tsb;
    if (!make_tmap(&ta, A8, (uint64_t)K, (uint64_t)M, 1, (uint64_t)lda, (uint64_t)lda * (uint64_t)M, 128, BM,
                   CU_TENSOR_MAP_DATA_TYPE_UINT8) ||
        !make_tmap(&tb, Bt8, (uint64_t)K, (uint64_t)N, 1, (uint64_t)ldb, (uint64_t)ldb * (uint64_t)N, 128, bn(MODE_FP8) / 2,
                   CU_TENSOR_MAP_DATA_TYPE_UINT8) ||
        // scale blocks: [row block][k-block] of 128 words, [column tile][k-block] of 256 words
        !make_tmap(&tsa, sfa, 128, (uint64_t)(mb * kb), 1, 512, (uint64_t)(512 * mb * kb), 128, 1,
                   CU_TENSOR_MAP_DATA_TYPE_UINT32, CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !make_tmap(&tsb, sfb, 256, (uint64_t)(tn * kb), 1, 1024, (uint64_t)(1024 * tn * kb), 256, 1,
                   CU_TENSOR_MAP_DATA_TYPE_UINT32, CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorInvalidValue;
    PairParams p{};
    p.M = M, p.N = N, p.K = K;
    p.kblocks = (int)kb;
    p.n_terms = 1;
    p.D = D, p.ldd = ldd;
    p.vec_store = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0);
    CUtensorMap td;
    std::memset(&td, 0, sizeof(td));
    p.bits_out = bits_out;
    p.tma_store = bits_out ? 0 : d_tmap(&td, D, ldd, M, N);
    p.d_evict_first = d_evict_first();
    return launch_pair<MODE_FP8>(ta, tb, td, tsa, tsb, p, s);
}

cudaError_t tc_gemm_pair_launch(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, int n_terms,
                                uint32_t term_a, uint32_t term_b, float *D, int64_t ldd, bool promote, cudaStream_t s,
                                bool i32_out, bool fp16) {
    if (promote && i32_out) return cudaErrorInvalidValue;
    PairParams p{};
    p.ab_fmt = ptx::idesc_ab_f16(fp16);
    p.i32_out = i32_out ? 1 : 0;
    p.M = M, p.N = N, p.K = K;
    p.kblocks = (K + bk(MODE_STORE) - 1) / bk(MODE_STORE);
    p.n_terms = n_terms;
    p.term_a = term_a, p.term_b = term_b;
    p.D = D, p.ldd = ldd;
    p.vec_store = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0);
    CUtensorMap td;
    p.tma_store = d_tmap(&td, D, ldd, M, N);
    p.d_evict_first = d_evict_first();
    return promote ? launch_pair<MODE_PROMOTE>(ta, tb, td, td, td, p, s) : launch_pair<MODE_STORE>(ta, tb, td, td, td, p, s);
}

cudaError_t tc_gemm_pair_ozaki_launch(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, int S, int beta,
                                      int lsb, int chunk_kblocks, int acc_pairs, const uint64_t *row_max,
                                      const uint64_t *col_max, double *D, int64_t ldd, void *scratch, cudaStream_t s) {
    PairParams p{};
    p.acc_pairs = acc_pairs;
    p.ab_fmt = ptx::idesc_ab_f16(false);
    p.rs = (float2 *)scratch;
    p.M = M, p.N = N, p.K = K;
    p.kblocks = (K + bk(MODE_OZAKI) - 1) / bk(MODE_OZAKI);
    p.n_terms = S * (S + 1) / 2;
    p.slices = S, p.beta = beta, p.lsb = lsb, p.chunk = chunk_kblocks;
    p.D64 = D, p.ldd = ldd, p.row_max = row_max, p.col_max = col_max;
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));
    return launch_pair<MODE_OZAKI>(ta, tb, none, none, none, p, s);
}

size_t pair_ozaki_scratch_bytes() {  // one 128 x 256 strip of (hi, lo) pairs per CTA
    return (size_t)pair_sms() * BM * bn(MODE_OZAKI) * sizeof(float2);
}

cudaError_t pair_read_and_clear_status(uint32_t *flags) {
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_pair_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    const uint32_t zero = 0;
    return cudaMemcpyToSymbol(g_pair_status, &zero, sizeof(uint32_t));
}

}  // namespace moa
