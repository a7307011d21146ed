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

#include "common.cuh"
#include "internal.h"
#include "tc.h"
#include "tc_ptx.cuh"

namespace moa {

__device__ uint32_t g_pair_status;

namespace {

constexpr int BM = 128;                // rows per CTA; the pair covers 2 * BM
constexpr int BN = 256;                // columns per pair tile; each CTA holds BN / 2 of B
constexpr int BK = 64;                 // bf16 per k-block: one 128-B swizzle row
constexpr int UK = 16;                 // contraction depth of one MMA
constexpr int STAGES = 6;
// Epilogue warps: one per TMEM lane quarter when the accumulator is stored
// as it is (4), two per quarter when every k-block is added into registers
// (8; each thread then holds 128 running sums).
__host__ __device__ constexpr int epi_warps(int mode) { return mode == 1 ? 8 : 4; }
__host__ __device__ constexpr int threads(int mode) { return 64 + 32 * epi_warps(mode); }
constexpr int A_BYTES = BM * BK * 2;   // 16 KB
constexpr int BOX_BYTES = BK * 128;    // 64 k-rows x 64 columns x 2 B
constexpr int B_BYTES = (BN / 2) * BK * 2;  // 16 KB: two boxes
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int STG_BYTES = 32 * 32 * 4;  // an epilogue warp's staging tile: 32 rows x 32 FP32
constexpr int NBARS = 2 * STAGES + 5;
constexpr int SMEM = STAGES * STAGE_BYTES + 8 * STG_BYTES + 1024 + 1024;  // staging for up to 8 warps
constexpr int ACC_STRIDE = BN;
constexpr int TMEM_COLS = 2 * ACC_STRIDE;
constexpr uint32_t IDESC = ptx::idesc_bf16_f32(2 * BM, BN, 1);
constexpr uint16_t kPair = 3;          // multicast mask: both CTAs
constexpr int MODE_STORE = 0, MODE_PROMOTE = 1;
static_assert(NBARS * 8 + 16 <= 1024, "barrier area");
static_assert(TMEM_COLS <= 512, "TMEM has 512 columns");
static_assert(SMEM <= 227 * 1024, "shared memory per CTA");

struct PairParams {
    int M, N, K;
    int tiles_m, tiles_n;  // pair tiles: ceil(M / 256) x ceil(N / 256)
    int kblocks, n_terms;
    uint32_t term_a, term_b;  // plane of A / B for term i in bits 4i..4i+3
    float *D;
    int64_t ldd;
    int vec_store;
    int tma_store;  // D written through per-warp staging tiles and TMA stores
};

// Groups of 16 row tiles, column tiles within a group: the A and B panels
// in flight stay resident in L2.
MOA_DEV void pair_tile_of(int t, int tiles_m, int tiles_n, int &tm, int &tn) {
    constexpr int GM = 16;
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
                 const __grid_constant__ CUtensorMap tmD, const PairParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES + 8 * STG_BYTES);
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
    const int num_tiles = p.tiles_m * p.tiles_n;
    const int kiters = p.kblocks * p.n_terms;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs; one elected lane issues)
        int stage = 0;
        uint32_t phase = 0, issued = 0, last_par = 0;
        bool ok = true;
        for (int t = cfirst; t < num_tiles && ok; t += cstride) {
            int tm, tn;
            pair_tile_of(t, p.tiles_m, p.tiles_n, tm, tn);
            const int row0 = tm * 2 * BM + crank * BM;
            const int col0 = tn * BN + crank * (BN / 2);
            for (int it = 0; it < kiters; ++it) {
                const int kb = it / p.n_terms;
                const int term = it - kb * p.n_terms;
                const int pa = (int)((p.term_a >> (4 * term)) & 15u);
                const int pb = (int)((p.term_b >> (4 * term)) & 15u);
                if (!ptx::mbar_wait_warp(empty(stage), phase ^ 1u, abort_flag, &g_pair_status)) {
                    ok = false;
                    break;
                }
                if (ptx::elect_one()) {
                    const uint32_t sa = tiles0 + stage * STAGE_BYTES, sb = sa + A_BYTES;
                    const uint32_t fbar = ptx::mapa(full(stage), 0);
                    if (leader) ptx::mbar_arrive_expect_tx(full(stage), 2 * STAGE_BYTES);
                    ptx::tma_load_3d_pair(sa, &tmA, fbar, kb * BK, row0, pa);
                    ptx::tma_load_3d_pair(sb, &tmB, fbar, col0, kb * BK, pb);
                    ptx::tma_load_3d_pair(sb + BOX_BYTES, &tmB, fbar, col0 + 64, kb * BK, pb);
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
        int stage = 0, abuf = 0;
        uint32_t phase = 0, aphase = 0;
        bool ok = true, any = false;
        // descriptors of stage 0, k-step 0; A steps +32 B along the swizzled
        // K row, B +UK rows of 128 B, a stage +STAGE_BYTES (offsets >> 4)
        const ptx::DescHalves a0 = ptx::desc_halves(ptx::smem_desc_sw128(tiles0, 16, 1024));
        const ptx::DescHalves b0 = ptx::desc_halves(ptx::smem_desc_sw128(tiles0 + A_BYTES, BOX_BYTES, 1024));
        for (int t = cfirst; t < num_tiles && ok; t += cstride) {
            for (int it = 0; it < kiters; ++it) {
                int j, last;  // position inside the current accumulator; whether it is its last step
                if constexpr (MODE == MODE_STORE) {
                    j = it;
                    last = it == kiters - 1;
                } else {
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
#pragma unroll
                    for (int k = 0; k < BK / UK; ++k)
                        ptx::mma_bf16_pair_h(dacc, a0.lo + so + k * (32 >> 4), a0.hi, b0.lo + so + k * (UK * 128 >> 4),
                                             b0.hi, IDESC, (j > 0 || k > 0) ? 1u : 0u);
                    ptx::mma_commit_pair_mc(empty(stage), kPair);
                    if (last) ptx::mma_commit_pair_mc(tfull(abuf), kPair);
                }
                __syncwarp();
                any = true;
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
    } else if (warp >= 2) {
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
        for (int t = cfirst; t < num_tiles && ok; t += cstride) {
            int tm, tn;
            pair_tile_of(t, p.tiles_m, p.tiles_n, tm, tn);
            const int64_t row = (int64_t)tm * 2 * BM + crank * BM + q * 32 + lane;
            const int64_t colh = (int64_t)tn * BN + half * HC;
            const uint32_t lanes = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * HC);
            if constexpr (MODE == MODE_PROMOTE) {
                float acc[HC];
#pragma unroll
                for (int j = 0; j < HC; ++j) acc[j] = 0.0f;
                for (int kb = 0; kb < p.kblocks; ++kb) {
                    if (!wait_acc()) {
                        ok = false;
                        break;
                    }
                    const uint32_t tb = lanes + (uint32_t)(abuf * ACC_STRIDE);
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
                const uint32_t tb = lanes + (uint32_t)(abuf * ACC_STRIDE);
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

int pair_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 2;
    }
    return n;
}

template <int MODE>
cudaError_t launch_pair(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &td, PairParams &p,
                        cudaStream_t s) {
    auto kern = tc_gemm_pair<MODE>;
    static int max_clusters = -1;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2, at[0].val.clusterDim.y = 1, at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(threads(MODE)), cfg.dynamicSmemBytes = SMEM;
    cfg.attrs = at, cfg.numAttrs = 1;
    if (max_clusters < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        max_clusters = pair_sms() / 2;
        cfg.gridDim = dim3(2 * max_clusters);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0 && n < max_clusters) max_clusters = n;
        cudaGetLastError();
    }
    p.tiles_m = (p.M + 2 * BM - 1) / (2 * BM);
    p.tiles_n = (p.N + BN - 1) / BN;
    const int tiles = p.tiles_m * p.tiles_n;
    const int clusters = tiles < max_clusters ? tiles : max_clusters;
    cfg.gridDim = dim3(2 * clusters);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, kern, ta, tb, td, p);
}

}  // namespace

// MOA_TMA_STORE=0 makes the epilogue store D directly from registers.
static bool tma_store_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("MOA_TMA_STORE");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

bool pair_mma_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = std::getenv("MOA_PAIR_MMA");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

cudaError_t tc_gemm_pair_launch(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, int n_terms,
                                uint32_t term_a, uint32_t term_b, float *D, int64_t ldd, bool promote, cudaStream_t s) {
    PairParams p{};
    p.M = M, p.N = N, p.K = K;
    p.kblocks = (K + BK - 1) / BK;
    p.n_terms = n_terms;
    p.term_a = term_a, p.term_b = term_b;
    p.D = D, p.ldd = ldd;
    p.vec_store = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0);
    // TMA store rules: 16-byte aligned base and row stride
    CUtensorMap td;
    std::memset(&td, 0, sizeof(td));
    p.tma_store = p.vec_store && tma_store_enabled() &&
                  make_tmap(&td, D, (uint64_t)N, (uint64_t)M, 1, (uint64_t)ldd * 4, (uint64_t)ldd * 4 * (uint64_t)M, 32, 32,
                            CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
    return promote ? launch_pair<MODE_PROMOTE>(ta, tb, td, p, s) : launch_pair<MODE_STORE>(ta, tb, td, p, s);
}

cudaError_t pair_read_and_clear_status(uint32_t *flags) {
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_pair_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    const uint32_t zero = 0;
    return cudaMemcpyToSymbol(g_pair_status, &zero, sizeof(uint32_t));
}

}  // namespace moa
