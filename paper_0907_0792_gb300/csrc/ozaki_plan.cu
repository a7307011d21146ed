// The Ozaki form's two size choices (Eq. 2 in its matrix-multiply case, on
// bf16 digit slices): how many slices each operand is cut into and how many
// k-blocks of the contraction one exact FP32 chunk of the slice-pair GEMM
// covers.  Both set the work and the data each launch of that GEMM moves, so
// they sit apart from the pre-pass kernels in ozaki.cu.
#include <cstdlib>

#include "common.cuh"
#include "tc.h"

namespace moa {

namespace {
constexpr int kMaxSlices = 10;
constexpr int kChunkKBlocks = 16;  // 16 x 64 = 1024 products (each at most 2^14) per exact FP32 chunk
}  // namespace

// k-blocks of 64 per chunk of the contraction: 16 up to K = 6144, 8 above
// (MOA_OZAKI_CHUNK overrides, 1..16); an accumulator takes 16 / chunk slice
// pairs of a chunk, so it holds at most 1024 products of 2^14.  Measured on
// one box, effective FP64 TFLOP/s, chunk 8 / 16: n = 2048 35.7 / 37.1, 3072
// 46.1 / 47.9, 4096 59.6 / 61.6, 6144 69.0 / 70.3; at 8192 (power capped)
// chunk 8 72.3 against 69.7 for 16, since the shorter chunk's smaller working
// set cuts DRAM traffic and leaves more of the power budget to the SMs
// (earlier, with 7 slices: 16 51.5-52.0, 8 54.3-54.5, 4 52.0-52.4).
int ozaki_chunk(int64_t K) {
    static const int forced = [] {
        const char *e = std::getenv("MOA_OZAKI_CHUNK");
        const int v = e ? std::atoi(e) : 0;
        return (v < 1 || v > kChunkKBlocks) ? 0 : v;
    }();
    return forced ? forced : (K <= 6144 ? 16 : 8);
}

int ozaki_acc_pairs(int chunk) { return kChunkKBlocks / chunk; }

// Slices per operand for a contraction of length K (MOA_OZAKI_SLICES overrides, 4..10).
int ozaki_slices(int64_t K) {
    static const int forced = [] {  // read once, thread-safe
        const char *e = std::getenv("MOA_OZAKI_SLICES");
        const int v = e ? std::atoi(e) : 0;
        return (v < 4 || v > kMaxSlices) ? 0 : v;
    }();
    if (forced) return forced;
    return K <= 64 ? 10 : (K <= 256 ? 8 : (K < 4096 ? 7 : 6));
}

}  // namespace moa

extern "C" int moa_ozaki_slices(int64_t K) { return K < 0 ? 0 : moa::ozaki_slices(K); }
