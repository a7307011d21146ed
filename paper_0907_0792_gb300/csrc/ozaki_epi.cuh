// Device pieces of the Ozaki-sliced FP64 form shared by the tensor-core
// kernels (tc_gemm.cu, tc_gemm_pair.cu): the order in which the slice-pair
// products run, the fold of a weight class's exact integer sum into the
// double-float running sum, and the final conversion to FP64.
//
// Slices: A = sum_s 2^(e_row - (s+1) beta) A_s and B likewise with digit
// planes A_s, B_u of balanced beta-bit integers; the product keeps the pairs
// s + u < S, grouped by weight class g = s + u.  Accumulators count units of
// 2^(e_row + e_col - lsb).
#pragma once

#include "common.cuh"

namespace moa {
namespace ozaki {

// Iteration order: weight class g from S-1 (lightest) down to 0, then
// chunk c of the contraction (`chunk` k-blocks, the last one shorter), then
// the class's slice pairs (s, g - s), s = 0..g, then the k-blocks of the
// chunk.  One exact FP32 accumulator takes `ap` consecutive pairs of a
// (class, chunk) (fewer for the class's last group), so it sums at most
// ap * chunk k-blocks of digit products; a class's sum is complete, and
// folded once, after its last chunk.  Running the class's pairs chunk by
// chunk keeps the slice panels of one chunk in L2 while every tile of a
// wave uses them; a short chunk makes that working set small, and grouping
// its pairs keeps the accumulators (one epilogue pass each) few.
struct Iter {
    int g = 0, c = 0, s = 0, kk = 0, clen = 0, ap = 1;
    int sg = 0;   // index of pair s inside its group of ap pairs
    int pos = 0;  // k-blocks of the current accumulator before this one
    MOA_DEV void start(int S, int chunk, int kblocks, int pairs_per_acc = 1) {
        g = S - 1;
        c = s = kk = sg = pos = 0;
        clen = min(chunk, kblocks);
        ap = pairs_per_acc;
    }
    MOA_DEV int kb(int chunk) const { return c * chunk + kk; }
    // position of the current k-block inside its accumulator, and whether it
    // is the accumulator's last (both before next()); kept incrementally, no
    // division in the issuing thread's loop
    MOA_DEV int acc_pos() const { return pos; }
    MOA_DEV bool acc_last() const { return kk == clen - 1 && (sg == ap - 1 || s == g); }
    MOA_DEV void next(int chunk, int kblocks) {
        pos = acc_last() ? 0 : pos + 1;
        if (++kk < clen) return;
        kk = 0;
        if (++s <= g) {
            if (++sg == ap) sg = 0;
            return;
        }
        s = sg = 0;
        if (++c * chunk < kblocks) {
            clen = min(chunk, kblocks - c * chunk);
            return;
        }
        c = 0;
        clen = min(chunk, kblocks);
        --g;
    }
};

// Accumulators the epilogue receives for class g: per chunk, its g + 1 pairs
// in groups of ap.
MOA_DEV int accs_in_class(int g, int chunks, int ap) { return chunks * ((g + ap) / ap); }

// Exponent e with |x| < 2^(e-1) for the largest |x| of a row / column, from
// its FP64 bit pattern (0 for an all-zero row): the scaled values lie below
// 1/2, which leaves the balanced top digit its carry.
MOA_DEV int scale_exponent(uint64_t maxbits) {
    const int be = (int)((maxbits >> 52) & 0x7FF);
    if (be == 0) return maxbits == 0 ? 0 : -1021;
    return be - 1021;
}

// The power-of-two weight of class g in accumulator units, exact in FP32.
MOA_DEV float class_weight(int g, int lsb, int beta) { return __int_as_float((127 + lsb - (g + 2) * beta) << 23); }

// (hi, lo) + w * q for an int32 q and a power of two w: q split exactly into
// two FP32 parts and scaled exactly, TwoSum of hi and the scaled high part,
// the low parts added into the error, then a FastTwoSum renormalisation:
// ~48 bits relative to the running sum.
MOA_DEV float2 add_scaled(float2 hl, int q, float w) {
    const float xh = __int2float_rn(q);
    const float xl = __int2float_rn(q - __float2int_rn(xh));  // exact remainder
    const float ah = __fmul_rn(xh, w), al = __fmul_rn(xl, w);  // exact scaling
    const float H = hl.x, L = hl.y;
    const float sum = __fadd_rn(H, ah);  // TwoSum(H, ah)
    const float bv = __fsub_rn(sum, H);
    float e = __fadd_rn(__fsub_rn(H, __fsub_rn(sum, bv)), __fsub_rn(ah, bv));
    e = __fadd_rn(e, __fadd_rn(L, al));
    const float nh = __fadd_rn(sum, e);  // FastTwoSum renormalisation
    return make_float2(nh, __fsub_rn(e, __fsub_rn(nh, sum)));
}

// End of a class: running sum (hi, lo) += w * qacc for this thread's HC
// columns of one row, the pair kept in the row's FP64 slots (drow[col] holds
// the FP32 pair until the tile is finished); `first` means no sum stored
// yet.  16 columns at a time, all loads issued before any store.
template <int HC>
MOA_DEV void fold(const int (&qacc)[HC], float w, double *drow, int64_t colh, int64_t N, bool first) {
#pragma unroll
    for (int c0 = 0; c0 < HC; c0 += 16) {
        float2 old[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int64_t col = colh + c0 + j;
            old[j] = (!first && col < N) ? *reinterpret_cast<const float2 *>(drow + col) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            old[j] = add_scaled(old[j], qacc[c0 + j], w);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int64_t col = colh + c0 + j;
            if (col < N) *reinterpret_cast<float2 *>(drow + col) = old[j];
        }
    }
}

// End of the tile: each (hi, lo) pair -> FP64, scaled by 2^(e_row + e_col - lsb).
template <int HC>
MOA_DEV void finish(double *drow, int64_t colh, int64_t N, uint64_t row_maxbits, const uint64_t *col_max, int lsb) {
    const int er = scale_exponent(row_maxbits);
#pragma unroll 4
    for (int j = 0; j < HC; ++j) {
        const int64_t col = colh + j;
        if (col >= N) break;
        const float2 v = *reinterpret_cast<const float2 *>(drow + col);
        const int ec = scale_exponent(col_max[col]);
        drow[col] = ldexp((double)v.x + (double)v.y, er + ec - lsb);
    }
}

// The same two steps with the running sums in a per-thread scratch strip
// instead of D's slots: element j of the thread at rs[32 j] (the 32 lanes of
// a warp interleaved), so every warp access is 256 contiguous bytes.
template <int HC>
MOA_DEV void fold_rs(const int (&qacc)[HC], float w, float2 *rs, bool first) {
#pragma unroll
    for (int c0 = 0; c0 < HC; c0 += 16) {
        float2 old[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) old[j] = first ? make_float2(0.0f, 0.0f) : rs[32 * (c0 + j)];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            old[j] = add_scaled(old[j], qacc[c0 + j], w);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) rs[32 * (c0 + j)] = old[j];
    }
}

template <int HC>
MOA_DEV void finish_rs(const float2 *rs, double *drow, int64_t colh, int64_t N, uint64_t row_maxbits,
                       const uint64_t *col_max, int lsb) {
    const int er = scale_exponent(row_maxbits);
#pragma unroll 4
    for (int j = 0; j < HC; ++j) {
        const int64_t col = colh + j;
        if (col >= N) break;
        const float2 v = rs[32 * j];
        const int ec = scale_exponent(col_max[col]);
        drow[col] = ldexp((double)v.x + (double)v.y, er + ec - lsb);
    }
}

}  // namespace ozaki
}  // namespace moa
