// Element operators of the CUDA-core generalized inner product, Eq. (2)
// with a general (reduce, combine) pair (Sec. I): identity of the reduce,
// one step acc = reduce(acc, a combine b), and a two-step form that uses the
// three-input min / max of sm_100+.  Shared by the single-problem kernels
// (semiring.cu) and the grouped batch kernel (batch.cu).
#pragma once

#include "common.cuh"

namespace moa {
namespace sr {

// Packed FP32 pairs (sm_100+ add / mul / fma .rn.f32x2): two IEEE
// round-to-nearest operations per instruction, lane by lane, so results are
// identical to the scalar forms.  (x, x) + (y0, y1), (x, x) * (y0, y1) and
// (x, x) - (y0, y1):
MOA_DEV void add2(float x, float y0, float y1, float &r0, float &r1) {
    asm("{\n\t.reg .b64 pa, pb;\n\tmov.b64 pa, {%2, %2};\n\tmov.b64 pb, {%3, %4};\n\t"
        "add.rn.f32x2 pa, pa, pb;\n\tmov.b64 {%0, %1}, pa;\n\t}"
        : "=f"(r0), "=f"(r1)
        : "f"(x), "f"(y0), "f"(y1));
}
MOA_DEV void mul2(float x, float y0, float y1, float &r0, float &r1) {
    asm("{\n\t.reg .b64 pa, pb;\n\tmov.b64 pa, {%2, %2};\n\tmov.b64 pb, {%3, %4};\n\t"
        "mul.rn.f32x2 pa, pa, pb;\n\tmov.b64 {%0, %1}, pa;\n\t}"
        : "=f"(r0), "=f"(r1)
        : "f"(x), "f"(y0), "f"(y1));
}
MOA_DEV void sub2(float x, float y0, float y1, float &r0, float &r1) {
    asm("{\n\t.reg .b64 pa, pb;\n\tmov.b64 pa, {%2, %2};\n\tmov.b64 pb, {%3, %4};\n\t"
        "sub.rn.f32x2 pa, pa, pb;\n\tmov.b64 {%0, %1}, pa;\n\t}"
        : "=f"(r0), "=f"(r1)
        : "f"(x), "f"(y0), "f"(y1));
}
// (c0, c1) = fma((x, x), (y0, y1), (c0, c1))
MOA_DEV void fma2(float x, float y0, float y1, float &c0, float &c1) {
    asm("{\n\t.reg .b64 pa, pb, pc;\n\tmov.b64 pa, {%2, %2};\n\tmov.b64 pb, {%3, %4};\n\t"
        "mov.b64 pc, {%0, %1};\n\tfma.rn.f32x2 pc, pa, pb, pc;\n\tmov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(c0), "+f"(c1)
        : "f"(x), "f"(y0), "f"(y1));
}

struct F32PlusTimes {
    using T = float;
    static MOA_DEV float identity() { return 0.0f; }
    static MOA_DEV float red(float x, float y) { return __fadd_rn(x, y); }
    static MOA_DEV float step(float acc, float a, float b) { return fmaf(a, b, acc); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmaf(a1, b1, fmaf(a0, b0, acc));
    }
    // two adjacent columns (c0: b*0, c1: b*1), two contraction steps
    static constexpr bool kPacked = true;
    static MOA_DEV void step2x2(float &c0, float &c1, float a0, float b00, float b01, float a1, float b10, float b11) {
        fma2(a0, b00, b01, c0, c1);
        fma2(a1, b10, b11, c0, c1);
    }
};
struct F64PlusTimes {
    using T = double;
    static constexpr bool kPacked = false;
    static MOA_DEV double identity() { return 0.0; }
    static MOA_DEV double step(double acc, double a, double b) { return fma(a, b, acc); }
    static MOA_DEV double step2(double acc, double a0, double b0, double a1, double b1) {
        return fma(a1, b1, fma(a0, b0, acc));
    }
};
struct I32PlusTimes {
    using T = int32_t;
    static constexpr bool kPacked = false;
    static MOA_DEV int32_t identity() { return 0; }
    static MOA_DEV int32_t step(int32_t acc, int32_t a, int32_t b) {
        return (int32_t)((uint32_t)acc + (uint32_t)a * (uint32_t)b);
    }
    static MOA_DEV int32_t step2(int32_t acc, int32_t a0, int32_t b0, int32_t a1, int32_t b1) {
        return step(step(acc, a0, b0), a1, b1);
    }
};
// reduce min or max with combine +, -, *, min or max over FP32: shortest,
// longest, most reliable, widest (max, min) and minimax (min, max) paths.
enum Combine { C_ADD, C_SUB, C_MUL, C_MIN, C_MAX };
template <bool kMax, int kComb> struct F32MinMax {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(kMax ? 0xff800000 : 0x7f800000); }
    static MOA_DEV float comb(float a, float b) {
        if constexpr (kComb == C_ADD) return __fadd_rn(a, b);
        else if constexpr (kComb == C_SUB) return __fsub_rn(a, b);
        else if constexpr (kComb == C_MUL) return __fmul_rn(a, b);
        else if constexpr (kComb == C_MIN) return fminf(a, b);
        else return fmaxf(a, b);
    }
    static MOA_DEV float red(float x, float y) { return kMax ? fmaxf(x, y) : fminf(x, y); }
    static MOA_DEV float red3(float x, float y, float z) { return kMax ? fmax3(x, y, z) : fmin3(x, y, z); }
    static MOA_DEV float step(float acc, float a, float b) { return red(acc, comb(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return red3(acc, comb(a0, b0), comb(a1, b1));
    }
    // arithmetic combines of two adjacent columns in one packed instruction
    static constexpr bool kPacked = kComb == C_ADD || kComb == C_SUB || kComb == C_MUL;
    static MOA_DEV void pair(float a, float b0, float b1, float &s0, float &s1) {
        if constexpr (kComb == C_ADD) add2(a, b0, b1, s0, s1);
        else if constexpr (kComb == C_SUB) sub2(a, b0, b1, s0, s1);
        else mul2(a, b0, b1, s0, s1);
    }
    static MOA_DEV void step2x2(float &c0, float &c1, float a0, float b00, float b01, float a1, float b10, float b11) {
        float s00, s01, s10, s11;
        pair(a0, b00, b01, s00, s01);
        pair(a1, b10, b11, s10, s11);
        c0 = red3(c0, s00, s10);
        c1 = red3(c1, s01, s11);
    }
};
using F32MinPlus = F32MinMax<false, C_ADD>;
using F32MaxPlus = F32MinMax<true, C_ADD>;
using F32MinTimes = F32MinMax<false, C_MUL>;
using F32MaxTimes = F32MinMax<true, C_MUL>;

}  // namespace sr
}  // namespace moa
