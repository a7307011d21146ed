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
// identical to the scalar forms.  (x, x) + (y0, y1) and (x, x) * (y0, y1):
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
struct F32MinPlus {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(0x7f800000); }
    static MOA_DEV float step(float acc, float a, float b) { return fminf(acc, __fadd_rn(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmin3(acc, __fadd_rn(a0, b0), __fadd_rn(a1, b1));
    }
    static constexpr bool kPacked = true;
    static MOA_DEV void step2x2(float &c0, float &c1, float a0, float b00, float b01, float a1, float b10, float b11) {
        float s00, s01, s10, s11;
        add2(a0, b00, b01, s00, s01);
        add2(a1, b10, b11, s10, s11);
        c0 = fmin3(c0, s00, s10);
        c1 = fmin3(c1, s01, s11);
    }
};
struct F32MaxPlus {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(0xff800000); }
    static MOA_DEV float step(float acc, float a, float b) { return fmaxf(acc, __fadd_rn(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmax3(acc, __fadd_rn(a0, b0), __fadd_rn(a1, b1));
    }
    static constexpr bool kPacked = true;
    static MOA_DEV void step2x2(float &c0, float &c1, float a0, float b00, float b01, float a1, float b10, float b11) {
        float s00, s01, s10, s11;
        add2(a0, b00, b01, s00, s01);
        add2(a1, b10, b11, s10, s11);
        c0 = fmax3(c0, s00, s10);
        c1 = fmax3(c1, s01, s11);
    }
};
struct F32MinTimes {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(0x7f800000); }
    static MOA_DEV float step(float acc, float a, float b) { return fminf(acc, __fmul_rn(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmin3(acc, __fmul_rn(a0, b0), __fmul_rn(a1, b1));
    }
    static constexpr bool kPacked = true;
    static MOA_DEV void step2x2(float &c0, float &c1, float a0, float b00, float b01, float a1, float b10, float b11) {
        float s00, s01, s10, s11;
        mul2(a0, b00, b01, s00, s01);
        mul2(a1, b10, b11, s10, s11);
        c0 = fmin3(c0, s00, s10);
        c1 = fmin3(c1, s01, s11);
    }
};
struct F32MaxTimes {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(0xff800000); }
    static MOA_DEV float step(float acc, float a, float b) { return fmaxf(acc, __fmul_rn(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmax3(acc, __fmul_rn(a0, b0), __fmul_rn(a1, b1));
    }
    static constexpr bool kPacked = true;
    static MOA_DEV void step2x2(float &c0, float &c1, float a0, float b00, float b01, float a1, float b10, float b11) {
        float s00, s01, s10, s11;
        mul2(a0, b00, b01, s00, s01);
        mul2(a1, b10, b11, s10, s11);
        c0 = fmax3(c0, s00, s10);
        c1 = fmax3(c1, s01, s11);
    }
};

}  // namespace sr
}  // namespace moa
