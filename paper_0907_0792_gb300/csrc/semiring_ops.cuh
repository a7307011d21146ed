// Element operators of the CUDA-core generalized inner product, Eq. (2)
// with a general (reduce, combine) pair (Sec. I): identity of the reduce,
// one step acc = reduce(acc, a combine b), and a two-step form that uses the
// three-input min / max of sm_100+.  Shared by the single-problem kernels
// (semiring.cu) and the grouped batch kernel (batch.cu).
#pragma once

#include "common.cuh"

namespace moa {
namespace sr {

struct F32PlusTimes {
    using T = float;
    static MOA_DEV float identity() { return 0.0f; }
    static MOA_DEV float step(float acc, float a, float b) { return fmaf(a, b, acc); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmaf(a1, b1, fmaf(a0, b0, acc));
    }
};
struct F64PlusTimes {
    using T = double;
    static MOA_DEV double identity() { return 0.0; }
    static MOA_DEV double step(double acc, double a, double b) { return fma(a, b, acc); }
    static MOA_DEV double step2(double acc, double a0, double b0, double a1, double b1) {
        return fma(a1, b1, fma(a0, b0, acc));
    }
};
struct I32PlusTimes {
    using T = int32_t;
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
};
struct F32MaxPlus {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(0xff800000); }
    static MOA_DEV float step(float acc, float a, float b) { return fmaxf(acc, __fadd_rn(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmax3(acc, __fadd_rn(a0, b0), __fadd_rn(a1, b1));
    }
};
struct F32MinTimes {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(0x7f800000); }
    static MOA_DEV float step(float acc, float a, float b) { return fminf(acc, __fmul_rn(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmin3(acc, __fmul_rn(a0, b0), __fmul_rn(a1, b1));
    }
};
struct F32MaxTimes {
    using T = float;
    static MOA_DEV float identity() { return __int_as_float(0xff800000); }
    static MOA_DEV float step(float acc, float a, float b) { return fmaxf(acc, __fmul_rn(a, b)); }
    static MOA_DEV float step2(float acc, float a0, float b0, float a1, float b1) {
        return fmax3(acc, __fmul_rn(a0, b0), __fmul_rn(a1, b1));
    }
};

}  // namespace sr
}  // namespace moa
