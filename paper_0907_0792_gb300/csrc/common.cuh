// Shared device helpers of libmoa: element operators of the generalized
// inner / outer product (Sec. I allows any binary operation in both) and
// small inline-PTX wrappers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "moa.h"

#define MOA_DEV __device__ __forceinline__

namespace moa {

// ---------------------------------------------------------------- scalar ops
// Every combine is one correctly rounded IEEE operation (explicit _rn
// intrinsics, so the compiler cannot contract a combine and a reduce into an
// FMA where the result must be bit-exact).
MOA_DEV float op_apply(int op, float a, float b) {
    switch (op) {
    case MOA_OP_ADD: return __fadd_rn(a, b);
    case MOA_OP_SUB: return __fsub_rn(a, b);
    case MOA_OP_MUL: return __fmul_rn(a, b);
    case MOA_OP_DIV: return __fdiv_rn(a, b);
    case MOA_OP_MIN: return fminf(a, b);
    case MOA_OP_MAX: return fmaxf(a, b);
    }
    return __int_as_float(0x7fc00000);
}
MOA_DEV double op_apply(int op, double a, double b) {
    switch (op) {
    case MOA_OP_ADD: return __dadd_rn(a, b);
    case MOA_OP_SUB: return __dsub_rn(a, b);
    case MOA_OP_MUL: return __dmul_rn(a, b);
    case MOA_OP_DIV: return __ddiv_rn(a, b);
    case MOA_OP_MIN: return fmin(a, b);
    case MOA_OP_MAX: return fmax(a, b);
    }
    return __longlong_as_double(0x7ff8000000000000ll);
}
MOA_DEV int32_t op_apply(int op, int32_t a, int32_t b) {
    uint32_t x = (uint32_t)a, y = (uint32_t)b;  // two's-complement wraparound
    switch (op) {
    case MOA_OP_ADD: return (int32_t)(x + y);
    case MOA_OP_SUB: return (int32_t)(x - y);
    case MOA_OP_MUL: return (int32_t)(x * y);
    }
    return 0;
}

// Three-input min / max (one instruction on sm_100+); NaN inputs are
// ignored as with fminf / fmaxf.
MOA_DEV float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
MOA_DEV float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ------------------------------------------------------- bounded waits
// Device status word written by any kernel whose bounded wait gives up
// (one per translation unit that waits; the host reads each of them).
constexpr uint32_t kStatusTimeout = 1u;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

MOA_DEV uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace moa
