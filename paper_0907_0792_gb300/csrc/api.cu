// C ABI of libmoa (include/moa.h): argument validation, psi-flattening and
// dispatch of the generalized inner product (Eq. 2) and outer product
// (Eq. 1), plus the per-stream scratch workspace.
//
// psi-flattening (Fig. 1; the appendix addresses element (i, p) of A at
// i*K + p, (p, j) of B at p*N + j and (i, j) of the result at i*N + j): for rho A =
// <a_0 .. a_{r-2}, p> and rho B = <p, b_1 .. b_{s-1}>, the row-major element
// vectors already are an M x K and a K x N row-major matrix with
// M = prod a, K = p, N = prod b, and D's element vector is the M x N
// row-major product.  No data moves; only the three extents are computed.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "internal.h"
#include "tc.h"

namespace moa {

static constexpr int kMaxRank = 8;
static constexpr unsigned kMaxDtype = MOA_F16;  // largest moa_dtype code

// ------------------------------------------------------------- validation
static moa_status count_elems(int rank, const int64_t *shape, int64_t *count) {
    int64_t n = 1;
    for (int k = 0; k < rank; ++k) {
        const int64_t e = shape[k];
        if (e < 0) return MOA_ERR_OVERFLOW;
        if (e != 0 && n > INT64_MAX / e) return MOA_ERR_OVERFLOW;
        n *= e;
    }
    *count = n;
    return MOA_OK;
}

static size_t elem_bytes(moa_dtype t) {
    switch (t) {
    case MOA_F64: return 8;
    case MOA_F32: return 4;
    case MOA_BF16: return 2;
    case MOA_FP8E4M3: return 1;
    case MOA_I32: return 4;
    case MOA_B1_U32: return 4;
    case MOA_F16: return 2;
    }
    return 0;
}

static bool aligned_to(const void *p, size_t a) { return a == 0 || ((uintptr_t)p % a) == 0; }

static moa_status from_cuda(cudaError_t e) { return e == cudaSuccess ? MOA_OK : MOA_ERR_CUDA; }

moa_status check_device_ptrs(const void *const *ptrs, int n) {
    int dev = -1;
    bool have_dev = false;
    for (int i = 0; i < n; ++i) {
        if (!ptrs[i]) continue;
        if (!have_dev) {
            if (cudaGetDevice(&dev) != cudaSuccess) {
                cudaGetLastError();
                return MOA_ERR_NOT_DEVICE;
            }
            have_dev = true;
        }
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptrs[i]) != cudaSuccess) {
            cudaGetLastError();  // not an address the runtime knows: not device memory
            return MOA_ERR_NOT_DEVICE;
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return MOA_ERR_NOT_DEVICE;
    }
    return MOA_OK;
}

// Fault injection for tests: MOA_FAULT_INJECT=workspace makes every
// workspace allocation fail (read once per process).
static bool inject_workspace_failure() {
    static const bool on = [] {  // read once, thread-safe
        const char *e = std::getenv("MOA_FAULT_INJECT");
        return e && std::strcmp(e, "workspace") == 0;
    }();
    return on;
}

// ------------------------------------------------------------- workspace
namespace {
struct WsKey {
    int device;
    cudaStream_t stream;
    int slot;
    bool operator<(const WsKey &o) const {
        if (device != o.device) return device < o.device;
        if (stream != o.stream) return stream < o.stream;
        return slot < o.slot;
    }
};
struct WsBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_ws_mu;
std::map<WsKey, WsBuf> g_ws;
}  // namespace

void *workspace_get(cudaStream_t stream, size_t bytes, moa_status *st, int slot) {
    *st = MOA_OK;
    if (bytes == 0) return nullptr;
    if (inject_workspace_failure()) {
        *st = MOA_ERR_WORKSPACE;
        return nullptr;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *st = MOA_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_ws_mu);
    WsBuf &b = g_ws[WsKey{dev, stream, slot}];
    if (b.bytes >= bytes) return b.ptr;
    // grow: stream-ordered free + allocation, so work already queued on this
    // stream keeps its buffer until it has finished with it
    if (b.ptr) cudaFreeAsync(b.ptr, stream);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 4;  // head-room against repeated small growth
    want = (want + 255) & ~(size_t)255;
    void *p = nullptr;
    if (cudaMallocAsync(&p, want, stream) != cudaSuccess) {
        cudaGetLastError();
        *st = MOA_ERR_WORKSPACE;
        return nullptr;
    }
    b.ptr = p;
    b.bytes = want;
    return p;
}

static moa_status workspace_release_all() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MOA_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return MOA_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (auto it = g_ws.begin(); it != g_ws.end();) {
        if (it->first.device == dev) {
            if (it->second.ptr) cudaFree(it->second.ptr);
            it = g_ws.erase(it);
        } else {
            ++it;
        }
    }
    return MOA_OK;
}

// ------------------------------------------------------------- inner
struct InnerPlan {
    int64_t M, K, N;
};

static moa_status inner_validate(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                                 const int64_t *shapeA, const void *A, int rankB, const int64_t *shapeB, const void *B,
                                 const void *out, moa_dtype out_dtype, InnerPlan *pl, int ptr_checks = 2) {
    // ptr_checks: 0 shapes and types only, 1 also null and alignment, 2 also device memory
    if (rankA < 1 || rankB < 1 || rankA > kMaxRank || rankB > kMaxRank) return MOA_ERR_RANK;
    if (!shapeA || !shapeB) return MOA_ERR_NULL;
    if ((unsigned)reduce > MOA_OP_AND || (unsigned)combine > MOA_OP_AND || (unsigned)dtype > kMaxDtype ||
        (unsigned)out_dtype > kMaxDtype || (unsigned)form > MOA_FORM_F16)
        return MOA_ERR_INVALID;
    int64_t nA, nB;
    moa_status st;
    if ((st = count_elems(rankA, shapeA, &nA)) != MOA_OK) return st;
    if ((st = count_elems(rankB, shapeB, &nB)) != MOA_OK) return st;
    // Eq. (2): the contracted axes must have the same length
    if (shapeA[rankA - 1] != shapeB[0]) return MOA_ERR_SHAPE_MISMATCH;
    int64_t M, N;
    if ((st = count_elems(rankA - 1, shapeA, &M)) != MOA_OK) return st;
    if ((st = count_elems(rankB - 1, shapeB + 1, &N)) != MOA_OK) return st;
    const int64_t K = shapeA[rankA - 1];
    if (M != 0 && N > INT64_MAX / M) return MOA_ERR_OVERFLOW;

    // supported (reduce, combine, dtype, out_dtype, form) tuples
    bool ok = false;
    if (reduce == MOA_OP_ADD && combine == MOA_OP_MUL) {
        ok = (dtype == MOA_F64 && out_dtype == MOA_F64 && (form == MOA_FORM_NATIVE || form == MOA_FORM_OZAKI)) ||
             (dtype == MOA_F32 && out_dtype == MOA_F32 &&
              (form == MOA_FORM_NATIVE || form == MOA_FORM_BF16 || form == MOA_FORM_F16 || form == MOA_FORM_BF16X3 ||
               form == MOA_FORM_FP8_T128)) ||
             ((dtype == MOA_BF16 || dtype == MOA_F16 || dtype == MOA_FP8E4M3) && out_dtype == MOA_F32 &&
              form == MOA_FORM_NATIVE) ||
             (dtype == MOA_I32 && out_dtype == MOA_I32 && form == MOA_FORM_NATIVE);
    } else if ((reduce == MOA_OP_MIN || reduce == MOA_OP_MAX) &&
               (combine == MOA_OP_ADD || combine == MOA_OP_SUB || combine == MOA_OP_MUL || combine == MOA_OP_MIN ||
                combine == MOA_OP_MAX)) {
        ok = dtype == MOA_F32 && out_dtype == MOA_F32 && form == MOA_FORM_NATIVE;
    } else if (reduce == MOA_OP_OR && combine == MOA_OP_AND) {
        ok = dtype == MOA_B1_U32 && out_dtype == MOA_B1_U32 && form == MOA_FORM_NATIVE;
    }
    if (!ok) return MOA_ERR_UNSUPPORTED;

    pl->M = M, pl->K = K, pl->N = N;
    if (ptr_checks == 0) return MOA_OK;
    if (M * N > 0) {
        if (!out) return MOA_ERR_NULL;
        if (M * K > 0 && !A) return MOA_ERR_NULL;
        if (K * N > 0 && !B) return MOA_ERR_NULL;
    }
    if (!aligned_to(A, elem_bytes(dtype)) || !aligned_to(B, elem_bytes(dtype)) ||
        !aligned_to(out, elem_bytes(out_dtype)))
        return MOA_ERR_ALIGNMENT;
    if (ptr_checks >= 2 && M * N > 0) {  // only operands the call reads, and the result it writes
        const void *used[3] = {M * K > 0 ? A : nullptr, K * N > 0 ? B : nullptr, out};
        if ((st = check_device_ptrs(used, 3)) != MOA_OK) return st;
    }
    return MOA_OK;
}

static moa_status inner_identity_fill(moa_op reduce, moa_dtype out_dtype, void *out, int64_t M, int64_t N,
                                      cudaStream_t s) {
    if (out_dtype == MOA_F64) return from_cuda(launch_fill64((uint64_t *)out, 0ull, M * N, s));  // +0.0
    if (out_dtype == MOA_B1_U32) return from_cuda(launch_fill32((uint32_t *)out, 0u, (M * N + 31) / 32, s));
    uint32_t v = 0u;  // F32 +0.0 and I32 0
    if (out_dtype == MOA_F32 && reduce == MOA_OP_MIN) v = 0x7f800000u;
    if (out_dtype == MOA_F32 && reduce == MOA_OP_MAX) v = 0xff800000u;
    return from_cuda(launch_fill32((uint32_t *)out, v, M * N, s));
}

static moa_status inner_run(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, const void *A,
                            const void *B, void *out, moa_dtype out_dtype, const InnerPlan &pl, cudaStream_t s) {
    const int64_t M = pl.M, K = pl.K, N = pl.N;
    if (M == 0 || N == 0) return MOA_OK;
    if (K == 0) return inner_identity_fill(reduce, out_dtype, out, M, N, s);

    if (reduce == MOA_OP_OR) {
        moa_status st;
        if (or_and_tc_applies(M, N, K)) {  // tensor cores, exact counting
            void *ws = workspace_get(s, or_and_tc_workspace_bytes(M, N, K), &st);
            if (st != MOA_OK) return st;
            return from_cuda(launch_or_and_tc((const uint32_t *)A, (const uint32_t *)B, (uint32_t *)out, M, N, K, ws, s));
        }
        void *ws = workspace_get(s, bits_workspace_bytes(M, N, K), &st);
        if (st != MOA_OK) return st;
        return from_cuda(launch_or_and((const uint32_t *)A, (const uint32_t *)B, (uint32_t *)out, M, N, K, ws, s));
    }
    if (reduce == MOA_OP_MIN || reduce == MOA_OP_MAX) {
        const bool mx = reduce == MOA_OP_MAX;
        SemiringKind k;
        switch (combine) {
        case MOA_OP_ADD: k = mx ? SR_F32_MAX_PLUS : SR_F32_MIN_PLUS; break;
        case MOA_OP_SUB: k = mx ? SR_F32_MAX_MINUS : SR_F32_MIN_MINUS; break;
        case MOA_OP_MUL: k = mx ? SR_F32_MAX_TIMES : SR_F32_MIN_TIMES; break;
        case MOA_OP_MIN: k = mx ? SR_F32_MAX_MIN : SR_F32_MIN_MIN; break;
        case MOA_OP_MAX: k = mx ? SR_F32_MAX_MAX : SR_F32_MIN_MAX; break;
        default: return MOA_ERR_UNSUPPORTED;
        }
        return from_cuda(launch_semiring(k, A, B, out, M, N, K, s));
    }
    // (add, mul)
    switch (dtype) {
    case MOA_I32:
        if (i32_tc_applies(M, N, K)) {  // tensor cores when the values are int8-range, checked on the device
            moa_status st;
            void *ws = workspace_get(s, i32_tc_workspace_bytes(M, N, K), &st);
            if (st != MOA_OK) return st;
            return tc_inner_i32((const int32_t *)A, (const int32_t *)B, (int32_t *)out, M, N, K, ws, s);
        }
        return from_cuda(launch_semiring(SR_I32_PLUS_TIMES, A, B, out, M, N, K, s));
    case MOA_F64:
        if (form == MOA_FORM_OZAKI) return tc_inner_ozaki((const double *)A, (const double *)B, (double *)out, M, N, K, s);
        if (skinny_applies(M, N, K)) return from_cuda(launch_skinny(true, A, B, out, M, N, K, s));
        return from_cuda(launch_semiring(SR_F64_PLUS_TIMES, A, B, out, M, N, K, s));
    case MOA_F32:
        if (form == MOA_FORM_NATIVE) {
            if (skinny_applies(M, N, K)) return from_cuda(launch_skinny(false, A, B, out, M, N, K, s));
            return from_cuda(launch_semiring(SR_F32_PLUS_TIMES, A, B, out, M, N, K, s));
        }
        return tc_inner_f32(form, (const float *)A, (const float *)B, (float *)out, M, N, K, s);
    case MOA_BF16: return tc_inner_bf16((const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, (float *)out, M, N, K, s);
    case MOA_F16: return tc_inner_f16((const __half *)A, (const __half *)B, (float *)out, M, N, K, s);
    case MOA_FP8E4M3: return tc_inner_e4m3((const uint8_t *)A, (const uint8_t *)B, (float *)out, M, N, K, s);
    default: break;
    }
    return MOA_ERR_UNSUPPORTED;
}

size_t dtype_bytes(moa_dtype t) { return elem_bytes(t); }

// Validation of moa_inner (all pointer checks when `launch`, none
// otherwise: moa_inner_host validates its host pointers itself) and, with
// `launch`, the run on `stream`; the psi-flattened extents are returned.
moa_status inner_checked(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                         const int64_t *shapeA, const void *A, int rankB, const int64_t *shapeB, const void *B,
                         void *out, moa_dtype out_dtype, cudaStream_t stream, int64_t *M, int64_t *K, int64_t *N,
                         bool launch) {
    InnerPlan pl;
    moa_status st = inner_validate(reduce, combine, dtype, form, rankA, shapeA, A, rankB, shapeB, B, out, out_dtype, &pl,
                                   launch ? 2 : 0);
    if (st != MOA_OK) return st;
    *M = pl.M, *K = pl.K, *N = pl.N;
    return launch ? inner_run(reduce, combine, dtype, form, A, B, out, out_dtype, pl, stream) : MOA_OK;
}

}  // namespace moa

using namespace moa;

extern "C" {

moa_status moa_inner_shape(int rankA, const int64_t *shapeA, int rankB, const int64_t *shapeB, int *rankD,
                           int64_t *shapeD) {
    if (rankA < 1 || rankB < 1 || rankA > kMaxRank || rankB > kMaxRank) return MOA_ERR_RANK;
    if (!shapeA || !shapeB || !rankD || (rankA + rankB - 2 > 0 && !shapeD)) return MOA_ERR_NULL;
    int64_t n;
    moa_status st;
    if ((st = count_elems(rankA, shapeA, &n)) != MOA_OK) return st;
    if ((st = count_elems(rankB, shapeB, &n)) != MOA_OK) return st;
    if (shapeA[rankA - 1] != shapeB[0]) return MOA_ERR_SHAPE_MISMATCH;
    int r = 0;
    for (int k = 0; k < rankA - 1; ++k) shapeD[r++] = shapeA[k];
    for (int k = 1; k < rankB; ++k) shapeD[r++] = shapeB[k];
    *rankD = r;
    return MOA_OK;
}

moa_status moa_outer_shape(int rankA, const int64_t *shapeA, int rankB, const int64_t *shapeB, int *rankC,
                           int64_t *shapeC) {
    if (rankA < 0 || rankB < 0 || rankA > kMaxRank || rankB > kMaxRank) return MOA_ERR_RANK;
    if ((rankA > 0 && !shapeA) || (rankB > 0 && !shapeB) || !rankC || (rankA + rankB > 0 && !shapeC))
        return MOA_ERR_NULL;
    int64_t nA, nB;
    moa_status st;
    if ((st = count_elems(rankA, shapeA, &nA)) != MOA_OK) return st;
    if ((st = count_elems(rankB, shapeB, &nB)) != MOA_OK) return st;
    if (nA != 0 && nB > INT64_MAX / nA) return MOA_ERR_OVERFLOW;
    int r = 0;
    for (int k = 0; k < rankA; ++k) shapeC[r++] = shapeA[k];
    for (int k = 0; k < rankB; ++k) shapeC[r++] = shapeB[k];
    *rankC = r;
    return MOA_OK;
}

moa_status moa_inner(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA, const int64_t *shapeA,
                     const void *A, int rankB, const int64_t *shapeB, const void *B, void *out, moa_dtype out_dtype,
                     moa_stream stream) {
    InnerPlan pl;
    moa_status st = inner_validate(reduce, combine, dtype, form, rankA, shapeA, A, rankB, shapeB, B, out, out_dtype, &pl);
    if (st != MOA_OK) return st;
    return inner_run(reduce, combine, dtype, form, A, B, out, out_dtype, pl, (cudaStream_t)stream);
}

moa_status moa_inner_e4m3_scaled(int rankA, const int64_t *shapeA, const void *A, const float *scale_a, int rankB,
                                 const int64_t *shapeB, const void *B, const float *scale_b, float *out,
                                 moa_stream stream) {
    InnerPlan pl;
    moa_status st = inner_validate(MOA_OP_ADD, MOA_OP_MUL, MOA_FP8E4M3, MOA_FORM_NATIVE, rankA, shapeA, A, rankB, shapeB,
                                   B, out, MOA_F32, &pl);
    if (st != MOA_OK) return st;
    const int64_t M = pl.M, K = pl.K, N = pl.N;
    if (M == 0 || N == 0) return MOA_OK;
    const cudaStream_t s = (cudaStream_t)stream;
    if (K == 0) return inner_identity_fill(MOA_OP_ADD, MOA_F32, out, M, N, s);
    if (!scale_a || !scale_b) return MOA_ERR_NULL;
    if (!aligned_to(scale_a, 4) || !aligned_to(scale_b, 4)) return MOA_ERR_ALIGNMENT;
    const void *used[2] = {scale_a, scale_b};
    if ((st = check_device_ptrs(used, 2)) != MOA_OK) return st;
    return tc_inner_e4m3((const uint8_t *)A, (const uint8_t *)B, out, M, N, K, s, scale_a, scale_b);
}

moa_status moa_transpose(moa_dtype dtype, int rank, const int64_t *shape, const int *perm, const void *A, void *out,
                         moa_stream stream) {
    if (rank < 0 || rank > kMaxRank) return MOA_ERR_RANK;
    if (rank > 0 && (!shape || !perm)) return MOA_ERR_NULL;
    if ((unsigned)dtype > kMaxDtype) return MOA_ERR_INVALID;
    if (dtype == MOA_B1_U32) return MOA_ERR_UNSUPPORTED;  // a packed bit stream has no per-element address
    bool seen[kMaxRank] = {};
    for (int k = 0; k < rank; ++k) {
        if (perm[k] < 0 || perm[k] >= rank || seen[perm[k]]) return MOA_ERR_INVALID;
        seen[perm[k]] = true;
    }
    int64_t n;
    moa_status st;
    if ((st = count_elems(rank, shape, &n)) != MOA_OK) return st;
    if (n == 0) return MOA_OK;
    if (!A || !out) return MOA_ERR_NULL;
    if (A == out) return MOA_ERR_INVALID;
    if (!aligned_to(A, elem_bytes(dtype)) || !aligned_to(out, elem_bytes(dtype))) return MOA_ERR_ALIGNMENT;
    const void *used[2] = {A, out};
    if ((st = check_device_ptrs(used, 2)) != MOA_OK) return st;
    return from_cuda(launch_transpose(elem_bytes(dtype), rank, shape, perm, A, out, (cudaStream_t)stream));
}

moa_status moa_inner_axes(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                          const int64_t *shapeA, const void *A, int axisA, int rankB, const int64_t *shapeB,
                          const void *B, int axisB, void *out, moa_dtype out_dtype, moa_stream stream) {
    if (rankA < 1 || rankB < 1 || rankA > kMaxRank || rankB > kMaxRank) return MOA_ERR_RANK;
    if (!shapeA || !shapeB) return MOA_ERR_NULL;
    if (axisA < 0 || axisA >= rankA || axisB < 0 || axisB >= rankB) return MOA_ERR_INVALID;
    // A with axisA moved last, B with axisB moved first: the form of Eq. (2)
    int64_t sa[kMaxRank], sb[kMaxRank];
    int pa[kMaxRank], pb[kMaxRank];
    int r = 0;
    for (int k = 0; k < rankA; ++k)
        if (k != axisA) pa[r] = k, sa[r++] = shapeA[k];
    pa[r] = axisA, sa[r] = shapeA[axisA];
    pb[0] = axisB, sb[0] = shapeB[axisB];
    r = 1;
    for (int k = 0; k < rankB; ++k)
        if (k != axisB) pb[r] = k, sb[r++] = shapeB[k];
    InnerPlan pl;
    moa_status st = inner_validate(reduce, combine, dtype, form, rankA, sa, A, rankB, sb, B, out, out_dtype, &pl, 1);
    if (st != MOA_OK) return st;
    const bool moveA = axisA != rankA - 1, moveB = axisB != 0;
    const bool empty = pl.M == 0 || pl.N == 0 || pl.K == 0;  // nothing to read
    if (dtype == MOA_B1_U32 && (moveA || moveB) && !empty) return MOA_ERR_UNSUPPORTED;  // bit streams are not transposed
    if (pl.M * pl.N > 0) {
        const void *used[3] = {pl.M * pl.K > 0 ? A : nullptr, pl.K * pl.N > 0 ? B : nullptr, out};
        if ((st = check_device_ptrs(used, 3)) != MOA_OK) return st;
    }
    if ((!moveA && !moveB) || empty)
        return inner_run(reduce, combine, dtype, form, A, B, out, out_dtype, pl, (cudaStream_t)stream);
    // transposed copies in the stream's second workspace slot (the inner
    // product may use the first itself)
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t es = elem_bytes(dtype);
    const size_t bytesA = moveA ? (size_t)(pl.M * pl.K) * es : 0, bytesB = moveB ? (size_t)(pl.K * pl.N) * es : 0;
    const size_t offB = (bytesA + 255) & ~(size_t)255;
    void *tmp = workspace_get(s, offB + bytesB, &st, 1);
    if (st != MOA_OK) return st;
    const void *a = A, *b = B;
    cudaError_t e = cudaSuccess;
    if (moveA) {
        e = launch_transpose(es, rankA, shapeA, pa, A, tmp, s);
        a = tmp;
    }
    if (moveB && e == cudaSuccess) {
        e = launch_transpose(es, rankB, shapeB, pb, B, (uint8_t *)tmp + offB, s);
        b = (uint8_t *)tmp + offB;
    }
    return e == cudaSuccess ? inner_run(reduce, combine, dtype, form, a, b, out, out_dtype, pl, s) : MOA_ERR_CUDA;
}

moa_status moa_outer(moa_op op, moa_dtype dtype, int rankA, const int64_t *shapeA, const void *A, int rankB,
                     const int64_t *shapeB, const void *B, void *out, moa_dtype out_dtype, moa_stream stream) {
    if (rankA < 0 || rankB < 0 || rankA > kMaxRank || rankB > kMaxRank) return MOA_ERR_RANK;
    if ((rankA > 0 && !shapeA) || (rankB > 0 && !shapeB)) return MOA_ERR_NULL;
    if ((unsigned)op > MOA_OP_AND || (unsigned)dtype > kMaxDtype || (unsigned)out_dtype > kMaxDtype)
        return MOA_ERR_INVALID;
    int64_t M, N;
    moa_status st;
    if ((st = count_elems(rankA, shapeA, &M)) != MOA_OK) return st;
    if ((st = count_elems(rankB, shapeB, &N)) != MOA_OK) return st;
    if (M != 0 && N > INT64_MAX / M) return MOA_ERR_OVERFLOW;
    const bool float_op = op <= MOA_OP_MAX;
    bool ok = false;
    if (float_op && ((dtype == MOA_F64 && out_dtype == MOA_F64) || (dtype == MOA_F32 && out_dtype == MOA_F32) ||
                     (dtype == MOA_BF16 && (out_dtype == MOA_BF16 || out_dtype == MOA_F32))))
        ok = true;
    if (dtype == MOA_I32 && out_dtype == MOA_I32 && (op == MOA_OP_ADD || op == MOA_OP_SUB || op == MOA_OP_MUL)) ok = true;
    if (!ok) return MOA_ERR_UNSUPPORTED;
    if (M == 0 || N == 0) return MOA_OK;
    if (!A || !B || !out) return MOA_ERR_NULL;
    if (!aligned_to(A, elem_bytes(dtype)) || !aligned_to(B, elem_bytes(dtype)) ||
        !aligned_to(out, elem_bytes(out_dtype)))
        return MOA_ERR_ALIGNMENT;
    const void *used[3] = {A, B, out};
    if ((st = check_device_ptrs(used, 3)) != MOA_OK) return st;
    return from_cuda(launch_outer(op, dtype, out_dtype, A, B, out, M, N, (cudaStream_t)stream));
}

const char *moa_status_string(moa_status s) {
    switch (s) {
    case MOA_OK: return "ok";
    case MOA_ERR_NULL: return "null pointer";
    case MOA_ERR_RANK: return "rank out of range";
    case MOA_ERR_SHAPE_MISMATCH: return "shape mismatch: last axis of A differs from first axis of B";
    case MOA_ERR_OVERFLOW: return "negative extent or element count overflow";
    case MOA_ERR_UNSUPPORTED: return "unsupported operator / dtype / form combination";
    case MOA_ERR_WORKSPACE: return "workspace allocation failed";
    case MOA_ERR_CUDA: return "CUDA error";
    case MOA_ERR_TIMEOUT: return "device wait timed out";
    case MOA_ERR_INTERNAL: return "internal error";
    case MOA_ERR_ALIGNMENT: return "misaligned pointer";
    case MOA_ERR_INVALID: return "invalid argument";
    case MOA_ERR_SCRATCH_LIMIT: return "problem needs more scratch than the fixed no-allocation buffer holds";
    case MOA_ERR_NOT_DEVICE: return "pointer is not device memory of the current device";
    }
    return "unknown status";
}

moa_status moa_device_status(moa_stream stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return MOA_ERR_CUDA;
    uint32_t flags = 0, bflags = 0, pflags = 0;
    if (tc_read_and_clear_status(&flags) != cudaSuccess) return MOA_ERR_CUDA;
    if (batch_read_and_clear_status(&bflags) != cudaSuccess) return MOA_ERR_CUDA;
    if (pair_read_and_clear_status(&pflags) != cudaSuccess) return MOA_ERR_CUDA;
    if ((flags | bflags | pflags) & kStatusTimeout) return MOA_ERR_TIMEOUT;
    return MOA_OK;
}

moa_status moa_release_workspace(void) { return workspace_release_all(); }

moa_status moa_selftest_wait_timeout(uint32_t limit_us, moa_stream stream) {
    if (limit_us == 0 || limit_us > 1000000u) return MOA_ERR_INVALID;
    return from_cuda(tc_wait_probe((uint64_t)limit_us * 1000ull, (cudaStream_t)stream));
}

int moa_version(void) { return 0x000100; }

}  // extern "C"
