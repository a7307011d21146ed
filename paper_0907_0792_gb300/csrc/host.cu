// moa_inner_host: the generalized inner product (Eq. 2) of arrays held in
// host memory.  The call copies A and B to the device, runs the same path as
// moa_inner there and copies D back, all ordered on the caller's stream.
//
// For a result of many rows the copies overlap the computation: the
// psi-flattened rows of A and D (Fig. 1: row i of D needs row i of A and all
// of B) are cut into up to four blocks; B and the first block of A go in
// first, then block b computes while block b+1 of A comes in on the upload
// streams and block b-1 of D goes out on the download streams.  Two device
// buffers per operand block alternate.  Every copy is split in two halves on
// two streams of its direction, so two copy engines share it (one engine
// alone reaches about half of the host link).  The copy streams belong to the
// library (one set per device and caller stream) and wait on, and are waited
// on by, the caller's stream through events, so the whole call is ordered on
// `stream` like every other call.  In the Ozaki form B's column maxima and
// digit planes are made once, not once per block.
#include <cstring>
#include <map>
#include <mutex>

#include "internal.h"
#include "tc.h"

namespace moa {

moa_status inner_checked(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                         const int64_t *shapeA, const void *A, int rankB, const int64_t *shapeB, const void *B,
                         void *out, moa_dtype out_dtype, cudaStream_t stream, int64_t *M, int64_t *K, int64_t *N,
                         bool launch);
size_t dtype_bytes(moa_dtype t);

namespace {

constexpr int kBufs = 2;
constexpr int kMaxBlocks = 4;
constexpr int kLanes = 2;  // copy streams per direction

struct CopyStreams {
    cudaStream_t up[kLanes] = {}, down[kLanes] = {};
    cudaEvent_t start = nullptr;
    cudaEvent_t b_in[kLanes] = {}, finished[kLanes] = {};
    cudaEvent_t a_in[kBufs][kLanes] = {}, computed[kBufs] = {}, d_out[kBufs][kLanes] = {};
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, CopyStreams> g_streams;

moa_status copy_streams(cudaStream_t s, CopyStreams **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MOA_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_streams.find({dev, s});
    if (it == g_streams.end()) {
        CopyStreams c;
        auto ev = [](cudaEvent_t *e) { return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess; };
        bool ok = ev(&c.start);
        for (int l = 0; l < kLanes && ok; ++l)
            ok = cudaStreamCreateWithFlags(&c.up[l], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaStreamCreateWithFlags(&c.down[l], cudaStreamNonBlocking) == cudaSuccess && ev(&c.b_in[l]) &&
                 ev(&c.finished[l]);
        for (int i = 0; i < kBufs && ok; ++i) {
            ok = ev(&c.computed[i]);
            for (int l = 0; l < kLanes && ok; ++l) ok = ev(&c.a_in[i][l]) && ev(&c.d_out[i][l]);
        }
        if (!ok) {
            cudaGetLastError();
            return MOA_ERR_CUDA;
        }
        it = g_streams.emplace(std::make_pair(dev, s), c).first;
    }
    *out = &it->second;
    return MOA_OK;
}

bool host_memory(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace
}  // namespace moa

using namespace moa;

extern "C" moa_status moa_inner_host(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                                     const int64_t *shapeA, const void *A, int rankB, const int64_t *shapeB,
                                     const void *B, void *out, moa_dtype out_dtype, moa_stream stream) {
    int64_t M = 0, K = 0, N = 0;
    // validation of everything but where the memory lives
    moa_status st = inner_checked(reduce, combine, dtype, form, rankA, shapeA, nullptr, rankB, shapeB, nullptr,
                                  nullptr, out_dtype, nullptr, &M, &K, &N, false);
    if (st != MOA_OK) return st;
    if (M == 0 || N == 0) return MOA_OK;
    if (!out || (M * K > 0 && !A) || (K * N > 0 && !B)) return MOA_ERR_NULL;
    if (!host_memory(out) || (M * K > 0 && !host_memory(A)) || (K * N > 0 && !host_memory(B))) return MOA_ERR_INVALID;
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t ea = dtype_bytes(dtype), ed = dtype_bytes(out_dtype);
    // blocks of rows (whole result for packed bits, whose rows need not start on a word)
    int nb = 1;
    if (dtype != MOA_B1_U32) {
        nb = (int)(M / 512);
        nb = nb < 1 ? 1 : (nb > kMaxBlocks ? kMaxBlocks : nb);
    }
    const int64_t rows = (M + nb - 1) / nb;
    const size_t bytesB = dtype == MOA_B1_U32 ? (size_t)((K * N + 31) / 32) * 4 : (size_t)(K * N) * ea;
    const size_t bytesA = dtype == MOA_B1_U32 ? (size_t)((M * K + 31) / 32) * 4 : (size_t)(rows * K) * ea;
    const size_t bytesD = out_dtype == MOA_B1_U32 ? (size_t)((M * N + 31) / 32) * 4 : (size_t)(rows * N) * ed;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t offA = up(bytesB), offD = offA + kBufs * up(bytesA), total = offD + kBufs * up(bytesD);
    uint8_t *ws = (uint8_t *)workspace_get(s, total, &st, 2);
    if (st != MOA_OK) return st;
    CopyStreams *c = nullptr;
    if ((st = copy_streams(s, &c)) != MOA_OK) return st;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // one copy as two halves (split on a 256-byte boundary), one per stream of `lanes`
    auto copy2 = [&](void *dst, const void *src, size_t n, cudaMemcpyKind kind, cudaStream_t *lanes) -> bool {
        const size_t h = n < 512 ? n : (n / 2 + 255) & ~(size_t)255;
        if (h && !ok(cudaMemcpyAsync(dst, src, h, kind, lanes[0]))) return false;
        return n == h || ok(cudaMemcpyAsync((uint8_t *)dst + h, (const uint8_t *)src + h, n - h, kind, lanes[1]));
    };
    // the copy streams start after the work already queued on `stream` (which
    // may still read the buffers of an earlier call)
    if (!ok(cudaEventRecord(c->start, s))) return MOA_ERR_CUDA;
    for (int l = 0; l < kLanes; ++l)
        if (!ok(cudaStreamWaitEvent(c->up[l], c->start, 0)) || !ok(cudaStreamWaitEvent(c->down[l], c->start, 0)))
            return MOA_ERR_CUDA;
    uint8_t *dB = ws, *dA[kBufs], *dD[kBufs];
    for (int i = 0; i < kBufs; ++i) dA[i] = ws + offA + i * up(bytesA), dD[i] = ws + offD + i * up(bytesD);
    if (bytesB && !copy2(dB, B, bytesB, cudaMemcpyHostToDevice, c->up)) return MOA_ERR_CUDA;
    for (int l = 0; l < kLanes; ++l)
        if (!ok(cudaEventRecord(c->b_in[l], c->up[l]))) return MOA_ERR_CUDA;
    auto upload = [&](int b) -> bool {
        const int64_t r0 = b * rows, r1 = (r0 + rows < M) ? r0 + rows : M;
        const size_t n = dtype == MOA_B1_U32 ? bytesA : (size_t)((r1 - r0) * K) * ea;
        const uint8_t *src = (const uint8_t *)A + (dtype == MOA_B1_U32 ? 0 : (size_t)(r0 * K) * ea);
        for (int l = 0; l < kLanes; ++l)  // the buffer is free once block b - kBufs is computed
            if (b >= kBufs && !ok(cudaStreamWaitEvent(c->up[l], c->computed[b % kBufs], 0))) return false;
        if (n && !copy2(dA[b % kBufs], src, n, cudaMemcpyHostToDevice, c->up)) return false;
        for (int l = 0; l < kLanes; ++l)
            if (!ok(cudaEventRecord(c->a_in[b % kBufs][l], c->up[l]))) return false;
        return true;
    };
    if (!upload(0)) return MOA_ERR_CUDA;
    for (int l = 0; l < kLanes; ++l)
        if (!ok(cudaStreamWaitEvent(s, c->b_in[l], 0))) return MOA_ERR_CUDA;
    // The Ozaki form prepares B (column maxima, digit planes) once for all
    // row blocks, while the first block of A is still coming in.
    const bool ozaki_blocks = reduce == MOA_OP_ADD && combine == MOA_OP_MUL && dtype == MOA_F64 &&
                              form == MOA_FORM_OZAKI && K > 0;
    OzakiB ob{};
    void *oz_rows_ws = nullptr;
    if (ozaki_blocks) {
        void *oz_b_ws = workspace_get(s, ozaki_b_bytes(K, N), &st, 3);
        if (st != MOA_OK) return st;
        oz_rows_ws = workspace_get(s, ozaki_rows_bytes(rows, K), &st, 0);
        if (st != MOA_OK) return st;
        if ((st = ozaki_prepare_b((const double *)dB, K, N, oz_b_ws, &ob, s)) != MOA_OK) return st;
    }
    for (int b = 0; b < nb; ++b) {
        const int64_t r0 = b * rows, r1 = (r0 + rows < M) ? r0 + rows : M;
        if (b + 1 < nb && !upload(b + 1)) return MOA_ERR_CUDA;
        for (int l = 0; l < kLanes; ++l) {
            if (!ok(cudaStreamWaitEvent(s, c->a_in[b % kBufs][l], 0))) return MOA_ERR_CUDA;
            if (b >= kBufs && !ok(cudaStreamWaitEvent(s, c->d_out[b % kBufs][l], 0))) return MOA_ERR_CUDA;  // D free
        }
        // the block as its own inner product: rho A = <rows, K>, rho B = <K, N>
        const int64_t sa[2] = {r1 - r0, K}, sb[2] = {K, N};
        int64_t m, k, n;
        if (ozaki_blocks)
            st = ozaki_rows((const double *)dA[b % kBufs], r1 - r0, ob, (double *)dD[b % kBufs], oz_rows_ws, s);
        else
            st = inner_checked(reduce, combine, dtype, form, 2, sa, dA[b % kBufs], 2, sb, dB, dD[b % kBufs], out_dtype,
                               s, &m, &k, &n, true);
        if (st != MOA_OK) return st;
        if (!ok(cudaEventRecord(c->computed[b % kBufs], s))) return MOA_ERR_CUDA;
        for (int l = 0; l < kLanes; ++l)
            if (!ok(cudaStreamWaitEvent(c->down[l], c->computed[b % kBufs], 0))) return MOA_ERR_CUDA;
        const size_t nd = out_dtype == MOA_B1_U32 ? bytesD : (size_t)((r1 - r0) * N) * ed;
        uint8_t *dst = (uint8_t *)out + (out_dtype == MOA_B1_U32 ? 0 : (size_t)(r0 * N) * ed);
        if (nd && !copy2(dst, dD[b % kBufs], nd, cudaMemcpyDeviceToHost, c->down)) return MOA_ERR_CUDA;
        for (int l = 0; l < kLanes; ++l)
            if (!ok(cudaEventRecord(c->d_out[b % kBufs][l], c->down[l]))) return MOA_ERR_CUDA;
    }
    // `stream` is done with the call once the last result has left the device
    for (int l = 0; l < kLanes; ++l)
        if (!ok(cudaEventRecord(c->finished[l], c->down[l])) || !ok(cudaStreamWaitEvent(s, c->finished[l], 0)) ||
            !ok(cudaStreamWaitEvent(s, c->a_in[(nb - 1) % kBufs][l], 0)))
            return MOA_ERR_CUDA;
    return MOA_OK;
}
