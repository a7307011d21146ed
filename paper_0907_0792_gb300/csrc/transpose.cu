// Transpose of a multi-dimensional array: out[i_perm[0], .., i_perm[r-1]] =
// in[i_0, .., i_{r-1}], i.e. output axis k is input axis perm[k].  It moves a
// contraction axis into the place Eq. (2) contracts (the last axis of A, the
// first of B), so that the generalized inner product runs over any pair of
// axes of equal length.  Pure data movement: HBM-bound, bit-exact.
//
// Host planning first drops axes of extent 1 and merges input axes that stay
// adjacent and in order in the output (their elements then move as one run).
// Two kernels remain:
//   * the input's innermost axis stays innermost: each row of that axis is
//     copied as a contiguous run, reads and writes coalesced;
//   * otherwise a 32 x 32 tile over (input innermost axis x, the input axis y
//     that becomes the output's innermost) goes through shared memory, so the
//     reads run along x and the writes along y; the remaining axes index
//     independent tiles.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace moa {
namespace {

constexpr int kMaxDims = 8;

// Independent axes (outer loop) with their input and output strides.
struct Outer {
    int nd = 0;
    int64_t ext[kMaxDims], is[kMaxDims], os[kMaxDims];
};

MOA_DEV void outer_offsets(const Outer &o, int64_t b, int64_t &in_off, int64_t &out_off) {
    in_off = 0, out_off = 0;
    for (int k = o.nd - 1; k >= 0; --k) {
        const int64_t e = o.ext[k], q = b / e, i = b - q * e;
        in_off += i * o.is[k];
        out_off += i * o.os[k];
        b = q;
    }
}

// Rows of n contiguous elements; rows indexed over `o`.
template <typename T>
__global__ void __launch_bounds__(256) copy_rows(const T *__restrict__ in, T *__restrict__ out, Outer o, int64_t rows,
                                                 int64_t n) {
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        int64_t ib, ob;
        outer_offsets(o, r, ib, ob);
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) out[ob + c] = __ldg(in + ib + c);
    }
}

// 32 x 32 tiles of the (y, x) plane: in[y * isy + x] -> out[x * osx + y].
template <typename T>
__global__ void __launch_bounds__(256) tile_transpose(const T *__restrict__ in, T *__restrict__ out, Outer o,
                                                      int64_t nb, int64_t nx, int64_t ny, int64_t isy, int64_t osx) {
    __shared__ T t[32][33];
    const int64_t tx = (nx + 31) / 32, ty = (ny + 31) / 32, tiles = nb * tx * ty;
    for (int64_t id = blockIdx.x; id < tiles; id += gridDim.x) {
        const int64_t b = id / (tx * ty), rem = id - b * (tx * ty);
        const int64_t y0 = (rem / tx) * 32, x0 = (rem % tx) * 32;
        int64_t ib, ob;
        outer_offsets(o, b, ib, ob);
        const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;  // 32 x 8 threads
        for (int j = ly; j < 32; j += 8) {
            const int64_t y = y0 + j, x = x0 + lx;
            if (y < ny && x < nx) t[j][lx] = __ldg(in + ib + y * isy + x);
        }
        __syncthreads();
        for (int j = ly; j < 32; j += 8) {
            const int64_t x = x0 + j, y = y0 + lx;
            if (x < nx && y < ny) out[ob + x * osx + y] = t[lx][j];
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t run(const void *in, void *out, const Outer &o, bool rows_case, int64_t nb, int64_t nx, int64_t ny,
                int64_t isy, int64_t osx, cudaStream_t s) {
    constexpr int64_t kMaxGrid = 152 * 32;
    if (rows_case) {
        copy_rows<T><<<(unsigned)std::min<int64_t>(nb, kMaxGrid), 256, 0, s>>>((const T *)in, (T *)out, o, nb, nx);
    } else {
        const int64_t tiles = nb * ((nx + 31) / 32) * ((ny + 31) / 32);
        tile_transpose<T><<<(unsigned)std::min<int64_t>(tiles, kMaxGrid), 256, 0, s>>>((const T *)in, (T *)out, o, nb,
                                                                                        nx, ny, isy, osx);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transpose(size_t elem_bytes, int rank, const int64_t *shape, const int *perm, const void *in,
                             void *out, cudaStream_t s) {
    int64_t total = 1;
    for (int k = 0; k < rank; ++k) total *= shape[k];
    if (total == 0) return cudaSuccess;
    // input axes with extent > 1, in output order; an axis that follows the
    // previous one in the input too (extent-1 axes between them aside)
    // merges into it
    int64_t ext[kMaxDims];   // merged axes, output order
    int first[kMaxDims], last[kMaxDims];  // their first and last input axes
    int n = 0;
    for (int k = 0; k < rank; ++k) {
        const int a = perm[k];
        if (shape[a] == 1) continue;
        if (n > 0) {
            int nxt = last[n - 1] + 1;
            while (nxt < rank && shape[nxt] == 1) ++nxt;
            if (nxt == a) {
                ext[n - 1] *= shape[a];
                last[n - 1] = a;
                continue;
            }
        }
        ext[n] = shape[a], first[n] = last[n] = a, ++n;
    }
    if (n == 0) return cudaMemcpyAsync(out, in, elem_bytes, cudaMemcpyDeviceToDevice, s);
    // the merged axes in input order give the input strides
    int order[kMaxDims];
    for (int k = 0; k < n; ++k) order[k] = k;
    std::sort(order, order + n, [&](int x, int y) { return first[x] < first[y]; });
    int64_t is[kMaxDims], os[kMaxDims];
    int64_t st = 1;
    for (int k = n - 1; k >= 0; --k) is[order[k]] = st, st *= ext[order[k]];
    st = 1;
    for (int k = n - 1; k >= 0; --k) os[k] = st, st *= ext[k];
    if (n == 1) return cudaMemcpyAsync(out, in, (size_t)total * elem_bytes, cudaMemcpyDeviceToDevice, s);

    const int xin = order[n - 1];  // merged axis innermost in the input
    const int yout = n - 1;        // merged axis innermost in the output
    Outer o;
    bool rows_case = xin == yout;
    int64_t nb = 1, nx = ext[xin], ny = rows_case ? 1 : ext[yout];
    for (int k = 0; k < n; ++k) {
        if (k == xin || k == yout) continue;
        o.ext[o.nd] = ext[k], o.is[o.nd] = is[k], o.os[o.nd] = os[k], ++o.nd;
        nb *= ext[k];
    }
    const int64_t isy = rows_case ? 0 : is[yout], osx = os[xin];
    switch (elem_bytes) {
    case 1: return run<uint8_t>(in, out, o, rows_case, nb, nx, ny, isy, osx, s);
    case 2: return run<uint16_t>(in, out, o, rows_case, nb, nx, ny, isy, osx, s);
    case 4: return run<uint32_t>(in, out, o, rows_case, nb, nx, ny, isy, osx, s);
    case 8: return run<uint64_t>(in, out, o, rows_case, nb, nx, ny, isy, osx, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace moa
