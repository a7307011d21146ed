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
//     copied as a contiguous run (16-byte vectors where aligned), reads and
//     writes coalesced, the rows' offsets stepped without division;
//   * otherwise a square tile (64 x 64, 32 x 32 for 8-byte elements) over
//     (input innermost axis x, the input axis y that becomes the output's
//     innermost) goes through shared memory, so the reads run along x and the
//     writes along y; the remaining axes index independent tiles.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "transpose_plan.h"

namespace moa {
namespace {

constexpr int kMaxDims = kTransposeMaxDims;

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

// The multi-index of a row over the outer axes and its two offsets,
// advanced by a fixed step with carries (no division after the start).
struct Odometer {
    int64_t idx[kMaxDims];
    int64_t in_off, out_off;
    // loops unrolled over the fixed maximum so that idx stays in registers
    MOA_DEV void start(const Outer &o, int64_t b) {
        in_off = 0, out_off = 0;
#pragma unroll
        for (int k = kMaxDims - 1; k >= 0; --k) {
            idx[k] = 0;
            if (k >= o.nd) continue;
            const int64_t e = o.ext[k], q = b / e;
            idx[k] = b - q * e;
            in_off += idx[k] * o.is[k];
            out_off += idx[k] * o.os[k];
            b = q;
        }
    }
    MOA_DEV void advance(const Outer &o, int64_t step) {
#pragma unroll
        for (int k = kMaxDims - 1; k >= 0; --k) {
            if (k >= o.nd || step == 0) continue;
            const int64_t e = o.ext[k];
            int64_t v = idx[k] + step;
            step = 0;
            while (v >= e) v -= e, ++step;  // step is small: the carry into the next axis
            in_off += (v - idx[k]) * o.is[k];
            out_off += (v - idx[k]) * o.os[k];
            idx[k] = v;
        }
    }
};

// Rows of n contiguous units (U: the element type, or 16-byte vectors when
// every row start is 16-byte aligned).  A block copies a contiguous range of
// rows, W threads per row and 256 / W rows at a time; each thread walks its
// rows with an odometer.
template <typename U>
__global__ void __launch_bounds__(256, 4) copy_rows(const U *__restrict__ in, U *__restrict__ out, Outer o, int64_t rows,
                                                 int64_t n, int W, int64_t per_block) {
    const int R = 256 / W, tr = threadIdx.x / W, lane = threadIdx.x % W;
    const int64_t r0 = (int64_t)blockIdx.x * per_block, r1 = min(rows, r0 + per_block);
    int64_t r = r0 + tr;
    if (r >= r1) return;
    Odometer od;
    od.start(o, r);
    for (;;) {  // two rows per pass: both rows' loads in flight before the stores
        const bool two = r + R < r1;
        const int64_t i0 = od.in_off, o0 = od.out_off;
        if (two) od.advance(o, R);
        for (int64_t k = lane; k < n; k += W) {
            const U v0 = __ldg(in + i0 + k);
            if (two) {
                const U v1 = __ldg(in + od.in_off + k);
                out[o0 + k] = v0;
                out[od.out_off + k] = v1;
            } else {
                out[o0 + k] = v0;
            }
        }
        r += 2 * R;
        if (r >= r1) break;
        od.advance(o, R);
    }
}

// TS x TS tiles of the (y, x) plane: in[y * isy + x] -> out[x * osx + y],
// 32 x 8 threads, TS * TS / 256 elements per thread in flight; blockIdx.x /
// y / z: tile column, tile row, independent plane.
template <typename T, int TS>
__global__ void __launch_bounds__(256) tile_transpose(const T *__restrict__ in, T *__restrict__ out, Outer o,
                                                      int64_t nb, int64_t nx, int64_t ny, int64_t isy, int64_t osx) {
    __shared__ T t[TS][TS + 1];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    for (int64_t b = blockIdx.z; b < nb; b += gridDim.z) {
        int64_t ib, ob;
        outer_offsets(o, b, ib, ob);
        for (int64_t y0 = (int64_t)blockIdx.y * TS; y0 < ny; y0 += (int64_t)gridDim.y * TS) {
            for (int64_t x0 = (int64_t)blockIdx.x * TS; x0 < nx; x0 += (int64_t)gridDim.x * TS) {
#pragma unroll
                for (int j = 0; j < TS; j += 8) {
#pragma unroll
                    for (int i = 0; i < TS; i += 32) {
                        const int64_t y = y0 + j + ly, x = x0 + i + lx;
                        if (y < ny && x < nx) t[j + ly][i + lx] = __ldg(in + ib + y * isy + x);
                    }
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < TS; j += 8) {
#pragma unroll
                    for (int i = 0; i < TS; i += 32) {
                        const int64_t x = x0 + j + ly, y = y0 + i + lx;
                        if (x < nx && y < ny) out[ob + x * osx + y] = t[i + lx][j + ly];
                    }
                }
                __syncthreads();
            }
        }
    }
}

unsigned clamp_grid(int64_t v, int64_t lim) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(v, lim)); }

template <typename T>
cudaError_t run(const void *in, void *out, Outer o, bool rows_case, int64_t nb, int64_t nx, int64_t ny, int64_t isy,
                int64_t osx, cudaStream_t s) {
    if (rows_case) {
        // 16-byte units when the row length, every row start and both bases allow
        bool vec = sizeof(T) < 16 && (nx * (int64_t)sizeof(T)) % 16 == 0 && (uintptr_t)in % 16 == 0 &&
                   (uintptr_t)out % 16 == 0;
        for (int k = 0; k < o.nd && vec; ++k)
            vec = (o.is[k] * (int64_t)sizeof(T)) % 16 == 0 && (o.os[k] * (int64_t)sizeof(T)) % 16 == 0;
        int64_t n = nx;
        if (vec) {
            const int64_t f = 16 / (int64_t)sizeof(T);
            n = nx / f;
            for (int k = 0; k < o.nd; ++k) o.is[k] /= f, o.os[k] /= f;
        }
        int W = 32;  // threads per row: the row length rounded up to a power of two, 32..256
        while (W < 256 && W < n) W *= 2;
        const int64_t blocks = std::min<int64_t>((nb + 256 / W - 1) / (256 / W), 152 * 16);
        const int64_t per_block = (nb + blocks - 1) / blocks;
        const unsigned grid = (unsigned)((nb + per_block - 1) / per_block);
        if (vec)
            copy_rows<uint4><<<grid, 256, 0, s>>>((const uint4 *)in, (uint4 *)out, o, nb, n, W, per_block);
        else
            copy_rows<T><<<grid, 256, 0, s>>>((const T *)in, (T *)out, o, nb, n, W, per_block);
    } else {
        constexpr int TS = sizeof(T) == 8 ? 32 : 64;
        const dim3 grid(clamp_grid((nx + TS - 1) / TS, 1 << 30), clamp_grid((ny + TS - 1) / TS, 65535),
                        clamp_grid(nb, 65535));
        tile_transpose<T, TS><<<grid, 256, 0, s>>>((const T *)in, (T *)out, o, nb, nx, ny, isy, osx);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transpose(size_t elem_bytes, int rank, const int64_t *shape, const int *perm, const void *in,
                             void *out, cudaStream_t s) {
    TransposePlan pl;
    if (!plan_transpose(rank, shape, perm, &pl)) return cudaErrorInvalidValue;
    if (pl.total == 0) return cudaSuccess;
    if (pl.n <= 1) return cudaMemcpyAsync(out, in, (size_t)pl.total * elem_bytes, cudaMemcpyDeviceToDevice, s);
    Outer o;  // every merged axis but the two the kernels walk
    int64_t nb = 1;
    for (int k = 0; k < pl.n; ++k) {
        if (k == pl.xin || k == pl.yout) continue;
        o.ext[o.nd] = pl.ext[k], o.is[o.nd] = pl.is[k], o.os[o.nd] = pl.os[k], ++o.nd;
        nb *= pl.ext[k];
    }
    const int64_t nx = pl.ext[pl.xin], ny = pl.rows_case ? 1 : pl.ext[pl.yout];
    const int64_t isy = pl.rows_case ? 0 : pl.is[pl.yout], osx = pl.os[pl.xin];
    switch (elem_bytes) {
    case 1: return run<uint8_t>(in, out, o, pl.rows_case, nb, nx, ny, isy, osx, s);
    case 2: return run<uint16_t>(in, out, o, pl.rows_case, nb, nx, ny, isy, osx, s);
    case 4: return run<uint32_t>(in, out, o, pl.rows_case, nb, nx, ny, isy, osx, s);
    case 8: return run<uint64_t>(in, out, o, pl.rows_case, nb, nx, ny, isy, osx, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace moa
