// Host planning of a multi-dimensional transpose (output axis k = input axis
// perm[k]) for the kernels of transpose.cu: plain C++, no CUDA, so it also
// builds into a CPU test.
//
// Axes of extent 1 are dropped; input axes that stay adjacent and in order
// in the output merge into one.  The merged axes (output order) carry their
// extents and their strides in the input and in the output (row-major,
// elements).  `xin` is the merged axis innermost in the input (input stride
// 1), `yout` the one innermost in the output (output stride 1); when they are
// the same axis the copy runs along contiguous rows, otherwise through
// square tiles of the (yout, xin) plane.  The remaining axes are "outer":
// independent rows or planes.
#pragma once

#include <stdint.h>

namespace moa {

constexpr int kTransposeMaxDims = 8;

struct TransposePlan {
    int64_t total = 0;  // elements
    int n = 0;          // merged axes (0: one element; 1: a plain copy)
    int64_t ext[kTransposeMaxDims], is[kTransposeMaxDims], os[kTransposeMaxDims];
    int xin = 0, yout = 0;
    bool rows_case = false;
};

// False when rank, shape or perm are out of range (callers validate first).
inline bool plan_transpose(int rank, const int64_t *shape, const int *perm, TransposePlan *p) {
    if (rank < 0 || rank > kTransposeMaxDims) return false;
    p->total = 1;
    for (int k = 0; k < rank; ++k) p->total *= shape[k];
    p->n = 0;
    if (p->total == 0) return true;
    int first[kTransposeMaxDims], last[kTransposeMaxDims];  // first and last input axes of each merged axis
    int n = 0;
    for (int k = 0; k < rank; ++k) {
        const int a = perm[k];
        if (a < 0 || a >= rank) return false;
        if (shape[a] == 1) continue;
        if (n > 0) {  // a follows the previous merged axis in the input too (extent-1 axes aside)?
            int nxt = last[n - 1] + 1;
            while (nxt < rank && shape[nxt] == 1) ++nxt;
            if (nxt == a) {
                p->ext[n - 1] *= shape[a];
                last[n - 1] = a;
                continue;
            }
        }
        p->ext[n] = shape[a], first[n] = last[n] = a, ++n;
    }
    p->n = n;
    if (n == 0) return true;
    int order[kTransposeMaxDims];  // merged axes in input order (insertion sort of at most 8)
    for (int k = 0; k < n; ++k) {
        int j = k;
        for (; j > 0 && first[order[j - 1]] > first[k]; --j) order[j] = order[j - 1];
        order[j] = k;
    }
    int64_t st = 1;
    for (int k = n - 1; k >= 0; --k) p->is[order[k]] = st, st *= p->ext[order[k]];
    st = 1;
    for (int k = n - 1; k >= 0; --k) p->os[k] = st, st *= p->ext[k];
    p->xin = order[n - 1];
    p->yout = n - 1;
    p->rows_case = p->xin == p->yout;
    return true;
}

}  // namespace moa
