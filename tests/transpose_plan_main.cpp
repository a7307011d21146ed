// Prints the host transpose plan (csrc/transpose_plan.h) for each input line
// "rank d_0 .. d_{rank-1} p_0 .. p_{rank-1}", for tests/test_transpose_plan.py.
#include <cstdio>
#include <iostream>

#include "transpose_plan.h"

int main() {
    int rank;
    while (std::cin >> rank) {
        int64_t shape[moa::kTransposeMaxDims] = {};
        int perm[moa::kTransposeMaxDims] = {};
        for (int k = 0; k < rank; ++k) std::cin >> shape[k];
        for (int k = 0; k < rank; ++k) std::cin >> perm[k];
        moa::TransposePlan p;
        if (!moa::plan_transpose(rank, shape, perm, &p)) {
            std::printf("invalid\n");
            continue;
        }
        std::printf("%lld %d %d %d %d", (long long)p.total, p.n, p.xin, p.yout, p.rows_case ? 1 : 0);
        for (int k = 0; k < p.n; ++k) std::printf(" %lld %lld %lld", (long long)p.ext[k], (long long)p.is[k], (long long)p.os[k]);
        std::printf("\n");
    }
    return 0;
}
