// Batched execution of many inner / outer products (placeholder until the
// grouped persistent kernel lands).
#include "common.cuh"
#include "internal.h"

struct moa_batch_plan {
    int count;
};

extern "C" {

moa_status moa_batch_plan_create(int count, const moa_problem *problems, moa_batch_plan **plan, int *bad_index) {
    (void)count;
    (void)problems;
    if (plan) *plan = nullptr;
    if (bad_index) *bad_index = -1;
    return MOA_ERR_UNSUPPORTED;
}

moa_status moa_batch_execute(moa_batch_plan *plan, moa_stream stream) {
    (void)plan;
    (void)stream;
    return MOA_ERR_UNSUPPORTED;
}

moa_status moa_batch_plan_info(const moa_batch_plan *plan, int64_t *n_problems, int64_t *n_launches, int64_t *n_tiles,
                               double *work_flops) {
    (void)plan, (void)n_problems, (void)n_launches, (void)n_tiles, (void)work_flops;
    return MOA_ERR_UNSUPPORTED;
}

void moa_batch_plan_destroy(moa_batch_plan *plan) { delete plan; }

}  // extern "C"
