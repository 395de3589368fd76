// sx_batch.cu -- placeholder until the persistent batched launcher is built.
#include "sx_internal.h"

using namespace sx;

extern "C" {
int sx_batch_create(sx_target *, const sx_batch_item *, size_t, const sx_batch_cfg *, sx_batch **) {
    return fail(SX_ERR_STATE, "batched launcher not available in this build");
}
int sx_batch_launch(sx_batch *) { return fail(SX_ERR_STATE, "not available"); }
int sx_batch_launch_percall(sx_batch *, const sx_launch_cfg *) { return fail(SX_ERR_STATE, "not available"); }
int sx_batch_set_record(sx_batch *, int) { return fail(SX_ERR_STATE, "not available"); }
int sx_batch_completion_ns(sx_batch *, uint64_t *, size_t) { return fail(SX_ERR_STATE, "not available"); }
int sx_batch_info(const sx_batch *, sx_batch_cfg *, uint64_t *, uint64_t *) { return fail(SX_ERR_STATE, "not available"); }
int sx_batch_destroy(sx_batch *) { return fail(SX_ERR_STATE, "not available"); }
int sx_tune_batch(sx_batch *, sx_batch_cfg *, float *) { return fail(SX_ERR_STATE, "not available"); }
}
