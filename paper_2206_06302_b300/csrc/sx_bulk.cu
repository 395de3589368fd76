// sx_bulk.cu -- TMA bulk-copy staging family of the STREAM kernels (placeholder until built).
#include "sx_internal.h"

namespace sx {

int validate_bulk_cfg(const sx_target *, int, const sx_launch_cfg &) {
    return fail(SX_ERR_INVALID, "BULK variant not available in this build");
}

int launch_bulk_op(const sx_target *, cudaStream_t, int, int, const void *, const void *, void *,
                   size_t, double, const sx_launch_cfg &) {
    return fail(SX_ERR_INVALID, "BULK variant not available in this build");
}

}  // namespace sx
