// sx_server.cpp -- placeholder until the serving loop is built.
#include "sx_internal.h"

using namespace sx;

extern "C" {
int sx_server_create(sx_target *, const sx_server_cfg *, sx_server **) { return fail(SX_ERR_STATE, "not available"); }
int sx_server_submit(sx_server *, const sx_request *, uint64_t *) { return fail(SX_ERR_STATE, "not available"); }
int sx_server_poll(sx_server *, uint64_t, sx_request_status *) { return fail(SX_ERR_STATE, "not available"); }
int sx_server_wait(sx_server *, uint64_t, int64_t, sx_request_status *) { return fail(SX_ERR_STATE, "not available"); }
int sx_server_read(sx_server *, uint64_t, int, void *, size_t) { return fail(SX_ERR_STATE, "not available"); }
int sx_server_release(sx_server *, uint64_t) { return fail(SX_ERR_STATE, "not available"); }
int sx_server_stats_get(sx_server *, sx_server_stats *) { return fail(SX_ERR_STATE, "not available"); }
int sx_server_destroy(sx_server *) { return fail(SX_ERR_STATE, "not available"); }
}
