// temporary: tuning and serving entry points are built in later commits
#include "internal.h"
using namespace si;
extern "C" {
si_status si_tune_mesh(si_mesh_t, const int32_t *, int64_t, int32_t, float, float, int32_t *, int32_t, si_schedule *,
                       double *, si_stream) { set_error("not built"); return SI_ERR_INVALID; }
si_status si_tune_lookup(int32_t, int64_t, int64_t, si_schedule *) { set_error("no tuning entry"); return SI_ERR_INVALID; }
si_status si_tune_save(const char *) { return SI_ERR_INVALID; }
si_status si_tune_load(const char *) { return SI_ERR_INVALID; }
si_status si_tune_clear(void) { return SI_OK; }
si_status si_serve_create(size_t, int32_t, si_server_t *) { return SI_ERR_INVALID; }
si_status si_serve_add_mesh(si_server_t, si_mesh_t, int32_t *) { return SI_ERR_INVALID; }
si_status si_serve_submit(si_server_t, const si_batch_item *, uint64_t *) { return SI_ERR_INVALID; }
si_status si_serve_poll(si_server_t, uint64_t, int32_t *) { return SI_ERR_INVALID; }
si_status si_serve_wait(si_server_t, uint64_t, int32_t) { return SI_ERR_INVALID; }
si_status si_serve_result(si_server_t, uint64_t, int32_t **, double *) { return SI_ERR_INVALID; }
si_status si_serve_release(si_server_t, uint64_t) { return SI_ERR_INVALID; }
si_status si_serve_destroy(si_server_t) { return SI_ERR_INVALID; }
}
