// serve.cu - continuous-batching request loop.
#include "darm.h"
#include "darm_internal.h"

extern "C" {
int darm_sort_serve_start(const darm_serve_cfg*) { return DARM_ERR_NOT_FOUND; }
int darm_sort_serve_submit(void*, uint32_t*, size_t, int, int, uint64_t*) { return DARM_ERR_NOT_FOUND; }
int darm_sort_serve_poll(uint64_t, int*) { return DARM_ERR_NOT_FOUND; }
int darm_sort_serve_wait(uint64_t, int) { return DARM_ERR_NOT_FOUND; }
int darm_sort_serve_stats(double*, double*, double*, uint64_t*) { return DARM_ERR_NOT_FOUND; }
int darm_sort_serve_stop(void) { return DARM_OK; }
int darm_autotune(int, size_t, int, const char*) { return DARM_ERR_NOT_FOUND; }
int darm_load_tune_db(const char*) { return DARM_ERR_NOT_FOUND; }
}
