// serve.cu -- placeholder until the serving engine lands.
#include "internal.h"
namespace mmhost {
void serve_shutdown(mm_handle_s*) {}
}
int mm_serve_submit(mm_handle, const mm_request*, uint64_t*) { return MM_ERR_UNSUPPORTED; }
int mm_serve_poll(mm_handle, uint64_t, mm_req_status*) { return MM_ERR_UNSUPPORTED; }
int mm_serve_drain(mm_handle) { return MM_ERR_UNSUPPORTED; }
