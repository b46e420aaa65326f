// grouped.cu -- placeholder until the grouped launch lands.
#include "internal.h"
namespace mmhost {
void grouped_release(mm_handle_s*) {}
}
int mm_gemm_grouped(mm_handle, int, const mm_problem*, int, void*) { return MM_ERR_UNSUPPORTED; }
