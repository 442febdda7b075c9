// batch.cpp -- request contexts, batched submission and polling.
#include <cuda_runtime.h>

#include "runtime.h"

extern "C" {

int tl_ctx_create(size_t, int32_t, int32_t, tl_ctx** out)
{
    if (out) *out = nullptr;
    return TL_EUNSUPPORTED;
}
int tl_ctx_destroy(tl_ctx*) { return TL_OK; }
int tl_batch_submit(tl_ctx*, const tl_op*, size_t, uint64_t*) { return TL_EUNSUPPORTED; }
int tl_poll(tl_ctx*, uint64_t, int32_t*, double*) { return TL_EUNSUPPORTED; }
int tl_wait(tl_ctx*, uint64_t, double, int32_t*, double*) { return TL_EUNSUPPORTED; }
int tl_cancel(tl_ctx*, uint64_t) { return TL_EUNSUPPORTED; }

}  // extern "C"
