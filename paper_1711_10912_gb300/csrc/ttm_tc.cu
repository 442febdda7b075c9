// ttm_tc.cu -- tcgen05 tensor-core ttm (placeholder until the kernel lands).
#include <cuda_runtime.h>

#include "kernels.h"

namespace tl {

int launch_ttm_tc(const TtmPlan&, const void*, const void*, void*, int, int, cudaStream_t)
{
    return TL_EUNSUPPORTED;
}

int ttm_tc_launches(const TtmPlan&) { return 0; }

}  // namespace tl
