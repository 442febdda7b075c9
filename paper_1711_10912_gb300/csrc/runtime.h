// runtime.h -- shared host-side pieces of the C ABI: device properties, the
// per-stream workspace and the validated "prepare" step of each operation
// (used by the direct entry points and by the batch / serving runtime).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdlib>

#include "plan.h"

namespace tl {

// An NVTX range named after an entry point, pushed when the environment
// variable TL_NVTX is set (read once per process), so profilers can attribute
// kernels to the ABI calls that launched them.
struct NvtxRange {
    bool on;
    explicit NvtxRange(const char* name) : on(enabled())
    {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxRange()
    {
        if (on) nvtxRangePop();
    }
    static bool enabled()
    {
        static const bool e = std::getenv("TL_NVTX") != nullptr;
        return e;
    }
};

int device_sms();
// TL_EBOUNDS if a bounds-checked build recorded an out-of-range mapped offset
// since the last cleared check, else TL_OK (TL_ECUDA if a word could not be read).
int bounds_status(bool clear);
// Raises `func`'s dynamic shared-memory limit to `bytes` on the current
// device, once per (device, kernel): the attribute applies to the device that
// is current when it is set, so a process that launches on several devices
// needs it on each.  Returns TL_OK, or TL_ECUDA if the runtime refused.
int smem_optin(const void* func, int bytes);
// Adds n to the process-wide launch counter reported by tl_launch_count().
void count_launches(int n);
void* workspace(cudaStream_t st, size_t bytes);
// Independent per-(device, stream) buffers: slot 0 holds kernel partial sums
// and converted operands; slot 1 the intermediates of operation sequences;
// slot 2 small results of sequences (norms).
void* workspace_slot(cudaStream_t st, size_t bytes, int slot);

int prepare_ttv(const tl_tensor* A, const void* b, int64_t incb, uint32_t q, const tl_tensor* C,
                int num_sms, Tensor& At, Tensor& Ct, TtvPlan& P);
int prepare_ttm(const tl_tensor* A, const void* B, int64_t J, int64_t ldb_row, int64_t ldb_col,
                uint32_t q, const tl_tensor* C, int32_t precision, Tensor& At, Tensor& Ct,
                TtmPlan& P);
int prepare_entrywise(int32_t op, const tl_tensor* A, const tl_tensor* B, const tl_tensor* C,
                      Tensor& At, Tensor& Bt, Tensor& Ct, bool& hasB, EwPlan& P);
int ttm_launches(const TtmPlan& P);
int run_ttm(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate, int sms,
            cudaStream_t st);

}  // namespace tl
