// kernels.h -- launchers of the CUDA kernels, called by the C ABI (api.cpp).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "plan.h"

namespace tl {

size_t ttv_workspace_bytes(const TtvPlan& P);
// TL_ETIMEOUT if a bounded wait of a pipelined ttv kernel gave up (see ttm_tc_status).
int ttv_status(bool clear);
int launch_ttv(const TtvPlan& P, const void* A, const void* b, void* C, void* ws,
               int accumulate, int num_sms, cudaStream_t st);

int launch_entrywise(const EwPlan& P, const void* A, const void* B, double alpha, void* C,
                     int num_sms, cudaStream_t st);
int launch_ew_tma(const EwPlan& P, const void* A, const void* B, double alpha, void* C,
                  int num_sms, cudaStream_t st);
// TL_ETIMEOUT if a bounded wait of the TMA entrywise kernel gave up.
int ew_status(bool clear);

// k splits of the SIMT ttm (1 = none) and the k values per split; the
// workspace of the partial sums; kernels one call launches.
int64_t ttm_simt_splits(const TtmPlan& P, int num_sms, int64_t* kchunk);
// a few rows over a long contraction: the split-K skinny kernel takes the call
bool ttm_skinny(const TtmPlan& P);
size_t ttm_simt_workspace_bytes(const TtmPlan& P, int num_sms);
int ttm_simt_launches(const TtmPlan& P, int num_sms);
// FP32 register-tiled ttm (ttm_sgemm.cu): output tiles of the plan, and the
// launch with `splits` k ranges of `kchunk` (splits > 1 writes the partial
// sums to ws, which ttm_splitk_reduce adds into C).
int64_t sgemm_tiles(const TtmPlan& P);
// JSON object naming how the FP32 kernel reads A and B (k4: 16-byte vectors
// along k, r4: along four contiguous rows, scalar) and writes C (j4, m4,
// scalar; ws4 / ws1: split-K partials), for tl_plan_describe.
std::string ttm_sgemm_describe(const TtmPlan& P, const void* A, const void* C, bool split);
int launch_ttm_sgemm(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                     void* ws, int64_t splits, int64_t kchunk, int num_sms, cudaStream_t st);
int launch_ttm_simt(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                    void* ws, int num_sms, cudaStream_t st);

// Deterministic FP64 sum-of-squares reduction over a collapsed space with
// operand 0 = X (dtype dx) and, when R != nullptr, operand 1 = R (dtype dr):
// writes {sqrt(num/den), sqrt(num), sqrt(den)} with num = sum (x-r)^2 and
// den = sum r^2 (R == nullptr: num = sum x^2, den = 0, result[0] = sqrt(num)).
// partials must hold 2 * norm_partial_blocks(...) doubles.
int norm_partial_blocks(int64_t count, int num_sms);
int launch_norm(const Space& sp, int dx, const void* X, int dr, const void* R, double* partials,
                int nblocks, double* result, cudaStream_t st);

}  // namespace tl

namespace tl {
int launch_ttm_tc(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                  int num_sms, cudaStream_t st);
// kernels one launch_ttm_tc call enqueues
int ttm_tc_launches(const TtmPlan& P);
// JSON object with the tensor-core kernel's launch configuration for P and an
// output at C (host only: ring depths, B residency, shared memory, threads,
// whether C is written by TMA stores)
std::string ttm_tc_describe(const TtmPlan& P, const void* C);
// TL_ETIMEOUT if a bounded wait in a tensor-core kernel gave up since the
// last cleared check, else TL_OK (reads the device status word).
int ttm_tc_status(bool clear);
// Launches the bounded-wait self test (see tl_selftest_wait_timeout).
int selftest_wait_timeout(double limit_us, cudaStream_t st);
}  // namespace tl
