// probe.cu -- FMA throughput probe: measures the SIMT pipes' FP32 FMA and
// FP64 DFMA rates on the current device, the peaks that the FP32 and FP64
// operations of this library are judged against (the paper has no such
// measurement; GB300's FP64 rate is sharply reduced and is measured rather
// than taken from a datasheet).  Changes no clock, power or other device
// setting: it only runs arithmetic.
#include <cuda_runtime.h>

#include "../../include/tlgb.h"
#include "runtime.h"

namespace tl {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;   // independent FMA chains per thread

// Each thread runs kChains independent chains x <- x * a + b for `iters`
// rounds (16 rounds per loop trip, so loop control is a small fraction of
// the issued instructions).  The result is stored only if it equals a value
// no chain reaches, which the compiler cannot prove, so nothing is removed.
// The multiplier and addend are formed in registers (from a block index
// term that is zero at run time but unknown to the compiler): DFMA with
// operands taken from the constant bank measured 1.06 instead of 1.26 TF/s.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int64_t iters, T a0, T b0, T* sink)
{
    const T a = a0 + T(blockIdx.x >> 30), b = b0 + T(blockIdx.x >> 30);
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
    for (int64_t it = 0; it < iters; it += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == T(1.0e30)) *sink = s;
}

}  // namespace

}  // namespace tl

extern "C" int tl_fma_peak_probe(int32_t dtype, int64_t iters, void* sink, double* flops,
                                 void* stream)
{
    using namespace tl;
    if (!sink || !flops || iters < 16 || iters % 16 || (dtype != TL_F32 && dtype != TL_F64))
        return TL_EINVAL;
    const int sms = device_sms();
    if (sms <= 0) return TL_ECUDA;
    const int blocks = sms * 8;   // 64 warps per SM
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == TL_F32)
        fma_probe_kernel<float><<<blocks, kProbeThreads, 0, st>>>(iters, 0.999f, 1e-4f,
                                                                  static_cast<float*>(sink));
    else
        fma_probe_kernel<double><<<blocks, kProbeThreads, 0, st>>>(iters, 0.999, 1e-4,
                                                                   static_cast<double*>(sink));
    if (cudaGetLastError() != cudaSuccess) return TL_ECUDA;
    count_launches(1);
    *flops = 2.0 * kChains * (double)iters * (double)blocks * kProbeThreads;
    return TL_OK;
}
