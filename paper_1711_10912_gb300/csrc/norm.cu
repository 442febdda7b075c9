// norm.cu -- Frobenius norm (Sec. 5.2 Table 3, norm) and the relative
// Frobenius error ||X - R||_F / ||R||_F, accumulated in FP64.
//
// Two passes make the result deterministic: pass 1 gives each CTA a fixed
// contiguous chunk of the linear index range and reduces it in a fixed order
// to one (num, den) pair in a partials array; pass 2 is one CTA that adds the
// partials in a fixed order.  The chunking depends only on the element count,
// not on the GPU.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace tl {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxPartials = 1024;
constexpr int64_t kPerBlock = 8192;

struct NormArgs {
    const void* X;
    const void* R;
    DevSpace sp;        // operands 0 = X, 1 = R
    int64_t N, chunk;
};

template <typename T>
__device__ __forceinline__ double ld64(const void* p, int64_t off)
{
    return (double)__ldg(static_cast<const T*>(p) + off);
}

__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh)
{
#pragma unroll
    for (int m = 16; m >= 1; m /= 2) {
        a += __shfl_xor_sync(0xffffffffu, a, m);
        b += __shfl_xor_sync(0xffffffffu, b, m);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
    __syncthreads();
    if (w == 0) {
        a = l < kThreads / 32 ? sh[2 * l] : 0.0;
        b = l < kThreads / 32 ? sh[2 * l + 1] : 0.0;
#pragma unroll
        for (int m = 16; m >= 1; m /= 2) {
            a += __shfl_xor_sync(0xffffffffu, a, m);
            b += __shfl_xor_sync(0xffffffffu, b, m);
        }
    }
}

template <typename TX, typename TR, bool HAS_R>
__global__ void __launch_bounds__(kThreads) norm_partial_kernel(const NormArgs a, double* partials)
{
    __shared__ double sh[2 * (kThreads / 32)];
    const int64_t lo = (int64_t)blockIdx.x * a.chunk;
    const int64_t hi = min(a.N, lo + a.chunk);
    double num = 0.0, den = 0.0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) {
        int64_t off[2];
        map_offsets<2>(a.sp, e, 1, off);
        double x = ld64<TX>(a.X, off[0]);
        if (HAS_R) {
            double r = ld64<TR>(a.R, off[1]);
            double d = x - r;
            num = fma(d, d, num);
            den = fma(r, r, den);
        } else {
            num = fma(x, x, num);
        }
    }
    block_sum2(num, den, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = num;
        partials[2 * blockIdx.x + 1] = den;
    }
}

__global__ void __launch_bounds__(kThreads) norm_final_kernel(const double* partials, int nblocks,
                                                              int has_r, double* result)
{
    __shared__ double sh[2 * (kThreads / 32)];
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) {
        num += partials[2 * i];
        den += partials[2 * i + 1];
    }
    block_sum2(num, den, sh);
    if (threadIdx.x == 0) {
        double rn = sqrt(num), rd = sqrt(den);
        result[0] = has_r ? (den > 0.0 ? sqrt(num / den) : rn) : rn;
        result[1] = rn;
        result[2] = rd;
    }
}

template <typename TX, typename TR, bool HAS_R>
void launch_pass1(const NormArgs& a, int nblocks, double* partials, cudaStream_t st)
{
    norm_partial_kernel<TX, TR, HAS_R><<<nblocks, kThreads, 0, st>>>(a, partials);
}

}  // namespace

int norm_partial_blocks(int64_t count, int /*num_sms*/)
{
    int64_t b = (count + kPerBlock - 1) / kPerBlock;
    if (b > kMaxPartials) b = kMaxPartials;
    return (int)(b < 1 ? 1 : b);
}

int launch_norm(const Space& sp, int dx, const void* X, int dr, const void* R, double* partials,
                int nblocks, double* result, cudaStream_t st)
{
    NormArgs a{};
    a.X = X;
    a.R = R;
    a.sp = to_dev(sp);
    a.N = sp.count();
    a.chunk = (a.N + nblocks - 1) / nblocks;
    if (a.N == 0) a.chunk = 1;
    const bool f64x = dx == TL_F64, f64r = dr == TL_F64;
    if (!R) {
        if (f64x) launch_pass1<double, double, false>(a, nblocks, partials, st);
        else launch_pass1<float, float, false>(a, nblocks, partials, st);
    } else if (f64x && f64r) {
        launch_pass1<double, double, true>(a, nblocks, partials, st);
    } else if (f64x) {
        launch_pass1<double, float, true>(a, nblocks, partials, st);
    } else if (f64r) {
        launch_pass1<float, double, true>(a, nblocks, partials, st);
    } else {
        launch_pass1<float, float, true>(a, nblocks, partials, st);
    }
    norm_final_kernel<<<1, kThreads, 0, st>>>(partials, nblocks, R ? 1 : 0, result);
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

}  // namespace tl
