// ttm_simt.cu -- mode-q tensor-times-matrix on the SIMT pipes (FP32 FMA or
// FP64 DFMA), Sec. 5.2 Eq. 25:
//   C(i with i_q = j) = sum_{k < n_q} A(i with i_q = k) * B(j, k).
//
// The non-contracted modes of A (and C) are collapsed into a row space of M
// rows, so the product is one M x J x n_q matrix product whose row m has its
// own A and C offsets (from the mapper) and whose k stride is w_q of A: the
// paper's "slice-times-matrix" reading of ttm (Sec. 5.2), with all slices
// batched into one launch.  Each CTA computes a 64 x 64 (m, j) tile with a
// 16-deep k slab staged in shared memory; each thread holds 4 x 4 outputs.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace tl {

namespace {

constexpr int BM = 64, BJ = 64, BK = 16, kThreads = 256;

struct TtmArgs {
    const void* A;
    const void* B;
    void* C;
    DevSpace rows;      // operands 0 = A, 1 = C
    int64_t M, J, nq, saq, scq, ldb_row, ldb_col;
    int64_t tiles_m, tiles_j;
    int accumulate;
};

template <typename T>
__global__ void __launch_bounds__(kThreads) ttm_simt_kernel(const TtmArgs a)
{
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BJ + 1];
    __shared__ int64_t offA[BM], offC[BM];
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const int tid = threadIdx.x;
    const int tm = tid & 15, tj = tid >> 4;
    const bool a_kfast = (a.saq == 1);
    const bool b_kfast = (a.ldb_col == 1);
    const int64_t ntiles = a.tiles_m * a.tiles_j;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t m0 = (tile % a.tiles_m) * BM;
        const int64_t j0 = (tile / a.tiles_m) * BJ;
        __syncthreads();
        if (tid < BM) {
            int64_t m = m0 + tid;
            int64_t off[2] = {0, 0};
            if (m < a.M) map_offsets<2>(a.rows, m, 1, off);
            offA[tid] = off[0];
            offC[tid] = off[1];
        }
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        for (int64_t k0 = 0; k0 < a.nq; k0 += BK) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < (BM * BK) / kThreads; ++r) {
                int e = tid + r * kThreads;
                int mm, kk;
                if (a_kfast) { kk = e % BK; mm = e / BK; }
                else { mm = e % BM; kk = e / BM; }
                int64_t m = m0 + mm, k = k0 + kk;
                As[kk][mm] = (m < a.M && k < a.nq) ? __ldg(A + offA[mm] + k * a.saq) : T(0);
            }
#pragma unroll
            for (int r = 0; r < (BJ * BK) / kThreads; ++r) {
                int e = tid + r * kThreads;
                int jj, kk;
                if (b_kfast) { kk = e % BK; jj = e / BK; }
                else { jj = e % BJ; kk = e / BJ; }
                int64_t j = j0 + jj, k = k0 + kk;
                Bs[kk][jj] = (j < a.J && k < a.nq) ? __ldg(B + j * a.ldb_row + k * a.ldb_col) : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[kk][tm + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tj + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int64_t m = m0 + tm + 16 * i;
            if (m >= a.M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t jg = j0 + tj + 16 * j;
                if (jg >= a.J) continue;
                T* c = C + offC[tm + 16 * i] + jg * a.scq;
                *c = a.accumulate ? *c + acc[i][j] : acc[i][j];
            }
        }
    }
}

template <typename T>
int launch_typed(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                 int num_sms, cudaStream_t st)
{
    TtmArgs a{};
    a.A = A;
    a.B = B;
    a.C = C;
    a.rows = to_dev(P.rows);
    a.M = P.M;
    a.J = P.J;
    a.nq = P.nq;
    a.saq = P.saq;
    a.scq = P.scq;
    a.ldb_row = P.ldb_row;
    a.ldb_col = P.ldb_col;
    a.tiles_m = (P.M + BM - 1) / BM;
    a.tiles_j = (P.J + BJ - 1) / BJ;
    a.accumulate = accumulate;
    int64_t ntiles = a.tiles_m * a.tiles_j;
    int64_t cap = (int64_t)num_sms * 4;
    int grid = (int)(ntiles < cap ? ntiles : cap);
    ttm_simt_kernel<T><<<grid, kThreads, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

}  // namespace

int launch_ttm_simt(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                    int num_sms, cudaStream_t st)
{
    if (P.dtype == TL_F64) return launch_typed<double>(P, A, B, C, accumulate, num_sms, st);
    return launch_typed<float>(P, A, B, C, accumulate, num_sms, st);
}

}  // namespace tl
