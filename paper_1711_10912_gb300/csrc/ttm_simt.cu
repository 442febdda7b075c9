// ttm_simt.cu -- mode-q tensor-times-matrix on the SIMT pipes (FP32 FMA or
// FP64 DFMA), Sec. 5.2 Eq. 25:
//   C(i with i_q = j) = sum_{k < n_q} A(i with i_q = k) * B(j, k).
//
// The non-contracted modes of A (and C) are collapsed into a row space of M
// rows, so the product is one M x J x n_q matrix product whose row m has its
// own A and C offsets (from the mapper) and whose k stride is w_q of A: the
// paper's "slice-times-matrix" reading of ttm (Sec. 5.2), with all slices
// batched into one launch.  For FP64 each CTA computes a 64 x 64 (m, j)
// tile with a 16-deep k slab staged in shared memory, each thread 4 x 4
// outputs; FP32 runs on the 128 x 128 register-tiled kernel of
// ttm_sgemm.cu (ttm_rows_kernel below takes short contractions of either).
// When the (m, j) tiles cannot fill the GPU and n_q is long (a few rows of a
// matrix-like tensor contracted over most of its elements), the k range is
// split across CTAs: split s writes its partial M x J block to a workspace
// and a second kernel adds the splits in order (deterministic) into C.
#include <cuda_runtime.h>

#include <algorithm>

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
    DevDiv rdiv;        // ttm_rows: division by the row extents
    int idx32;          // ttm_rows: item indices fit in 31 bits
    FastDiv fdM, fdG;   // ttm_rows: division by M and by the column groups
    int64_t M, J, nq, saq, scq, ldb_row, ldb_col;
    int64_t tiles_m, tiles_j;
    int accumulate;
    int64_t splits, kchunk;   // k splits; > 1: partials go to ws[s][m][j]
    void* ws;
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
    for (int64_t w = blockIdx.x; w < ntiles * a.splits; w += gridDim.x) {
        const int64_t tile = w % ntiles, split = w / ntiles;
        const int64_t m0 = (tile % a.tiles_m) * BM;
        const int64_t j0 = (tile / a.tiles_m) * BJ;
        const int64_t kb = split * a.kchunk;
        const int64_t ke = min(a.nq, kb + a.kchunk);
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
        for (int64_t k0 = kb; k0 < ke; k0 += BK) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < (BM * BK) / kThreads; ++r) {
                int e = tid + r * kThreads;
                int mm, kk;
                if (a_kfast) { kk = e % BK; mm = e / BK; }
                else { mm = e % BM; kk = e / BM; }
                int64_t m = m0 + mm, k = k0 + kk;
                As[kk][mm] = (m < a.M && k < ke) ? __ldg(A + offA[mm] + k * a.saq) : T(0);
            }
#pragma unroll
            for (int r = 0; r < (BJ * BK) / kThreads; ++r) {
                int e = tid + r * kThreads;
                int jj, kk;
                if (b_kfast) { kk = e % BK; jj = e / BK; }
                else { jj = e % BJ; kk = e / BJ; }
                int64_t j = j0 + jj, k = k0 + kk;
                Bs[kk][jj] = (j < a.J && k < ke) ? __ldg(B + j * a.ldb_row + k * a.ldb_col) : T(0);
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
                if (a.splits > 1) {
                    static_cast<T*>(a.ws)[(split * a.M + m) * a.J + jg] = acc[i][j];
                } else {
                    T* c = C + offC[tm + 16 * i] + jg * a.scq;
                    *c = a.accumulate ? *c + acc[i][j] : acc[i][j];
                }
            }
        }
    }
}

// Short contractions (n_q <= 64) with the whole matrix in shared memory: each
// work item is one row of A and a group of JB columns (JB = 16 when the rows
// alone fill the GPU, down to 1 for few rows, so small problems still use
// every SM); its outputs are accumulated in registers, k streams in groups of
// 8 loads, B is read as shared-memory broadcasts.  Rows are contiguous in C
// whenever j is not: then the items are numbered row-fastest, so a warp's 32
// threads write 32 consecutive rows of one column (128 bytes for FP32) instead
// of 8 rows of four column groups; when j is contiguous in C the threads of a
// row stay together.
template <typename T, int JB>
__global__ void __launch_bounds__(kThreads) ttm_rows_kernel(const TtmArgs a)
{
    extern __shared__ __align__(16) uint8_t smem_rows[];
    T* Bs = reinterpret_cast<T*>(smem_rows);     // [n_q][Jp], zero beyond J
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const int nq = (int)a.nq, J = (int)a.J;
    const int Jp = (J + JB - 1) / JB * JB;
    const int groups = Jp / JB;
    for (int e = threadIdx.x; e < nq * Jp; e += kThreads) {
        const int k = e / Jp, j = e - k * Jp;
        Bs[e] = j < J ? __ldg(B + j * a.ldb_row + k * a.ldb_col) : T(0);
    }
    __syncthreads();
    const int64_t items = a.M * groups;
    for (int64_t it = (int64_t)blockIdx.x * kThreads + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * kThreads) {
        int64_t m;
        int j0;
        if (a.idx32) {
            const uint32_t u = (uint32_t)it;
            if (a.scq != 1) {
                const uint32_t g = fast_div(u, a.fdM);
                m = u - g * (uint32_t)a.M;
                j0 = (int)g * JB;
            } else {
                const uint32_t mm = fast_div(u, a.fdG);
                m = mm;
                j0 = (int)(u - mm * (uint32_t)groups) * JB;
            }
        } else if (a.scq != 1) {
            const int64_t g = it / a.M;
            m = it - g * a.M;
            j0 = (int)g * JB;
        } else {
            m = it / groups;
            j0 = (int)(it - m * groups) * JB;
        }
        int64_t off[2];
        map_offsets_fast<2>(a.rows, a.rdiv, m, 1, off);
        const T* pa = A + off[0];
        T* pc = C + off[1];
        T acc[JB];
#pragma unroll
        for (int j = 0; j < JB; ++j) acc[j] = T(0);
        row_dot<T, JB>(pa, a.saq, nq, Bs + j0, Jp, acc);
        pc += (int64_t)j0 * a.scq;
        if (!a.accumulate && j0 + JB <= J) {
#pragma unroll
            for (int j = 0; j < JB; ++j) pc[(int64_t)j * a.scq] = acc[j];
        } else {
#pragma unroll
            for (int j = 0; j < JB; ++j) {
                if (j0 + j < J) {
                    T* c = pc + (int64_t)j * a.scq;
                    *c = a.accumulate ? *c + acc[j] : acc[j];
                }
            }
        }
    }
}

// C(m, j) (+)= sum over splits s = 0, 1, ... of ws[s][m][j].
// Skinny ttm: a few rows (M <= 16) contracted over a long mode (n_q >= 2048)
// into at most 64 columns (M x J <= 512 outputs), where any GEMM tile would be
// almost all idle.  The k range is split across the CTAs; per 64-deep k tile
// a CTA stages the M rows of A and the J rows of B in shared memory (every
// load of the tile issued before the stores) and each thread accumulates one
// or two (m, j) dot products over ascending k; the partial M x J blocks go
// to ws[s][m][j] and ttm_splitk_reduce adds them.
constexpr int kSkinnyKT = 64;

template <typename T>
__global__ void __launch_bounds__(kThreads) ttm_skinny_kernel(const TtmArgs a)
{
    constexpr int KT = kSkinnyKT;
    constexpr int kLoadsA = 16 * KT / kThreads, kLoadsB = 64 * KT / kThreads;
    __shared__ T As[16][KT + 1];
    __shared__ T Bs[64][KT + 1];
    __shared__ int64_t offA[16];
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ ws = static_cast<T*>(a.ws);
    const int tid = threadIdx.x;
    const int M = (int)a.M, J = (int)a.J, pairs = M * J;
    if (tid < M) {
        int64_t off[2];
        map_offsets<2>(a.rows, tid, 1, off);
        offA[tid] = off[0];
    }
    const int p0 = tid, p1 = tid + kThreads;
    const int m0 = p0 / J, j0 = p0 - m0 * J, m1 = p1 / J, j1 = p1 - m1 * J;
    __syncthreads();
    for (int64_t s = blockIdx.x; s < a.splits; s += gridDim.x) {
        const int64_t kb = s * a.kchunk, ke = min(a.nq, kb + a.kchunk);
        T acc0 = T(0), acc1 = T(0);
        for (int64_t k0 = kb; k0 < ke; k0 += KT) {
            const int kn = (int)min((int64_t)KT, ke - k0);
            T va[kLoadsA], vb[kLoadsB];
#pragma unroll
            for (int it = 0; it < kLoadsA; ++it) {
                const int e = tid + kThreads * it, m = e / KT, kk = e % KT;
                va[it] = (m < M && kk < kn) ? __ldg(A + offA[m] + (k0 + kk) * a.saq) : T(0);
            }
#pragma unroll
            for (int it = 0; it < kLoadsB; ++it) {
                const int e = tid + kThreads * it, j = e / KT, kk = e % KT;
                vb[it] = (j < J && kk < kn) ? __ldg(B + j * a.ldb_row + (k0 + kk) * a.ldb_col) : T(0);
            }
            __syncthreads();      // the previous tile's readers are done
#pragma unroll
            for (int it = 0; it < kLoadsA; ++it) {
                const int e = tid + kThreads * it;
                As[e / KT][e % KT] = va[it];
            }
#pragma unroll
            for (int it = 0; it < kLoadsB; ++it) {
                const int e = tid + kThreads * it;
                Bs[e / KT][e % KT] = vb[it];
            }
            __syncthreads();
            if (p0 < pairs) {
#pragma unroll 8
                for (int kk = 0; kk < KT; ++kk) acc0 = fma(As[m0][kk], Bs[j0][kk], acc0);
            }
            if (p1 < pairs) {
#pragma unroll 8
                for (int kk = 0; kk < KT; ++kk) acc1 = fma(As[m1][kk], Bs[j1][kk], acc1);
            }
        }
        if (p0 < pairs) ws[(s * M + m0) * J + j0] = acc0;
        if (p1 < pairs) ws[(s * M + m1) * J + j1] = acc1;
    }
}

// Adds the split partials ws[s][m][j] into C: in split order by one thread
// per output, or, with WARP (many splits), by a warp per output whose lanes
// each add every 32nd split in order and combine by a fixed butterfly
// (deterministic either way).
template <typename T, bool WARP>
__global__ void __launch_bounds__(kThreads) ttm_splitk_reduce(const TtmArgs a)
{
    const T* __restrict__ ws = static_cast<const T*>(a.ws);
    T* __restrict__ C = static_cast<T*>(a.C);
    const int64_t total = a.M * a.J;
    constexpr int kPer = WARP ? 32 : 1;
    const int lane = threadIdx.x & 31;
    for (int64_t e = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / kPer; e < total;
         e += (int64_t)gridDim.x * kThreads / kPer) {
        const int64_t m = e / a.J, j = e - m * a.J;
        T acc = T(0);
        if constexpr (WARP) {
            for (int64_t s = lane; s < a.splits; s += 32) acc += ws[s * total + e];
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
            if (lane != 0) continue;
        } else {
            for (int64_t s = 0; s < a.splits; ++s) acc += ws[s * total + e];
        }
        int64_t off[2];
        map_offsets<2>(a.rows, m, 1, off);
        T* c = C + off[1] + j * a.scq;
        *c = a.accumulate ? *c + acc : acc;
    }
}

template <typename T>
int launch_typed(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                 void* ws, int num_sms, cudaStream_t st)
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
    int64_t kchunk = 0;
    a.splits = ttm_simt_splits(P, num_sms, &kchunk);
    a.kchunk = a.splits > 1 ? kchunk : P.nq;
    a.ws = ws;
    if (a.splits > 1 && !ws) return TL_ENOMEM;
    int64_t cap = (int64_t)num_sms * 4;
    if (P.kernel == K_TTM_ROWS) {
        a.rdiv = make_devdiv(P.rows, 1);
        // columns per work item: as many as keep at least two CTAs per SM busy
        const int64_t want = (int64_t)num_sms * 2 * kThreads;
        int jb = 16;
        while (jb > 1 && P.M * ((P.J + jb - 1) / jb) < want) jb /= 2;
        const int Jp = (int)((P.J + jb - 1) / jb * jb);
        const size_t smem = (size_t)P.nq * Jp * sizeof(T);
        const int64_t items = P.M * (Jp / jb);
        a.idx32 = items < (int64_t(1) << 31) ? 1 : 0;
        a.fdM = make_fastdiv(a.idx32 ? (uint32_t)P.M : 1u);
        a.fdG = make_fastdiv((uint32_t)(Jp / jb));
        int64_t blocks = (items + kThreads - 1) / kThreads;
        const int64_t rcap = (int64_t)num_sms * 8;
        if (blocks > rcap) blocks = rcap;
        switch (jb) {
        case 16: ttm_rows_kernel<T, 16><<<(int)blocks, kThreads, smem, st>>>(a); break;
        case 8: ttm_rows_kernel<T, 8><<<(int)blocks, kThreads, smem, st>>>(a); break;
        case 4: ttm_rows_kernel<T, 4><<<(int)blocks, kThreads, smem, st>>>(a); break;
        case 2: ttm_rows_kernel<T, 2><<<(int)blocks, kThreads, smem, st>>>(a); break;
        default: ttm_rows_kernel<T, 1><<<(int)blocks, kThreads, smem, st>>>(a); break;
        }
        return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
    }
    if (ttm_skinny(P)) {
        const int grid = (int)(a.splits < cap ? a.splits : cap);
        ttm_skinny_kernel<T><<<grid, kThreads, 0, st>>>(a);
    } else if constexpr (sizeof(T) == 4) {
        // FP32: the register-tiled kernel of ttm_sgemm.cu
        const int rc = launch_ttm_sgemm(P, A, B, C, accumulate, ws, a.splits, a.kchunk, num_sms, st);
        if (rc != TL_OK) return rc;
    } else {
        int64_t work = a.tiles_m * a.tiles_j * a.splits;
        int grid = (int)(work < cap ? work : cap);
        ttm_simt_kernel<T><<<grid, kThreads, 0, st>>>(a);
    }
    if (a.splits >= 64) {
        int64_t blocks = (P.M * P.J * 32 + kThreads - 1) / kThreads;
        if (blocks > cap) blocks = cap;
        ttm_splitk_reduce<T, true><<<(int)blocks, kThreads, 0, st>>>(a);
    } else if (a.splits > 1) {
        int64_t blocks = (P.M * P.J + kThreads - 1) / kThreads;
        if (blocks > cap) blocks = cap;
        ttm_splitk_reduce<T, false><<<(int)blocks, kThreads, 0, st>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

}  // namespace

bool ttm_skinny(const TtmPlan& P)
{
    return P.kernel == K_TTM_SIMT && P.M <= 16 && P.J <= 64 && P.M * P.J <= 512 && P.nq >= 2048;
}

int64_t ttm_simt_splits(const TtmPlan& P, int num_sms, int64_t* kchunk)
{
    if (P.kernel == K_TTM_ROWS) {
        if (kchunk) *kchunk = P.nq;
        return 1;
    }
    if (ttm_skinny(P)) {
        // chunks of at least 512 k (whole 64-deep tiles), up to 4 per SM
        int64_t splits = std::min<int64_t>((P.nq + 511) / 512, (int64_t)num_sms * 4);
        int64_t kc = (P.nq + splits - 1) / splits;
        kc = (kc + kSkinnyKT - 1) / kSkinnyKT * kSkinnyKT;
        if (kchunk) *kchunk = kc;
        return (P.nq + kc - 1) / kc;
    }
    // split k when the tiles cover less than half of the resident CTAs (one
    // per SM for the FP32 256-thread tiles, four for the FP64 64 x 64 ones)
    // and each split still gets at least 16 k slabs of 16; the partials stay
    // below 256 MB
    const bool f32 = P.dtype != TL_F64;
    const int64_t tiles = f32 ? sgemm_tiles(P) : ((P.M + BM - 1) / BM) * ((P.J + BJ - 1) / BJ);
    const int64_t target = (int64_t)num_sms * (f32 ? 1 : 4);
    int64_t splits = 1;
    if (tiles * 2 < target && P.nq >= 2 * 16 * BK) {
        splits = (target + tiles - 1) / tiles;
        const int64_t most = P.nq / (16 * BK);
        if (splits > most) splits = most;
        const int64_t elem = P.dtype == TL_F64 ? 8 : 4;
        const int64_t per = P.M * P.J * elem;
        while (splits > 1 && splits * per > (int64_t(256) << 20)) splits /= 2;
    }
    if (splits < 1) splits = 1;
    // the FP32 kernel counts k within a split in 32-bit arithmetic
    if (f32 && P.nq >= (int64_t(1) << 30)) splits = std::max<int64_t>(splits, (P.nq >> 29) + 1);
    int64_t kc = (P.nq + splits - 1) / splits;
    kc = (kc + BK - 1) / BK * BK;
    if (kchunk) *kchunk = kc;
    return splits > 1 ? (P.nq + kc - 1) / kc : 1;
}

size_t ttm_simt_workspace_bytes(const TtmPlan& P, int num_sms)
{
    const int64_t splits = ttm_simt_splits(P, num_sms, nullptr);
    if (splits <= 1) return 0;
    return (size_t)splits * P.M * P.J * (P.dtype == TL_F64 ? 8 : 4);
}

int ttm_simt_launches(const TtmPlan& P, int num_sms)
{
    return ttm_simt_splits(P, num_sms, nullptr) > 1 ? 2 : 1;
}

int launch_ttm_simt(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                    void* ws, int num_sms, cudaStream_t st)
{
    if (P.dtype == TL_F64) return launch_typed<double>(P, A, B, C, accumulate, ws, num_sms, st);
    return launch_typed<float>(P, A, B, C, accumulate, ws, num_sms, st);
}

}  // namespace tl
