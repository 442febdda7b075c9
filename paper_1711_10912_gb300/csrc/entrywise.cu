// entrywise.cu -- layout-mixed entrywise operations, Sec. 5.1:
//   Eq. 23  C(i) = A(i) op B(i),  op in {+, -, *, /}
//   Eq. 22  C(i) = alpha * A(i)   (SCALE), and C(i) = A(i) (COPY, a relayout
//           when C's layout differs, Sec. 3.2)
// for every multi-index i; each operand follows its own strides.
//
// Three kernels, chosen by the collapsed space (plan.cpp):
//   ew_flat     A, B and C share one contiguous layout: a flat stream with
//               16-byte vectors.
//   ew_tile     an input's fastest dim t differs from C's fastest dim 0: a
//               32 x 32 tile over dims (0, t) is read along t (coalesced for
//               that input), transposed in shared memory and written along
//               dim 0 (coalesced for C); an input already contiguous along
//               dim 0 is read directly in the write phase.
//   ew_rows     every operand is contiguous along dim 0 but the other dims
//               are ordered differently: one offset decode per 16-byte vector.
//   ew_generic  anything else: each element's offsets come from the mapper.
// FP32 cases of ew_tile and ew_rows that a tensor map can describe run on the
// TMA-staged kernel of ew_tma.cu instead.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace tl {

namespace {

struct EwArgs {
    const void* A;
    const void* B;
    void* C;
    double alpha;
    int op;
    int tdim;
    int64_t N;
    DevSpace sp;        // operands 0 = A, 1 = B, 2 = C
};

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T apply(int op, T a, T b, T alpha)
{
    switch (op) {
    case TL_ADD: return a + b;
    case TL_SUB: return a - b;
    case TL_MUL: return a * b;
    case TL_DIV: return a / b;
    case TL_COPY: return a;
    default: return alpha * a;
    }
}

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) ew_flat_kernel(const EwArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int64_t nvec = a.N / VEC;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    // two vectors per thread per iteration keep more loads in flight
    for (; i + stride < nvec; i += 2 * stride) {
        T x0[VEC], y0[VEC], x1[VEC], y1[VEC], r0[VEC], r1[VEC];
        vload_stream<T, VEC>(A + i * VEC, x0);
        vload_stream<T, VEC>(A + (i + stride) * VEC, x1);
        if (!unary) {
            vload_stream<T, VEC>(B + i * VEC, y0);
            vload_stream<T, VEC>(B + (i + stride) * VEC, y1);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            r0[v] = apply<T>(a.op, x0[v], unary ? T(0) : y0[v], alpha);
            r1[v] = apply<T>(a.op, x1[v], unary ? T(0) : y1[v], alpha);
        }
        vstore<T, VEC>(C + i * VEC, r0);
        vstore<T, VEC>(C + (i + stride) * VEC, r1);
    }
    for (; i < nvec; i += stride) {
        T x[VEC], y[VEC], r[VEC];
        vload_stream<T, VEC>(A + i * VEC, x);
        if (!unary) vload_stream<T, VEC>(B + i * VEC, y);
#pragma unroll
        for (int v = 0; v < VEC; ++v) r[v] = apply<T>(a.op, x[v], unary ? T(0) : y[v], alpha);
        vstore<T, VEC>(C + i * VEC, r);
    }
    // scalar tail
    const int64_t tail0 = nvec * VEC;
    for (int64_t e = tail0 + (int64_t)blockIdx.x * kThreads + threadIdx.x; e < a.N; e += stride) {
        C[e] = apply<T>(a.op, A[e], unary ? T(0) : B[e], alpha);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) ew_generic_kernel(const EwArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < a.N; e += stride) {
        int64_t off[3];
        map_offsets<3>(a.sp, e, 1, off);
        T x = __ldg(A + off[0]);
        T y = unary ? T(0) : __ldg(B + off[1]);
        C[off[2]] = apply<T>(a.op, x, y, alpha);
    }
}

// All operands unit-stride along dim 0 but laid out differently in the other
// dims: one offset decode per 16-byte vector along dim 0, vector loads and
// stores (dim 0's extent and every other stride are multiples of VEC).  Each
// thread issues the loads of U vectors before their stores, so a resident
// SM keeps enough bytes in flight to cover the HBM latency.
template <typename T, int VEC, int U>
__global__ void __launch_bounds__(kThreads, 4) ew_rows_kernel(const EwArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int64_t nvec = a.N / VEC;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    for (; g + (U - 1) * stride < nvec; g += U * stride) {
        int64_t off[U][3];
        T x[U][VEC], y[U][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u) map_offsets<3>(a.sp, g + u * stride, VEC, off[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            vload_stream<T, VEC>(A + off[u][0], x[u]);
            if (!unary) vload_stream<T, VEC>(B + off[u][1], y[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            T r[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                r[v] = apply<T>(a.op, x[u][v], unary ? T(0) : y[u][v], alpha);
            vstore<T, VEC>(C + off[u][2], r);
        }
    }
    for (; g < nvec; g += stride) {
        int64_t off[3];
        map_offsets<3>(a.sp, g, VEC, off);
        T x[VEC], y[VEC], r[VEC];
        vload_stream<T, VEC>(A + off[0], x);
        if (!unary) vload_stream<T, VEC>(B + off[1], y);
#pragma unroll
        for (int v = 0; v < VEC; ++v) r[v] = apply<T>(a.op, x[v], unary ? T(0) : y[v], alpha);
        vstore<T, VEC>(C + off[2], r);
    }
}

// Tile over dims 0 (fastest in C) and t.  Block = 32 x 8 threads; each
// thread handles 4 rows of the 32 x 32 tile in each phase.
constexpr int kTile = 32;

template <typename T>
__global__ void __launch_bounds__(kThreads) ew_tile_kernel(const EwArgs a, int64_t tiles0,
                                                           int64_t tiles1, int64_t batch)
{
    __shared__ T tA[kTile][kTile + 1];
    __shared__ T tB[kTile][kTile + 1];
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int t = a.tdim;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t n0 = a.sp.n[0], nt = a.sp.n[t];
    // an input is staged when dim t is its faster dim of the two
    const bool stageA = a.sp.s[0][t] < a.sp.s[0][0];
    const bool stageB = !unary && a.sp.s[1][t] < a.sp.s[1][0];
    const int64_t total = tiles0 * tiles1 * batch;
    for (int64_t blk = blockIdx.x; blk < total; blk += gridDim.x) {
        int64_t bt0 = blk % tiles0;
        int64_t rest = blk / tiles0;
        int64_t bt1 = rest % tiles1;
        int64_t bz = rest / tiles1;
        // base offsets of the batch index over the remaining dims
        int64_t base[3] = {0, 0, 0};
        {
            int64_t g = bz;
            for (int d = 1; d < a.sp.nd; ++d) {
                if (d == t) continue;
                int64_t i = g % a.sp.n[d];
                g /= a.sp.n[d];
#pragma unroll
                for (int o = 0; o < 3; ++o) base[o] += i * a.sp.s[o][d];
            }
        }
        const int64_t i0b = bt0 * kTile, itb = bt1 * kTile;
        __syncthreads();
        // load phase: lanes run along dim t
        if (stageA || stageB) {
#pragma unroll
            for (int r = 0; r < kTile; r += 8) {
                int64_t i0 = i0b + ty + r, it = itb + tx;
                if (i0 < n0 && it < nt) {
                    if (stageA) tA[ty + r][tx] = __ldcs(A + base[0] + i0 * a.sp.s[0][0] + it * a.sp.s[0][t]);
                    if (stageB) tB[ty + r][tx] = __ldcs(B + base[1] + i0 * a.sp.s[1][0] + it * a.sp.s[1][t]);
                }
            }
        }
        __syncthreads();
        // write phase: lanes run along dim 0
#pragma unroll
        for (int r = 0; r < kTile; r += 8) {
            int64_t i0 = i0b + tx, it = itb + ty + r;
            if (i0 < n0 && it < nt) {
                T x = stageA ? tA[tx][ty + r]
                             : __ldcs(A + base[0] + i0 * a.sp.s[0][0] + it * a.sp.s[0][t]);
                T y = T(0);
                if (!unary)
                    y = stageB ? tB[tx][ty + r]
                               : __ldcs(B + base[1] + i0 * a.sp.s[1][0] + it * a.sp.s[1][t]);
                C[base[2] + i0 * a.sp.s[2][0] + it * a.sp.s[2][t]] = apply<T>(a.op, x, y, alpha);
            }
        }
    }
}

// Vectorised variant of the tile kernel: TILE x TILE elements (64 for FP32,
// 32 for FP64), 16-byte global accesses along each operand's unit-stride
// dim, and every global load of a tile issued before the shared-memory
// hand-off.  Chosen by the planner when extents and strides allow 16-byte
// vectors for all three operands.
template <typename T>
__global__ void __launch_bounds__(kThreads, 4) ew_tile_vec_kernel(const EwArgs a, int64_t tiles0,
                                                               int64_t tiles1, int64_t batch)
{
    constexpr int VEC = 16 / sizeof(T);
    constexpr int TILE = 16 * VEC;
    constexpr int CH = TILE / VEC;          // vectors per tile row (16)
    constexpr int RPP = kThreads / CH;      // tile rows per pass (16)
    constexpr int NP = TILE / RPP;          // passes
    __shared__ T tA[TILE][TILE + 1];
    __shared__ T tB[TILE][TILE + 1];
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int t = a.tdim;
    const int ch = threadIdx.x % CH, rr = threadIdx.x / CH;
    const int64_t n0 = a.sp.n[0], nt = a.sp.n[t];
    const bool stageA = a.sp.s[0][t] < a.sp.s[0][0];
    const bool stageB = !unary && a.sp.s[1][t] < a.sp.s[1][0];
    const int64_t total = tiles0 * tiles1 * batch;
    for (int64_t blk = blockIdx.x; blk < total; blk += gridDim.x) {
        int64_t bt0 = blk % tiles0;
        int64_t rest = blk / tiles0;
        int64_t bt1 = rest % tiles1;
        int64_t bz = rest / tiles1;
        int64_t base[3] = {0, 0, 0};
        {
            int64_t g = bz;
            for (int d = 1; d < a.sp.nd; ++d) {
                if (d == t) continue;
                int64_t i = g % a.sp.n[d];
                g /= a.sp.n[d];
#pragma unroll
                for (int o = 0; o < 3; ++o) base[o] += i * a.sp.s[o][d];
            }
        }
        const int64_t i0b = bt0 * TILE, itb = bt1 * TILE;
        T xa[NP][VEC], xb[NP][VEC];
        __syncthreads();
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            // staged operands: vectors along t; direct operands: along dim 0
            const int64_t i0s = i0b + rr + p * RPP, its = itb + ch * VEC;
            const int64_t i0d = i0b + ch * VEC, itd = itb + rr + p * RPP;
            if (stageA) {
                if (i0s < n0 && its < nt) {
                    T x[VEC];
                    vload_stream<T, VEC>(A + base[0] + i0s * a.sp.s[0][0] + its, x);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) tA[ch * VEC + e][rr + p * RPP] = x[e];
                }
            } else if (i0d < n0 && itd < nt) {
                vload_stream<T, VEC>(A + base[0] + i0d + itd * a.sp.s[0][t], xa[p]);
            }
            if (!unary) {
                if (stageB) {
                    if (i0s < n0 && its < nt) {
                        T x[VEC];
                        vload_stream<T, VEC>(B + base[1] + i0s * a.sp.s[1][0] + its, x);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) tB[ch * VEC + e][rr + p * RPP] = x[e];
                    }
                } else if (i0d < n0 && itd < nt) {
                    vload_stream<T, VEC>(B + base[1] + i0d + itd * a.sp.s[1][t], xb[p]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int64_t i0 = i0b + ch * VEC, it = itb + rr + p * RPP;
            if (i0 < n0 && it < nt) {
                T r[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    T x = stageA ? tA[rr + p * RPP][ch * VEC + e] : xa[p][e];
                    T y = unary ? T(0) : (stageB ? tB[rr + p * RPP][ch * VEC + e] : xb[p][e]);
                    r[e] = apply<T>(a.op, x, y, alpha);
                }
                vstore<T, VEC>(C + base[2] + i0 + it * a.sp.s[2][t], r);
            }
        }
    }
}

int grid_for(int64_t threads, int num_sms)
{
    int64_t blocks = (threads + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms * (2048 / kThreads);
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

template <typename T>
int launch_typed(const EwPlan& P, const void* A, const void* B, double alpha, void* C,
                 int num_sms, cudaStream_t st)
{
    EwArgs a{};
    a.A = A;
    a.B = B ? B : A;
    a.C = C;
    a.alpha = alpha;
    a.op = P.op;
    a.tdim = P.tdim;
    a.N = P.N;
    a.sp = to_dev(P.sp);
    constexpr int V = 16 / sizeof(T);
    if (P.kernel == K_EW_FLAT) {
        int grid = grid_for((P.N / P.vec + 1) / 2, num_sms);
        if (P.vec == V) ew_flat_kernel<T, V><<<grid, kThreads, 0, st>>>(a);
        else ew_flat_kernel<T, 1><<<grid, kThreads, 0, st>>>(a);
    } else if (P.kernel == K_EW_TILE) {
        const int tile = P.vec > 1 ? 16 * V : kTile;
        int64_t tiles0 = (P.sp.d[0].n + tile - 1) / tile;
        int64_t tiles1 = (P.sp.d[P.tdim].n + tile - 1) / tile;
        int64_t batch = P.N / (P.sp.d[0].n * P.sp.d[P.tdim].n);
        int64_t total = tiles0 * tiles1 * batch;
        int64_t cap = (int64_t)num_sms * 8;
        int grid = (int)(total < cap ? total : cap);
        if (P.vec > 1) ew_tile_vec_kernel<T><<<grid, kThreads, 0, st>>>(a, tiles0, tiles1, batch);
        else ew_tile_kernel<T><<<grid, kThreads, 0, st>>>(a, tiles0, tiles1, batch);
    } else if (P.kernel == K_EW_ROWS) {
        ew_rows_kernel<T, V, 2><<<grid_for((P.N / V + 1) / 2, num_sms), kThreads, 0, st>>>(a);
    } else {
        ew_generic_kernel<T><<<grid_for(P.N, num_sms), kThreads, 0, st>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

}  // namespace

int launch_entrywise(const EwPlan& P, const void* A, const void* B, double alpha, void* C,
                     int num_sms, cudaStream_t st)
{
    if (P.N == 0) return TL_OK;
    if (P.kernel == K_EW_TMA) return launch_ew_tma(P, A, B, alpha, C, num_sms, st);
    if (P.dtype == TL_F64) return launch_typed<double>(P, A, B, alpha, C, num_sms, st);
    return launch_typed<float>(P, A, B, alpha, C, num_sms, st);
}

}  // namespace tl
