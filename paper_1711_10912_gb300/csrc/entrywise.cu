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
//               tile over dims (0, t) is read along t (coalesced for that
//               input), transposed in shared memory and written along dim 0
//               (coalesced for C); an input already contiguous along dim 0
//               is read directly.  16-byte vectors and one 64 x 64 (FP32) or
//               32 x 32 (FP64) tile per CTA when extents and strides allow,
//               else 32 x 32 element tiles.
//   ew_rows     every operand is contiguous along dim 0 but the other dims
//               are ordered differently: one offset decode per 16-byte vector.
//   ew_generic  anything else: each element's offsets come from the mapper.
// FP32 tiles that the vector kernel cannot take (a ragged extent in a padded
// view) but a tensor map can describe run on the TMA-staged kernel of
// ew_tma.cu instead.
#include <cuda_runtime.h>

#include <cstdint>

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
    DevDiv dv;          // ew_rows: division by the extents (dim 0 in vectors)
    // tile kernels: the tile index is (tile along dim 0, tile along t, batch
    // dims); idx32 when it fits in 31 bits (multiply-high division)
    int idx32;
    uint32_t ntile0, ntile1;
    FastDiv ft0, ft1;
    int nb;
    uint32_t bext[kMaxDims];
    FastDiv fb[kMaxDims];
    int64_t bs[3][kMaxDims];   // operands' strides along the batch dims
};

constexpr int kThreads = 256;

// Decodes tile index blk into its tile coordinates along dim 0 and t and the
// operands' offsets of its batch index.  NB >= 0 is the number of batch dims
// known at compile time (the loop unrolls and reads its tables at fixed
// offsets; a bound with a run-time count instead measured 15 % slower on the
// 128^4 adds); NB < 0 takes any number.
template <int NB>
__device__ __forceinline__ void tile_decode(const EwArgs& a, int64_t blk, int64_t& bt0,
                                            int64_t& bt1, int64_t* base)
{
    constexpr int KMAX = NB >= 0 ? NB : kMaxDims;
    const int nb = NB >= 0 ? NB : a.nb;
    base[0] = base[1] = base[2] = 0;
    if (a.idx32) {
        uint32_t r = (uint32_t)blk;
        uint32_t q = fast_div(r, a.ft0);
        bt0 = r - q * a.ntile0;
        r = q;
        q = fast_div(r, a.ft1);
        bt1 = r - q * a.ntile1;
        r = q;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k >= nb) break;
            uint32_t i = r;
            if (k < nb - 1) {
                q = fast_div(r, a.fb[k]);
                i = r - q * a.bext[k];
                r = q;
            }
#pragma unroll
            for (int o = 0; o < 3; ++o) base[o] += (int64_t)i * a.bs[o][k];
        }
        return;
    }
    bt0 = blk % a.ntile0;
    int64_t g = blk / a.ntile0;
    bt1 = g % a.ntile1;
    g /= a.ntile1;
    for (int k = 0; k < nb; ++k) {
        const int64_t i = g % a.bext[k];
        g /= a.bext[k];
#pragma unroll
        for (int o = 0; o < 3; ++o) base[o] += i * a.bs[o][k];
    }
}

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

// Flat stream: U vectors of VEC elements per thread (kThreads apart, so a
// warp's accesses stay contiguous), all loads issued before the stores, and a
// grid of one such chunk per thread (grid-stride only beyond the largest
// grid).  Many short-lived CTAs keep more loads in flight than a persistent
// grid: an FP32 add of 1 GiB operands ran at 7.1 TB/s this way against 6.65
// with a grid of 8 CTAs per SM looping over the stream.
template <typename T, int VEC, int U>
__global__ void __launch_bounds__(kThreads) ew_flat_kernel(const EwArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int64_t nvec = a.N / VEC;
    const int64_t step = (int64_t)gridDim.x * kThreads * U;
    for (int64_t g0 = (int64_t)blockIdx.x * kThreads * U + threadIdx.x; g0 < nvec; g0 += step) {
        T x[U][VEC], y[U][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = g0 + (int64_t)u * kThreads;
            if (g < nvec) {
                vload_stream<T, VEC>(A + g * VEC, x[u]);
                if (!unary) vload_stream<T, VEC>(B + g * VEC, y[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = g0 + (int64_t)u * kThreads;
            if (g < nvec) {
                T r[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) r[v] = apply<T>(a.op, x[u][v], unary ? T(0) : y[u][v], alpha);
                vstore<T, VEC>(C + g * VEC, r);
            }
        }
    }
    // scalar tail (fewer than VEC elements)
    if (blockIdx.x == 0) {
        const int64_t e = nvec * VEC + threadIdx.x;
        if (e < a.N) C[e] = apply<T>(a.op, A[e], unary ? T(0) : B[e], alpha);
    }
}

// Any strides: each element's offsets come from the layout function, with
// multiply-high division and (ND > 0) the collapsed dim count known at
// compile time, so the decode unrolls; U elements per thread (kThreads
// apart: C's writes stay contiguous along dim 0), all loads before the
// stores, one such chunk per thread.
template <typename T, int ND, int U>
__global__ void __launch_bounds__(kThreads) ew_generic_kernel(const EwArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int64_t step = (int64_t)gridDim.x * kThreads * U;
    for (int64_t g0 = (int64_t)blockIdx.x * kThreads * U + threadIdx.x; g0 < a.N; g0 += step) {
        int64_t off[U][3];
        T x[U], y[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = g0 + (int64_t)u * kThreads;
            if (e < a.N) {
                if constexpr (ND > 0) map_offsets_nd<ND, 3>(a.sp, a.dv, e, 1, off[u]);
                else map_offsets_fast<3>(a.sp, a.dv, e, 1, off[u]);
                x[u] = __ldg(A + off[u][0]);
                y[u] = unary ? T(0) : __ldg(B + off[u][1]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = g0 + (int64_t)u * kThreads;
            if (e < a.N) C[off[u][2]] = apply<T>(a.op, x[u], y[u], alpha);
        }
    }
}

// All operands unit-stride along dim 0 but laid out differently in the other
// dims: one offset decode per 16-byte vector along dim 0 (multiply-high
// division), vector loads and stores (dim 0's extent and every other stride
// are multiples of VEC).  Each thread issues the loads of its U vectors
// (kThreads apart) before their stores, one such chunk per thread as in
// ew_flat.  ND > 0 is the collapsed dim count, known at compile time so the
// decode unrolls: on permuted rows of 128^4 FP32 tensors that took the add
// from 6.0 to 6.9 TB/s and the copy from 4.4 to 5.9 (the decode's latency
// sits in front of every load).
template <typename T, int VEC, int U, int ND>
__global__ void __launch_bounds__(kThreads) ew_rows_kernel(const EwArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int64_t nvec = a.N / VEC;
    const int64_t step = (int64_t)gridDim.x * kThreads * U;
    for (int64_t g0 = (int64_t)blockIdx.x * kThreads * U + threadIdx.x; g0 < nvec; g0 += step) {
        int64_t off[U][3];
        T x[U][VEC], y[U][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = g0 + (int64_t)u * kThreads;
            if (g < nvec) {
                if constexpr (ND > 0) map_offsets_nd<ND, 3>(a.sp, a.dv, g, VEC, off[u]);
                else map_offsets_fast<3>(a.sp, a.dv, g, VEC, off[u]);
                vload_stream<T, VEC>(A + off[u][0], x[u]);
                if (!unary) vload_stream<T, VEC>(B + off[u][1], y[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = g0 + (int64_t)u * kThreads;
            if (g < nvec) {
                T r[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    r[v] = apply<T>(a.op, x[u][v], unary ? T(0) : y[u][v], alpha);
                vstore<T, VEC>(C + off[u][2], r);
            }
        }
    }
}

// Tile over dims 0 (fastest in C) and t with element accesses, for extents
// or strides that rule out 16-byte vectors: a T0 x TT tile of 1024 elements
// (16 x 64, 32 x 32, 64 x 16 or 128 x 8, whichever the ragged edges fill
// best: an extent of 9 along t fills a 128 x 8 tile's rows at 9 / 16 instead
// of 9 / 32), 256 threads with 4 elements each per phase, one tile per CTA.
// Staged inputs (faster along t) are read with lanes along t into a padded
// [dim 0][t] shared tile; C and direct inputs go along dim 0.
constexpr int kTileElems = 1024;

template <typename T, int T0>
__global__ void __launch_bounds__(kThreads) ew_tile_kernel(const EwArgs a, int64_t total)
{
    constexpr int TT = kTileElems / T0;
    __shared__ T tA[T0][TT + 1];
    __shared__ T tB[T0][TT + 1];
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const bool unary = (a.op == TL_COPY || a.op == TL_SCALE);
    const int t = a.tdim;
    const int64_t n0 = a.sp.n[0], nt = a.sp.n[t];
    // an input is staged when dim t is its faster dim of the two
    const bool stageA = a.sp.s[0][t] < a.sp.s[0][0];
    const bool stageB = !unary && a.sp.s[1][t] < a.sp.s[1][0];
    const int lt = threadIdx.x % TT, lr = threadIdx.x / TT;     // load phase
    const int lx = threadIdx.x % T0, ly = threadIdx.x / T0;     // write phase
    for (int64_t blk = blockIdx.x; blk < total; blk += gridDim.x) {
        int64_t bt0, bt1, base[3];
        tile_decode<-1>(a, blk, bt0, bt1, base);
        const int64_t i0b = bt0 * T0, itb = bt1 * TT;
        __syncthreads();          // the previous tile's readers are done
        if (stageA || stageB) {
#pragma unroll
            for (int r = 0; r < T0; r += kThreads / TT) {
                const int64_t i0 = i0b + lr + r, it = itb + lt;
                if (i0 < n0 && it < nt) {
                    if (stageA)
                        tA[lr + r][lt] = __ldcs(A + checked_off(a.sp, 0, base[0] + i0 * a.sp.s[0][0] +
                                                                     it * a.sp.s[0][t], 1));
                    if (stageB)
                        tB[lr + r][lt] = __ldcs(B + checked_off(a.sp, 1, base[1] + i0 * a.sp.s[1][0] +
                                                                     it * a.sp.s[1][t], 1));
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < TT; r += kThreads / T0) {
            const int64_t i0 = i0b + lx, it = itb + ly + r;
            if (i0 < n0 && it < nt) {
                T x = stageA ? tA[lx][ly + r]
                             : __ldcs(A + checked_off(a.sp, 0, base[0] + i0 * a.sp.s[0][0] +
                                                                   it * a.sp.s[0][t], 1));
                T y = T(0);
                if (!unary)
                    y = stageB ? tB[lx][ly + r]
                               : __ldcs(B + checked_off(a.sp, 1, base[1] + i0 * a.sp.s[1][0] +
                                                                     it * a.sp.s[1][t], 1));
                C[checked_off(a.sp, 2, base[2] + i0 * a.sp.s[2][0] + it * a.sp.s[2][t], 1)] =
                    apply<T>(a.op, x, y, alpha);
            }
        }
    }
}

// Threads of a vector-tile CTA for a T0 x TT tile: four 16-byte vectors per
// thread and operand for FP32, two for FP64.
template <typename T>
__host__ __device__ constexpr int tile_threads(int t0, int tt)
{
    return t0 * tt / (16 / (int)sizeof(T)) / (sizeof(T) == 4 ? 4 : 2);
}

// Vectorised tile kernel: TILE x TILE elements over dims (0, t), TILE = 64
// for FP32 and 32 for FP64 (256-byte rows either way), one tile per CTA
// (a grid-stride loop only when the tiles outnumber the largest grid).
// Chosen when extents and strides allow 16-byte vectors for all operands.
// SA / SB say which inputs are staged (unit stride along t); UN marks the
// unary operations (COPY, SCALE: B absent); NB is the number of batch dims
// when known at compile time (tile_decode).  Phase 1 reads a staged input as
// 16-byte vectors along t into a padded [dim 0][t] shared tile and a direct
// input (unit stride along dim 0) as 16-byte vectors along dim 0 into
// registers, in the positions phase 2 writes.  Phase 2 writes C along dim 0:
// eight lanes cover 128 contiguous bytes and a warp four t-rows, so the
// staged values it reads from shared memory (column t, rows x..x+VEC-1) fall
// in distinct banks.  Small CTAs, one tile each, keep many tiles' loads in
// flight per SM; binary operations issue every global load of the tile
// before any shared-memory store (up to 4 CTAs per SM), unary ones store each
// load as it arrives (6 CTAs per SM).  On 128^4 FP32 tensors, every
// transposed layout pair: adds 6.6-7.1 TB/s, copies 6.3-7.0; the TMA-staged
// kernel ran them at 5.0-6.8 (its boxes of 128 rows 8 MB apart are the slow
// case), and storing each load at once, or capping binary operations at 6
// CTAs per SM, left the add of the reversed layouts at 5.3-6.0.
template <typename T, int T0, int TT, bool SA, bool SB, bool UN, int NB>
__global__ void __launch_bounds__(tile_threads<T>(T0, TT), (UN ? 1536 : 1024) / tile_threads<T>(T0, TT))
ew_tile_vec_kernel(const EwArgs a, int64_t total)
{
    constexpr int VEC = 16 / sizeof(T);
    constexpr int NT = tile_threads<T>(T0, TT);          // threads of the CTA
    constexpr int LD = TT + 1;                            // padded shared row
    constexpr int NV = T0 * TT / VEC / NT;                // vectors per thread and operand
    constexpr int HALVES = T0 / (8 * VEC);                // 128-byte pieces of a dim-0 row
    static_assert(NV * VEC * NT == T0 * TT && (HALVES == 1 || HALVES == 2), "tile shape");
    extern __shared__ __align__(16) unsigned char ew_smem[];
    T* const tA = reinterpret_cast<T*>(ew_smem);
    T* const tB = tA + (SA ? T0 * LD : 0);
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ B = static_cast<const T*>(a.B);
    T* __restrict__ C = static_cast<T*>(a.C);
    const T alpha = (T)a.alpha;
    const int t = a.tdim;
    const int64_t n0 = a.sp.n[0], nt = a.sp.n[t];
    const int64_t sA0 = a.sp.s[0][0], sAt = a.sp.s[0][t], sB0 = a.sp.s[1][0], sBt = a.sp.s[1][t];
    const int64_t sCt = a.sp.s[2][t];
    for (int64_t blk = blockIdx.x; blk < total; blk += gridDim.x) {
        int64_t bt0, bt1, base[3];
        tile_decode<NB>(a, blk, bt0, bt1, base);
        const int64_t i0b = bt0 * T0, itb = bt1 * TT;
        T xa[SA ? 1 : NV][VEC], xb[(SB || UN) ? 1 : NV][VEC];
        if constexpr (UN) {
            // unary (one staged input): each load is followed by its
            // shared-memory store
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const int v = threadIdx.x + NT * k;
                const int ts = (v % (TT / VEC)) * VEC, xs = v / (TT / VEC);
                const int64_t i0s = i0b + xs, its = itb + ts;
                if (i0s < n0 && its < nt) {
                    T x[VEC];
                    vload_stream<T, VEC>(A + checked_off(a.sp, 0, base[0] + i0s * sA0 + its, VEC), x);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) tA[xs * LD + ts + e] = x[e];
                }
            }
            __syncthreads();
        } else {
            T ya[SA ? NV : 1][VEC], yb[SB ? NV : 1][VEC];   // staged values on their way to smem
            bool oks[NV];
            // every global load of the tile first, then the shared-memory stores
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const int v = threadIdx.x + NT * k;
                // staged order: TT / VEC vectors along t per dim-0 row
                const int ts = (v % (TT / VEC)) * VEC, xs = v / (TT / VEC);
                // write order: 8 vectors along dim 0, 4 t-rows, the 128-byte
                // pieces of dim 0
                const int xd = ((v >> 5) % HALVES) * 8 * VEC + (v & 7) * VEC;
                const int td = (v >> 5) / HALVES * 4 + ((v >> 3) & 3);
                const int64_t i0s = i0b + xs, its = itb + ts, i0d = i0b + xd, itd = itb + td;
                oks[k] = i0s < n0 && its < nt;
                const bool okd = i0d < n0 && itd < nt;
                if constexpr (SA) {
                    if (oks[k])
                        vload_stream<T, VEC>(A + checked_off(a.sp, 0, base[0] + i0s * sA0 + its, VEC),
                                             ya[k]);
                } else if (okd) {
                    vload_stream<T, VEC>(A + checked_off(a.sp, 0, base[0] + i0d + itd * sAt, VEC),
                                         xa[k]);
                }
                if constexpr (SB) {
                    if (oks[k])
                        vload_stream<T, VEC>(B + checked_off(a.sp, 1, base[1] + i0s * sB0 + its, VEC),
                                             yb[k]);
                } else if constexpr (!UN) {
                    if (okd)
                        vload_stream<T, VEC>(B + checked_off(a.sp, 1, base[1] + i0d + itd * sBt, VEC),
                                             xb[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const int v = threadIdx.x + NT * k;
                const int ts = (v % (TT / VEC)) * VEC, xs = v / (TT / VEC);
                if (oks[k]) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        if constexpr (SA) tA[xs * LD + ts + e] = ya[k][e];
                        if constexpr (SB) tB[xs * LD + ts + e] = yb[k][e];
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int v = threadIdx.x + NT * k;
            const int xd = ((v >> 5) % HALVES) * 8 * VEC + (v & 7) * VEC;
            const int td = (v >> 5) / HALVES * 4 + ((v >> 3) & 3);
            const int64_t i0 = i0b + xd, it = itb + td;
            if (i0 < n0 && it < nt) {
                T r[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const T x = SA ? tA[(xd + e) * LD + td] : xa[SA ? 0 : k][e];
                    T y = T(0);
                    if constexpr (SB) y = tB[(xd + e) * LD + td];
                    else if constexpr (!UN) y = xb[k][e];
                    r[e] = apply<T>(a.op, x, y, alpha);
                }
                vstore<T, VEC>(C + checked_off(a.sp, 2, base[2] + i0 + it * sCt, VEC), r);
            }
        }
        __syncthreads();   // the next tile (grid-stride case) reuses the shared tiles
    }
}

// Launches the vector tile kernel for staging kind vkind (0 unary, 1 both
// inputs staged, 2 A staged, 3 B staged), a T0 x TT tile and NB batch dims
// (-1: any number).
template <typename T, int T0, int TT, int NB>
void launch_tile_vec(int vkind, int grid, size_t smem, cudaStream_t st, const EwArgs& a,
                     int64_t total)
{
    constexpr int NT = tile_threads<T>(T0, TT);
    switch (vkind) {
    case 0: ew_tile_vec_kernel<T, T0, TT, true, false, true, NB><<<grid, NT, smem, st>>>(a, total); break;
    case 1: ew_tile_vec_kernel<T, T0, TT, true, true, false, NB><<<grid, NT, smem, st>>>(a, total); break;
    case 2: ew_tile_vec_kernel<T, T0, TT, true, false, false, NB><<<grid, NT, smem, st>>>(a, total); break;
    default: ew_tile_vec_kernel<T, T0, TT, false, true, false, NB><<<grid, NT, smem, st>>>(a, total); break;
    }
}

template <typename T, int T0, int TT>
void launch_tile_vec_nb(int nb, int vkind, int grid, size_t smem, cudaStream_t st,
                        const EwArgs& a, int64_t total)
{
    switch (nb) {
    case 0: launch_tile_vec<T, T0, TT, 0>(vkind, grid, smem, st, a, total); break;
    case 1: launch_tile_vec<T, T0, TT, 1>(vkind, grid, smem, st, a, total); break;
    case 2: launch_tile_vec<T, T0, TT, 2>(vkind, grid, smem, st, a, total); break;
    case 3: launch_tile_vec<T, T0, TT, 3>(vkind, grid, smem, st, a, total); break;
    default: launch_tile_vec<T, T0, TT, -1>(vkind, grid, smem, st, a, total); break;
    }
}

// Dim-0 edge of the element tile kernel's T0 x (1024 / T0) tile: the shape
// (16 x 64, 32 x 32, 64 x 16 or 128 x 8) whose ragged edges leave the fewest
// idle slots, 32 x 32 on ties.
int scalar_tile_t0(int64_t n0, int64_t nt)
{
    auto fill = [](int64_t n, int64_t e) { return (double)n / (double)((n + e - 1) / e * e); };
    int best = 32;
    double bf = fill(n0, 32) * fill(nt, 32);
    for (int t0 : {16, 64, 128}) {
        const double f = fill(n0, t0) * fill(nt, kTileElems / t0);
        if (f > bf + 1e-9) {
            bf = f;
            best = t0;
        }
    }
    return best;
}

// Tile edge (elements) along one dim: 256 bytes, or 128 when that fills the
// ragged last tile better (an extent of 96 FP32 elements: three 32-element
// tiles instead of two of 64, the second half empty).
template <typename T>
int tile_edge(int64_t n)
{
    const int64_t big = 256 / sizeof(T), small = 128 / sizeof(T);
    const int64_t tb = (n + big - 1) / big * big, ts = (n + small - 1) / small * small;
    return (int)(ts < tb ? small : big);
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
    constexpr int U = 2;   // vectors per thread (flat, rows)
    auto chunk_grid = [](int64_t nvec) {
        const int64_t g = (nvec + (int64_t)kThreads * U - 1) / ((int64_t)kThreads * U);
        return (int)(g < 1 ? 1 : (g < INT32_MAX ? g : INT32_MAX));
    };
    if (P.kernel == K_EW_FLAT) {
        if (P.vec == V) ew_flat_kernel<T, V, U><<<chunk_grid(P.N / V), kThreads, 0, st>>>(a);
        else ew_flat_kernel<T, 1, U><<<chunk_grid(P.N), kThreads, 0, st>>>(a);
    } else if (P.kernel == K_EW_TILE) {
        const bool unary = P.op == TL_COPY || P.op == TL_SCALE;
        const bool sa = P.sp.d[P.tdim].s[0] < P.sp.d[0].s[0];
        const bool sb = !unary && P.sp.d[P.tdim].s[1] < P.sp.d[0].s[1];
        const bool vec = P.vec > 1 && (sa || sb);
        const int st0 = scalar_tile_t0(P.sp.d[0].n, P.sp.d[P.tdim].n);
        const int t0 = vec ? tile_edge<T>(P.sp.d[0].n) : st0;
        const int tt = vec ? tile_edge<T>(P.sp.d[P.tdim].n) : kTileElems / st0;
        int64_t tiles0 = (P.sp.d[0].n + t0 - 1) / t0;
        int64_t tiles1 = (P.sp.d[P.tdim].n + tt - 1) / tt;
        int64_t batch = P.N / (P.sp.d[0].n * P.sp.d[P.tdim].n);
        int64_t total = tiles0 * tiles1 * batch;
        {
            // tile decode tables: tiles along dim 0 and t, then the batch dims
            a.ntile0 = (uint32_t)tiles0;
            a.ntile1 = (uint32_t)tiles1;
            a.idx32 = total < (int64_t(1) << 31) ? 1 : 0;
            a.ft0 = make_fastdiv(a.idx32 ? a.ntile0 : 1);
            a.ft1 = make_fastdiv(a.idx32 ? a.ntile1 : 1);
            a.nb = 0;
            for (int d = 1; d < P.sp.nd; ++d) {
                if (d == P.tdim) continue;
                a.bext[a.nb] = (uint32_t)P.sp.d[d].n;
                a.fb[a.nb] = make_fastdiv(a.idx32 ? a.bext[a.nb] : 1);
                for (int o = 0; o < 3; ++o) a.bs[o][a.nb] = P.sp.d[d].s[o];
                ++a.nb;
            }
            if (!a.idx32 && (tiles0 >= (int64_t(1) << 32) || tiles1 >= (int64_t(1) << 32)))
                return TL_EUNSUPPORTED;
        }
        const int grid = (int)(total < INT32_MAX ? total : INT32_MAX);
        if (vec) {
            // one tile per CTA; an input is staged when dim t is its faster
            // dim of the two (the planner's vector conditions make it unit
            // stride there)
            const size_t smem = (size_t)((sa ? 1 : 0) + (sb ? 1 : 0)) * t0 * (tt + 1) * sizeof(T);
            const int vkind = unary ? 0 : (sa && sb) ? 1 : sa ? 2 : 3;
            const int nb = a.idx32 ? a.nb : -1;
            constexpr int B = 256 / sizeof(T), S = 128 / sizeof(T);
            if (t0 == B && tt == B) launch_tile_vec_nb<T, B, B>(nb, vkind, grid, smem, st, a, total);
            else if (t0 == B) launch_tile_vec_nb<T, B, S>(nb, vkind, grid, smem, st, a, total);
            else if (tt == B) launch_tile_vec_nb<T, S, B>(nb, vkind, grid, smem, st, a, total);
            else launch_tile_vec_nb<T, S, S>(nb, vkind, grid, smem, st, a, total);
        } else {
            switch (st0) {
            case 16: ew_tile_kernel<T, 16><<<grid, kThreads, 0, st>>>(a, total); break;
            case 64: ew_tile_kernel<T, 64><<<grid, kThreads, 0, st>>>(a, total); break;
            case 128: ew_tile_kernel<T, 128><<<grid, kThreads, 0, st>>>(a, total); break;
            default: ew_tile_kernel<T, 32><<<grid, kThreads, 0, st>>>(a, total); break;
            }
        }
    } else if (P.kernel == K_EW_ROWS) {
        a.dv = make_devdiv(P.sp, V);
        const int grid = chunk_grid(P.N / V);
        switch (a.sp.small ? P.sp.nd : 0) {
        case 2: ew_rows_kernel<T, V, U, 2><<<grid, kThreads, 0, st>>>(a); break;
        case 3: ew_rows_kernel<T, V, U, 3><<<grid, kThreads, 0, st>>>(a); break;
        case 4: ew_rows_kernel<T, V, U, 4><<<grid, kThreads, 0, st>>>(a); break;
        case 5: ew_rows_kernel<T, V, U, 5><<<grid, kThreads, 0, st>>>(a); break;
        default: ew_rows_kernel<T, V, U, 0><<<grid, kThreads, 0, st>>>(a); break;
        }
    } else {
        a.dv = make_devdiv(P.sp, 1);
        const int grid = chunk_grid(P.N);
        switch (a.sp.small ? P.sp.nd : 0) {
        case 1: ew_generic_kernel<T, 1, U><<<grid, kThreads, 0, st>>>(a); break;
        case 2: ew_generic_kernel<T, 2, U><<<grid, kThreads, 0, st>>>(a); break;
        case 3: ew_generic_kernel<T, 3, U><<<grid, kThreads, 0, st>>>(a); break;
        case 4: ew_generic_kernel<T, 4, U><<<grid, kThreads, 0, st>>>(a); break;
        case 5: ew_generic_kernel<T, 5, U><<<grid, kThreads, 0, st>>>(a); break;
        case 6: ew_generic_kernel<T, 6, U><<<grid, kThreads, 0, st>>>(a); break;
        case 7: ew_generic_kernel<T, 7, U><<<grid, kThreads, 0, st>>>(a); break;
        default: ew_generic_kernel<T, 0, U><<<grid, kThreads, 0, st>>>(a); break;
        }
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
