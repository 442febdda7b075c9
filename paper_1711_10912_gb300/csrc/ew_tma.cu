// ew_tma.cu -- the layout-mixed entrywise operation of Sec. 5.1 (Eqs. 22-23) for
// FP32 tensors whose layouts differ, staged through shared memory by TMA.
//
// The collapsed space (plan.cpp) has C unit-stride along dim 0.  The kernel
// walks tiles of up to 128 (dim 0) x 32 (t) elements over dims (0, t), times
// the remaining (batch) dims.  Each input is either
//   transposed  unit stride along t: one TMA box of 32 t-values (128 bytes)
//               x up to 128 dim-0 rows lands as [dim 0][t], or
//   direct      unit stride along dim 0: up to four 32 x 32 boxes land as
//               [t][dim 0], one per 32 rows of dim 0.
// Boxes use the 128-byte swizzle (16-byte chunk index XOR row mod 8), which
// keeps the transposed read free of bank conflicts (the direct read: 2-way).
//
// Warp 8 is the producer: for every tile of the CTA it waits for a free
// stage, arms the stage's barrier with the tile's bytes and issues the TMA
// loads.  Warps 0-7 consume: warp w owns t = 4w..4w+3 of the tile.  For each
// 32-row block m, lane l = 4g + j reads 16 bytes of a transposed input at row
// 32m + l, chunk w; a 4 x 4 transpose among lanes 4g..4g+3 (four shuffles)
// leaves lane l holding dim-0 rows 32m + 4g..4g+3 at t = 4w + j, one 16-byte
// vector of C, and the eight lanes with the same j write 128 contiguous bytes
// of C.  Direct inputs are read at that final position.  The operation is a
// template parameter.  All mbarrier waits are bounded; a CTA that gives up
// sets g_ew_status and drains its in-flight copies.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cstdint>

#include "kernels.h"
#include "runtime.h"
#include "pipeline.cuh"
#include "plan.h"

namespace tl {

__device__ unsigned int g_ew_status = 0;

namespace {

constexpr int kTB = 32;                    // box edge (elements): 128 bytes of FP32
constexpr int kMaxBlocks = 4;              // 32-row blocks of dim 0 per tile
constexpr int kConsumers = 8;
constexpr int kThreadsTma = (kConsumers + 1) * 32;
constexpr uint32_t kBoxBytes = kTB * kTB * 4;

struct TmaArgs {
    float* C;
    int op;
    float alpha;
    int nin;                // inputs loaded (1 for COPY / SCALE, else 2)
    int transposed[2];      // input o has unit stride along t (else along dim 0)
    int nb;                 // batch dims (0..3)
    int64_t n0, nt;
    int64_t tiles0, tilest, ntiles;
    int64_t bn[3];          // batch extents
    int64_t sct;            // C's stride along t
    int64_t scb[3];         // C's strides along the batch dims
    int nstages;
    int blocks;             // 32-row blocks of dim 0 per tile (1..4)
    uint32_t in_bytes;      // bytes of one input's tile in shared memory
    uint32_t stage_bytes;
    uint32_t off_bar;
};

template <int OP>
__device__ __forceinline__ float apply_op(float a, float b, float alpha)
{
    if constexpr (OP == TL_ADD) return a + b;
    else if constexpr (OP == TL_SUB) return a - b;
    else if constexpr (OP == TL_MUL) return a * b;
    else if constexpr (OP == TL_DIV) return a / b;
    else if constexpr (OP == TL_COPY) return a;
    else return alpha * a;
}

template <int OP>
__device__ __forceinline__ float4 apply4(float4 x, float4 y, float alpha)
{
    return make_float4(apply_op<OP>(x.x, y.x, alpha), apply_op<OP>(x.y, y.y, alpha),
                       apply_op<OP>(x.z, y.z, alpha), apply_op<OP>(x.w, y.w, alpha));
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int nd,
                                         const int* c, uint32_t bar)
{
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    switch (nd) {
    case 2:
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst), "l"(m), "r"(c[0]), "r"(c[1]), "r"(bar)
            : "memory");
        break;
    case 3:
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst), "l"(m), "r"(c[0]), "r"(c[1]),
            "r"(c[2]), "r"(bar)
            : "memory");
        break;
    case 4:
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst), "l"(m), "r"(c[0]), "r"(c[1]),
            "r"(c[2]), "r"(c[3]), "r"(bar)
            : "memory");
        break;
    default:
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst), "l"(m), "r"(c[0]),
            "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(bar)
            : "memory");
        break;
    }
}

// Mixed-radix tile coordinates (tile along dim 0, tile along t, batch
// indices), decoded in 32-bit arithmetic (tile counts and extents are below
// 2^31).
struct TileCoord {
    uint32_t b0, bt, bi[3];
};

__device__ __forceinline__ TileCoord decode_tile(const TmaArgs& a, int64_t tile)
{
    TileCoord c;
    uint32_t r = (uint32_t)tile;
    c.b0 = r % (uint32_t)a.tiles0;
    r /= (uint32_t)a.tiles0;
    c.bt = r % (uint32_t)a.tilest;
    r /= (uint32_t)a.tilest;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d < a.nb) {
            c.bi[d] = r % (uint32_t)a.bn[d];
            r /= (uint32_t)a.bn[d];
        } else {
            c.bi[d] = 0;
        }
    }
    return c;
}

// Byte offset of the 16-byte chunk `chunk` of row `row` in a 128-byte-swizzled
// tile whose rows are 128 bytes.
__device__ __forceinline__ uint32_t swz(int row, int chunk)
{
    return (uint32_t)(row * 128 + ((chunk ^ (row & 7)) << 4));
}

// 4 x 4 transpose among the lanes 4g..4g+3: on entry lane j holds row j
// (x[i] = M[j][i]); on exit it holds column j (x[i] = M[i][j]).
__device__ __forceinline__ void transpose4(float4& v, int j)
{
    const bool odd = j & 1, hi = j & 2;
    const float r0 = __shfl_xor_sync(0xffffffffu, odd ? v.x : v.y, 1);
    const float r1 = __shfl_xor_sync(0xffffffffu, odd ? v.z : v.w, 1);
    // rows {j & ~1, j | 1} x columns {j & 1, (j & 1) + 2}
    const float u00 = odd ? r0 : v.x, u01 = odd ? r1 : v.z;
    const float u10 = odd ? v.y : r0, u11 = odd ? v.w : r1;
    const float q0 = __shfl_xor_sync(0xffffffffu, hi ? u00 : u01, 2);
    const float q1 = __shfl_xor_sync(0xffffffffu, hi ? u10 : u11, 2);
    if (hi) {
        v = make_float4(q0, q1, u01, u11);
    } else {
        v = make_float4(u00, u10, q0, q1);
    }
}

template <int OP>
__global__ void __launch_bounds__(kThreadsTma, 2)
ew_tma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const TmaArgs a, int ndA, int ndB)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // TMA's 128-byte swizzle wants 1024-byte aligned destinations
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = pipe::smem_u32(smem);
    const uint32_t full = base + a.off_bar, empty = full + 8 * a.nstages;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.nstages; ++s) {
            pipe::mbar_init(full + 8 * s, 1);
            pipe::mbar_init(empty + 8 * s, kConsumers);
        }
        pipe::mbar_init_fence();
        pipe::fence_proxy_async();
    }
    __syncthreads();
    const int rows = a.blocks * kTB;      // dim-0 extent of a tile

    if (warp == kConsumers) {
        if (lane == 0) {
            pipe::Ring r;
            bool ok = true;
            uint32_t armed = 0, par = 0;
            for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
                if (!(ok = pipe::mbar_wait(empty + 8 * r.idx, r.phase ^ 1u, &g_ew_status))) break;
                const TileCoord tc = decode_tile(a, tile);
                const uint32_t bar = full + 8 * r.idx;
                pipe::mbar_arrive_tx(bar, a.stage_bytes);
                const uint32_t dst = base + r.idx * a.stage_bytes;
                int c[5];
                c[2] = (int)tc.bi[0];
                c[3] = (int)tc.bi[1];
                c[4] = (int)tc.bi[2];
                for (int o = 0; o < a.nin; ++o) {
                    const CUtensorMap* map = o == 0 ? &mapA : &mapB;
                    const int nd = o == 0 ? ndA : ndB;
                    if (a.transposed[o]) {
                        // one box: 32 t-values x `rows` dim-0 rows
                        c[0] = (int)(tc.bt * kTB);
                        c[1] = (int)(tc.b0 * rows);
                        tma_load(dst + o * a.in_bytes, map, nd, c, bar);
                    } else {
                        // per 32-row block m of dim 0: a 32 x 32 box
                        for (int m = 0; m < a.blocks; ++m) {
                            c[0] = (int)(tc.b0 * rows + m * kTB);
                            c[1] = (int)(tc.bt * kTB);
                            tma_load(dst + o * a.in_bytes + m * kBoxBytes, map, nd, c, bar);
                        }
                    }
                }
                armed |= 1u << r.idx;
                par = (par & ~(1u << r.idx)) | (r.phase << r.idx);
                r.next(a.nstages);
            }
            if (!ok)
                for (int s = 0; s < a.nstages; ++s)
                    if (armed & (1u << s)) pipe::mbar_drain(full + 8 * s, (par >> s) & 1u);
        }
        return;
    }

    const int g = lane >> 2, j = lane & 3;
    const bool tA = a.transposed[0], tB = a.nin == 2 && a.transposed[1];
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    pipe::Ring r;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        if (!pipe::mbar_wait(full + 8 * r.idx, r.phase, &g_ew_status)) break;
        const uint8_t* st = smem + r.idx * a.stage_bytes;
        float4 res[kMaxBlocks];
#pragma unroll
        for (int m = 0; m < kMaxBlocks; ++m) {
            if (m < a.blocks) {
                // transposed tiles: row 32m + lane, chunk warp; direct: box m,
                // row 4 warp + j, chunk g
                const uint32_t ot = swz(m * kTB + lane, warp);
                const uint32_t od = m * kBoxBytes + swz(4 * warp + j, g);
                if (a.nin == 1) {
                    float4 x = *reinterpret_cast<const float4*>(st + (tA ? ot : od));
                    if (tA) transpose4(x, j);
                    res[m] = apply4<OP>(x, zero, a.alpha);
                } else if (tA && tB) {
                    const float4 x = *reinterpret_cast<const float4*>(st + ot);
                    const float4 y = *reinterpret_cast<const float4*>(st + a.in_bytes + ot);
                    float4 v = apply4<OP>(x, y, a.alpha);
                    transpose4(v, j);
                    res[m] = v;
                } else {
                    float4 x = *reinterpret_cast<const float4*>(st + (tA ? ot : od));
                    float4 y = *reinterpret_cast<const float4*>(st + a.in_bytes + (tB ? ot : od));
                    if (tA) transpose4(x, j);
                    if (tB) transpose4(y, j);
                    res[m] = apply4<OP>(x, y, a.alpha);
                }
            }
        }
        __syncwarp();
        if (lane == 0) pipe::mbar_arrive(empty + 8 * r.idx);
        r.next(a.nstages);
        const TileCoord tc = decode_tile(a, tile);
        const int64_t it = (int64_t)tc.bt * kTB + 4 * warp + j;
        if (it < a.nt) {
            int64_t off = it * a.sct;
            for (int d = 0; d < a.nb; ++d) off += (int64_t)tc.bi[d] * a.scb[d];
#pragma unroll
            for (int m = 0; m < kMaxBlocks; ++m) {
                const int64_t i0 = (int64_t)tc.b0 * rows + m * kTB + 4 * g;
                if (m < a.blocks && i0 < a.n0) {
                    float* pc = a.C + off + i0;
                    const float4 v = res[m];
                    if (i0 + 3 < a.n0) {
                        *reinterpret_cast<float4*>(pc) = v;
                    } else {
                        const float e[4] = {v.x, v.y, v.z, v.w};
                        for (int q = 0; q < 4 && i0 + q < a.n0; ++q) pc[q] = e[q];
                    }
                }
            }
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static std::atomic<void*> fn{nullptr};
    void* p = fn.load();
    if (!p) {
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn.store(p);
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
}

}  // namespace

// The planner's conditions (plan.cpp, K_EW_TMA) guarantee that every map
// below is encodable; a failure is reported as TL_ECUDA.
int launch_ew_tma(const EwPlan& P, const void* A, const void* B, double alpha, void* C,
                  int num_sms, cudaStream_t st)
{
    const Space& sp = P.sp;
    const int t = P.tdim;
    TmaArgs a{};
    a.C = static_cast<float*>(C);
    a.op = P.op;
    a.alpha = (float)alpha;
    a.nin = (P.op == TL_COPY || P.op == TL_SCALE) ? 1 : 2;
    a.n0 = sp.d[0].n;
    a.nt = sp.d[t].n;
    a.blocks = (int)((a.n0 + kTB - 1) / kTB);
    if (a.blocks > kMaxBlocks) a.blocks = kMaxBlocks;
    const int64_t rows = (int64_t)a.blocks * kTB;
    a.tiles0 = (a.n0 + rows - 1) / rows;
    a.tilest = (a.nt + kTB - 1) / kTB;
    a.sct = sp.d[t].s[2];
    a.nb = 0;
    int bdim[3];
    for (int d = 1; d < sp.nd; ++d) {
        if (d == t) continue;
        bdim[a.nb] = d;
        a.bn[a.nb] = sp.d[d].n;
        a.scb[a.nb] = sp.d[d].s[2];
        ++a.nb;
    }
    a.ntiles = a.tiles0 * a.tilest;
    for (int d = 0; d < a.nb; ++d) a.ntiles *= a.bn[d];
    if (a.ntiles == 0) return TL_OK;

    auto enc = encoder();
    if (!enc) return TL_ECUDA;
    CUtensorMap maps[2];
    int nds[2] = {0, 0};
    for (int o = 0; o < a.nin; ++o) {
        const void* ptr = o == 0 ? A : B;
        a.transposed[o] = sp.d[t].s[o] == 1 && sp.d[0].s[o] != 1;
        const int first = a.transposed[o] ? t : 0, second = a.transposed[o] ? 0 : t;
        cuuint64_t gdim[5], gstr[4];
        cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
        gdim[0] = (cuuint64_t)sp.d[first].n;
        gdim[1] = (cuuint64_t)sp.d[second].n;
        gstr[0] = (cuuint64_t)sp.d[second].s[o] * 4;
        box[0] = kTB;
        box[1] = a.transposed[o] ? (cuuint32_t)rows : kTB;
        for (int d = 0; d < a.nb; ++d) {
            gdim[2 + d] = (cuuint64_t)sp.d[bdim[d]].n;
            gstr[1 + d] = (cuuint64_t)sp.d[bdim[d]].s[o] * 4;
            box[2 + d] = 1;
        }
        nds[o] = 2 + a.nb;
        // no promotion beyond the 128-byte box rows: with 256-byte L2 fills
        // a transposed input whose rows are 512 bytes apart (its t-tiles
        // read by neighbouring CTAs at the same time) copies at 4.75 TB/s
        // instead of 6.06 (128^4 FP32, C in (2,3,4,1) order)
        CUresult cr = enc(&maps[o], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nds[o], const_cast<void*>(ptr),
                          gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return TL_ECUDA;
    }
    if (a.nin == 1) {
        maps[1] = maps[0];
        nds[1] = nds[0];
    }
    a.in_bytes = (uint32_t)a.blocks * kBoxBytes;
    a.stage_bytes = (uint32_t)a.nin * a.in_bytes;
    // 2 resident CTAs per SM with 3 stages for one input (96 KB of tiles in
    // flight per SM) and 2 for two (128 KB): on 128^4 FP32 tensors the
    // two-input add with one operand in (2,4,1,3) order runs at 6.4 TB/s with
    // 2 stages and 5.7 with 3, the fully reversed one at 5.0 with either; a
    // grid larger than the resident CTAs measured slower
    const int ctas = 2;
    a.nstages = a.nin == 2 ? 2 : 3;
    a.off_bar = a.nstages * a.stage_bytes;
    const uint32_t smem = a.off_bar + 16 * a.nstages + 1024;
    int rc;
    switch (a.op) {
    case TL_ADD: rc = smem_optin(reinterpret_cast<const void*>(ew_tma_kernel<TL_ADD>), (int)smem); break;
    case TL_SUB: rc = smem_optin(reinterpret_cast<const void*>(ew_tma_kernel<TL_SUB>), (int)smem); break;
    case TL_MUL: rc = smem_optin(reinterpret_cast<const void*>(ew_tma_kernel<TL_MUL>), (int)smem); break;
    case TL_DIV: rc = smem_optin(reinterpret_cast<const void*>(ew_tma_kernel<TL_DIV>), (int)smem); break;
    case TL_COPY: rc = smem_optin(reinterpret_cast<const void*>(ew_tma_kernel<TL_COPY>), (int)smem); break;
    default: rc = smem_optin(reinterpret_cast<const void*>(ew_tma_kernel<TL_SCALE>), (int)smem); break;
    }
    if (rc != TL_OK) return TL_ECUDA;
    const int64_t cap = (int64_t)num_sms * ctas;
    const int grid = (int)(a.ntiles < cap ? a.ntiles : cap);
    switch (a.op) {
    case TL_ADD: ew_tma_kernel<TL_ADD><<<grid, kThreadsTma, smem, st>>>(maps[0], maps[1], a, nds[0], nds[1]); break;
    case TL_SUB: ew_tma_kernel<TL_SUB><<<grid, kThreadsTma, smem, st>>>(maps[0], maps[1], a, nds[0], nds[1]); break;
    case TL_MUL: ew_tma_kernel<TL_MUL><<<grid, kThreadsTma, smem, st>>>(maps[0], maps[1], a, nds[0], nds[1]); break;
    case TL_DIV: ew_tma_kernel<TL_DIV><<<grid, kThreadsTma, smem, st>>>(maps[0], maps[1], a, nds[0], nds[1]); break;
    case TL_COPY: ew_tma_kernel<TL_COPY><<<grid, kThreadsTma, smem, st>>>(maps[0], maps[1], a, nds[0], nds[1]); break;
    default: ew_tma_kernel<TL_SCALE><<<grid, kThreadsTma, smem, st>>>(maps[0], maps[1], a, nds[0], nds[1]); break;
    }
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

int ew_status(bool clear)
{
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_ew_status, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return TL_ECUDA;
    }
    if (v && clear) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_ew_status, &z, sizeof z);
    }
    return v ? TL_ETIMEOUT : TL_OK;
}

}  // namespace tl
