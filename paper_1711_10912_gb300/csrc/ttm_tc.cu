// ttm_tc.cu -- mode-q tensor-times-matrix on the tcgen05 tensor cores,
// Sec. 5.2 Eq. 25:  C(i with i_q = j) = sum_k A(i with i_q = k) * B(j, k).
//
// The rows of the product are the non-contracted elements of A (m), the
// columns are j and the reduction runs over k = i_q, i.e. the paper's
// slice-times-matrix reading of ttm with every slice batched into one GEMM.
// Two row orientations are supported (chosen by the planner):
//   ROW  w_q = 1: row m of A is contiguous in k (A is M x n_q, row stride
//        lda), loaded by a 2-D TMA box of 128 rows x 32 k (128-byte swizzle);
//   COL  the fastest output mode i has unit stride in A and w_q > 1: the
//        rows of one tile are 128 consecutive i of one outer index o, loaded
//        by a 3-D TMA box of 128 i x 32 k x 1 o.
// FP32 data is converted on chip: eight converter warps read the FP32 tile,
// round it to TF32, to BF16, or split it into BF16 hi + lo (hi = RN(a),
// lo = RN(a - hi)), and write the tensor-core operand in the K-major,
// no-swizzle canonical layout (8-row x 16-byte core matrices).  B is
// converted once per call into the same layout in global scratch; up to
// 64 KB of it stays in shared memory for the whole launch, a larger one is
// streamed per k stage with bulk copies by a warp of its own.
// Split-BF16x3 issues hi*hi + hi*lo + lo*hi; every product accumulates in
// FP32 in TMEM.
//
// Warp roles (608 threads, one CTA per SM, persistent over tiles):
//   warp 0       TMA producer of the FP32 A tiles (one thread)
//   warp 1       TMEM allocator and MMA issuer (one thread)
//   warps 2-9    converters: two threads per operand row, each converting
//                half of the stage's 32 k values
//   warps 10-17  epilogue: TMEM -> registers -> C; warp w reads the TMEM
//                lane quarter w % 4 and every other 32-column chunk
//   warp 18      B stream (one thread; idle when B is resident)
// Eight + eight warps rather than four + four: the conversion and drain
// chains are latency-bound, and more warps in flight keep the HBM stream
// busy (measured on GB300).
// Every mbarrier wait is bounded: after about two seconds without progress
// the thread records a timeout in a status word, the CTA drains its TMA copies,
// frees its TMEM and returns, and tl_device_status() reports TL_ETIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "kernels.h"
#include "pipeline.cuh"
#include "runtime.h"

namespace tl {

__device__ unsigned int g_tc_status;

namespace {

constexpr int BM = 128;
constexpr int BK = 32;                 // k per stage
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 8;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kEpiWarp0 = 2 + kConvWarps;
constexpr int kBWarp = kEpiWarp0 + kEpiWarps;   // streams B when it is not resident
constexpr int kThreads = 32 * (kBWarp + 1);
constexpr int kTmemCols = 512;

enum Variant { V_NONE = 0, V_ROW = 1, V_COL = 2 };

// ------------------------------------------------------------ PTX helpers --

// mbarriers, bulk copies, TMA loads and proxy fences come from pipeline.cuh;
// this kernel's bounded waits report into g_tc_status.
using pipe::bulk_load;
using pipe::fence_proxy_async;
using pipe::kTimeoutCycles;
using pipe::mbar_arrive;
using pipe::mbar_arrive_tx;
using pipe::mbar_init;
using pipe::mbar_try;
using pipe::smem_u32;
using pipe::tma_load_2d;
using pipe::tma_load_3d;

// Bounded wait: false (and the status word set) after `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = kTimeoutCycles)
{
    return pipe::mbar_wait(bar, parity, &g_tc_status, limit);
}

// One thread waits on a barrier whose phase never completes (its arrival
// count is 2 and only one arrival happens); the bounded wait gives up.
__global__ void selftest_wait_kernel(long long limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        const uint32_t b = smem_u32(&bar);
        mbar_init(b, 2);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_arrive(b);
        mbar_wait(b, 0u, limit);
    }
}

// TMA stores of a shared-memory box into C (bulk-group completion, issued and
// waited on by one thread)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z,
                                             uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the source of every committed store has been read (its shared memory may be reused)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// UMMA shared-memory descriptor, K-major, no swizzle: 8-row x 16-byte core
// matrices; lbo = byte distance between core matrices along K, sbo = byte
// distance between 8-row groups.
// Shared-memory matrix descriptor of a K-major swizzled operand: rows of
// `row` bytes (64: 64-byte swizzle, 128: 128-byte swizzle), 8-row groups
// `sbo` bytes apart; the leading byte offset is unused for K-major swizzled
// layouts (set to 16 bytes).  `addr` may point inside a swizzle atom along K
// (the k sub-steps of a stage): the swizzle is a function of the address bits,
// and every atom starts at a multiple of its size (base offset 0).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t row, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;            // leading byte offset 16 (unused)
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
    d |= (uint64_t)(row == 128 ? 2u : 4u) << 61;   // layout: 128-byte / 64-byte swizzle
    return d;
}

// Byte offset of 16-byte chunk c of row r in a K-major swizzled operand with
// rows of `row` bytes: the chunk index is XORed with the row's position in
// the swizzle pattern (128-byte swizzle: r mod 8; 64-byte swizzle: (r / 2)
// mod 4), which spreads the rows of an 8-row group over all banks.
__host__ __device__ __forceinline__ uint32_t sw_off(uint32_t r, uint32_t c, uint32_t row)
{
    const uint32_t f = row == 128 ? (r & 7u) : ((r >> 1) & 3u);
    return r * row + ((c ^ f) << 4);
}

// Instruction descriptor: D = F32, A/B format (1 = BF16, 2 = TF32), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t fmt, uint32_t M, uint32_t N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accum)
{
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    }
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// FP32 -> TF32 rounded to nearest, ties to even (the same rule as the BF16
// conversions), so TF32 results do not drift away from zero on ties
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rn.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------ parameters --

struct TcArgs {
    float* C;
    const uint8_t* bimg;     // converted B, [ks][part][Jp x BK] canonical tiles
    int variant;
    int prec;                // TL_P_TF32, TL_P_BF16, TL_P_BF16X3
    int nparts;              // 1 or 2 (hi, lo)
    int esize;               // operand element bytes (4 tf32, 2 bf16)
    int J, Jp, nks;
    int ns_stg, ns_op;
    int nacc;                // TMEM accumulator buffers (2 when Jp <= 256)
    int accumulate;
    int vec_out;             // j contiguous in C, 16-byte aligned rows: float4 stores
    int vec_rows;            // rows contiguous in C (COL), 16-byte aligned: float4 along rows
    int tma_out;             // C written by TMA stores of 32 x 32 boxes (no accumulation)
    int64_t ntiles;
    int64_t M;               // ROW: rows; COL: inner extent
    int64_t tiles_per_o;     // COL
    int64_t sc_m;            // ROW: C stride of m; COL: C stride of i
    int64_t sc_o;            // COL: C stride of o
    int64_t scq;             // C stride of j
    uint32_t a_stage_bytes;  // FP32 staging tile
    uint32_t opa_part_bytes, opb_part_bytes;
    uint32_t off_stg, off_op, op_stage_bytes, off_bar, off_epi;
    int b_resident;          // the whole converted B stays in shared memory at off_b
    uint32_t off_b, b_bytes;
};

struct Bars {
    uint32_t stg_full, stg_empty, op_full, op_empty, acc_full, acc_empty, b_full, tmem_slot;
};

__device__ __forceinline__ Bars bar_layout(uint32_t base, const TcArgs& a)
{
    Bars b;
    b.stg_full = base;
    b.stg_empty = b.stg_full + 8 * a.ns_stg;
    b.op_full = b.stg_empty + 8 * a.ns_stg;
    b.op_empty = b.op_full + 8 * a.ns_op;
    b.acc_full = b.op_empty + 8 * a.ns_op;
    b.acc_empty = b.acc_full + 16;
    b.b_full = b.acc_empty + 16;
    b.tmem_slot = b.b_full + 8;
    return b;
}

// Pipeline position: stage index and the parity of its current phase.
struct Pipe {
    int idx = 0;
    uint32_t phase = 0;
    __device__ void next(int n)
    {
        if (++idx == n) { idx = 0; phase ^= 1u; }
    }
};

// ---------------------------------------------------------------- kernel --

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
ttm_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap cmap,
              const TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // align the dynamic shared memory base to 1024 bytes (128-byte swizzle atoms)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sbase = smem_raw + (base - raw);
    const Bars bars = bar_layout(base + a.off_bar, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool kTF32 = (PREC == TL_P_TF32);
    constexpr int kParts = (PREC == TL_P_BF16X3) ? 2 : 1;
    constexpr int kKmma = kTF32 ? 8 : 16;           // k per MMA instruction
    constexpr int kSubs = BK / kKmma;
    constexpr int kChunks = BK * (kTF32 ? 4 : 2) / 16;   // 16-byte chunks per operand row
    constexpr uint32_t kRow = kChunks * 16;         // operand row bytes (= swizzle width)
    constexpr uint32_t kSbo = kChunks * 128;        // bytes per 8-row group
    constexpr uint32_t kSubBytes = kKmma * (kTF32 ? 4 : 2);   // k bytes per MMA instruction

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.ns_stg; ++s) {
            mbar_init(bars.stg_full + 8 * s, 1);
            mbar_init(bars.stg_empty + 8 * s, kConvThreads);
        }
        for (int s = 0; s < a.ns_op; ++s) {
            mbar_init(bars.op_full + 8 * s, (a.b_resident ? 0 : 1) + kConvThreads);
            mbar_init(bars.op_empty + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(bars.acc_full + 8 * s, 1);
            mbar_init(bars.acc_empty + 8 * s, kEpiThreads);
        }
        mbar_init(bars.b_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(bars.tmem_slot), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(sbase + (bars.tmem_slot - base));
    const uint32_t acc_cols = a.nacc == 2 ? 256u : 512u;

    auto op_a = [&](int stage, int part) -> uint32_t {
        return base + a.off_op + stage * a.op_stage_bytes + part * a.opa_part_bytes;
    };
    // streamed B: in the operand stage after A's parts; resident B: the image
    // tile of k stage `ks` (passed as `stage`)
    auto op_b = [&](int stage, int part) -> uint32_t {
        if (a.b_resident) return base + a.off_b + (uint32_t)(stage * kParts + part) * a.opb_part_bytes;
        return base + a.off_op + stage * a.op_stage_bytes + kParts * a.opa_part_bytes +
               part * a.opb_part_bytes;
    };

    if (warp == 0) {
        // ------------------------------------------------------ producer
        if (lane == 0) {
            Pipe st;
            bool ok = true;
            // parity of the last arm of each stage, to drain on exit
            uint32_t stg_armed = 0, stg_par = 0;
            if (a.b_resident) {
                // the whole converted B, once per CTA, in 64 KB pieces
                mbar_arrive_tx(bars.b_full, a.b_bytes);
                for (uint32_t o = 0; o < a.b_bytes; o += 65536u) {
                    const uint32_t n = a.b_bytes - o < 65536u ? a.b_bytes - o : 65536u;
                    bulk_load(base + a.off_b + o, a.bimg + o, n, bars.b_full);
                }
            }
            for (int64_t tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
                int64_t o = 0, r0;
                if (a.variant == V_COL) {
                    o = tile / a.tiles_per_o;
                    r0 = (tile % a.tiles_per_o) * BM;
                } else {
                    r0 = tile * BM;
                }
                for (int ks = 0; ks < a.nks && ok; ++ks) {
                    if (!(ok = mbar_wait(bars.stg_empty + 8 * st.idx, st.phase ^ 1u))) break;
                    uint32_t sb = bars.stg_full + 8 * st.idx;
                    mbar_arrive_tx(sb, a.a_stage_bytes);
                    uint32_t dst = base + a.off_stg + st.idx * a.a_stage_bytes;
                    if (a.variant == V_COL)
                        tma_load_3d(dst, &tmap, (int)r0, ks * BK, (int)o, sb);
                    else
                        tma_load_2d(dst, &tmap, ks * BK, (int)r0, sb);
                    stg_armed |= 1u << st.idx;
                    stg_par = (stg_par & ~(1u << st.idx)) | (st.phase << st.idx);
                    st.next(a.ns_stg);
                }
            }
            if (!ok || a.b_resident) {
                // the resident B must have landed before the CTA can exit
                if (a.b_resident) {
                    long long t0 = clock64();
                    while (!mbar_try(bars.b_full, 0u) && clock64() - t0 < kTimeoutCycles) {}
                }
            }
            if (!ok) {
                // drain: every copy issued must land before the CTA exits
                for (int s = 0; s < a.ns_stg; ++s)
                    if (stg_armed & (1u << s)) {
                        long long t0 = clock64();
                        while (!mbar_try(bars.stg_full + 8 * s, (stg_par >> s) & 1u) &&
                               clock64() - t0 < kTimeoutCycles) {}
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            Pipe op, acc;
            bool ok = true;
            const int nchunks = (a.Jp + 255) / 256;
            // One thread issues every MMA, so its instruction stream is the
            // issue rate: the descriptors are built once per operand stage
            // and each MMA only adds its k sub-step (and 256-column chunk) to
            // their start-address fields (16-byte units; shared addresses stay
            // below 2^18 bytes, so the 14-bit field never carries).  Building
            // both descriptors per MMA from the stage addresses held
            // split-BF16x3 at J = 64 (three MMAs of N = 64 per k sub-step) to
            // about 210 cycles per MMA with the tensor pipe 18 % busy.
            const uint32_t idesc_full = umma_idesc(kTF32 ? 2u : 1u, BM, 256u);
            const uint32_t idesc_last =
                umma_idesc(kTF32 ? 2u : 1u, BM, (uint32_t)(a.Jp - 256 * (nchunks - 1)));
            const uint64_t dhi = umma_desc(0u, kRow, kSbo);   // every field but the address
            constexpr uint64_t kSubStep = kSubBytes >> 4;
            constexpr uint64_t kChunkStep = ((256u / 8u) * kSbo) >> 4;
            auto dsc = [&](uint32_t addr) -> uint64_t { return dhi | (uint64_t)((addr >> 4) & 0x3FFFu); };
            if (a.b_resident) ok = mbar_wait(bars.b_full, 0u);
            if (ok) tc_fence_after();
            for (int64_t tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
                if (!(ok = mbar_wait(bars.acc_empty + 8 * acc.idx, acc.phase ^ 1u))) break;
                tc_fence_after();
                const uint32_t dcol = tmem_base + acc.idx * acc_cols;
                for (int ks = 0; ks < a.nks && ok; ++ks) {
                    if (!(ok = mbar_wait(bars.op_full + 8 * op.idx, op.phase))) break;
                    tc_fence_after();
                    const int bs = a.b_resident ? ks : op.idx;
                    const uint64_t da0 = dsc(op_a(op.idx, 0)), da1 = dsc(op_a(op.idx, kParts - 1));
                    const uint64_t db0 = dsc(op_b(bs, 0)), db1 = dsc(op_b(bs, kParts - 1));
#pragma unroll
                    for (int sub = 0; sub < kSubs; ++sub) {
                        for (int c = 0; c < nchunks; ++c) {
                            const uint32_t idesc = c == nchunks - 1 ? idesc_last : idesc_full;
                            const uint64_t sa = sub * kSubStep;
                            const uint64_t sb = sub * kSubStep + (uint64_t)c * kChunkStep;
                            const uint32_t d = dcol + 256u * c;
                            const uint32_t accum = (ks > 0 || sub > 0) ? 1u : 0u;
                            umma<kTF32>(d, da0 + sa, db0 + sb, idesc, accum);
                            if constexpr (kParts == 2) {
                                umma<kTF32>(d, da0 + sa, db1 + sb, idesc, 1u);
                                umma<kTF32>(d, da1 + sa, db0 + sb, idesc, 1u);
                            }
                        }
                    }
                    umma_commit(bars.op_empty + 8 * op.idx);
                    op.next(a.ns_op);
                }
                if (!ok) break;
                umma_commit(bars.acc_full + 8 * acc.idx);
                acc.next(a.nacc);
            }
        }
    } else if (warp < kEpiWarp0) {
        // ------------------------------------------------------ converters
        const int tc = threadIdx.x - 64;
        const int t = tc & (BM - 1);             // operand row 0..127
        const int kh = tc >> 7;                  // which half of the 32 k values
        constexpr int KH = BK / 2;
        Pipe st, op;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
            for (int ks = 0; ks < a.nks && ok; ++ks) {
                if (!(ok = mbar_wait(bars.stg_full + 8 * st.idx, st.phase))) break;
                if (!(ok = mbar_wait(bars.op_empty + 8 * op.idx, op.phase ^ 1u))) break;
                const float* stg = reinterpret_cast<const float*>(
                    sbase + a.off_stg + st.idx * a.a_stage_bytes);
                float x[KH];
                if (a.variant == V_COL) {
                    // staging is [BK k][128 i]: column t, k in this half
#pragma unroll
                    for (int k = 0; k < KH; ++k) x[k] = stg[(kh * KH + k) * BM + t];
                } else {
                    // staging is [128 m][BK k] with 128-byte swizzle
                    const float4* row = reinterpret_cast<const float4*>(stg + t * BK);
#pragma unroll
                    for (int c = 0; c < KH / 4; ++c) {
                        float4 v = row[(kh * (KH / 4) + c) ^ (t & 7)];
                        x[4 * c] = v.x;
                        x[4 * c + 1] = v.y;
                        x[4 * c + 2] = v.z;
                        x[4 * c + 3] = v.w;
                    }
                }
                uint8_t* pa0 = sbase + (op_a(op.idx, 0) - base);
                if constexpr (kTF32) {
#pragma unroll
                    for (int c = 0; c < KH / 4; ++c) {
                        uint4 v = make_uint4(to_tf32(x[4 * c]), to_tf32(x[4 * c + 1]),
                                             to_tf32(x[4 * c + 2]), to_tf32(x[4 * c + 3]));
                        *reinterpret_cast<uint4*>(pa0 + sw_off(t, kh * (KH / 4) + c, kRow)) = v;
                    }
                } else {
                    uint8_t* pa1 = sbase + (op_a(op.idx, kParts - 1) - base);
#pragma unroll
                    for (int c = 0; c < KH / 8; ++c) {
                        float h[8], l[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            h[e] = __bfloat162float(__float2bfloat16_rn(x[8 * c + e]));
                            l[e] = x[8 * c + e] - h[e];
                        }
                        const int oc = kh * (KH / 8) + c;
                        uint4 vh = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]),
                                              pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
                        *reinterpret_cast<uint4*>(pa0 + sw_off(t, oc, kRow)) = vh;
                        if constexpr (kParts == 2) {
                            uint4 vl = make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]),
                                                  pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
                            *reinterpret_cast<uint4*>(pa1 + sw_off(t, oc, kRow)) = vl;
                        }
                    }
                }
                fence_proxy_async();
                mbar_arrive(bars.stg_empty + 8 * st.idx);
                mbar_arrive(bars.op_full + 8 * op.idx);
                st.next(a.ns_stg);
                op.next(a.ns_op);
            }
        }
    } else if (warp == kBWarp) {
        // ------------------------------------------------------ B stream
        // a B too large to stay resident is copied into each operand stage as
        // soon as the tensor cores free it, ahead of the conversion of that
        // stage, so neither the A producer nor the converters wait on it
        if (lane == 0 && !a.b_resident) {
            Pipe op;
            bool ok = true;
            uint32_t op_armed = 0, op_par = 0;   // stages with a copy in flight (for the drain)
            for (int64_t tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
                for (int ks = 0; ks < a.nks && ok; ++ks) {
                    if (!(ok = mbar_wait(bars.op_empty + 8 * op.idx, op.phase ^ 1u))) break;
                    const uint32_t ob = bars.op_full + 8 * op.idx;
                    mbar_arrive_tx(ob, kParts * a.opb_part_bytes);
                    for (int part = 0; part < kParts; ++part)
                        bulk_load(op_b(op.idx, part),
                                  a.bimg + ((size_t)ks * kParts + part) * a.opb_part_bytes,
                                  a.opb_part_bytes, ob);
                    op_armed |= 1u << op.idx;
                    op_par = (op_par & ~(1u << op.idx)) | (op.phase << op.idx);
                    op.next(a.ns_op);
                }
            }
            if (!ok) {
                // drain: every copy issued must land before the CTA exits
                for (int s2 = 0; s2 < a.ns_op; ++s2)
                    if (op_armed & (1u << s2)) {
                        long long t0 = clock64();
                        while (!mbar_try(bars.op_full + 8 * s2, (op_par >> s2) & 1u) &&
                               clock64() - t0 < kTimeoutCycles) {}
                    }
            }
        }
    } else {
        // ------------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int chalf = (warp - kEpiWarp0) >> 2;   // this warp's 32-column chunks
        // per-warp 32 x 33 staging tile: rows are TMEM lanes, columns j
        float* tile = reinterpret_cast<float*>(sbase + a.off_epi) + (warp - kEpiWarp0) * 32 * 33;
        // TMA-store path: per-warp 32 x 32 box image (4 KB, 1024-byte aligned)
        float* const box = reinterpret_cast<float*>(sbase + a.off_epi) + (warp - kEpiWarp0) * 32 * 32;
        const uint32_t box_addr = base + a.off_epi + (uint32_t)(warp - kEpiWarp0) * 4096u;
        // j contiguous in C (and not i): transpose so that lanes run along j
        const bool j_fast = (a.scq == 1);
        Pipe acc;
        bool ok = true;
        for (int64_t tile_id = blockIdx.x; tile_id < a.ntiles && ok; tile_id += gridDim.x) {
            if (!(ok = mbar_wait(bars.acc_full + 8 * acc.idx, acc.phase))) break;
            tc_fence_after();
            int64_t rbase, obase = 0, nrows, o = 0;
            if (a.variant == V_COL) {
                o = tile_id / a.tiles_per_o;
                rbase = (tile_id % a.tiles_per_o) * BM + quarter * 32;
                obase = o * a.sc_o;
            } else {
                rbase = tile_id * BM + quarter * 32;
            }
            nrows = a.M - rbase;               // rows of this warp that exist (may be <= 0)
            const uint32_t tcol = tmem_base + ((uint32_t)(quarter * 32) << 16) + acc.idx * acc_cols;
            for (int c0 = 32 * chalf; c0 < a.Jp; c0 += 64) {
                float v[32];
                tmem_ld32(tcol + c0, v);
                if (a.tma_out) {
                    // the box goes to C by one TMA store, which clips the rows
                    // past M and the columns past J
                    if (nrows > 0 && c0 < a.J) {
                        if (lane == 0) bulk_wait_read();   // the previous store has read the box
                        __syncwarp();
                        if (a.variant == V_COL) {
                            // [column][row]: rows contiguous in C
#pragma unroll
                            for (int j = 0; j < 32; ++j) box[j * 32 + lane] = v[j];
                        } else {
                            // [row][column], 16-byte chunks placed the way the
                            // map's 128-byte swizzle reads them (conflict-free)
                            float4* b4 = reinterpret_cast<float4*>(box);
#pragma unroll
                            for (int c = 0; c < 8; ++c)
                                b4[lane * 8 + (c ^ (lane & 7))] =
                                    make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                        }
                        fence_proxy_async();
                        __syncwarp();
                        if (lane == 0) {
                            if (a.variant == V_COL) tma_store_3d(&cmap, (int)rbase, c0, (int)o, box_addr);
                            else tma_store_2d(&cmap, c0, (int)rbase, box_addr);
                            bulk_commit();
                        }
                    }
                } else if (j_fast && a.vec_out) {
                    // 32 x 32 tile with 16-byte chunks XOR-swizzled by row: both the
                    // row-wise writes and the chunk-wise reads are conflict-free
                    float4* t4 = reinterpret_cast<float4*>(tile);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        t4[lane * 8 + (c ^ (lane & 7))] =
                            make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                    __syncwarp();
                    const int cc = lane & 7;
                    const int jg = c0 + 4 * cc;
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int r = it * 4 + (lane >> 3);
                        float4 x = t4[r * 8 + (cc ^ (r & 7))];
                        if (r < nrows && jg < a.J) {
                            float4* p = reinterpret_cast<float4*>(a.C + obase + (rbase + r) * a.sc_m + jg);
                            if (a.accumulate) {
                                float4 o = *p;
                                x.x += o.x; x.y += o.y; x.z += o.z; x.w += o.w;
                            }
                            *p = x;
                        }
                    }
                    __syncwarp();
                } else if (j_fast) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = v[j];
                    __syncwarp();
                    const int jg = c0 + lane;
                    if (jg < a.J) {
                        for (int r = 0; r < 32 && r < nrows; ++r) {
                            float* p = a.C + obase + (rbase + r) * a.sc_m + jg;
                            float x = tile[r * 33 + lane];
                            *p = a.accumulate ? *p + x : x;
                        }
                    }
                    __syncwarp();
                } else if (a.vec_rows) {
                    // rows contiguous in C: the warp's 32 rows x 32 columns go
                    // through its shared-memory tile as [column][row] (32
                    // conflict-free 4-byte stores per lane); each quarter-warp
                    // then reads one column's 32 rows (8 x 16 bytes, conflict
                    // free) and writes them as 128 contiguous bytes of C
#pragma unroll
                    for (int j = 0; j < 32; ++j) tile[j * 32 + lane] = v[j];
                    __syncwarp();
                    const int g = lane & 7, jj = lane >> 3;     // rows 4g..4g+3 of column 4*it+jj
                    const int64_t nr = a.M - (rbase + 4 * g);   // rows of this vector that exist
                    float* const pbase = a.C + obase + rbase + 4 * g;
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int col = 4 * it + jj;
                        const int jg = c0 + col;
                        float4 x = *reinterpret_cast<const float4*>(tile + col * 32 + 4 * g);
                        if (jg < a.J && nr > 0) {
                            float* p = pbase + (int64_t)jg * a.scq;
                            if (nr >= 4) {
                                float4* p4 = reinterpret_cast<float4*>(p);
                                if (a.accumulate) {
                                    const float4 o = *p4;
                                    x.x += o.x; x.y += o.y; x.z += o.z; x.w += o.w;
                                }
                                *p4 = x;
                            } else {
                                const float e[4] = {x.x, x.y, x.z, x.w};
                                for (int q = 0; q < nr; ++q) p[q] = a.accumulate ? p[q] + e[q] : e[q];
                            }
                        }
                    }
                    __syncwarp();
                } else if (lane < nrows) {
                    float* pc = a.C + obase + (rbase + lane) * a.sc_m;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        int jg = c0 + j;
                        if (jg < a.J) {
                            float* p = pc + (int64_t)jg * a.scq;
                            *p = a.accumulate ? *p + v[j] : v[j];
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(bars.acc_empty + 8 * acc.idx);
            acc.next(a.nacc);
        }
        if (a.tma_out && lane == 0) bulk_wait_all();
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(kTmemCols));
    }
}

// B(j, k) -> canonical K-major tiles [ks][part][Jp rows x BK], 16 bytes per thread.
template <int PREC>
__global__ void ttm_tc_prep_b(const float* __restrict__ B, int64_t ldb_row, int64_t ldb_col, int J,
                              int Jp, int64_t nq, int nks, uint8_t* __restrict__ img,
                              uint32_t part_bytes)
{
    constexpr bool kTF32 = (PREC == TL_P_TF32);
    constexpr int kParts = (PREC == TL_P_BF16X3) ? 2 : 1;
    constexpr int kEl = kTF32 ? 4 : 8;                  // elements per 16-byte chunk
    constexpr int kChunks = BK / kEl;
    constexpr uint32_t kRow = kChunks * 16;
    const int64_t total = (int64_t)nks * Jp * kChunks;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % kChunks);
        const int j = (int)((t / kChunks) % Jp);
        const int ks = (int)(t / ((int64_t)kChunks * Jp));
        float x[kEl];
#pragma unroll
        for (int e = 0; e < kEl; ++e) {
            int64_t k = (int64_t)ks * BK + c * kEl + e;
            x[e] = (j < J && k < nq) ? B[j * ldb_row + k * ldb_col] : 0.f;
        }
        const uint32_t off = sw_off((uint32_t)j, (uint32_t)c, kRow);
        uint8_t* p0 = img + ((size_t)ks * kParts) * part_bytes + off;
        if constexpr (kTF32) {
            *reinterpret_cast<uint4*>(p0) =
                make_uint4(to_tf32(x[0]), to_tf32(x[1]), to_tf32(x[2]), to_tf32(x[3]));
        } else {
            float h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                h[e] = __bfloat162float(__float2bfloat16_rn(x[e]));
                l[e] = x[e] - h[e];
            }
            *reinterpret_cast<uint4*>(p0) = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]),
                                                       pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
            if constexpr (kParts == 2) {
                uint8_t* p1 = p0 + part_bytes;
                *reinterpret_cast<uint4*>(p1) =
                    make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]),
                               pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
            }
        }
    }
}

// --------------------------------------------------------------- host side --

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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

struct Layout {
    int nparts, esize, Jp, nks, ns_stg, ns_op, nacc, b_resident;
    uint32_t a_stage, opa_part, opb_part, op_stage, off_stg, off_op, off_epi, off_bar, smem;
    uint32_t off_b, b_bytes;
};

Layout layout_for(const TtmPlan& P)
{
    Layout L{};
    L.nparts = P.precision == TL_P_BF16X3 ? 2 : 1;
    L.esize = P.precision == TL_P_TF32 ? 4 : 2;
    L.Jp = (int)((P.J + 15) / 16 * 16);
    L.nks = (int)((P.nq + BK - 1) / BK);
    L.nacc = L.Jp <= 256 ? 2 : 1;
    L.a_stage = BM * BK * 4;
    L.opa_part = BM * BK * L.esize;
    L.opb_part = (uint32_t)L.Jp * BK * L.esize;
    // a converted B of at most 64 KB stays in shared memory for the whole
    // launch (loaded once per CTA) instead of streaming with every k stage
    L.b_bytes = (uint32_t)L.nks * L.nparts * L.opb_part;
    L.b_resident = L.b_bytes <= 64u * 1024u ? 1 : 0;
    L.op_stage = L.nparts * (L.opa_part + (L.b_resident ? 0 : L.opb_part));
    const uint32_t epi = kEpiWarps * 32 * 33 * 4;        // epilogue transpose tiles
    const uint32_t budget = 227 * 1024 - 1024 - 512 - epi -
                            (L.b_resident ? L.b_bytes : 0);   // alignment slack + barriers
    // FP32 staging keeps the HBM bytes in flight; the operand ring only has
    // to cover the convert -> MMA hand-off
    for (L.ns_op = 3; L.ns_op >= 2; --L.ns_op) {
        int64_t room = (int64_t)budget - (int64_t)L.ns_op * L.op_stage;
        L.ns_stg = room > 0 ? (int)(room / L.a_stage) : 0;
        if (L.ns_stg > 8) L.ns_stg = 8;
        if (L.ns_stg >= 2) break;
    }
    // Depth of the A ring. Where C is about as large as A (J >= n_q), more
    // than about 64 KB of A in flight per SM lowers the DRAM throughput (the
    // reads crowd out the write-back of C: on 128^4, 96^4 and 64^5 FP32
    // tensors 4 stages run at 6.2-6.9 TB/s, 5-8 stages at 5.3-6.4); the less
    // of C there is per byte of A, the deeper the ring pays (J = n_q / 4 and
    // n_q / 8 run fastest with 6-8 stages). COL tiles past a short inner
    // extent load only the rows that exist, so their stages hold fewer bytes.
    {
        int want = 4;
        if (P.J < P.nq) want += (int)(4 * (P.nq - P.J) / P.nq);
        const int64_t rows = P.tc_variant == V_COL && P.rows.d[0].n < BM ? P.rows.d[0].n : BM;
        want = (int)((want * BM + rows - 1) / rows);
        if (L.ns_stg > want) L.ns_stg = want < 2 ? 2 : want;
    }
    L.off_stg = 0;
    L.off_op = L.ns_stg * L.a_stage;
    L.off_b = L.off_op + L.ns_op * L.op_stage;
    L.off_epi = L.off_b + (L.b_resident ? L.b_bytes : 0);
    L.off_bar = L.off_epi + epi;
    L.smem = L.off_bar + 8 * (2 * L.ns_stg + 2 * L.ns_op + 5) + 16 + 1024;
    // more than half of the SM's shared memory keeps one CTA per SM, so no
    // two CTAs ever wait on each other for the 512 TMEM columns
    if (L.smem < 116 * 1024) L.smem = 116 * 1024;
    return L;
}

// The tensor map C is written through when the epilogue stores by TMA: 16-byte
// aligned base and strides, coordinates in 32 bits, no accumulation (a TMA
// store overwrites).  ROW: 2-D {J, M}, 32 x 32 boxes with 128-byte swizzle;
// COL: 3-D {inner, J, outer}, 32 x 32 x 1 boxes.
struct StoreMap {
    bool ok = false;
    int rank = 0;
    cuuint64_t gdim[3] = {0, 0, 0}, gstr[2] = {0, 0};
    cuuint32_t box[3] = {32, 32, 1};
};

StoreMap store_map(const TtmPlan& P, const Layout& L, const void* C, int accumulate)
{
    StoreMap m;
    if (accumulate || (reinterpret_cast<uintptr_t>(C) % 16) != 0 || (L.off_epi % 1024) != 0 ||
        P.J >= (1LL << 31))
        return m;
    if (P.tc_variant == V_ROW && P.scq == 1) {
        const int64_t M = P.M, sc_m = P.rows.nd ? P.rows.d[0].s[1] : 0;
        const int64_t ld = M > 1 ? sc_m : (P.J + 3) / 4 * 4;
        if (M < (1LL << 31) && ld % 4 == 0 && ld > 0 && ld * 4 < (1LL << 40)) {
            m.rank = 2;
            m.gdim[0] = (cuuint64_t)P.J;
            m.gdim[1] = (cuuint64_t)M;
            m.gstr[0] = (cuuint64_t)ld * 4;
            m.ok = true;
        }
    } else if (P.tc_variant == V_COL && P.rows.d[0].s[1] == 1) {
        const int64_t inner = P.rows.d[0].n;
        const int64_t outer = P.rows.nd == 2 ? P.rows.d[1].n : 1;
        const int64_t so = outer > 1 ? P.rows.d[1].s[1] : P.scq * P.J;
        if (inner < (1LL << 31) && outer < (1LL << 31) && P.scq % 4 == 0 && P.scq > 0 &&
            so % 4 == 0 && so > 0 && P.scq * 4 < (1LL << 40) && so * 4 < (1LL << 40)) {
            m.rank = 3;
            m.gdim[0] = (cuuint64_t)inner;
            m.gdim[1] = (cuuint64_t)P.J;
            m.gdim[2] = (cuuint64_t)outer;
            m.gstr[0] = (cuuint64_t)P.scq * 4;
            m.gstr[1] = (cuuint64_t)so * 4;
            m.ok = true;
        }
    }
    return m;
}

template <int PREC>
int launch_prec(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate, int sms,
                cudaStream_t st)
{
    const Layout L = layout_for(P);
    if (L.smem > 227 * 1024 || L.ns_stg < 2 || L.ns_op < 2) return TL_EUNSUPPORTED;
    auto enc = encode_fn();
    if (!enc) return TL_ECUDA;

    TcArgs a{};
    a.C = static_cast<float*>(C);
    a.variant = P.tc_variant;
    a.prec = PREC;
    a.nparts = L.nparts;
    a.esize = L.esize;
    a.J = (int)P.J;
    a.Jp = L.Jp;
    a.nks = L.nks;
    a.ns_stg = L.ns_stg;
    a.ns_op = L.ns_op;
    a.nacc = L.nacc;
    a.accumulate = accumulate;
    a.scq = P.scq;
    a.a_stage_bytes = L.a_stage;
    {
        const int64_t scm = P.tc_variant == V_ROW ? (P.rows.nd ? P.rows.d[0].s[1] : 0)
                                                  : P.rows.d[0].s[1];
        a.vec_out = (P.scq == 1 && P.J % 4 == 0 && scm % 4 == 0 &&
                     (P.tc_variant != V_COL || P.rows.nd < 2 || P.rows.d[1].s[1] % 4 == 0) &&
                     (reinterpret_cast<uintptr_t>(C) % 16) == 0) ? 1 : 0;
        a.vec_rows = (P.tc_variant == V_COL && scm == 1 && P.scq % 4 == 0 &&
                      (P.rows.nd < 2 || P.rows.d[1].s[1] % 4 == 0) &&
                      (reinterpret_cast<uintptr_t>(C) % 16) == 0) ? 1 : 0;
    }
    a.opa_part_bytes = L.opa_part;
    a.opb_part_bytes = L.opb_part;
    a.off_stg = L.off_stg;
    a.off_op = L.off_op;
    a.op_stage_bytes = L.op_stage;
    a.off_bar = L.off_bar;
    a.off_epi = L.off_epi;
    a.b_resident = L.b_resident;
    a.off_b = L.off_b;
    a.b_bytes = L.b_bytes;

    CUtensorMap map;
    CUresult cr;
    const cuuint32_t estr[3] = {1, 1, 1};
    if (P.tc_variant == V_ROW) {
        const int64_t lda = P.rows.nd ? P.rows.d[0].s[0] : P.nq;
        a.M = P.M;
        a.ntiles = (P.M + BM - 1) / BM;
        a.sc_m = P.rows.nd ? P.rows.d[0].s[1] : 0;
        const cuuint64_t gdim[2] = {(cuuint64_t)P.nq, (cuuint64_t)P.M};
        const cuuint64_t gstr[1] = {(cuuint64_t)lda * 4};
        const cuuint32_t box[2] = {BK, BM};
        cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(A), gdim, gstr, box,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const int64_t inner = P.rows.d[0].n;
        const int64_t outer = P.rows.nd == 2 ? P.rows.d[1].n : 1;
        const int64_t sa_o = P.rows.nd == 2 ? P.rows.d[1].s[0] : inner * P.nq;
        a.M = inner;
        a.tiles_per_o = (inner + BM - 1) / BM;
        a.ntiles = a.tiles_per_o * outer;
        a.sc_m = P.rows.d[0].s[1];
        a.sc_o = P.rows.nd == 2 ? P.rows.d[1].s[1] : 0;
        const cuuint64_t gdim[3] = {(cuuint64_t)inner, (cuuint64_t)P.nq, (cuuint64_t)outer};
        const cuuint64_t gstr[2] = {(cuuint64_t)P.saq * 4, (cuuint64_t)sa_o * 4};
        const cuuint32_t box[3] = {BM, BK, 1};
        cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(A), gdim, gstr, box,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (cr != CUDA_SUCCESS) return TL_EUNSUPPORTED;

    // C by TMA stores where its layout allows a tensor map; otherwise the
    // warps store
    CUtensorMap cmap{};
    a.tma_out = 0;
    const StoreMap sm = store_map(P, L, C, accumulate);
    if (sm.ok)
        a.tma_out = enc(&cmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sm.rank, C, sm.gdim, sm.gstr, sm.box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        sm.rank == 2 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;

    // converted B in the per-stream workspace
    const size_t img_bytes = (size_t)L.nks * L.nparts * L.opb_part;
    uint8_t* img = static_cast<uint8_t*>(workspace(st, img_bytes));
    if (!img) return TL_ENOMEM;
    a.bimg = img;
    {
        constexpr int kEl = PREC == TL_P_TF32 ? 4 : 8;
        int64_t total = (int64_t)L.nks * L.Jp * (BK / kEl);
        int grid = (int)((total + 255) / 256);
        if (grid > sms * 8) grid = sms * 8;
        ttm_tc_prep_b<PREC><<<grid, 256, 0, st>>>(static_cast<const float*>(B), P.ldb_row,
                                                  P.ldb_col, (int)P.J, L.Jp, P.nq, L.nks, img,
                                                  L.opb_part);
    }
    if (smem_optin(reinterpret_cast<const void*>(ttm_tc_kernel<PREC>), (int)L.smem) != TL_OK)
        return TL_ECUDA;
    int grid = (int)(a.ntiles < sms ? a.ntiles : sms);
    ttm_tc_kernel<PREC><<<grid, kThreads, L.smem, st>>>(map, cmap, a);
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

}  // namespace

int ttm_tc_launches(const TtmPlan&) { return 2; }

std::string ttm_tc_describe(const TtmPlan& P, const void* C)
{
    const Layout L = layout_for(P);
    const StoreMap sm = store_map(P, L, C, 0);
    char b[256];
    std::snprintf(b, sizeof b,
                  "{\"a_stages\":%d,\"op_stages\":%d,\"b_resident\":%d,\"smem\":%u,"
                  "\"threads\":%d,\"store\":\"%s\"}",
                  L.ns_stg, L.ns_op, L.b_resident, L.smem, kThreads, sm.ok ? "tma" : "warps");
    return b;
}

int launch_ttm_tc(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                  int num_sms, cudaStream_t st)
{
    switch (P.precision) {
    case TL_P_TF32: return launch_prec<TL_P_TF32>(P, A, B, C, accumulate, num_sms, st);
    case TL_P_BF16: return launch_prec<TL_P_BF16>(P, A, B, C, accumulate, num_sms, st);
    case TL_P_BF16X3: return launch_prec<TL_P_BF16X3>(P, A, B, C, accumulate, num_sms, st);
    default: return TL_EUNSUPPORTED;
    }
}

int selftest_wait_timeout(double limit_us, cudaStream_t st)
{
    if (!(limit_us > 0) || limit_us > 1e6) return TL_EINVAL;
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) khz = 2000000;
    const long long cycles = (long long)(limit_us * 1e-3 * khz);
    selftest_wait_kernel<<<1, 32, 0, st>>>(cycles);
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

int ttm_tc_status(bool clear)
{
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return TL_ECUDA;
    }
    if (clear && v) {
        unsigned int z = 0;
        cudaMemcpyToSymbol(g_tc_status, &z, sizeof z);
    }
    return v ? TL_ETIMEOUT : TL_OK;
}

}  // namespace tl
