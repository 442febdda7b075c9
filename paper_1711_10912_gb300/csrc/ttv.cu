// ttv.cu -- mode-q tensor-times-vector, Sec. 5.2 Eq. 24:
//   C(i without q) = sum_{k < n_q} A(i with i_q = k) * b(k).
//
// After collapsing (plan.cpp) the output modes form a space whose dim 0 is
// the output mode with the smallest stride in A.  Two kernels cover every
// layout:
//   ttv_row  the contracted mode is contiguous in A (w_q = 1, the paper's
//            "m = 0" special case of Sec. 5.2): a group of L lanes reads one
//            output's fiber with 16-byte loads and reduces it by warp
//            shuffles; each group keeps R fibers in flight.
//   ttv_col  the contracted mode is strided: threads run along the output
//            dims (coalesced when dim 0 is contiguous in A), each thread walks
//            k with stride w_q and keeps VEC sums in registers.
// When the outputs alone cannot fill the GPU, the k range is split across
// CTAs; each split writes FP partial sums to the workspace and a second
// kernel adds them in split order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "kernels.h"
#include "pipeline.cuh"
#include "runtime.h"

namespace tl {

// Set when a bounded wait of a pipelined ttv kernel gives up.
__device__ unsigned int g_ttv_status;

namespace {

struct TtvArgs {
    const void* A;
    const void* b;
    void* C;
    void* ws;
    DevSpace out;       // operands 0 = A, 1 = C
    int64_t nq, saq, incb, nout, kchunk;
    int splits, accumulate;
};

constexpr int kThreads = 256;

// Sums R (4 or 8) per-lane partials over groups of L lanes with a halving
// butterfly: at each of the first log2(R) levels a lane keeps the half of the
// rows its partner does not, so R = 8 over 32 lanes takes 9 shuffles instead
// of 40.  Afterwards the lane with sub-lane index s holds the total of row
// sum_l ((s & (L >> (l+1))) != 0) << (log2(R) - 1 - l).
template <typename T, int L, int R>
__device__ __forceinline__ T reduce_rows(T* v, int sub)
{
    int cnt = R;
#pragma unroll
    for (int lvl = 0; (R >> lvl) > 1; ++lvl) {
        const int h = L >> (lvl + 1);
        const bool up = (sub & h) != 0;
        const int half = cnt / 2;
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            if (i < half) {
                T send = up ? v[i] : v[i + half];
                T keep = up ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
        }
        cnt = half;
    }
    T r = v[0];
    constexpr int kLevels = (R == 8) ? 3 : 2;
#pragma unroll
    for (int m = (L >> kLevels) / 2; m >= 1; m /= 2) r += __shfl_xor_sync(0xffffffffu, r, m);
    return r;
}

template <typename T, int VEC, int L, int R, bool SPLIT>
__global__ void __launch_bounds__(kThreads) ttv_row_kernel(const TtvArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ b = static_cast<const T*>(a.b);
    const int lane = threadIdx.x & 31;
    const int sub = lane & (L - 1);
    const int64_t group = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / L;
    const int64_t ngroups = (int64_t)gridDim.x * kThreads / L;
    const int64_t step = (int64_t)R * ngroups;
    // Work items are (split, output) pairs, split-major, spread over every
    // group, so the splits of a long contraction run in parallel; each of a
    // group's R items in flight has its own k range (SPLIT; without it they
    // share one and one load of b, at fewer registers).  Every lane of a warp
    // runs the same iterations, so the shuffles always see a converged warp.
    const int64_t total = a.nout * (SPLIT ? a.splits : 1);
    const int64_t iters = (total + step - 1) / step;
    constexpr bool split = SPLIT;
    for (int64_t it = 0; it < iters; ++it) {
        int64_t row[R], offA[R], k0[R], klen[R], sp[R];
        bool ok[R];
        T acc[R];
        int64_t kmax = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t w = (it * R + r) * ngroups + group;
            ok[r] = w < total;
            sp[r] = split ? w / a.nout : 0;
            row[r] = w - sp[r] * a.nout;
            k0[r] = sp[r] * a.kchunk;
            klen[r] = ok[r] ? min(a.nq - k0[r], a.kchunk) : 0;
            kmax = max(kmax, klen[r]);
            acc[r] = T(0);
            int64_t off[1] = {0};
            if (ok[r]) map_offsets<1>(a.out, row[r], 1, off);
            offA[r] = off[0] + k0[r];
        }
        for (int64_t kk = (int64_t)sub * VEC; kk < kmax; kk += (int64_t)L * VEC) {
            T vb[SPLIT ? R : 1][VEC];
            if constexpr (!SPLIT) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) vb[0][v] = __ldg(b + (kk + v) * a.incb);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int v = 0; v < VEC; ++v)
                        vb[r][v] = kk < klen[r] ? __ldg(b + (k0[r] + kk + v) * a.incb) : T(0);
            }
            T va[R][VEC];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (kk < klen[r]) {
                    vload_stream<T, VEC>(A + offA[r] + kk, va[r]);
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) va[r][v] = T(0);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[r] = fma(va[r][v], vb[SPLIT ? r : 0][v], acc[r]);
        }
        const T tot = reduce_rows<T, L, R>(acc, sub);
        constexpr int kG = L / R;                 // lanes per row after the butterfly
        if ((sub & (kG - 1)) == 0) {
            const int rs = sub / kG;
            int64_t rw = 0, sw = 0;
            bool okw = false;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r == rs) { rw = row[r]; sw = sp[r]; okw = ok[r]; }
            if (okw) {
                if constexpr (SPLIT) {
                    static_cast<T*>(a.ws)[sw * a.nout + rw] = tot;
                } else {
                    int64_t off[2];
                    map_offsets<2>(a.out, rw, 1, off);
                    T* c = static_cast<T*>(a.C) + off[1];
                    *c = a.accumulate ? *c + tot : tot;
                }
            }
        }
    }
}

// Row case with dense rows (w_q = 1 and consecutive outputs n_q apart): the
// rows are one contiguous stream, so a producer thread moves blocks of rows
// with 1-D bulk copies into a 3-stage shared-memory ring (16 KB stages) and
// eight consumer warps reduce them from shared memory (b is staged once per
// CTA).  Three CTAs per SM: measured on GB300, the consumers of a single CTA
// per SM cannot keep up (3.1 TB/s) while three CTAs stream at 6.7 TB/s.
struct RowStageArgs {
    const void* A;
    const void* b;
    void* C;
    int64_t rows, nq, sc;
    int rows_per_stage, nstages;
    uint32_t stage_bytes, off_b, off_bar;
    int accumulate;
};

constexpr int kStageConsumers = 8;                      // consumer warps
constexpr int kStageThreads = 32 * (kStageConsumers + 1);

template <typename T>
__global__ void __launch_bounds__(kStageThreads, 3) ttv_row_staged_kernel(const RowStageArgs a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int VEC = 16 / sizeof(T);
    using VT = typename Vec<T, VEC>::type;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = pipe::smem_u32(smem);
    const uint32_t full = base + a.off_bar, empty = full + 8 * a.nstages;
    const T* sb = reinterpret_cast<const T*>(smem + a.off_b);
    const int64_t nchunks = (a.rows + a.rows_per_stage - 1) / a.rows_per_stage;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.nstages; ++s) {
            pipe::mbar_init(full + 8 * s, 1);
            pipe::mbar_init(empty + 8 * s, kStageConsumers);
        }
        pipe::mbar_init_fence();
        pipe::fence_proxy_async();
    }
    for (int64_t k = threadIdx.x; k < a.nq; k += kStageThreads)
        const_cast<T*>(sb)[k] = static_cast<const T*>(a.b)[k];
    __syncthreads();

    if (warp == kStageConsumers) {
        if (lane == 0) {
            pipe::Ring r;
            bool ok = true;
            uint32_t armed = 0, par = 0;
            const size_t row_bytes = (size_t)a.nq * sizeof(T);
            for (int64_t c = blockIdx.x; c < nchunks && ok; c += gridDim.x) {
                if (!(ok = pipe::mbar_wait(empty + 8 * r.idx, r.phase ^ 1u, &g_ttv_status))) break;
                const int64_t r0 = c * a.rows_per_stage;
                const int64_t nr = min((int64_t)a.rows_per_stage, a.rows - r0);
                const uint32_t bytes = (uint32_t)(nr * row_bytes);
                pipe::mbar_arrive_tx(full + 8 * r.idx, bytes);
                pipe::bulk_load(base + r.idx * a.stage_bytes,
                                static_cast<const T*>(a.A) + r0 * a.nq, bytes, full + 8 * r.idx);
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
    // consumers: warp w takes rows w, w + 8, ... of each staged block, four at a time
    pipe::Ring r;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        if (!pipe::mbar_wait(full + 8 * r.idx, r.phase, &g_ttv_status)) break;
        const int64_t r0 = c * a.rows_per_stage;
        const int nr = (int)min((int64_t)a.rows_per_stage, a.rows - r0);
        const T* st = reinterpret_cast<const T*>(smem + r.idx * a.stage_bytes);
        for (int g0 = warp * 4; g0 < nr; g0 += kStageConsumers * 4) {
            T acc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i] = T(0);
                const int row = g0 + i;
                if (row < nr) {
                    for (int64_t kk = (int64_t)lane * VEC; kk < a.nq; kk += 32 * VEC) {
                        VT x = *reinterpret_cast<const VT*>(st + (int64_t)row * a.nq + kk);
                        VT y = *reinterpret_cast<const VT*>(sb + kk);
                        const T* xe = reinterpret_cast<const T*>(&x);
                        const T* ye = reinterpret_cast<const T*>(&y);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[i] = fma(xe[v], ye[v], acc[i]);
                    }
                }
            }
            const T tot = reduce_rows<T, 32, 4>(acc, lane);
            if ((lane & 7) == 0) {
                const int row = g0 + (lane >> 3);
                if (row < nr) {
                    T* pc = static_cast<T*>(a.C) + (r0 + row) * a.sc;
                    *pc = a.accumulate ? *pc + tot : tot;
                }
            }
        }
        __syncwarp();
        if (lane == 0) pipe::mbar_arrive(empty + 8 * r.idx);
        r.next(a.nstages);
    }
}

template <typename T, int VEC, int U>
__global__ void __launch_bounds__(kThreads) ttv_col_kernel(const TtvArgs a)
{
    const T* __restrict__ A = static_cast<const T*>(a.A);
    const T* __restrict__ b = static_cast<const T*>(a.b);
    const int64_t items = a.nout / VEC;
    const int64_t work = items * a.splits;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < work; t += stride) {
        const int64_t g = t % items;
        const int64_t s = t / items;
        int64_t off[2];
        map_offsets<2>(a.out, g, VEC, off);
        const int64_t k0 = s * a.kchunk;
        const int64_t k1 = min(a.nq, k0 + a.kchunk);
        T acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = T(0);
        const T* pa = A + off[0];
        int64_t k = k0;
        for (; k + U <= k1; k += U) {
            T va[U][VEC];
            T vb[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                vload_stream<T, VEC>(pa + (k + u) * a.saq, va[u]);
                vb[u] = __ldg(b + (k + u) * a.incb);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] = fma(va[u][v], vb[u], acc[v]);
        }
        for (; k < k1; ++k) {
            T va[VEC];
            vload_stream<T, VEC>(pa + k * a.saq, va);
            T bk = __ldg(b + k * a.incb);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = fma(va[v], bk, acc[v]);
        }
        if (a.splits > 1) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) static_cast<T*>(a.ws)[s * a.nout + g * VEC + v] = acc[v];
        } else {
            T* pc = static_cast<T*>(a.C) + off[1];
            if (a.accumulate) {
                T old[VEC];
                if (VEC > 1) vload<T, VEC>(pc, old);
                else old[0] = *pc;
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] += old[v];
            }
            vstore<T, VEC>(pc, acc);
        }
    }
}

// Adds the split partial sums ws[s][e] and writes C: in split order by one
// thread per output, or, with WARP (many splits), by a warp per output whose
// lanes each add every 32nd split in order and combine by a fixed butterfly
// (deterministic either way).
template <typename T, bool WARP>
__global__ void __launch_bounds__(kThreads) ttv_splitk_reduce(const TtvArgs a)
{
    const T* ws = static_cast<const T*>(a.ws);
    constexpr int kPer = WARP ? 32 : 1;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kThreads / kPer;
    for (int64_t e = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / kPer; e < a.nout; e += stride) {
        T sum = T(0);
        if constexpr (WARP) {
            for (int s = lane; s < a.splits; s += 32) sum += ws[(int64_t)s * a.nout + e];
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, m);
            if (lane != 0) continue;
        } else {
            for (int s = 0; s < a.splits; ++s) sum += ws[(int64_t)s * a.nout + e];
        }
        int64_t off[2];
        map_offsets<2>(a.out, e, 1, off);
        T* c = static_cast<T*>(a.C) + off[1];
        *c = a.accumulate ? *c + sum : sum;
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
int launch_typed(const TtvPlan& P, const void* A, const void* b, void* C, void* ws,
                 int accumulate, int num_sms, cudaStream_t st)
{
    TtvArgs a{};
    a.A = A;
    a.b = b;
    a.C = C;
    a.ws = ws;
    a.out = to_dev(P.out);
    a.nq = P.nq;
    a.saq = P.saq;
    a.incb = P.incb;
    a.nout = P.nout;
    a.kchunk = P.kchunk;
    a.splits = P.splits;
    a.accumulate = accumulate;
    constexpr int V = 16 / sizeof(T);
    if (P.kernel == K_TTV_ROW && P.splits == 1 && P.vec == V && P.nq % (32 * V) == 0 &&
        P.out.nd == 1 && P.out.d[0].s[0] == P.nq && P.nq * (int64_t)sizeof(T) <= 8192 &&
        P.incb == 1 && aligned(b, 16)) {
        RowStageArgs r{};
        r.A = A;
        r.b = b;
        r.C = C;
        r.rows = P.nout;
        r.nq = P.nq;
        r.sc = P.out.d[0].s[1];
        r.accumulate = accumulate;
        const int64_t row_bytes = P.nq * (int64_t)sizeof(T);
        // about 16 KB per stage, a multiple of 4 rows (row_bytes <= 8 KB)
        r.rows_per_stage = (int)std::max<int64_t>(4, std::min<int64_t>(256, (16 * 1024) / row_bytes) / 4 * 4);
        r.nstages = 3;
        r.stage_bytes = (uint32_t)(r.rows_per_stage * row_bytes);
        r.off_b = r.nstages * r.stage_bytes;
        r.off_bar = r.off_b + (uint32_t)((row_bytes + 127) / 128 * 128);
        const uint32_t smem = r.off_bar + 16 * r.nstages;
        if (smem_optin(reinterpret_cast<const void*>(ttv_row_staged_kernel<T>), (int)smem) != TL_OK)
            return TL_ECUDA;
        const int64_t nchunks = (P.nout + r.rows_per_stage - 1) / r.rows_per_stage;
        const int grid = (int)std::min<int64_t>(nchunks, (int64_t)num_sms * 3);
        ttv_row_staged_kernel<T><<<grid, kStageThreads, smem, st>>>(r);
        return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
    }
    if (P.kernel == K_TTV_ROW) {
        // one group of `lanes` threads per 4 (split, output) items
        int64_t threads = (P.nout * P.splits + 3) / 4 * P.lanes;
        int grid = grid_for(threads, num_sms);
#define TL_ROW(VV, LL)                                                              \
    do {                                                                            \
        if (P.splits > 1) ttv_row_kernel<T, VV, LL, 4, true><<<grid, kThreads, 0, st>>>(a);  \
        else ttv_row_kernel<T, VV, LL, 4, false><<<grid, kThreads, 0, st>>>(a);            \
    } while (0)
        if (P.vec == V) {
            switch (P.lanes) {
            case 32: TL_ROW(V, 32); break;
            case 16: TL_ROW(V, 16); break;
            case 8: TL_ROW(V, 8); break;
            default: TL_ROW(V, 4); break;
            }
        } else {
            switch (P.lanes) {
            case 32: TL_ROW(1, 32); break;
            case 16: TL_ROW(1, 16); break;
            case 8: TL_ROW(1, 8); break;
            default: TL_ROW(1, 4); break;
            }
        }
#undef TL_ROW
    } else {
        int64_t threads = P.nout / P.vec * P.splits;
        int grid = grid_for(threads, num_sms);
        if (P.vec == V) ttv_col_kernel<T, V, 4><<<grid, kThreads, 0, st>>>(a);
        else ttv_col_kernel<T, 1, 4><<<grid, kThreads, 0, st>>>(a);
    }
    if (P.splits >= 64) {
        ttv_splitk_reduce<T, true><<<grid_for(P.nout * 32, num_sms), kThreads, 0, st>>>(a);
    } else if (P.splits > 1) {
        ttv_splitk_reduce<T, false><<<grid_for(P.nout, num_sms), kThreads, 0, st>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ECUDA;
}

}  // namespace

int ttv_status(bool clear)
{
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_ttv_status, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return TL_ECUDA;
    }
    if (clear && v) {
        unsigned int z = 0;
        cudaMemcpyToSymbol(g_ttv_status, &z, sizeof z);
    }
    return v ? TL_ETIMEOUT : TL_OK;
}

size_t ttv_workspace_bytes(const TtvPlan& P)
{
    if (P.splits <= 1) return 0;
    return (size_t)P.splits * (size_t)P.nout * (P.dtype == TL_F64 ? 8 : 4);
}

int launch_ttv(const TtvPlan& P, const void* A, const void* b, void* C, void* ws,
               int accumulate, int num_sms, cudaStream_t st)
{
    if (P.dtype == TL_F64) return launch_typed<double>(P, A, b, C, ws, accumulate, num_sms, st);
    return launch_typed<float>(P, A, b, C, ws, accumulate, num_sms, st);
}

}  // namespace tl

// ------------------------------------------------------------------------
// tl_ttv_noalloc: the same kernels with the split-K partial sums in a static
// device array instead of the library's per-stream workspace, so the call
// allocates no device memory (see tlgb.h for who needs this).
// ------------------------------------------------------------------------

#include <atomic>
#include <mutex>

static __device__ __align__(256) unsigned char g_ttv_noalloc_scratch[TL_TTV_NOALLOC_SCRATCH_BYTES];

namespace tl {
namespace {

constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of g_ttv_noalloc_scratch on the current device.  In host
// code the symbol names a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int noalloc_scratch(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TL_ECUDA;
    void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            cudaError_t e = cudaGetSymbolAddress(&p, g_ttv_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return TL_ECUDA;
            }
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return TL_OK;
}

}  // namespace
}  // namespace tl

extern "C" int tl_ttv_noalloc(const tl_tensor* A_, const void* b, int64_t incb, uint32_t q,
                              const tl_tensor* C_, int32_t accumulate, void* stream)
{
    using namespace tl;
    Tensor A, C;
    TtvPlan P;
    int sms = device_sms();
    if (sms <= 0) return TL_ECUDA;
    int rc = prepare_ttv(A_, b, incb, q, C_, sms, A, C, P);
    if (rc) return rc;
    size_t need = ttv_workspace_bytes(P);
    if (need > (size_t)TL_TTV_NOALLOC_SCRATCH_BYTES) return TL_ENOMEM;
    void* ws = nullptr;
    if (need) {
        rc = noalloc_scratch(&ws);
        if (rc) return rc;
    }
    rc = launch_ttv(P, A.data, b, C.data, ws, accumulate ? 1 : 0, sms,
                    static_cast<cudaStream_t>(stream));
    if (rc == TL_OK) count_launches(P.splits > 1 ? 2 : 1);
    return rc;
}
