// batch.cu -- many small ttv / ttm / entrywise operations (Sec. 5.2 Eqs. 24-25,
// Sec. 5.1 Eq. 23) of uneven order, extents and layout in ONE persistent
// launch.
//
// Each operation is planned on the host exactly as a single call would be
// (validation, Eq. 14 strides, joint mode collapse) and becomes a device
// descriptor.  Its outputs are cut into work units (a range of outputs for
// ttv and entrywise, a tile of rows for ttm); a prefix sum over the units of
// all operations forms one global unit index.  A persistent grid takes units
// from an atomic counter, looks the owning operation up by binary search and
// runs the unit with the whole CTA.  The unit size and the per-unit code
// variant of every shape class are chosen by an autotuner that times the
// candidates once and caches the winner on disk.  The launch (counter reset
// + kernel) can be captured into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "batch.h"
#include "device.cuh"
#include "kernels.h"
#include "runtime.h"

namespace tl {

namespace {

constexpr int kThreads = 256;
constexpr int kBD = 8;              // dims of a collapsed space in a batch descriptor

// Work-unit code variants.
enum : int32_t {
    BV_TTV_COL = 0,      // one thread per output, k loop
    BV_TTV_ROW4 = 1,     // 4 lanes per output (contraction contiguous)
    BV_TTV_ROW8 = 2,
    BV_TTV_ROW32 = 3,
    BV_TTM_32 = 4,       // smem-tiled GEMM tile of 32 rows
    BV_TTM_64 = 5,       // 64 rows
    BV_EW = 6,           // one thread per element
    BV_TTM_SMALL = 7,    // B in shared memory, a row per thread, J outputs in registers
    BV_TTV_VEC = 8,      // 16 bytes of consecutive outputs per thread (unit stride in A and C)
};

struct BOp {
    int32_t kind, dtype, variant, nd;
    int32_t eop, accumulate;
    int64_t count;       // outputs (ttv), rows (ttm) or elements (entrywise)
    int64_t unit;        // count per work unit
    int64_t ubegin;      // first global unit of this operation
    int64_t n[kBD], s0[kBD], s1[kBD], s2[kBD];
    int64_t nq, saq, incb, J, scq, ldb_row, ldb_col;
    double alpha;
    const void* A;
    const void* B;       // b (ttv), B (ttm), second operand (entrywise)
    void* C;
    int32_t idx32;       // every linear index fits 32 bits: decode with fd[]
    FastDiv fd[kBD];     // multiply-high division by n[d]
    int64_t lim[3];      // operand limits (Space::limit), checked in bounds-checked builds
};

// Bounds-checked builds: a decoded offset outside its operand's limit is
// recorded and replaced by 0 (product builds compile this away).
__device__ __forceinline__ void bcheck(const BOp& op, int64_t& o0, int64_t& o1, int64_t& o2)
{
#ifdef TL_CHECK_BOUNDS
    int64_t* o[3] = {&o0, &o1, &o2};
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (op.lim[k] > 0 && (*o[k] < 0 || *o[k] >= op.lim[k])) {
            bounds_record(*o[k]);
            *o[k] = 0;
        }
#endif
}

__device__ __forceinline__ void bdecode(const BOp& op, int64_t g, int64_t& o0, int64_t& o1,
                                        int64_t& o2)
{
    o0 = o1 = o2 = 0;
    if (op.idx32) {
        uint32_t r = (uint32_t)g;
        for (int d = 0; d < op.nd; ++d) {
            uint32_t i = r;
            if (d < op.nd - 1) {
                const FastDiv f = op.fd[d];
                const uint32_t t = __umulhi(f.mul, r);
                const uint32_t qd = (t + ((r - t) >> f.sh1)) >> f.sh2;
                i = r - qd * (uint32_t)op.n[d];
                r = qd;
            }
            o0 += (int64_t)i * op.s0[d];
            o1 += (int64_t)i * op.s1[d];
            o2 += (int64_t)i * op.s2[d];
        }
        bcheck(op, o0, o1, o2);
        return;
    }
    for (int d = 0; d < op.nd; ++d) {
        int64_t i;
        if (d == op.nd - 1) {
            i = g;
        } else {
            int64_t q = g / op.n[d];
            i = g - q * op.n[d];
            g = q;
        }
        o0 += i * op.s0[d];
        o1 += i * op.s1[d];
        o2 += i * op.s2[d];
    }
    bcheck(op, o0, o1, o2);
}

// Loads of A per chunk of a strided dot product: 8 FP32 / 4 FP64 keep the
// persistent kernel within its 64 registers.
template <typename T>
constexpr int dot_chunk_len()
{
    return sizeof(T) == 4 ? 8 : 4;
}

template <typename T>
__device__ void unit_ttv_col(const BOp& op, int64_t e0, int64_t e1)
{
    const T* A = static_cast<const T*>(op.A);
    const T* b = static_cast<const T*>(op.B);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
        int64_t oa, oc, unused;
        bdecode(op, e, oa, oc, unused);
        const T acc = dot_strided<T, dot_chunk_len<T>()>(A + oa, op.saq, b, op.incb, op.nq, T(0));
        T* pc = static_cast<T*>(op.C) + oc;
        *pc = op.accumulate ? *pc + acc : acc;
    }
}

template <typename T>
__device__ __forceinline__ bool ttv_vec_ok(const BOp& op)
{
    constexpr int64_t V = 16 / sizeof(T);
    if (op.nd < 1 || op.s0[0] != 1 || op.s1[0] != 1 || op.n[0] % V || op.saq % V ||
        op.unit % V)
        return false;
    for (int d = 1; d < op.nd; ++d)
        if (op.s0[d] % V || op.s1[d] % V) return false;
    return ((reinterpret_cast<uintptr_t>(op.A) | reinterpret_cast<uintptr_t>(op.C)) & 15) == 0;
}

// acc[v] += sum over u < NQ of a[u * sa + v] * b[u * sb], u ascending: the
// chunk's 16-byte loads of A all issued before the first product.
template <typename T, int NQ>
__device__ __forceinline__ void vec_chunk(const T* __restrict__ a, int64_t sa, const T* __restrict__ b,
                                          int64_t sb, T* acc)
{
    constexpr int V = 16 / sizeof(T);
    using VT = typename Vec<T, V>::type;
    VT x[NQ];
    T y[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
        x[u] = __ldg(reinterpret_cast<const VT*>(a + u * sa));
        y[u] = __ldg(b + u * sb);
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
        const T* xe = reinterpret_cast<const T*>(&x[u]);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma(xe[v], y[u], acc[v]);
    }
}

// Outputs contiguous in A and C along the collapsed dim 0 (its extent and
// every other stride multiples of the vector width, 16-byte aligned bases):
// each thread takes 16 bytes of consecutive outputs and streams A with
// 16-byte loads, 128 bytes per thread at a time and the remainder as one
// chunk.
template <typename T>
__device__ void unit_ttv_vec(const BOp& op, int64_t e0, int64_t e1)
{
    constexpr int V = 16 / sizeof(T);
    using VT = typename Vec<T, V>::type;
    const T* A = static_cast<const T*>(op.A);
    const T* b = static_cast<const T*>(op.B);
    for (int64_t e = e0 + (int64_t)V * threadIdx.x; e < e1; e += (int64_t)V * kThreads) {
        int64_t oa, oc, unused;
        bdecode(op, e, oa, oc, unused);
        const T* pa = A + oa;
        T acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = T(0);
        // chunks of 128 bytes of A per thread (8 FP32 / 4 FP64 vectors) fit
        // the kernel's 64 registers
        constexpr int CH = sizeof(T) == 8 ? 4 : 8;
        int64_t k = 0;
        for (; k + CH <= op.nq; k += CH)
            vec_chunk<T, CH>(pa + k * op.saq, op.saq, b + k * op.incb, op.incb, acc);
        const T* at = pa + k * op.saq;
        const T* bt = b + k * op.incb;
        switch ((int)(op.nq - k)) {
        case 1: vec_chunk<T, 1>(at, op.saq, bt, op.incb, acc); break;
        case 2: vec_chunk<T, 2>(at, op.saq, bt, op.incb, acc); break;
        case 3: vec_chunk<T, 3>(at, op.saq, bt, op.incb, acc); break;
        case 4: vec_chunk<T, CH == 8 ? 4 : 1>(at, op.saq, bt, op.incb, acc); break;
        case 5: vec_chunk<T, CH == 8 ? 5 : 1>(at, op.saq, bt, op.incb, acc); break;
        case 6: vec_chunk<T, CH == 8 ? 6 : 1>(at, op.saq, bt, op.incb, acc); break;
        case 7: vec_chunk<T, CH == 8 ? 7 : 1>(at, op.saq, bt, op.incb, acc); break;
        default: break;
        }
        T* pc = static_cast<T*>(op.C) + oc;
        if (op.accumulate) {
            const VT o = *reinterpret_cast<const VT*>(pc);
            const T* oe = reinterpret_cast<const T*>(&o);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += oe[v];
        }
        *reinterpret_cast<VT*>(pc) = *reinterpret_cast<const VT*>(acc);
    }
}

template <typename T, int L>
__device__ void unit_ttv_row(const BOp& op, int64_t e0, int64_t e1)
{
    const T* A = static_cast<const T*>(op.A);
    const T* b = static_cast<const T*>(op.B);
    const int g = threadIdx.x / L, sub = threadIdx.x % L;
    constexpr int G = kThreads / L;
    // uniform trip count so every shuffle sees a converged warp
    for (int64_t base = e0; base < e1; base += G) {
        const int64_t e = base + g;
        const bool ok = e < e1;
        T acc = T(0);
        int64_t oa = 0, oc = 0, unused;
        if (ok) {
            bdecode(op, e, oa, oc, unused);
            // this lane's k = sub, sub + L, ... in ascending order
            if (sub < op.nq)
                acc = dot_strided<T, dot_chunk_len<T>()>(A + oa + sub * op.saq, L * op.saq,
                                                         b + sub * op.incb, L * op.incb,
                                                         (op.nq - sub + L - 1) / L, T(0));
        }
#pragma unroll
        for (int m = L / 2; m >= 1; m /= 2) acc += __shfl_xor_sync(0xffffffffu, acc, m);
        if (ok && sub == 0) {
            T* pc = static_cast<T*>(op.C) + oc;
            *pc = op.accumulate ? *pc + acc : acc;
        }
    }
}

// Rows [m0, m0 + BM) x all J columns; k staged 16 deep in shared memory.
template <typename T, int BM>
__device__ void unit_ttm(const BOp& op, int64_t m0, uint8_t* smem)
{
    constexpr int BJ = 64, BK = 16;
    T (*As)[BM + 1] = reinterpret_cast<T (*)[BM + 1]>(smem);
    T (*Bs)[BJ + 1] = reinterpret_cast<T (*)[BJ + 1]>(smem + sizeof(T) * BK * (BM + 1));
    int64_t* offA = reinterpret_cast<int64_t*>(smem + sizeof(T) * BK * (BM + 1 + BJ + 1));
    int64_t* offC = offA + BM;
    const T* A = static_cast<const T*>(op.A);
    const T* B = static_cast<const T*>(op.B);
    T* C = static_cast<T*>(op.C);
    const int tid = threadIdx.x, tm = tid & 15, tj = tid >> 4;
    constexpr int RM = BM / 16;
    const bool a_kfast = op.saq == 1, b_kfast = op.ldb_col == 1;
    if (tid < BM) {
        int64_t oa = 0, oc = 0, unused;
        if (m0 + tid < op.count) bdecode(op, m0 + tid, oa, oc, unused);
        offA[tid] = oa;
        offC[tid] = oc;
    }
    for (int64_t j0 = 0; j0 < op.J; j0 += BJ) {
        T acc[RM][4];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        for (int64_t k0 = 0; k0 < op.nq; k0 += BK) {
            __syncthreads();
            for (int e = tid; e < BM * BK; e += kThreads) {
                int mm, kk;
                if (a_kfast) { kk = e % BK; mm = e / BK; }
                else { mm = e % BM; kk = e / BM; }
                int64_t k = k0 + kk;
                As[kk][mm] = (m0 + mm < op.count && k < op.nq) ? __ldg(A + offA[mm] + k * op.saq) : T(0);
            }
            for (int e = tid; e < BJ * BK; e += kThreads) {
                int jj, kk;
                if (b_kfast) { kk = e % BK; jj = e / BK; }
                else { jj = e % BJ; kk = e / BJ; }
                int64_t j = j0 + jj, k = k0 + kk;
                Bs[kk][jj] = (j < op.J && k < op.nq) ? __ldg(B + j * op.ldb_row + k * op.ldb_col) : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T av[RM], bv[4];
#pragma unroll
                for (int i = 0; i < RM; ++i) av[i] = As[kk][tm + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tj + 16 * j];
#pragma unroll
                for (int i = 0; i < RM; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
        }
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const int mm = tm + 16 * i;
            if (m0 + mm >= op.count) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t jg = j0 + tj + 16 * j;
                if (jg >= op.J) continue;
                T* p = C + offC[mm] + jg * op.scq;
                *p = op.accumulate ? *p + acc[i][j] : acc[i][j];
            }
        }
    }
    __syncthreads();
}

// ttm with the whole J x n_q matrix in shared memory (n_q <= 64, J <= 64 for
// FP32, J <= 32 for FP64): one row of A per thread, JB <= 16 of its outputs
// kept in registers per pass (further passes re-read the row, from L1/L2,
// when J > 16: on the 4096-operation batch recipe that ran the small ttm
// operations in 1.69 ms against 1.84 with 32 columns per pass), the row's
// loads issued in chunks of 8 and a remainder chunk of exact length (row_dot)
// so that a short contraction waits for one memory latency, B read as
// 16-byte broadcasts.
template <typename T, int JB>
__device__ void unit_ttm_small(const BOp& op, int64_t e0, int64_t e1, uint8_t* smem)
{
    const T* A = static_cast<const T*>(op.A);
    const T* B = static_cast<const T*>(op.B);
    T* C = static_cast<T*>(op.C);
    const int nq = (int)op.nq, J = (int)op.J;
    const int JT = (J + JB - 1) / JB * JB;        // padded columns held in shared memory
    T* Bs = reinterpret_cast<T*>(smem);           // [n_q][JT], zero beyond J
    for (int e = threadIdx.x; e < nq * JT; e += kThreads) {
        const int k = e / JT, j = e - k * JT;
        Bs[e] = j < J ? __ldg(B + j * op.ldb_row + k * op.ldb_col) : T(0);
    }
    __syncthreads();
    for (int64_t m = e0 + threadIdx.x; m < e1; m += kThreads) {
        int64_t oa, oc, unused;
        bdecode(op, m, oa, oc, unused);
        const T* pa = A + oa;
        T* pc = C + oc;
        for (int j0 = 0; j0 < J; j0 += JB) {
            T acc[JB];
#pragma unroll
            for (int j = 0; j < JB; ++j) acc[j] = T(0);
            row_dot<T, JB>(pa, op.saq, nq, Bs + j0, JT, acc);
            T* pj = pc + (int64_t)j0 * op.scq;
            if (!op.accumulate && j0 + JB <= J) {
#pragma unroll
                for (int j = 0; j < JB; ++j) pj[(int64_t)j * op.scq] = acc[j];
            } else {
#pragma unroll
                for (int j = 0; j < JB; ++j) {
                    if (j0 + j < J) {
                        T* p = pj + (int64_t)j * op.scq;
                        *p = op.accumulate ? *p + acc[j] : acc[j];
                    }
                }
            }
        }
    }
    __syncthreads();          // Bs is rewritten by the next unit
}

template <typename T>
__device__ void unit_ew(const BOp& op, int64_t e0, int64_t e1)
{
    const T* A = static_cast<const T*>(op.A);
    const T* B = static_cast<const T*>(op.B);
    T* C = static_cast<T*>(op.C);
    const bool unary = op.eop == TL_COPY || op.eop == TL_SCALE;
    const T alpha = (T)op.alpha;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
        int64_t oa, ob, oc;
        bdecode(op, e, oa, ob, oc);
        T x = __ldg(A + oa);
        T y = unary ? T(0) : __ldg(B + ob);
        T r;
        switch (op.eop) {
        case TL_ADD: r = x + y; break;
        case TL_SUB: r = x - y; break;
        case TL_MUL: r = x * y; break;
        case TL_DIV: r = x / y; break;
        case TL_COPY: r = x; break;
        default: r = alpha * x; break;
        }
        C[oc] = r;
    }
}

template <typename T>
__device__ void run_unit(const BOp& op, int64_t u, uint8_t* smem)
{
    const int64_t e0 = (u - op.ubegin) * op.unit;
    const int64_t e1 = min(op.count, e0 + op.unit);
    switch (op.variant) {
    case BV_TTV_COL: unit_ttv_col<T>(op, e0, e1); break;
    case BV_TTV_ROW4: unit_ttv_row<T, 4>(op, e0, e1); break;
    case BV_TTV_ROW8: unit_ttv_row<T, 8>(op, e0, e1); break;
    case BV_TTV_ROW32: unit_ttv_row<T, 32>(op, e0, e1); break;
    case BV_TTV_VEC:
        // the host only assigns this unit where it applies; the check keeps a
        // stale or foreign assignment from issuing misaligned vector loads
        if (ttv_vec_ok<T>(op)) unit_ttv_vec<T>(op, e0, e1);
        else unit_ttv_col<T>(op, e0, e1);
        break;
    case BV_TTM_32:
        for (int64_t m0 = e0; m0 < e1; m0 += 32) unit_ttm<T, 32>(op, m0, smem);
        break;
    case BV_TTM_64:
        for (int64_t m0 = e0; m0 < e1; m0 += 64) unit_ttm<T, 64>(op, m0, smem);
        break;
    case BV_TTM_SMALL:
        // the matrix must fit the static shared memory (as the host checks);
        // anything else takes the tiled unit, one 64-row tile at a time
        if (op.nq > 64 || op.J > (sizeof(T) == 8 ? 32 : 64)) {
            for (int64_t m0 = e0; m0 < e1; m0 += 64) unit_ttm<T, 64>(op, m0, smem);
        } else if (op.J <= 4) unit_ttm_small<T, 4>(op, e0, e1, smem);
        else if (op.J <= 8) unit_ttm_small<T, 8>(op, e0, e1, smem);
        else if (op.J <= 16) unit_ttm_small<T, 16>(op, e0, e1, smem);
        else unit_ttm_small<T, 16>(op, e0, e1, smem);
        break;
    default: unit_ew<T>(op, e0, e1); break;
    }
}

constexpr size_t kSmem = 8 * 16 * (64 + 1 + 64 + 1) + 2 * 64 * 8;   // FP64 ttm tile

__global__ void __launch_bounds__(kThreads, 4) batch_kernel(const BOp* __restrict__ ops, int nops,
                                                         int64_t total_units,
                                                         unsigned long long* counter)
{
    __shared__ __align__(16) uint8_t smem[kSmem];
    __shared__ __align__(16) BOp sop;
    __shared__ int64_t s_unit;
    __shared__ int s_op;
    int cur = -1;                        // operation held in sop (same in every thread)
    int hint = 0;                        // thread 0: search start
    for (;;) {
        if (threadIdx.x == 0) {
            int64_t u = (int64_t)atomicAdd(counter, 1ull);
            s_unit = u;
            if (u < total_units) {
                // the counter only grows, so the owner of u is at or after the
                // owner of this CTA's previous unit: scan forward, then bisect
                int lo = hint;
                if (lo + 1 < nops && ops[lo + 1].ubegin <= u) {
                    int hi = nops - 1;
                    while (lo < hi) {
                        int mid = (lo + hi + 1) / 2;
                        if (ops[mid].ubegin <= u) lo = mid;
                        else hi = mid - 1;
                    }
                }
                s_op = lo;
                hint = lo;
            }
        }
        __syncthreads();
        const int64_t u = s_unit;
        if (u >= total_units) break;
        if (s_op != cur) {
            cur = s_op;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(ops + cur);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sop);
            for (int i = threadIdx.x; i < (int)(sizeof(BOp) / 4); i += kThreads) dst[i] = src[i];
            __syncthreads();
        }
        if (sop.dtype == TL_F64) run_unit<double>(sop, u, smem);
        else run_unit<float>(sop, u, smem);
        __syncthreads();
    }
}

// -------------------------------------------------------------- autotuner --

struct Candidate {
    int32_t variant;
    int64_t unit;
};

// The vectorised ttv unit needs outputs contiguous in A and C along dim 0,
// vector-aligned addresses for every output group, and whole vectors per unit.
bool vec_ttv_host(const BOp& op)
{
    if (op.kind != TL_OP_TTV || op.nd < 1) return false;
    const int64_t V = op.dtype == TL_F64 ? 2 : 4;
    if (op.s0[0] != 1 || op.s1[0] != 1 || op.n[0] % V || op.saq % V) return false;
    for (int d = 1; d < op.nd; ++d)
        if (op.s0[d] % V || op.s1[d] % V) return false;
    return (reinterpret_cast<uintptr_t>(op.A) % 16) == 0 && (reinterpret_cast<uintptr_t>(op.C) % 16) == 0;
}

// The shared-memory ttm unit takes B whole: n_q <= 64 and J <= 64 (FP32) or
// 32 (FP64), so B fits the kernel's static shared memory.
bool small_ttm_host(const BOp& op)
{
    return op.kind == TL_OP_TTM && op.nq <= 64 && op.J <= (op.dtype == TL_F64 ? 32 : 64);
}

std::string class_key(const BOp& op)
{
    auto lg = [](int64_t x) { int b = 0; while ((int64_t(1) << b) < x) ++b; return b; };
    char buf[160];
    // the key records which optional units apply, so a choice cached for one
    // operation never lands on an operation the unit does not fit
    std::snprintf(buf, sizeof buf, "k%d|d%d|row%d|nq%d|J%d|cnt%d|v%d|s%d", op.kind, op.dtype,
                  op.kind == TL_OP_TTV && op.saq == 1 ? 1 : 0, lg(op.nq), lg(op.J), lg(op.count),
                  vec_ttv_host(op) ? 1 : 0, small_ttm_host(op) ? 1 : 0);
    return buf;
}

std::vector<Candidate> candidates(const BOp& op)
{
    std::vector<Candidate> c;
    if (op.kind == TL_OP_TTV) {
        if (op.saq == 1) {
            for (int32_t v : {BV_TTV_ROW4, BV_TTV_ROW8, BV_TTV_ROW32})
                for (int64_t u : {512, 4096}) c.push_back({v, u});
        }
        for (int64_t u : {1024, 4096, 16384}) c.push_back({BV_TTV_COL, u});
        if (vec_ttv_host(op))
            for (int64_t u : {1024, 4096, 16384}) c.push_back({BV_TTV_VEC, u});
    } else if (op.kind == TL_OP_TTM) {
        for (int64_t u : {256, 1024, 4096}) {
            c.push_back({BV_TTM_32, u});
            c.push_back({BV_TTM_64, u});
            if (small_ttm_host(op)) c.push_back({BV_TTM_SMALL, u});
        }
    } else {
        for (int64_t u : {8192, 65536}) c.push_back({BV_EW, u});
    }
    return c;
}

// Default choice when tuning is off.
Candidate heuristic(const BOp& op)
{
    if (op.kind == TL_OP_TTV) {
        if (op.saq == 1 && op.nq >= 32) return {BV_TTV_ROW8, 2048};
        if (vec_ttv_host(op)) return {BV_TTV_VEC, 4096};
        return {BV_TTV_COL, 4096};
    }
    if (op.kind == TL_OP_TTM) {
        if (small_ttm_host(op)) return {BV_TTM_SMALL, 1024};
        return op.count >= 4096 ? Candidate{BV_TTM_64, 1024} : Candidate{BV_TTM_32, 256};
    }
    return {BV_EW, 65536};
}

// A candidate from the cache (or from a representative operation) as it may
// be applied to `op`: variants of another kind, or optional units that do not
// fit the operation, fall back to the default choice.
Candidate sanitize(Candidate c, const BOp& op)
{
    bool ok = c.unit >= 1;
    if (op.kind == TL_OP_TTV)
        ok = ok && (c.variant == BV_TTV_COL || c.variant == BV_TTV_ROW4 || c.variant == BV_TTV_ROW8 ||
                    c.variant == BV_TTV_ROW32 || (c.variant == BV_TTV_VEC && vec_ttv_host(op) &&
                                                  c.unit % 4 == 0));
    else if (op.kind == TL_OP_TTM)
        ok = ok && (c.variant == BV_TTM_32 || c.variant == BV_TTM_64 ||
                    (c.variant == BV_TTM_SMALL && small_ttm_host(op)));
    else
        ok = ok && c.variant == BV_EW;
    return ok ? c : heuristic(op);
}

struct TuneCache {
    std::mutex mu;
    bool loaded = false;
    std::map<std::string, Candidate> table;
    std::string path;

    void load()
    {
        if (loaded) return;
        loaded = true;
        const char* p = std::getenv("TL_TUNE_CACHE");
        if (p && *p) {
            path = p;
        } else {
            const char* h = std::getenv("HOME");
            path = std::string(h ? h : "/tmp") + "/.cache/tlgb_tune.txt";
        }
        std::ifstream in(path);
        std::string key;
        Candidate c;
        while (in >> key >> c.variant >> c.unit) table[key] = c;
    }
    void save()
    {
        std::string dir = path.substr(0, path.find_last_of('/'));
        if (!dir.empty()) mkdir(dir.c_str(), 0755);   // best effort; may exist
        std::ofstream out(path);
        if (!out) return;
        for (auto& kv : table) out << kv.first << ' ' << kv.second.variant << ' ' << kv.second.unit << '\n';
    }
};

TuneCache g_tune;

std::string device_tag()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "dev?";
    std::string s = prop.name;
    for (auto& ch : s)
        if (ch == ' ') ch = '_';
    return s + "_sm" + std::to_string(prop.multiProcessorCount);
}

int grid_size()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel, kThreads, 0);
    if (per < 1) per = 1;
    int g = per * device_sms();
    if (dev >= 0 && dev < 64) cached[dev] = g;
    return g;
}

int64_t units_of(const BOp& op) { return op.count == 0 ? 0 : (op.count + op.unit - 1) / op.unit; }

}  // namespace

// ------------------------------------------------------------ batch object --

struct Batch {
    std::vector<BOp> host;
    BOp* dev_ops = nullptr;
    unsigned long long* counter = nullptr;
    int64_t total_units = 0;
    int32_t flags = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    size_t bytes = 0;            // algorithmic bytes of all operations
    int direct = 0;              // operations run by their own kernels
    std::vector<tl_op> direct_ops;
    // the direct operations run on a stream of their own, concurrently with
    // the persistent launch, between a fork and a join event
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Operations the persistent kernel does not take: a contraction this long
// would run serially inside one work unit (the split-K kernels spread it),
// and an operation this large amortises its own launch, so it runs on the
// kernel tuned for its layout (TMA tiles, staged rows, tensor cores).
constexpr int64_t kLongContraction = 4096;
constexpr size_t kDirectBytes = size_t(16) << 20;

// In a batch of many operations, a ttm that the row unit takes (its matrix
// fits shared memory) stays in the persistent launch up to 256 MB: the side
// stream cannot overlap a persistent launch that holds every register of
// every SM, and the 77 such operations of 16-64 MB in the 4096-operation
// recipe ran at 1.9 TB/s as their own launches (the whole batch 3.56 ms)
// against 3.24 ms for the batch with them as units.  Serving's slot
// launches keep the 16 MB rule: its large requests have a lane of their own.
constexpr size_t kDirectBytesRows = size_t(256) << 20;

static int fill_op(const tl_op& o, BOp& b, size_t& bytes, bool& direct, bool many = false)
{
    std::memset(&b, 0, sizeof b);
    b.kind = o.kind;
    b.accumulate = o.accumulate ? 1 : 0;
    direct = false;
    const int sms = device_sms() > 0 ? device_sms() : 152;
    if (o.kind == TL_OP_TTV) {
        Tensor A, C;
        TtvPlan P;
        int rc = prepare_ttv(&o.A, o.vec, o.incb, o.q, &o.C, sms, A, C, P);
        if (rc) return rc;
        const size_t mine = (size_t)(A.count() + C.count() + P.nq) * A.elem();
        if (P.out.nd > kBD || (P.splits > 1 && P.nq >= kLongContraction) || mine >= kDirectBytes) {
            direct = true;
            return TL_OK;
        }
        b.dtype = A.dtype;
        b.nd = P.out.nd;
        for (int d = 0; d < P.out.nd; ++d) {
            b.n[d] = P.out.d[d].n;
            b.s0[d] = P.out.d[d].s[0];
            b.s1[d] = P.out.d[d].s[1];
        }
        b.count = P.nout;
        b.nq = P.nq;
        b.saq = P.saq;
        b.incb = o.incb;
        b.lim[0] = debug_limit(P.out.limit[0]);
        b.lim[1] = debug_limit(P.out.limit[1]);
        b.A = A.data;
        b.B = o.vec;
        b.C = C.data;
        bytes += (size_t)(A.count() + C.count() + P.nq) * A.elem();
    } else if (o.kind == TL_OP_TTM) {
        Tensor A, C;
        TtmPlan P;
        int rc = prepare_ttm(&o.A, o.vec, o.J, o.ldb_row, o.ldb_col, o.q, &o.C, o.precision, A, C, P);
        if (rc) return rc;
        const size_t mine = (size_t)(A.count() + C.count() + P.J * P.nq) * A.elem();
        const bool rows_unit = P.nq <= 64 && P.J <= (A.dtype == TL_F64 ? 32 : 64);
        if (P.rows.nd > kBD || P.kernel == K_TTM_TC ||
            (ttm_simt_splits(P, sms, nullptr) > 1 && P.nq >= kLongContraction) ||
            mine >= (many && rows_unit ? kDirectBytesRows : kDirectBytes)) {
            direct = true;
            return TL_OK;
        }
        b.dtype = A.dtype;
        b.nd = P.rows.nd;
        for (int d = 0; d < P.rows.nd; ++d) {
            b.n[d] = P.rows.d[d].n;
            b.s0[d] = P.rows.d[d].s[0];
            b.s1[d] = P.rows.d[d].s[1];
        }
        b.count = P.M;
        b.nq = P.nq;
        b.saq = P.saq;
        b.lim[0] = debug_limit(P.rows.limit[0]);
        b.lim[1] = debug_limit(P.rows.limit[1]);
        b.J = P.J;
        b.scq = P.scq;
        b.ldb_row = P.ldb_row;
        b.ldb_col = P.ldb_col;
        b.A = A.data;
        b.B = o.vec;
        b.C = C.data;
        bytes += (size_t)(A.count() + C.count() + P.J * P.nq) * A.elem();
    } else if (o.kind == TL_OP_ENTRYWISE) {
        Tensor A, B, C;
        EwPlan P;
        bool hasB = false;
        bool unary = o.entry_op == TL_COPY || o.entry_op == TL_SCALE;
        int rc = prepare_entrywise(o.entry_op, &o.A, unary ? nullptr : &o.B, &o.C, A, B, C, hasB, P);
        if (rc) return rc;
        if (P.sp.nd > kBD || (size_t)((hasB ? 3 : 2) * A.count()) * A.elem() >= kDirectBytes) {
            direct = true;
            return TL_OK;
        }
        b.dtype = A.dtype;
        b.nd = P.sp.nd;
        for (int d = 0; d < P.sp.nd; ++d) {
            b.n[d] = P.sp.d[d].n;
            b.s0[d] = P.sp.d[d].s[0];
            b.s1[d] = P.sp.d[d].s[1];
            b.s2[d] = P.sp.d[d].s[2];
        }
        b.count = P.N;
        for (int k = 0; k < 3; ++k) b.lim[k] = debug_limit(P.sp.limit[k]);
        b.eop = o.entry_op;
        b.alpha = o.alpha;
        b.A = A.data;
        b.B = hasB ? B.data : A.data;
        b.C = C.data;
        bytes += (size_t)((hasB ? 3 : 2) * A.count()) * A.elem();
    } else {
        return TL_EINVAL;
    }
    // linear indices below 2^32: 32-bit multiply-high decoding
    b.idx32 = b.count <= (int64_t)0xffffffffLL ? 1 : 0;
    for (int d = 0; d < b.nd; ++d) b.fd[d] = make_fastdiv((uint32_t)(b.n[d] > 0 ? b.n[d] : 1));
    return TL_OK;
}

// Times one candidate on a one-operation table (milliseconds, best of 3).
// Device time of one persistent launch over `ops` (their variants and unit
// sizes as assigned; ubegin is recomputed here): the best of 3 launches after
// one warm-up.  dev holds room for ops.size() descriptors.
static float time_ops(std::vector<BOp>& ops, BOp* dev, unsigned long long* counter,
                      cudaStream_t st)
{
    int64_t units = 0;
    for (BOp& b : ops) {
        b.ubegin = units;
        units += units_of(b);
    }
    if (units == 0) return 0.f;
    if (cudaMemcpyAsync(dev, ops.data(), sizeof(BOp) * ops.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    const int grid = grid_size();
    for (int rep = 0; rep < 4; ++rep) {
        cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
        cudaEventRecord(e0, st);
        batch_kernel<<<grid, kThreads, 0, st>>>(dev, (int)ops.size(), units, counter);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return best;
}

int batch_create(const tl_op* ops, size_t count, int32_t flags, void* stream, Batch** out)
{
    if (!out || (!ops && count)) return TL_EINVAL;
    *out = nullptr;
    Batch* B = new Batch();
    B->flags = flags;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (size_t i = 0; i < count; ++i) {
        BOp b;
        bool direct = false;
        int rc = fill_op(ops[i], b, B->bytes, direct, true);
        if (rc) {
            delete B;
            return rc;
        }
        if (direct) {
            B->direct_ops.push_back(ops[i]);
            B->direct++;
            continue;
        }
        if (b.count > 0) B->host.push_back(b);
    }
    // large operations first, so the tail of the persistent launch is small units
    std::stable_sort(B->host.begin(), B->host.end(),
                     [](const BOp& x, const BOp& y) { return x.count * (x.kind == TL_OP_TTM ? x.J : 1) >
                                                             y.count * (y.kind == TL_OP_TTM ? y.J : 1); });
    // variant and unit size per operation: the default choice, or with
    // TL_BATCH_TUNE the choice of each shape class timed on all of the
    // batch's operations of that class launched together (cached on disk);
    // the tuned plan is kept only if the whole batch runs faster with it
    for (BOp& b : B->host) {
        const Candidate c = heuristic(b);
        b.variant = c.variant;
        b.unit = c.unit;
    }
    if ((flags & TL_BATCH_TUNE) && !B->host.empty()) {
        std::lock_guard<std::mutex> lk(g_tune.mu);
        g_tune.load();
        const std::string tag = device_tag();
        std::map<std::string, std::vector<size_t>> members;
        for (size_t i = 0; i < B->host.size(); ++i)
            members[tag + "|" + class_key(B->host[i])].push_back(i);
        size_t largest = 0;
        for (auto& kv : members) largest = std::max(largest, kv.second.size());
        BOp* dev = nullptr;
        unsigned long long* ctr = nullptr;
        if (cudaMalloc(&dev, sizeof(BOp) * B->host.size()) != cudaSuccess ||
            cudaMalloc(&ctr, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            if (dev) cudaFree(dev);
            batch_destroy(B);
            return TL_ENOMEM;
        }
        std::vector<BOp> tuned = B->host;
        bool saved = false;
        std::vector<BOp> sub;
        for (auto& kv : members) {
            Candidate pick;
            auto hit = g_tune.table.find(kv.first);
            if (hit != g_tune.table.end()) {
                pick = hit->second;
            } else {
                const BOp& rep = B->host[kv.second.front()];
                pick = heuristic(rep);
                float best_ms = 1e30f;
                for (Candidate c : candidates(rep)) {
                    sub.clear();
                    for (size_t i : kv.second) {
                        BOp t = B->host[i];
                        const Candidate s_ = sanitize(c, t);
                        t.variant = s_.variant;
                        t.unit = s_.unit;
                        sub.push_back(t);
                    }
                    const float ms = time_ops(sub, dev, ctr, st);
                    if (ms < best_ms) {
                        best_ms = ms;
                        pick = c;
                    }
                }
                g_tune.table[kv.first] = pick;
                saved = true;
            }
            for (size_t i : kv.second) {
                const Candidate s_ = sanitize(pick, tuned[i]);
                tuned[i].variant = s_.variant;
                tuned[i].unit = s_.unit;
            }
        }
        if (saved) g_tune.save();
        std::vector<BOp> plain = B->host;
        const float t_plain = time_ops(plain, dev, ctr, st);
        const float t_tuned = time_ops(tuned, dev, ctr, st);
        if (t_tuned < t_plain) B->host = tuned;
        cudaFree(dev);
        cudaFree(ctr);
    }
    int64_t u = 0;
    for (BOp& b : B->host) {
        b.ubegin = u;
        u += units_of(b);
    }
    B->total_units = u;
    if (!B->host.empty()) {
        if (cudaMalloc(&B->dev_ops, sizeof(BOp) * B->host.size()) != cudaSuccess ||
            cudaMalloc(&B->counter, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            batch_destroy(B);
            return TL_ENOMEM;
        }
        if (cudaMemcpyAsync(B->dev_ops, B->host.data(), sizeof(BOp) * B->host.size(),
                            cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            batch_destroy(B);
            return TL_ECUDA;
        }
    }
    *out = B;
    return TL_OK;
}

static int enqueue(Batch* B, cudaStream_t st)
{
    if (B->total_units > 0) {
        if (cudaMemsetAsync(B->counter, 0, sizeof(unsigned long long), st) != cudaSuccess) return TL_ECUDA;
        batch_kernel<<<grid_size(), kThreads, 0, st>>>(B->dev_ops, (int)B->host.size(),
                                                       B->total_units, B->counter);
        if (cudaGetLastError() != cudaSuccess) return TL_ECUDA;
    }
    return TL_OK;
}

int batch_launch(Batch* B, cudaStream_t st);

int batch_run(Batch* B, void* stream)
{
    if (!B) return TL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // operations the batch kernel does not take run through their own kernels,
    // on the side stream when there is a persistent launch to overlap them with
    const bool overlap = !B->direct_ops.empty() && B->total_units > 0;
    if (overlap && !B->side) {
        if (cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming) != cudaSuccess)
            return TL_ECUDA;
    }
    void* dstream = overlap ? static_cast<void*>(B->side) : stream;
    if (overlap && (cudaEventRecord(B->fork, st) != cudaSuccess ||
                    cudaStreamWaitEvent(B->side, B->fork, 0) != cudaSuccess))
        return TL_ECUDA;
    for (const tl_op& o : B->direct_ops) {
        int rc = TL_OK;
        if (o.kind == TL_OP_TTV) rc = tl_ttv(&o.A, o.vec, o.incb, o.q, &o.C, o.accumulate, dstream);
        else if (o.kind == TL_OP_TTM)
            rc = tl_ttm(&o.A, o.vec, o.J, o.ldb_row, o.ldb_col, o.q, &o.C, o.precision, o.accumulate,
                        dstream);
        else
            rc = tl_entrywise(o.entry_op, &o.A,
                              (o.entry_op == TL_COPY || o.entry_op == TL_SCALE) ? nullptr : &o.B,
                              o.alpha, &o.C, dstream);
        if (rc) return rc;
    }
    if (overlap && cudaEventRecord(B->join, B->side) != cudaSuccess) return TL_ECUDA;
    int rc = batch_launch(B, st);
    // the caller's stream waits for the direct operations as well
    if (overlap && cudaStreamWaitEvent(st, B->join, 0) != cudaSuccess) return TL_ECUDA;
    return rc;
}

// The persistent launch of a batch on st (from its CUDA graph when asked).
int batch_launch(Batch* B, cudaStream_t st)
{
    if (B->total_units == 0) return TL_OK;
    if (!(B->flags & TL_BATCH_GRAPH)) {
        int rc = enqueue(B, st);
        if (rc == TL_OK) count_launches(1);
        return rc;
    }
    if (!B->exec || B->graph_stream != st) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (B->graph) cudaGraphDestroy(B->graph);
        B->exec = nullptr;
        B->graph = nullptr;
        // capture on a private stream, then launch the graph on the caller's
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return TL_ECUDA;
        cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int rc = enqueue(B, cap);
        cudaError_t e = cudaStreamEndCapture(cap, &B->graph);
        cudaStreamDestroy(cap);
        if (rc || e != cudaSuccess) return TL_ECUDA;
        if (cudaGraphInstantiate(&B->exec, B->graph, 0) != cudaSuccess) return TL_ECUDA;
        B->graph_stream = st;
    }
    if (cudaGraphLaunch(B->exec, st) != cudaSuccess) return TL_ECUDA;
    count_launches(1);
    return TL_OK;
}

int batch_destroy(Batch* B)
{
    if (!B) return TL_OK;
    if (B->side) {
        cudaStreamSynchronize(B->side);
        cudaStreamDestroy(B->side);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->join) cudaEventDestroy(B->join);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->dev_ops) cudaFree(B->dev_ops);
    if (B->counter) cudaFree(B->counter);
    delete B;
    return TL_OK;
}

size_t batch_bytes(const Batch* B) { return B ? B->bytes : 0; }

int batch_set_variant(Batch* B, int32_t kind, int32_t variant, int64_t unit, void* stream)
{
    if (!B || unit < 1) return TL_EINVAL;
    const bool ok_kind =
        (kind == TL_OP_TTV && (variant == BV_TTV_COL || variant == BV_TTV_ROW4 ||
                               variant == BV_TTV_ROW8 || variant == BV_TTV_ROW32 ||
                               variant == BV_TTV_VEC)) ||
        (kind == TL_OP_TTM &&
         (variant == BV_TTM_32 || variant == BV_TTM_64 || variant == BV_TTM_SMALL)) ||
        (kind == TL_OP_ENTRYWISE && variant == BV_EW);
    if (!ok_kind) return TL_EINVAL;
    if (kind == TL_OP_TTM && variant != BV_TTM_SMALL) {   // whole row tiles
        const int64_t bm = variant == BV_TTM_32 ? 32 : 64;
        unit = (unit + bm - 1) / bm * bm;
    }
    if (variant == BV_TTV_VEC) unit = (unit + 3) / 4 * 4;   // whole vectors per unit
    for (BOp& b : B->host)
        if (b.kind == kind && (variant != BV_TTM_SMALL || small_ttm_host(b)) &&
            (variant != BV_TTV_VEC || vec_ttv_host(b))) {
            b.variant = variant;
            b.unit = unit;
        }
    int64_t u = 0;
    for (BOp& b : B->host) {
        b.ubegin = u;
        u += units_of(b);
    }
    B->total_units = u;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    if (B->host.empty()) return TL_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(B->dev_ops, B->host.data(), sizeof(BOp) * B->host.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TL_ECUDA;
    return TL_OK;
}

int batch_describe(const Batch* B, char* buf, size_t len)
{
    if (!B || !buf || !len) return TL_EINVAL;
    int hist[16] = {0};
    // operations whose recorded unit does not fit them (a cached choice that
    // escaped sanitize); the device-side checks are the second guard
    int unfit = 0;
    for (const BOp& b : B->host) {
        hist[b.variant & 15]++;
        const Candidate c{b.variant, b.unit};
        const Candidate s = sanitize(c, b);
        if (s.variant != c.variant || s.unit != c.unit) ++unfit;
    }
    std::snprintf(buf, len,
                  "{\"ops\":%zu,\"direct\":%d,\"units\":%lld,\"grid\":%d,\"bytes\":%zu,"
                  "\"unfit\":%d,"
                  "\"variants\":{\"ttv_col\":%d,\"ttv_row4\":%d,\"ttv_row8\":%d,\"ttv_row32\":%d,"
                  "\"ttm32\":%d,\"ttm64\":%d,\"ew\":%d,\"ttm_small\":%d,\"ttv_vec\":%d}}",
                  B->host.size(), B->direct, (long long)B->total_units, grid_size(), B->bytes, unfit,
                  hist[0], hist[1], hist[2], hist[3], hist[4], hist[5], hist[6], hist[7], hist[8]);
    return TL_OK;
}

// ------------------------------------------------------------------ slots --

struct Slot {
    size_t cap = 0;
    BOp* dev = nullptr;
    BOp* pinned = nullptr;
    unsigned long long* counter = nullptr;
};

Slot* slot_create(size_t capacity)
{
    Slot* s = new Slot();
    s->cap = capacity;
    if (cudaMalloc(&s->dev, sizeof(BOp) * capacity) != cudaSuccess ||
        cudaMallocHost(&s->pinned, sizeof(BOp) * capacity) != cudaSuccess ||
        cudaMalloc(&s->counter, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        slot_destroy(s);
        return nullptr;
    }
    return s;
}

void slot_destroy(Slot* s)
{
    if (!s) return;
    if (s->dev) cudaFree(s->dev);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->counter) cudaFree(s->counter);
    delete s;
}

int slot_launch(Slot* s, const tl_op* const* ops, size_t n, cudaStream_t st)
{
    size_t m = 0, bytes = 0;
    int64_t units = 0;
    int rc = TL_OK;
    for (size_t i = 0; i < n && rc == TL_OK; ++i) {
        BOp b;
        bool direct = false;
        rc = fill_op(*ops[i], b, bytes, direct);
        if (rc) break;
        if (direct || !s || m == s->cap) {
            const tl_op& o = *ops[i];
            if (o.kind == TL_OP_TTV) rc = tl_ttv(&o.A, o.vec, o.incb, o.q, &o.C, o.accumulate, st);
            else if (o.kind == TL_OP_TTM)
                rc = tl_ttm(&o.A, o.vec, o.J, o.ldb_row, o.ldb_col, o.q, &o.C, o.precision,
                            o.accumulate, st);
            else
                rc = tl_entrywise(o.entry_op, &o.A,
                                  (o.entry_op == TL_COPY || o.entry_op == TL_SCALE) ? nullptr : &o.B,
                                  o.alpha, &o.C, st);
            continue;
        }
        if (b.count == 0) continue;
        Candidate c = heuristic(b);
        {
            std::lock_guard<std::mutex> lk(g_tune.mu);
            if (g_tune.loaded) {
                auto it = g_tune.table.find(device_tag() + "|" + class_key(b));
                if (it != g_tune.table.end()) c = sanitize(it->second, b);
            }
        }
        b.variant = c.variant;
        b.unit = c.unit;
        b.ubegin = units;
        units += units_of(b);
        s->pinned[m++] = b;
    }
    if (rc) return rc;
    if (m == 0 || !s) return TL_OK;
    if (cudaMemcpyAsync(s->dev, s->pinned, sizeof(BOp) * m, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(s->counter, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return TL_ECUDA;
    batch_kernel<<<grid_size(), kThreads, 0, st>>>(s->dev, (int)m, units, s->counter);
    if (cudaGetLastError() != cudaSuccess) return TL_ECUDA;
    count_launches(1);
    return TL_OK;
}

long long op_bytes(const tl_op& o)
{
    BOp b;
    size_t bytes = 0;
    bool direct = false;
    int rc = fill_op(o, b, bytes, direct);
    return rc ? (long long)rc : (long long)bytes;
}

}  // namespace tl

using namespace tl;

extern "C" {

int tl_batch_create(const tl_op* ops, size_t count, int32_t flags, void* stream, tl_batch** out)
{
    return batch_create(ops, count, flags, stream, reinterpret_cast<Batch**>(out));
}

int tl_batch_run(tl_batch* b, void* stream)
{
    NvtxRange nvtx_range("tl_batch_run");
    return batch_run(reinterpret_cast<Batch*>(b), stream);
}

int tl_batch_destroy(tl_batch* b) { return batch_destroy(reinterpret_cast<Batch*>(b)); }

int tl_batch_set_variant(tl_batch* b, int32_t kind, int32_t variant, int64_t unit, void* stream)
{
    return batch_set_variant(reinterpret_cast<Batch*>(b), kind, variant, unit, stream);
}

int tl_batch_describe(const tl_batch* b, char* buf, size_t len)
{
    return batch_describe(reinterpret_cast<const Batch*>(b), buf, len);
}

}  // extern "C"
