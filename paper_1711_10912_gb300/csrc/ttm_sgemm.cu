// ttm_sgemm.cu -- FP32 mode-q tensor-times-matrix on the FMA pipes, Sec. 5.2
// Eq. 25:  C(i with i_q = j) = sum_{k < n_q} A(i with i_q = k) * B(j, k).
//
// As in ttm_simt.cu, the modes other than q are collapsed into M rows (each
// with its own A and C offset from the layout function, Eq. 17), so the call
// is one M x J x n_q matrix product.  This kernel is the FP32 one, built for
// the FMA issue rate:
//  - one CTA of 256 threads per SM computes a 128 x 256 (rows x j) tile when
//    J > 128, a 256 x 128 tile when 64 < J <= 128, and a 512 x 64 tile when
//    J <= 64 (no idle columns for small J); each thread holds an 8 x 16,
//    16 x 8 or 32 x 4 block of outputs in registers, built from 4 x 4
//    sub-blocks 64 apart so that its operands are 16-byte shared-memory
//    reads.  Each k step then reads 24 floats per thread for 128 FMAs (36
//    for the 512 x 64 tile): the SM's shared-memory port (32 lanes x 4 bytes
//    per cycle) delivers them in 3/4 of the time the FMA pipes (128 lanes per
//    cycle) take, where an 8 x 8 block would need all of it;
//  - k advances in slabs of 16: the next slab's A and B tiles are loaded from
//    global memory into registers while the current slab is multiplied out
//    of shared memory, then stored into the second of two shared-memory
//    buffers (one barrier per slab);
//  - A and B are read with 16-byte loads along whichever index is contiguous
//    (k, or four consecutive rows / columns) and stored k-major into shared
//    memory, padded so that the transposing stores do not conflict;
//  - C is written with 16-byte stores along j or along rows when the layout
//    allows it, else element by element;
//  - tiles are numbered with j fastest, so the CTAs in flight at one time
//    share their rows of A through L2;
//  - when the tiles cannot fill the GPU and n_q is long, k is split across
//    CTAs into a workspace, added in order by ttm_splitk_reduce (ttm_simt.cu).
#include <cuda_runtime.h>

#include <string>

#include "device.cuh"
#include "kernels.h"
#include "runtime.h"

namespace tl {

namespace {

constexpr int kThreads = 256;
constexpr int BK = 16;  // k per slab

// how an operand slab (rows x BK) is read from global memory
enum : int {
    LD_K4 = 0,      // 16-byte vectors along k (k contiguous)
    LD_R4 = 1,      // 16-byte vectors along four contiguous rows
    LD_SCALAR = 2,  // element loads (k or rows fastest across threads)
};
// how the output tile is written
enum : int {
    ST_J4 = 0,      // 16-byte vectors along j
    ST_M4 = 1,      // 16-byte vectors along rows
    ST_SCALAR = 2,
    ST_WS4 = 3,     // split-K partials ws[s][m][j], 16-byte vectors along j
    ST_WS1 = 4,     // split-K partials, element stores
};

struct SgArgs {
    const float* A;
    const float* B;
    float* C;
    float* ws;
    DevSpace rows;      // operands 0 = A, 1 = C
    int64_t M, J, nq, saq, scq, ldb_row, ldb_col;
    int64_t tiles_m, tiles_j, splits, kchunk;
    int bmode, cmode, accumulate;
};

// One operand slab of NR rows x BK k values, staged through registers: the
// NR * BK / 256 elements this thread moves.  Row i of the tile starts at
// base + rowoff(i); k steps by sk.
template <int MODE, int NR>
struct Slab {
    static constexpr int kElems = NR * BK / kThreads;   // 8 or 16
    float r[kElems];

    // LD_K4: vector v of this thread holds row k4_row(v), k = k4_k(v)..+3.
    // Each pass covers 128 rows (two threads per row, 8 k values apart from
    // the next pass's pair), so a warp's transposing stores touch rows 4
    // banks apart at two k values 4 apart: 32 distinct banks.  A 64-row slab
    // takes four threads per row instead (one pass covers its 64 rows x 16 k).
    static constexpr int kTpr = NR >= 128 ? 2 : 4;       // threads per row in a pass
    static_assert(NR >= 64 && NR % (kThreads / kTpr) == 0, "LD_K4 slab rows");
    __device__ __forceinline__ static int k4_row(int v)
    {
        return (v / (BK / (4 * kTpr))) * (kThreads / kTpr) + (int)threadIdx.x / kTpr;
    }
    __device__ __forceinline__ static int k4_k(int v)
    {
        return (v % (BK / (4 * kTpr))) * (4 * kTpr) + ((int)threadIdx.x % kTpr) * 4;
    }

    template <typename RowOff>
    __device__ __forceinline__ void load(const float* __restrict__ base, const RowOff& rowoff,
                                         int64_t sk, int nvalid, int k0, int kend, bool kfast)
    {
        const int tid = threadIdx.x;
        if constexpr (MODE == LD_K4) {
#pragma unroll
            for (int v = 0; v < kElems / 4; ++v) {
                const int i = k4_row(v), k = k0 + k4_k(v);
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < nvalid && k < kend)
                    x = __ldg(reinterpret_cast<const float4*>(base + rowoff(i) + k));
                r[4 * v] = x.x; r[4 * v + 1] = x.y; r[4 * v + 2] = x.z; r[4 * v + 3] = x.w;
            }
        } else if constexpr (MODE == LD_R4) {
#pragma unroll
            for (int v = 0; v < kElems / 4; ++v) {
                const int f = tid + v * kThreads;
                const int i = (f % (NR / 4)) * 4, k = k0 + f / (NR / 4);
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < nvalid && k < kend)
                    x = __ldg(reinterpret_cast<const float4*>(base + rowoff(i) + (int64_t)k * sk));
                r[4 * v] = x.x; r[4 * v + 1] = x.y; r[4 * v + 2] = x.z; r[4 * v + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < kElems; ++u) {
                const int e = tid + u * kThreads;
                const int i = kfast ? e / BK : e % NR;
                const int k = k0 + (kfast ? e % BK : e / NR);
                r[u] = (i < nvalid && k < kend) ? __ldg(base + rowoff(i) + (int64_t)k * sk) : 0.f;
            }
        }
    }

    // into the k-major shared tile t[k * ld + row] (ld = NR + 4: the padded
    // rows are 4 banks apart, so the transposing stores of a warp are
    // conflict-free)
    __device__ __forceinline__ void store(float* t, bool kfast) const
    {
        constexpr int ld = NR + 4;
        const int tid = threadIdx.x;
        if constexpr (MODE == LD_K4) {
#pragma unroll
            for (int v = 0; v < kElems / 4; ++v) {
                const int i = k4_row(v), kq = k4_k(v);
#pragma unroll
                for (int u = 0; u < 4; ++u) t[(kq + u) * ld + i] = r[4 * v + u];
            }
        } else if constexpr (MODE == LD_R4) {
#pragma unroll
            for (int v = 0; v < kElems / 4; ++v) {
                const int f = tid + v * kThreads;
                const int i = (f % (NR / 4)) * 4, kk = f / (NR / 4);
                *reinterpret_cast<float4*>(t + kk * ld + i) =
                    make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < kElems; ++u) {
                const int e = tid + u * kThreads;
                const int i = kfast ? e / BK : e % NR;
                const int kk = kfast ? e % BK : e / NR;
                t[kk * ld + i] = r[u];
            }
        }
    }
};

// A CTA computes a (64 RM4) x (64 RN4) tile of C; thread (tx, ty) of a 16 x
// 16 grid owns rows tx*4 + 64a + {0..3} (a < RM4) and columns ty*4 + 64b +
// {0..3} (b < RN4): 4 RM4 x 4 RN4 outputs in registers.  Per k step it reads
// RM4 + RN4 16-byte vectors from shared memory for 16 RM4 RN4 FMAs, so
// shared-memory bandwidth stays below the FMA rate when RM4 * RN4 >= 8.
template <int AMODE, int BMODE, int RM4, int RN4>
__global__ void __launch_bounds__(kThreads, 1) ttm_sgemm_kernel(const SgArgs a)
{
    constexpr int TM = 64 * RM4, TN = 64 * RN4;
    constexpr int LDA = TM + 4, LDB = TN + 4;
    extern __shared__ __align__(16) float sg_tiles[];   // A[2][BK][LDA], then B[2][BK][LDB]
    float* const As = sg_tiles;
    float* const Bs = sg_tiles + 2 * BK * LDA;
    __shared__ int64_t offA[TM], offC[TM];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // a warp covers 8 row groups x 4 column groups: its A reads are 128
    // contiguous bytes and its B reads 64, both broadcast across the warp
    const int tx = (warp & 1) * 8 + (lane & 7);
    const int ty = (warp >> 1) * 4 + (lane >> 3);
    const bool akf = a.saq == 1, bkf = a.ldb_col == 1;
    const int64_t ntiles = a.tiles_m * a.tiles_j;
    for (int64_t w = blockIdx.x; w < ntiles * a.splits; w += gridDim.x) {
        const int64_t tile = w % ntiles, split = w / ntiles;
        const int64_t j0 = (tile % a.tiles_j) * TN;
        const int64_t m0 = (tile / a.tiles_j) * TM;
        const int64_t kb = split * a.kchunk;
        const int kn = (int)(min(a.nq, kb + a.kchunk) - kb);   // < 2^30 by the split rule
        const int mvalid = (int)min((int64_t)TM, a.M - m0);
        const int jvalid = (int)min((int64_t)TN, a.J - j0);
        __syncthreads();   // the previous tile is done with offA / offC and the slabs
        for (int i = tid; i < TM; i += kThreads) {
            int64_t off[2] = {0, 0};
            if (i < mvalid) map_offsets<2>(a.rows, m0 + i, 1, off);
            offA[i] = off[0];
            offC[i] = off[1];
        }
        __syncthreads();
        const float* pa = a.A + kb * a.saq;
        const float* pb = a.B + j0 * a.ldb_row + kb * a.ldb_col;
        auto rowA = [&](int i) { return offA[i]; };
        auto rowB = [&](int i) { return (int64_t)i * a.ldb_row; };
        float acc[4 * RM4][4 * RN4];
#pragma unroll
        for (int i = 0; i < 4 * RM4; ++i)
#pragma unroll
            for (int j = 0; j < 4 * RN4; ++j) acc[i][j] = 0.f;
        Slab<AMODE, TM> sa;
        Slab<BMODE, TN> sb;
        sa.load(pa, rowA, a.saq, mvalid, 0, kn, akf);
        sb.load(pb, rowB, a.ldb_col, jvalid, 0, kn, bkf);
        sa.store(As, akf);
        sb.store(Bs, bkf);
        __syncthreads();
        for (int k0 = 0, buf = 0; k0 < kn; k0 += BK, buf ^= 1) {
            const bool more = k0 + BK < kn;
            if (more) {
                sa.load(pa, rowA, a.saq, mvalid, k0 + BK, kn, akf);
                sb.load(pb, rowB, a.ldb_col, jvalid, k0 + BK, kn, bkf);
            }
            const float* at = As + buf * (BK * LDA);
            const float* bt = Bs + buf * (BK * LDB);
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float av[4 * RM4], bv[4 * RN4];
#pragma unroll
                for (int g = 0; g < RM4; ++g) {
                    const float4 x = *reinterpret_cast<const float4*>(at + kk * LDA + 64 * g + tx * 4);
                    av[4 * g] = x.x; av[4 * g + 1] = x.y; av[4 * g + 2] = x.z; av[4 * g + 3] = x.w;
                }
#pragma unroll
                for (int g = 0; g < RN4; ++g) {
                    const float4 x = *reinterpret_cast<const float4*>(bt + kk * LDB + 64 * g + ty * 4);
                    bv[4 * g] = x.x; bv[4 * g + 1] = x.y; bv[4 * g + 2] = x.z; bv[4 * g + 3] = x.w;
                }
#pragma unroll
                for (int i = 0; i < 4 * RM4; ++i)
#pragma unroll
                    for (int j = 0; j < 4 * RN4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            if (more) {
                sa.store(As + (buf ^ 1) * (BK * LDA), akf);
                sb.store(Bs + (buf ^ 1) * (BK * LDB), bkf);
            }
            __syncthreads();
        }
        // epilogue: acc[i][j] is row 64 (i / 4) + 4 tx + i % 4 and column
        // 64 (j / 4) + 4 ty + j % 4 of the tile
        if (a.cmode == ST_J4 || a.cmode == ST_WS4) {
#pragma unroll
            for (int i = 0; i < 4 * RM4; ++i) {
                const int ri = 64 * (i >> 2) + tx * 4 + (i & 3);
                if (ri >= mvalid) continue;
#pragma unroll
                for (int h = 0; h < RN4; ++h) {
                    const int cj = 64 * h + ty * 4;
                    if (cj >= jvalid) continue;
                    float4 v = make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2],
                                           acc[i][4 * h + 3]);
                    float* p = a.cmode == ST_WS4 ? a.ws + (split * a.M + m0 + ri) * a.J + j0 + cj
                                                 : a.C + offC[ri] + j0 + cj;
                    if (a.accumulate && a.cmode == ST_J4) {
                        const float4 c = *reinterpret_cast<const float4*>(p);
                        v.x += c.x; v.y += c.y; v.z += c.z; v.w += c.w;
                    }
                    *reinterpret_cast<float4*>(p) = v;
                }
            }
        } else if (a.cmode == ST_M4) {
#pragma unroll
            for (int j = 0; j < 4 * RN4; ++j) {
                const int cj = 64 * (j >> 2) + ty * 4 + (j & 3);
                if (cj >= jvalid) continue;
#pragma unroll
                for (int h = 0; h < RM4; ++h) {
                    const int ri = 64 * h + tx * 4;
                    if (ri >= mvalid) continue;
                    float4 v = make_float4(acc[4 * h][j], acc[4 * h + 1][j], acc[4 * h + 2][j],
                                           acc[4 * h + 3][j]);
                    float* p = a.C + offC[ri] + (j0 + cj) * a.scq;
                    if (a.accumulate) {
                        const float4 c = *reinterpret_cast<const float4*>(p);
                        v.x += c.x; v.y += c.y; v.z += c.z; v.w += c.w;
                    }
                    *reinterpret_cast<float4*>(p) = v;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4 * RM4; ++i) {
                const int ri = 64 * (i >> 2) + tx * 4 + (i & 3);
                if (ri >= mvalid) continue;
#pragma unroll
                for (int j = 0; j < 4 * RN4; ++j) {
                    const int cj = 64 * (j >> 2) + ty * 4 + (j & 3);
                    if (cj >= jvalid) continue;
                    if (a.cmode == ST_WS1) {
                        a.ws[(split * a.M + m0 + ri) * a.J + j0 + cj] = acc[i][j];
                    } else {
                        float* p = a.C + offC[ri] + (j0 + cj) * a.scq;
                        *p = a.accumulate ? *p + acc[i][j] : acc[i][j];
                    }
                }
            }
        }
    }
}

bool all_multiple(const Space& sp, int op, int64_t v, int from)
{
    for (int d = from; d < sp.nd; ++d)
        if (sp.d[d].s[op] % v) return false;
    return true;
}

}  // namespace

int sgemm_amode(const TtmPlan& P, const void* A)
{
    const bool al = aligned(A, 16);
    if (P.saq == 1 && P.nq % 4 == 0 && al && all_multiple(P.rows, 0, 4, 0)) return LD_K4;
    if (P.rows.nd >= 1 && P.rows.d[0].s[0] == 1 && P.rows.d[0].n % 4 == 0 && P.saq % 4 == 0 &&
        al && all_multiple(P.rows, 0, 4, 1))
        return LD_R4;
    return LD_SCALAR;
}

int sgemm_bmode(const TtmPlan& P, const void* B)
{
    if (P.ldb_col == 1 && P.ldb_row % 4 == 0 && P.nq % 4 == 0 && aligned(B, 16)) return LD_K4;
    return LD_SCALAR;
}

// 128 x 256 tiles when J spans more than 128 columns, 512 x 64 when it spans
// at most 64, else 256 x 128
bool sgemm_wide(const TtmPlan& P) { return P.J > 128; }
bool sgemm_thin(const TtmPlan& P) { return P.J <= 64; }

void sgemm_tile(const TtmPlan& P, int64_t& tm, int64_t& tn)
{
    tm = sgemm_wide(P) ? 128 : sgemm_thin(P) ? 512 : 256;
    tn = sgemm_wide(P) ? 256 : sgemm_thin(P) ? 64 : 128;
}

int sgemm_cmode(const TtmPlan& P, const void* C, bool split)
{
    if (split) return P.J % 4 == 0 ? ST_WS4 : ST_WS1;
    const bool al = aligned(C, 16);
    if (P.scq == 1 && P.J % 4 == 0 && al && all_multiple(P.rows, 1, 4, 0)) return ST_J4;
    if (P.rows.nd >= 1 && P.rows.d[0].s[1] == 1 && P.rows.d[0].n % 4 == 0 && P.scq % 4 == 0 &&
        al && all_multiple(P.rows, 1, 4, 1))
        return ST_M4;
    return ST_SCALAR;
}

std::string ttm_sgemm_describe(const TtmPlan& P, const void* A, const void* C, bool split)
{
    static const char* ld[] = {"k4", "r4", "scalar"};
    static const char* stn[] = {"j4", "m4", "scalar", "ws4", "ws1"};
    // the matrix is taken as row-major (ldb_row = n_q, ldb_col = 1) when the
    // plan has no strides for it, and as 16-byte aligned (allocator pointers are)
    alignas(16) static const float aligned_b[4] = {0.f, 0.f, 0.f, 0.f};
    TtmPlan Q = P;
    if (Q.ldb_row == 0 && Q.ldb_col == 0) {
        Q.ldb_row = Q.nq;
        Q.ldb_col = 1;
    }
    return std::string("{\"a\":\"") + ld[sgemm_amode(P, A)] + "\",\"b\":\"" +
           ld[sgemm_bmode(Q, aligned_b)] + "\",\"c\":\"" + stn[sgemm_cmode(P, C, split)] +
           "\",\"tile\":[" + (sgemm_wide(P) ? "128,256" : sgemm_thin(P) ? "512,64" : "256,128") + "]}";
}

int64_t sgemm_tiles(const TtmPlan& P)
{
    int64_t tm, tn;
    sgemm_tile(P, tm, tn);
    return ((P.M + tm - 1) / tm) * ((P.J + tn - 1) / tn);
}

int launch_ttm_sgemm(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate,
                     void* ws, int64_t splits, int64_t kchunk, int num_sms, cudaStream_t st)
{
    const bool wide = sgemm_wide(P), thin = sgemm_thin(P);
    int64_t tm, tn;
    sgemm_tile(P, tm, tn);
    SgArgs a{};
    a.A = static_cast<const float*>(A);
    a.B = static_cast<const float*>(B);
    a.C = static_cast<float*>(C);
    a.ws = static_cast<float*>(ws);
    a.rows = to_dev(P.rows);
    a.M = P.M;
    a.J = P.J;
    a.nq = P.nq;
    a.saq = P.saq;
    a.scq = P.scq;
    a.ldb_row = P.ldb_row;
    a.ldb_col = P.ldb_col;
    a.tiles_m = (P.M + tm - 1) / tm;
    a.tiles_j = (P.J + tn - 1) / tn;
    a.splits = splits;
    a.kchunk = splits > 1 ? kchunk : P.nq;
    const int amode = sgemm_amode(P, A);
    a.bmode = sgemm_bmode(P, B);
    a.cmode = sgemm_cmode(P, C, splits > 1);
    a.accumulate = accumulate;
    if (splits > 1 && !ws) return TL_ENOMEM;
    const int64_t work = a.tiles_m * a.tiles_j * splits;
    const int64_t cap = num_sms;   // one CTA of 256 threads per SM (up to 255 registers each)
    const int grid = (int)(work < cap ? work : cap);
    if (grid <= 0) return TL_OK;
    using KernelFn = void (*)(SgArgs);
    static const KernelFn wide_k[3][2] = {
        {ttm_sgemm_kernel<LD_K4, LD_K4, 2, 4>, ttm_sgemm_kernel<LD_K4, LD_SCALAR, 2, 4>},
        {ttm_sgemm_kernel<LD_R4, LD_K4, 2, 4>, ttm_sgemm_kernel<LD_R4, LD_SCALAR, 2, 4>},
        {ttm_sgemm_kernel<LD_SCALAR, LD_K4, 2, 4>, ttm_sgemm_kernel<LD_SCALAR, LD_SCALAR, 2, 4>},
    };
    static const KernelFn tall_k[3][2] = {
        {ttm_sgemm_kernel<LD_K4, LD_K4, 4, 2>, ttm_sgemm_kernel<LD_K4, LD_SCALAR, 4, 2>},
        {ttm_sgemm_kernel<LD_R4, LD_K4, 4, 2>, ttm_sgemm_kernel<LD_R4, LD_SCALAR, 4, 2>},
        {ttm_sgemm_kernel<LD_SCALAR, LD_K4, 4, 2>, ttm_sgemm_kernel<LD_SCALAR, LD_SCALAR, 4, 2>},
    };
    static const KernelFn thin_k[3][2] = {
        {ttm_sgemm_kernel<LD_K4, LD_K4, 8, 1>, ttm_sgemm_kernel<LD_K4, LD_SCALAR, 8, 1>},
        {ttm_sgemm_kernel<LD_R4, LD_K4, 8, 1>, ttm_sgemm_kernel<LD_R4, LD_SCALAR, 8, 1>},
        {ttm_sgemm_kernel<LD_SCALAR, LD_K4, 8, 1>, ttm_sgemm_kernel<LD_SCALAR, LD_SCALAR, 8, 1>},
    };
    const int bi = a.bmode == LD_K4 ? 0 : 1;
    const KernelFn fn = wide ? wide_k[amode][bi] : thin ? thin_k[amode][bi] : tall_k[amode][bi];
    // double-buffered A and B slabs, rows padded by 4 floats
    const size_t smem = (size_t)2 * BK * ((tm + 4) + (tn + 4)) * sizeof(float);
    if (smem_optin(reinterpret_cast<const void*>(fn), (int)smem) != TL_OK) return TL_ECUDA;
    fn<<<grid, kThreads, smem, st>>>(a);
    return TL_OK;
}

}  // namespace tl
