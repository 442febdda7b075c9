// device.cuh -- small device helpers shared by the kernels: the offset mapper
// (linear index -> per-operand element offsets, the layout function of Sec. 3.2
// Eq. 17 applied to a collapsed iteration space) and 16-byte vector types.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdlib>

#include "plan.h"

namespace tl {

// Registers a reader of one file's bounds-violation word (bounds-checked
// builds); tl_device_status() calls every reader.
int register_bounds_reader(int (*reader)(bool clear));

#ifdef TL_CHECK_BOUNDS
// Bounds-checked build: each file that includes this header has its own word
// (no relocatable device code), holding 1 + the first offending offset.
static __device__ unsigned long long g_bounds_bad = 0;

__device__ __forceinline__ void bounds_record(int64_t off)
{
    atomicCAS(&g_bounds_bad, 0ull, 1ull + ((unsigned long long)off & 0x7fffffffffffffffull));
}

namespace {
int bounds_read(bool clear)
{
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_bad, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return TL_ECUDA;
    }
    if (v && clear) {
        const unsigned long long zero = 0;
        cudaMemcpyToSymbol(g_bounds_bad, &zero, sizeof zero);
    }
    return v ? TL_EBOUNDS : TL_OK;
}
[[maybe_unused]] const int g_bounds_registered = register_bounds_reader(&bounds_read);
}  // namespace

// Checked builds: TL_DEBUG_SHRINK_LIMITS set in the environment halves every
// limit handed to a kernel, so that in-range accesses are reported (and
// skipped) -- a way to show the check works without touching memory out of
// range.
inline int64_t debug_limit(int64_t lim)
{
    static const bool shrink = std::getenv("TL_DEBUG_SHRINK_LIMITS") != nullptr;
    return shrink && lim > 1 ? lim / 2 : lim;
}
#else
inline int64_t debug_limit(int64_t lim) { return lim; }
#endif

// Collapsed iteration space as kernel parameters: dims[0] varies fastest.
// small != 0 when every linear index fits in 31 bits, so the mapper can use
// 32-bit division.
struct DevSpace {
    int nd;
    int small;
    int64_t n[kMaxDims];
    int64_t s[3][kMaxDims];
    int64_t limit[3];   // see Space::limit (checked builds)
};

inline DevSpace to_dev(const Space& sp)
{
    DevSpace d{};
    d.nd = sp.nd;
    for (int i = 0; i < sp.nd; ++i) {
        d.n[i] = sp.d[i].n;
        for (int o = 0; o < 3; ++o) d.s[o][i] = sp.d[i].s[o];
    }
    d.small = sp.count() < (int64_t(1) << 31) ? 1 : 0;
    for (int o = 0; o < 3; ++o) d.limit[o] = debug_limit(sp.limit[o]);
    return d;
}

// Bounds-checked builds: an offset whose addressed elements (a vector of
// `vec0` along dim 0) fall outside the operand's limit is recorded and
// replaced by 0; product builds compile this away.
template <int NOPS>
__device__ __forceinline__ void check_offsets(const DevSpace& sp, int64_t vec0, int64_t* off)
{
#ifdef TL_CHECK_BOUNDS
#pragma unroll
    for (int o = 0; o < NOPS; ++o) {
        const int64_t last = off[o] + (vec0 - 1) * (sp.nd > 0 ? sp.s[o][0] : 0);
        if (sp.limit[o] > 0 && (off[o] < 0 || last >= sp.limit[o])) {
            bounds_record(off[o]);
            off[o] = 0;
        }
    }
#endif
}

// Bounds-checked builds: operand o's access of `vec` contiguous elements at
// `off` (kernels that compute their own offsets) is checked against the
// operand's limit, recorded and redirected to 0 when outside; product builds
// return `off` unchanged.
__device__ __forceinline__ int64_t checked_off(const DevSpace& sp, int o, int64_t off, int vec)
{
#ifdef TL_CHECK_BOUNDS
    if (sp.limit[o] > 0 && (off < 0 || off + vec - 1 >= sp.limit[o])) {
        bounds_record(off);
        return 0;
    }
#else
    (void)sp;
    (void)o;
    (void)vec;
#endif
    return off;
}

// Offsets of linear index g for operands 0..NOPS-1.  dim 0 is taken in units
// of `vec0` elements (g counts vectors along dim 0); the last dim needs no
// division because g is already below its extent.
template <int NOPS>
__device__ __forceinline__ void map_offsets(const DevSpace& sp, int64_t g, int64_t vec0,
                                            int64_t* off)
{
#pragma unroll
    for (int o = 0; o < NOPS; ++o) off[o] = 0;
    if (sp.small) {
        uint32_t gs = (uint32_t)g;
        for (int d = 0; d < sp.nd; ++d) {
            uint32_t ext = (uint32_t)(d == 0 ? sp.n[0] / vec0 : sp.n[d]);
            uint32_t i;
            if (d == sp.nd - 1) {
                i = gs;
            } else {
                uint32_t qd = gs / ext;
                i = gs - qd * ext;
                gs = qd;
            }
            int64_t ii = d == 0 ? (int64_t)i * vec0 : (int64_t)i;
#pragma unroll
            for (int o = 0; o < NOPS; ++o) off[o] += ii * sp.s[o][d];
        }
        check_offsets<NOPS>(sp, vec0, off);
        return;
    }
    for (int d = 0; d < sp.nd; ++d) {
        int64_t ext = d == 0 ? sp.n[0] / vec0 : sp.n[d];
        int64_t i;
        if (d == sp.nd - 1) {
            i = g;
        } else {
            int64_t qd = g / ext;
            i = g - qd * ext;
            g = qd;
        }
        if (d == 0) i *= vec0;
#pragma unroll
        for (int o = 0; o < NOPS; ++o) off[o] += i * sp.s[o][d];
    }
    check_offsets<NOPS>(sp, vec0, off);
}

// Quotient of a 32-bit index by an invariant divisor (FastDiv, plan.h).
__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f)
{
    const uint32_t t = __umulhi(f.mul, n);
    return (t + ((n - t) >> f.sh1)) >> f.sh2;
}

// Division tables of a collapsed space whose linear indices fit in 31 bits
// (DevSpace::small): fd[d] divides by dim d's extent, dim 0 counted in
// vectors of `vec0` elements.
struct DevDiv {
    FastDiv fd[kMaxDims];
    uint32_t ext[kMaxDims];
};

inline DevDiv make_devdiv(const Space& sp, int64_t vec0)
{
    DevDiv v{};
    for (int d = 0; d < sp.nd; ++d) {
        const int64_t ext = d == 0 ? sp.d[0].n / vec0 : sp.d[d].n;
        v.ext[d] = (uint32_t)(ext > 0 && ext < (int64_t(1) << 32) ? ext : 1);
        v.fd[d] = make_fastdiv(v.ext[d]);
    }
    return v;
}

// map_offsets with multiply-high division for spaces with 31-bit indices;
// others take the 64-bit path of map_offsets.
template <int NOPS>
__device__ __forceinline__ void map_offsets_fast(const DevSpace& sp, const DevDiv& dv, int64_t g,
                                                 int64_t vec0, int64_t* off)
{
    if (!sp.small) {
        map_offsets<NOPS>(sp, g, vec0, off);
        return;
    }
#pragma unroll
    for (int o = 0; o < NOPS; ++o) off[o] = 0;
    uint32_t r = (uint32_t)g;
    for (int d = 0; d < sp.nd; ++d) {
        uint32_t i = r;
        if (d < sp.nd - 1) {
            const uint32_t qd = fast_div(r, dv.fd[d]);
            i = r - qd * dv.ext[d];
            r = qd;
        }
        const int64_t ii = d == 0 ? (int64_t)i * vec0 : (int64_t)i;
#pragma unroll
        for (int o = 0; o < NOPS; ++o) off[o] += ii * sp.s[o][d];
    }
    check_offsets<NOPS>(sp, vec0, off);
}

// map_offsets_fast for a space of exactly ND dims with 31-bit indices: the
// decode unrolls and reads its tables at fixed offsets.
template <int ND, int NOPS>
__device__ __forceinline__ void map_offsets_nd(const DevSpace& sp, const DevDiv& dv, int64_t g,
                                               int64_t vec0, int64_t* off)
{
#pragma unroll
    for (int o = 0; o < NOPS; ++o) off[o] = 0;
    uint32_t r = (uint32_t)g;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        uint32_t i = r;
        if (d < ND - 1) {
            const uint32_t qd = fast_div(r, dv.fd[d]);
            i = r - qd * dv.ext[d];
            r = qd;
        }
        const int64_t ii = d == 0 ? (int64_t)i * vec0 : (int64_t)i;
#pragma unroll
        for (int o = 0; o < NOPS; ++o) off[o] += ii * sp.s[o][d];
    }
    check_offsets<NOPS>(sp, vec0, off);
}

template <typename T, int V> struct Vec;
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<float, 1> { using type = float; };
template <> struct Vec<double, 2> { using type = double2; };
template <> struct Vec<double, 1> { using type = double; };

template <typename T, int V>
__device__ __forceinline__ void vload(const T* p, T* r)
{
    if constexpr (V == 1) {
        r[0] = __ldg(p);
    } else {
        using VT = typename Vec<T, V>::type;
        VT v = __ldg(reinterpret_cast<const VT*>(p));
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) r[i] = e[i];
    }
}

// Streaming load: read-once data that should not displace L1 lines.
template <typename T, int V>
__device__ __forceinline__ void vload_stream(const T* p, T* r)
{
    if constexpr (V == 1) {
        r[0] = __ldcs(p);
    } else {
        using VT = typename Vec<T, V>::type;
        VT v = __ldcs(reinterpret_cast<const VT*>(p));
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) r[i] = e[i];
    }
}

template <typename T, int V>
__device__ __forceinline__ void vstore(T* p, const T* r)
{
    if constexpr (V == 1) {
        p[0] = r[0];
    } else {
        using VT = typename Vec<T, V>::type;
        VT v;
        T* e = reinterpret_cast<T*>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) e[i] = r[i];
        *reinterpret_cast<VT*>(p) = v;
    }
}

// One row of a row-by-matrix product (Eq. 25 with n_q small): acc[j] +=
// sum over u < NQ of a[u * sa] * b[u * ldb + j], u ascending.  All NQ loads
// of the row are issued before the first product, so a short contraction
// waits for one memory latency rather than NQ of them.
template <typename T, int JB, int NQ>
__device__ __forceinline__ void row_chunk(const T* __restrict__ a, int64_t sa, const T* b, int ldb,
                                          T* acc)
{
    T x[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) x[u] = __ldg(a + (int64_t)u * sa);
    // b's rows start at multiples of JB elements from a 16-byte aligned
    // base: 16-byte reads where JB elements fill whole vectors
    constexpr int V = 16 / (int)sizeof(T);
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
        if constexpr (JB % V == 0) {
            using VT = typename Vec<T, V>::type;
            const VT* br = reinterpret_cast<const VT*>(b + u * ldb);
#pragma unroll
            for (int c = 0; c < JB / V; ++c) {
                const VT v = br[c];
                const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
                for (int i = 0; i < V; ++i) acc[c * V + i] = fma(x[u], e[i], acc[c * V + i]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < JB; ++j) acc[j] = fma(x[u], b[u * ldb + j], acc[j]);
        }
    }
}

// The whole contraction of one row: chunks of 8, then the remainder as one
// chunk of its exact length (a warp-uniform branch on n_q).
template <typename T, int JB>
__device__ __forceinline__ void row_dot(const T* __restrict__ a, int64_t sa, int nq, const T* b,
                                        int ldb, T* acc)
{
    const int k8 = nq & ~7;
    for (int k0 = 0; k0 < k8; k0 += 8)
        row_chunk<T, JB, 8>(a + (int64_t)k0 * sa, sa, b + k0 * ldb, ldb, acc);
    const T* at = a + (int64_t)k8 * sa;
    const T* bt = b + k8 * ldb;
    switch (nq - k8) {
    case 1: row_chunk<T, JB, 1>(at, sa, bt, ldb, acc); break;
    case 2: row_chunk<T, JB, 2>(at, sa, bt, ldb, acc); break;
    case 3: row_chunk<T, JB, 3>(at, sa, bt, ldb, acc); break;
    case 4: row_chunk<T, JB, 4>(at, sa, bt, ldb, acc); break;
    case 5: row_chunk<T, JB, 5>(at, sa, bt, ldb, acc); break;
    case 6: row_chunk<T, JB, 6>(at, sa, bt, ldb, acc); break;
    case 7: row_chunk<T, JB, 7>(at, sa, bt, ldb, acc); break;
    default: break;
    }
}

// acc + sum over u < NQ of a[u * sa] * b[u * sb], u ascending, every load of
// a in the chunk issued before the first product (b, a short vector read by
// every output, comes from cache).
template <typename T, int NQ>
__device__ __forceinline__ T dot_chunk(const T* __restrict__ a, int64_t sa, const T* __restrict__ b,
                                       int64_t sb, T acc)
{
    T x[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) x[u] = __ldg(a + (int64_t)u * sa);
#pragma unroll
    for (int u = 0; u < NQ; ++u) acc = fma(x[u], __ldg(b + (int64_t)u * sb), acc);
    return acc;
}

// acc + the strided dot product of length n (Eq. 24 for one output), k
// ascending: chunks of CH, then the remainder as one chunk of its exact
// length.
template <typename T, int CH>
__device__ __forceinline__ T dot_strided(const T* __restrict__ a, int64_t sa,
                                         const T* __restrict__ b, int64_t sb, int64_t n, T acc)
{
    static_assert(CH == 4 || CH == 8, "chunk of 4 or 8");
    int64_t k = 0;
    for (; k + CH <= n; k += CH) acc = dot_chunk<T, CH>(a + k * sa, sa, b + k * sb, sb, acc);
    const T* at = a + k * sa;
    const T* bt = b + k * sb;
    switch ((int)(n - k)) {
    case 1: acc = dot_chunk<T, 1>(at, sa, bt, sb, acc); break;
    case 2: acc = dot_chunk<T, 2>(at, sa, bt, sb, acc); break;
    case 3: acc = dot_chunk<T, 3>(at, sa, bt, sb, acc); break;
    case 4: acc = dot_chunk<T, CH == 8 ? 4 : 1>(at, sa, bt, sb, acc); break;
    case 5: acc = dot_chunk<T, CH == 8 ? 5 : 1>(at, sa, bt, sb, acc); break;
    case 6: acc = dot_chunk<T, CH == 8 ? 6 : 1>(at, sa, bt, sb, acc); break;
    case 7: acc = dot_chunk<T, CH == 8 ? 7 : 1>(at, sa, bt, sb, acc); break;
    default: break;
    }
    return acc;
}

}  // namespace tl
