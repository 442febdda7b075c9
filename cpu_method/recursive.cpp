// recursive.cpp -- the plain CPU method of the TLib paper (arXiv 1711.10912):
// tensor functions that recurse over the modes of their operands, one level
// per mode, each level stepping along its mode with a stride iterator, the
// innermost level handing whole fibers to the C++ standard library:
//   cm_transform_f32  entrywise C = A op B, Sec. 5.1 Eq. 23 (std::transform
//                     on fibers of mode 1)
//   cm_ttv_f32        mode-m tensor-times-vector, Sec. 5.2 Eq. 24
//                     (std::inner_product of the mode-m fiber with b)
//   cm_ttm_f32        mode-m tensor-times-matrix, Sec. 5.2 Eq. 25 (the
//                     innermost level is a fiber-times-matrix product)
// Arithmetic is the element type's own (FP32), as in the paper's templates.
// This is a timed CPU baseline that sits beside the GPU library and shares
// nothing with it: the outermost recursion level is split across OpenMP
// threads, and a caller may restrict that level to its first `count` indices
// to time a bounded sample of a call.
//
// Conventions: modes are 0-based here; strides are in elements; for ttv the
// output strides wc are indexed by A's modes (wc[m] is not used), for ttm C
// has A's modes with extent J in mode m.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <iterator>
#include <numeric>
#include <type_traits>

#include <omp.h>

namespace {

// One fiber: a pointer that steps by a fixed stride.
template <class T>
struct StrideIt {
    using iterator_category = std::forward_iterator_tag;
    using value_type = std::remove_const_t<T>;
    using difference_type = std::ptrdiff_t;
    using pointer = T*;
    using reference = T&;
    T* p;
    int64_t s;
    T& operator*() const { return *p; }
    StrideIt& operator++()
    {
        p += s;
        return *this;
    }
    bool operator==(const StrideIt& o) const { return p == o.p; }
    bool operator!=(const StrideIt& o) const { return p != o.p; }
};

template <class T>
StrideIt<T> first(T* p, int64_t s) { return StrideIt<T>{p, s}; }
template <class T>
StrideIt<T> last(T* p, int64_t s, int64_t n) { return StrideIt<T>{p + n * s, s}; }

// ------------------------------------------------------------ transform ---

struct EwCtx {
    int op;
    const int64_t* n;
    const int64_t *wa, *wb, *wc;
};

template <class Op>
void transform_level(const EwCtx& c, int r, const float* A, const float* B, float* C, Op op)
{
    if (r == 0) {
        std::transform(first(A, c.wa[0]), last(A, c.wa[0], c.n[0]), first(B, c.wb[0]),
                       first(C, c.wc[0]), op);
        return;
    }
    for (int64_t i = 0; i < c.n[r]; ++i)
        transform_level(c, r - 1, A + i * c.wa[r], B + i * c.wb[r], C + i * c.wc[r], op);
}

template <class Op>
void transform_top(const EwCtx& c, int p, const float* A, const float* B, float* C,
                   int64_t count, Op op)
{
    const int top = p - 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < count; ++i) {
        if (top == 0) {
            C[i * c.wc[0]] = op(A[i * c.wa[0]], B[i * c.wb[0]]);
        } else {
            transform_level(c, top - 1, A + i * c.wa[top], B + i * c.wb[top], C + i * c.wc[top],
                            op);
        }
    }
}

// ------------------------------------------------------------------ ttv ---

struct TtvCtx {
    int m;          // contracted mode
    int lowest;     // the lowest free mode (the innermost loop)
    const int64_t* n;
    const int64_t *wa, *wc;
};

// Level r loops over mode r of A and C; the contracted mode is skipped (its
// fiber is consumed by the inner products of the innermost level).
void ttv_level(const TtvCtx& c, int r, const float* A, const float* b, float* C)
{
    if (r == c.m) {
        ttv_level(c, r - 1, A, b, C);
        return;
    }
    if (r == c.lowest) {
        const int64_t sm = c.wa[c.m], nm = c.n[c.m];
        for (int64_t i = 0; i < c.n[r]; ++i) {
            const float* a = A + i * c.wa[r];
            C[i * c.wc[r]] = std::inner_product(first(a, sm), last(a, sm, nm), b, 0.0f);
        }
        return;
    }
    for (int64_t i = 0; i < c.n[r]; ++i) ttv_level(c, r - 1, A + i * c.wa[r], b, C + i * c.wc[r]);
}

// ------------------------------------------------------------------ ttm ---

struct TtmCtx {
    int m, lowest;
    const int64_t* n;
    const int64_t *wa, *wc;
    const float* B;
    int64_t J, ldb_row, ldb_col;
};

// As ttv; the innermost level multiplies each mode-m fiber of A by every row
// of B (a fiber-times-matrix product) into the mode-m fiber of C.
void ttm_level(const TtmCtx& c, int r, const float* A, float* C)
{
    if (r == c.m) {
        ttm_level(c, r - 1, A, C);
        return;
    }
    if (r == c.lowest) {
        const int64_t sm = c.wa[c.m], nm = c.n[c.m];
        for (int64_t i = 0; i < c.n[r]; ++i) {
            const float* a = A + i * c.wa[r];
            float* out = C + i * c.wc[r];
            for (int64_t j = 0; j < c.J; ++j)
                out[j * c.wc[c.m]] = std::inner_product(first(a, sm), last(a, sm, nm),
                                                        first(c.B + j * c.ldb_row, c.ldb_col),
                                                        0.0f);
        }
        return;
    }
    for (int64_t i = 0; i < c.n[r]; ++i) ttm_level(c, r - 1, A + i * c.wa[r], C + i * c.wc[r]);
}

int lowest_free(int p, int m) { return m == 0 ? (p > 1 ? 1 : -1) : 0; }
int highest_free(int p, int m) { return m == p - 1 ? p - 2 : p - 1; }

int use_threads(int threads)
{
    if (threads > 0) omp_set_num_threads(threads);
    return omp_get_max_threads();
}

}  // namespace

extern "C" {

// Threads the parallel level uses (after an optional request, 0 = default).
int cm_threads(int threads) { return use_threads(threads); }

// C = A op B over the first `count` indices of mode p-1 (op 0..3: + - * /).
int cm_transform_f32(int p, const int64_t* n, int op, const float* A, const int64_t* wa,
                     const float* B, const int64_t* wb, float* C, const int64_t* wc,
                     int64_t count, int threads)
{
    if (p < 1 || op < 0 || op > 3 || count < 0 || count > n[p - 1]) return -1;
    use_threads(threads);
    const EwCtx c{op, n, wa, wb, wc};
    switch (op) {
    case 0: transform_top(c, p, A, B, C, count, std::plus<float>()); break;
    case 1: transform_top(c, p, A, B, C, count, std::minus<float>()); break;
    case 2: transform_top(c, p, A, B, C, count, std::multiplies<float>()); break;
    default: transform_top(c, p, A, B, C, count, std::divides<float>()); break;
    }
    return 0;
}

// C = A x_m b (Eq. 24) over the first `count` indices of the highest free mode.
int cm_ttv_f32(int p, const int64_t* n, const float* A, const int64_t* wa, int m,
               const float* b, float* C, const int64_t* wc, int64_t count, int threads)
{
    if (p < 2 || m < 0 || m >= p) return -1;
    const int top = highest_free(p, m);
    if (count < 0 || count > n[top]) return -1;
    use_threads(threads);
    const TtvCtx c{m, lowest_free(p, m), n, wa, wc};
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < count; ++i) {
        const float* a = A + i * wa[top];
        float* out = C + i * wc[top];
        if (top == c.lowest)
            *out = std::inner_product(first(a, wa[m]), last(a, wa[m], n[m]), b, 0.0f);
        else
            ttv_level(c, top - 1, a, b, out);
    }
    return 0;
}

// C = A x_m B (Eq. 25), B(j, k) at B[j * ldb_row + k * ldb_col], over the
// first `count` indices of the highest free mode.
int cm_ttm_f32(int p, const int64_t* n, const float* A, const int64_t* wa, int m,
               const float* B, int64_t J, int64_t ldb_row, int64_t ldb_col, float* C,
               const int64_t* wc, int64_t count, int threads)
{
    if (p < 2 || m < 0 || m >= p || J < 1) return -1;
    const int top = highest_free(p, m);
    if (count < 0 || count > n[top]) return -1;
    use_threads(threads);
    const TtmCtx c{m, lowest_free(p, m), n, wa, wc, B, J, ldb_row, ldb_col};
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < count; ++i) {
        const float* a = A + i * wa[top];
        float* out = C + i * wc[top];
        if (top == c.lowest) {
            for (int64_t j = 0; j < J; ++j)
                out[j * wc[m]] = std::inner_product(first(a, wa[m]), last(a, wa[m], n[m]),
                                                    first(B + j * ldb_row, ldb_col), 0.0f);
        } else {
            ttm_level(c, top - 1, a, out);
        }
    }
    return 0;
}

}  // extern "C"
