// plan.h -- host-side descriptor validation and iteration-space canonicalisation.
//
// A call's tensors are described by (p, n, pi, w) as in Sec. 3.1 of the TLib
// paper.  The planner turns them into a collapsed iteration space: a list of
// dims, each with one extent and one stride per operand, from which the kernels
// compute element offsets as sum_d i_d * s_d (the layout function, Sec. 3.2
// Eq. 17).  Collapsing never changes which elements are combined; it only
// merges modes that are adjacent in memory for every operand at once.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/tlgb.h"

namespace tl {

constexpr int kMaxDims = TL_MAX_ORDER;

struct Dim {
    int64_t n;
    int64_t s[3];   // stride of this dim for operand 0, 1, 2 (elements)
};

// An iteration space over up to kMaxDims dims and up to 3 operands.
// dims[0] is the fastest-varying dim of the linearised index.
struct Space {
    int nd = 0;
    int nops = 0;
    Dim d[kMaxDims];
    // exclusive bound on the offset of the last element a mapped index
    // addresses in each operand (its span less the planned extra offset along
    // the contraction or the output column); <= 0: not set.  Checked by the
    // mapper in builds with TL_CHECK_BOUNDS only.
    int64_t limit[3] = {0, 0, 0};
    int64_t count() const {
        int64_t c = 1;
        for (int i = 0; i < nd; ++i) c *= d[i].n;
        return c;
    }
};

// A validated tensor: extents and strides (derived by Eq. 14 when absent).
struct Tensor {
    uint32_t p = 0;
    int32_t dtype = TL_F32;
    int64_t n[kMaxDims];
    int64_t w[kMaxDims];
    void* data = nullptr;
    size_t elem() const { return dtype == TL_F64 ? 8 : 4; }
    int64_t count() const {
        int64_t c = 1;
        for (uint32_t r = 0; r < p; ++r) c *= n[r];
        return c;
    }
    // number of elements spanned in memory (largest offset + 1)
    int64_t span() const {
        int64_t s = 1;
        for (uint32_t r = 0; r < p; ++r) s += (n[r] - 1) * w[r];
        return s;
    }
};

// Validates a descriptor; fills t.  is_output additionally checks that no two
// elements share an address.  Returns TL_OK or TL_EINVAL.
int load_tensor(const tl_tensor* d, bool is_output, Tensor& t);

// Eq. 14: strides of the dense layout pi (1-based) for extents n.
void dense_strides(uint32_t p, const int64_t* n, const uint32_t* pi, int64_t* w);

// Drops extent-1 dims, sorts by the stride of operand `key` (ties by the
// others) and merges dim d+1 into d whenever s[d+1] == n[d]*s[d] holds for
// every operand.
void collapse(Space& sp, int key);

// Kernel choices recorded in plans (also reported by tl_plan_describe).
enum Kernel : int {
    K_NONE = 0,
    K_TTV_ROW,        // contraction contiguous in A: one lane group per output
    K_TTV_COL,        // contraction strided: threads along the output dims
    K_EW_FLAT,        // all operands share one contiguous layout
    K_EW_TILE,        // two fastest dims differ: smem-tiled transpose
    K_EW_GENERIC,     // any strides: per-element offset mapping
    K_EW_ROWS,        // all contiguous along dim 0, other dims permuted: per-vector mapping
    K_TTM_SIMT,       // register-tiled FP32 / FP64 batched GEMM
    K_TTM_TC,         // tcgen05 tensor-core batched GEMM
    K_EW_TMA,         // FP32, layouts differ, <= 5 dims: TMA-staged 32 x 32 tiles
    K_TTM_ROWS,       // SIMT ttm with n_q <= 32: a row per thread, B in shared memory
};

const char* kernel_name(int k);

struct TtvPlan {
    int32_t dtype;
    Space out;          // operands: 0 = A, 1 = C
    int64_t nq, saq, incb;
    int64_t nout;       // number of output elements
    int kernel;
    int vec;            // elements per vector access (1, 2, 4)
    int lanes;          // ROW: lanes per output row
    int splits;         // k-range splits (>1 uses the workspace)
    int64_t kchunk;     // k values per split
};

struct TtmPlan {
    int32_t dtype;
    int32_t precision;
    Space rows;         // all modes but q; operands: 0 = A, 1 = C
    int64_t nq, saq;    // contraction
    int64_t J, scq;     // output mode q in C
    int64_t ldb_row, ldb_col;
    int64_t M;          // rows.count()
    int kernel;
    int tc_variant;     // tensor-core path layout (see ttm_tc.cu)
};

struct EwPlan {
    int32_t dtype;
    int32_t op;
    Space sp;           // operands: 0 = A, 1 = B, 2 = C
    int64_t N;
    int kernel;
    int vec;
    int tdim;           // EW_TILE: the dim tiled against dims[0]
};

int plan_ttv(const Tensor& A, int64_t incb, uint32_t q, const Tensor& C, TtvPlan& P,
             int num_sms);
int plan_ttm(const Tensor& A, int64_t J, int64_t ldb_row, int64_t ldb_col, uint32_t q,
             const Tensor& C, int32_t precision, TtmPlan& P);
int plan_entrywise(int32_t op, const Tensor& A, const Tensor* B, const Tensor& C, EwPlan& P);

// Division of 32-bit unsigned indices by an invariant divisor d >= 1 with a
// multiply-high, an add and two shifts (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Fig. 4.1): with
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, sh1 = min(l, 1),
// sh2 = max(l - 1, 0):  n / d = (t + ((n - t) >> sh1)) >> sh2, t = mulhi(m, n).
struct FastDiv {
    uint32_t mul;
    uint32_t sh1, sh2;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while (l < 32 && (uint64_t(1) << l) < d) ++l;
    FastDiv f;
    f.mul = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    f.sh1 = l < 1 ? l : 1;
    f.sh2 = l > 1 ? l - 1 : 0;
    return f;
}

inline uint32_t fastdiv_host(uint32_t n, const FastDiv& f)
{
    const uint32_t t = (uint32_t)(((uint64_t)f.mul * n) >> 32);
    return (t + ((n - t) >> f.sh1)) >> f.sh2;
}

// Pointer alignment helper.
inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace tl
