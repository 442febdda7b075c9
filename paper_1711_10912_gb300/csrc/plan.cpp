// plan.cpp -- descriptor validation, stride derivation (Sec. 3.1 Eq. 14) and
// joint mode collapsing for ttv, ttm and entrywise calls.  Host only; no
// CUDA calls, no heap allocation, O(p^2) work.
#include "plan.h"

#include <algorithm>
#include <cstring>

namespace tl {

void dense_strides(uint32_t p, const int64_t* n, const uint32_t* pi, int64_t* w)
{
    // Eq. 14: w_{pi_1} = 1 and w_{pi_r} = w_{pi_{r-1}} * n_{pi_{r-1}}.
    int64_t run = 1;
    for (uint32_t r = 0; r < p; ++r) {
        uint32_t mode = pi ? pi[r] - 1 : r;
        w[mode] = run;
        run *= n[mode];
    }
}

static bool is_perm(uint32_t p, const uint32_t* pi)
{
    bool seen[kMaxDims] = {false};
    for (uint32_t r = 0; r < p; ++r) {
        if (pi[r] < 1 || pi[r] > p || seen[pi[r] - 1]) return false;
        seen[pi[r] - 1] = true;
    }
    return true;
}

// Distinct multi-indices map to distinct addresses when, in ascending stride
// order (extent-1 modes skipped), each stride exceeds the largest offset
// reachable with the faster modes alone.
static bool no_self_overlap(const Tensor& t)
{
    int idx[kMaxDims];
    int m = 0;
    for (uint32_t r = 0; r < t.p; ++r)
        if (t.n[r] > 1) idx[m++] = (int)r;
    for (int i = 1; i < m; ++i) {
        int x = idx[i], j = i - 1;
        while (j >= 0 && t.w[x] < t.w[idx[j]]) {
            idx[j + 1] = idx[j];
            --j;
        }
        idx[j + 1] = x;
    }
    int64_t reach = 0;
    for (int i = 0; i < m; ++i) {
        if (t.w[idx[i]] <= reach) return false;
        reach += (t.n[idx[i]] - 1) * t.w[idx[i]];
    }
    return true;
}

int load_tensor(const tl_tensor* d, bool is_output, Tensor& t)
{
    if (!d || d->p < 1 || d->p > (uint32_t)kMaxDims || !d->n || !d->data) return TL_EINVAL;
    if (d->dtype != TL_F32 && d->dtype != TL_F64) return TL_EINVAL;
    t.p = d->p;
    t.dtype = d->dtype;
    t.data = d->data;
    for (uint32_t r = 0; r < t.p; ++r) {
        if (d->n[r] < 1) return TL_EINVAL;
        t.n[r] = d->n[r];
    }
    if (d->pi && !is_perm(t.p, d->pi)) return TL_EINVAL;
    if (d->w) {
        for (uint32_t r = 0; r < t.p; ++r) {
            if (d->w[r] < 1) return TL_EINVAL;
            t.w[r] = d->w[r];
        }
    } else {
        dense_strides(t.p, t.n, d->pi, t.w);
    }
    if (is_output && !no_self_overlap(t)) return TL_EINVAL;
    return TL_OK;
}

void collapse(Space& sp, int key)
{
    // 1. drop extent-1 dims
    int m = 0;
    for (int i = 0; i < sp.nd; ++i)
        if (sp.d[i].n > 1) sp.d[m++] = sp.d[i];
    sp.nd = m;
    // 2. sort by the key operand's stride, ties by the other operands
    //    (insertion sort: stable, at most kMaxDims entries, no allocation)
    auto less = [&](const Dim& a, const Dim& b) {
        if (a.s[key] != b.s[key]) return a.s[key] < b.s[key];
        for (int o = 0; o < sp.nops; ++o)
            if (a.s[o] != b.s[o]) return a.s[o] < b.s[o];
        return false;
    };
    for (int i = 1; i < sp.nd; ++i) {
        Dim x = sp.d[i];
        int j = i - 1;
        while (j >= 0 && less(x, sp.d[j])) {
            sp.d[j + 1] = sp.d[j];
            --j;
        }
        sp.d[j + 1] = x;
    }
    // 3. merge neighbours that are adjacent in memory for every operand
    if (sp.nd == 0) return;
    int out = 0;
    for (int i = 1; i < sp.nd; ++i) {
        Dim& cur = sp.d[out];
        const Dim& nx = sp.d[i];
        bool mergeable = true;
        for (int o = 0; o < sp.nops; ++o)
            if (nx.s[o] != cur.n * cur.s[o]) { mergeable = false; break; }
        if (mergeable) cur.n *= nx.n;
        else sp.d[++out] = nx;
    }
    sp.nd = out + 1;
}

const char* kernel_name(int k)
{
    switch (k) {
    case K_TTV_ROW: return "ttv_row";
    case K_TTV_COL: return "ttv_col";
    case K_EW_FLAT: return "ew_flat";
    case K_EW_TILE: return "ew_tile";
    case K_EW_GENERIC: return "ew_generic";
    case K_EW_ROWS: return "ew_rows";
    case K_TTM_SIMT: return "ttm_simt";
    case K_TTM_TC: return "ttm_tc";
    case K_EW_TMA: return "ew_tma";
    case K_TTM_ROWS: return "ttm_rows";
    default: return "none";
    }
}

int plan_ttv(const Tensor& A, int64_t incb, uint32_t q, const Tensor& C, TtvPlan& P, int num_sms)
{
    if (A.p < 2 || q < 1 || q > A.p || incb < 1) return TL_EINVAL;
    if (C.p != A.p - 1 || C.dtype != A.dtype) return TL_EINVAL;
    for (uint32_t r = 0, c = 0; r < A.p; ++r) {
        if (r == q - 1) continue;
        if (C.n[c] != A.n[r]) return TL_EINVAL;
        ++c;
    }
    P = {};
    P.dtype = A.dtype;
    P.out.nops = 2;
    for (uint32_t r = 0, c = 0; r < A.p; ++r) {
        if (r == q - 1) continue;
        Dim& d = P.out.d[P.out.nd++];
        d.n = A.n[r];
        d.s[0] = A.w[r];
        d.s[1] = C.w[c];
        d.s[2] = 0;
        ++c;
    }
    collapse(P.out, 0);
    P.nq = A.n[q - 1];
    P.saq = A.w[q - 1];
    P.incb = incb;
    P.out.limit[0] = A.span() - (P.nq - 1) * P.saq;
    P.out.limit[1] = C.span();
    P.nout = P.out.count();
    const int es = (int)A.elem();
    const int V = 16 / es;   // elements per 16-byte vector
    P.splits = 1;
    P.kchunk = P.nq;

    if (P.saq == 1 && P.nq >= 8) {
        P.kernel = K_TTV_ROW;
        bool v = (P.nq % V == 0) && aligned(A.data, 16) && incb == 1;
        for (int i = 0; i < P.out.nd && v; ++i) v = (P.out.d[i].s[0] % V == 0);
        P.vec = v ? V : 1;
        int64_t chunks = (P.nq + P.vec - 1) / P.vec;
        P.lanes = chunks >= 32 ? 32 : chunks >= 16 ? 16 : chunks >= 8 ? 8 : 4;
    } else {
        P.kernel = K_TTV_COL;
        bool v = P.out.nd >= 1 && P.out.d[0].s[0] == 1 && P.out.d[0].s[1] == 1 &&
                 P.out.d[0].n % V == 0 && P.saq % V == 0 && aligned(A.data, 16) &&
                 aligned(C.data, 16);
        for (int i = 1; i < P.out.nd && v; ++i)
            v = (P.out.d[i].s[0] % V == 0) && (P.out.d[i].s[1] % V == 0);
        P.vec = v ? V : 1;
        P.lanes = 1;
    }
    // Split the k range across CTAs when the outputs alone cannot fill the
    // GPU (about 2048 resident threads per SM).
    int64_t threads = P.kernel == K_TTV_ROW ? P.nout * P.lanes : P.nout / P.vec;
    int64_t target = (int64_t)num_sms * 2048;
    int64_t kmin = P.kernel == K_TTV_ROW ? (int64_t)P.lanes * P.vec * 2 : 16;
    if (threads < target / 2 && P.nq >= 2 * kmin) {
        int64_t s = (target + threads - 1) / threads;
        s = std::min<int64_t>(s, P.nq / kmin);
        s = std::min<int64_t>(s, 4096);
        if (s > 1) {
            int64_t align = P.kernel == K_TTV_ROW ? (int64_t)P.lanes * P.vec : 4;
            int64_t chunk = (P.nq + s - 1) / s;
            chunk = (chunk + align - 1) / align * align;
            P.kchunk = chunk;
            P.splits = (int)((P.nq + chunk - 1) / chunk);
        }
    }
    return TL_OK;
}

int plan_ttm(const Tensor& A, int64_t J, int64_t ldb_row, int64_t ldb_col, uint32_t q,
             const Tensor& C, int32_t precision, TtmPlan& P)
{
    if (A.p < 2 || q < 1 || q > A.p || J < 1) return TL_EINVAL;
    if (C.p != A.p || C.dtype != A.dtype) return TL_EINVAL;
    for (uint32_t r = 0; r < A.p; ++r) {
        int64_t want = (r == q - 1) ? J : A.n[r];
        if (C.n[r] != want) return TL_EINVAL;
    }
    if (precision == TL_P_DEFAULT) precision = A.dtype == TL_F64 ? TL_P_F64 : TL_P_F32;
    if (precision < TL_P_F64 || precision > TL_P_BF16X3) return TL_EINVAL;
    if ((precision == TL_P_F64) != (A.dtype == TL_F64)) return TL_EUNSUPPORTED;
    P = {};
    P.dtype = A.dtype;
    P.precision = precision;
    P.rows.nops = 2;
    for (uint32_t r = 0; r < A.p; ++r) {
        if (r == q - 1) continue;
        Dim& d = P.rows.d[P.rows.nd++];
        d.n = A.n[r];
        d.s[0] = A.w[r];
        d.s[1] = C.w[r];
        d.s[2] = 0;
    }
    collapse(P.rows, 0);
    P.nq = A.n[q - 1];
    P.saq = A.w[q - 1];
    P.J = J;
    P.scq = C.w[q - 1];
    P.rows.limit[0] = A.span() - (P.nq - 1) * P.saq;
    P.rows.limit[1] = C.span() - (J - 1) * P.scq;
    P.ldb_row = ldb_row;
    P.ldb_col = ldb_col;
    P.M = P.rows.count();
    P.kernel = K_TTM_SIMT;
    P.tc_variant = 0;
    // short contractions, and narrow outputs (J <= 16) over enough rows to
    // fill the GPU: a row per thread with the matrix in shared memory (at
    // most 32 KB of it), unless the tensor-core path takes the call below.
    // The 64 x 64 tiles of the FP64 kernel would leave 48 of their 64 columns
    // idle at J <= 16 (an FP64 ttm of 438600 rows, n_q = 232, J = 6 took
    // 5.6 ms against a 0.49 ms DFMA bound).
    {
        const int64_t Jp = (J + 15) / 16 * 16;
        const bool fits = P.nq * Jp * (int64_t)A.elem() <= 32 * 1024;
        if (fits && (P.nq <= 64 || (J <= 16 && P.M >= 65536))) P.kernel = K_TTM_ROWS;
    }
    // Tensor-core path: FP32 data in a tensor-core precision, a contraction
    // and output width worth an MMA, and an A that a TMA box can describe
    // (16-byte aligned base and strides).
    const bool tc_prec = precision == TL_P_TF32 || precision == TL_P_BF16 ||
                         precision == TL_P_BF16X3;
    if (tc_prec && A.dtype == TL_F32 && J <= 512 && P.nq >= 16 && aligned(A.data, 16)) {
        if (P.saq == 1 && P.rows.nd == 1 && P.M >= 128 && P.rows.d[0].s[0] % 4 == 0) {
            P.kernel = K_TTM_TC;
            P.tc_variant = 1;   // rows contiguous in k
        } else if (P.saq > 1 && P.saq % 4 == 0 && P.rows.nd >= 1 && P.rows.nd <= 2 &&
                   P.rows.d[0].s[0] == 1 && P.rows.d[0].n >= 64 &&
                   (P.rows.nd == 1 || P.rows.d[1].s[0] % 4 == 0)) {
            P.kernel = K_TTM_TC;
            P.tc_variant = 2;   // rows contiguous in the fastest output mode
        }
    }
    return TL_OK;
}

int plan_entrywise(int32_t op, const Tensor& A, const Tensor* B, const Tensor& C, EwPlan& P)
{
    if (op < TL_ADD || op > TL_SCALE) return TL_EINVAL;
    bool unary = (op == TL_COPY || op == TL_SCALE);
    if (unary != (B == nullptr)) return TL_EINVAL;
    if (C.p != A.p || C.dtype != A.dtype) return TL_EINVAL;
    for (uint32_t r = 0; r < A.p; ++r)
        if (C.n[r] != A.n[r]) return TL_EINVAL;
    if (B) {
        if (B->p != A.p || B->dtype != A.dtype) return TL_EINVAL;
        for (uint32_t r = 0; r < A.p; ++r)
            if (B->n[r] != A.n[r]) return TL_EINVAL;
    }
    P = {};
    P.dtype = A.dtype;
    P.op = op;
    P.sp.nops = 3;
    for (uint32_t r = 0; r < A.p; ++r) {
        Dim& d = P.sp.d[P.sp.nd++];
        d.n = A.n[r];
        d.s[0] = A.w[r];
        d.s[1] = B ? B->w[r] : A.w[r];
        d.s[2] = C.w[r];
    }
    collapse(P.sp, 2);
    P.N = P.sp.count();
    P.sp.limit[0] = A.span();
    P.sp.limit[1] = B ? B->span() : A.span();
    P.sp.limit[2] = C.span();
    const int V = 16 / (int)A.elem();
    P.vec = 1;
    P.tdim = -1;
    if (P.sp.nd <= 1 && (P.sp.nd == 0 ||
                         (P.sp.d[0].s[0] == 1 && P.sp.d[0].s[1] == 1 && P.sp.d[0].s[2] == 1))) {
        P.kernel = K_EW_FLAT;
        bool v = aligned(A.data, 16) && aligned(C.data, 16) && (!B || aligned(B->data, 16));
        P.vec = v ? V : 1;
        return TL_OK;
    }
    // Tile the output's fastest dim against the fastest dim of an input whose
    // own fastest dim is another one (a transposed operand).
    int t = -1;
    for (int o = 0; o < (B ? 2 : 1) && t < 0; ++o) {
        int best = 0;
        for (int i = 1; i < P.sp.nd; ++i)
            if (P.sp.d[i].s[o] < P.sp.d[best].s[o]) best = i;
        if (best != 0) t = best;
    }
    if (t > 0 && P.sp.d[0].s[2] == 1) {
        P.kernel = K_EW_TILE;
        P.tdim = t;
        // 16-byte vectors: each operand contiguous along dim 0 (read in the
        // write phase) or along dim t (staged), every other stride and both
        // tiled extents multiples of the vector width, 16-byte aligned bases
        const Space& sp = P.sp;
        bool v = sp.d[0].n % V == 0 && sp.d[t].n % V == 0 && aligned(C.data, 16) &&
                 aligned(A.data, 16) && (!B || aligned(B->data, 16));
        for (int o = 0; o < 3 && v; ++o) {
            if (o == 1 && !B) continue;
            bool staged = o < 2 && sp.d[t].s[o] < sp.d[0].s[o];
            int unit = staged ? t : 0, other = staged ? 0 : t;
            v = sp.d[unit].s[o] == 1 && sp.d[other].s[o] % V == 0;
            for (int d = 1; d < sp.nd && v; ++d)
                if (d != t) v = sp.d[d].s[o] % V == 0;
        }
        P.vec = v ? V : 1;
    } else {
        P.kernel = K_EW_GENERIC;
        // every operand contiguous along dim 0: decode once per 16-byte vector
        const Space& sp = P.sp;
        bool v = sp.nd >= 1 && sp.d[0].n % V == 0 && aligned(A.data, 16) && aligned(C.data, 16) &&
                 (!B || aligned(B->data, 16));
        for (int o = 0; o < 3 && v; ++o) {
            if (o == 1 && !B) continue;
            v = sp.d[0].s[o] == 1;
            for (int d = 1; d < sp.nd && v; ++d) v = sp.d[d].s[o] % V == 0;
        }
        if (v) {
            P.kernel = K_EW_ROWS;
            P.vec = V;
        }
    }
    // Tiles over (dim 0, dim t) of 1024 elements (16 x 64 .. 128 x 8) that
    // even the best shape leaves mostly idle (high-order tensors with small
    // extents): map every element instead.
    if (P.kernel == K_EW_TILE) {
        auto fill = [](int64_t n, int64_t e) { return (double)n / (double)((n + e - 1) / e * e); };
        double best = 0.0;
        for (int64_t t0 : {16, 32, 64, 128})
            best = std::max(best, fill(P.sp.d[0].n, t0) * fill(P.sp.d[P.tdim].n, 1024 / t0));
        if (best < 0.2) {
            P.kernel = K_EW_GENERIC;
            P.vec = 1;
            P.tdim = -1;
            return TL_OK;
        }
    }
    // FP32 tiles whose extents rule out the 16-byte vector tile kernel (a
    // ragged extent in a padded view) go through TMA-staged 32 x 32 tiles
    // when every input is unit-stride along dim 0 or along the tiled dim t, C
    // along dim 0, there are at most 5 dims (the tensor-map rank), every
    // other stride is a multiple of 16 bytes and the bases are 16-byte
    // aligned.  Vector tiles and permuted rows stay on the SIMT kernels:
    // on 128^4 FP32 tensors they ran every layout pair faster than the TMA
    // kernel (its boxes of 128 rows 8 MB apart are the slow case).
    if (A.dtype == TL_F32 && P.kernel == K_EW_TILE && P.vec == 1 && P.sp.nd >= 2 &&
        P.sp.nd <= 5) {
        const Space& sp = P.sp;
        const int t = P.kernel == K_EW_TILE ? P.tdim : 1;
        bool ok = sp.d[0].s[2] == 1 && aligned(A.data, 16) && aligned(C.data, 16) &&
                  (!B || aligned(B->data, 16));
        for (int o = 0; o < 3 && ok; ++o) {
            if (o == 1 && !B) continue;
            const int unit = sp.d[0].s[o] == 1 ? 0 : (o < 2 && sp.d[t].s[o] == 1 ? t : -1);
            if (unit < 0) ok = false;
            for (int d = 0; d < sp.nd && ok; ++d)
                if (d != unit) ok = sp.d[d].s[o] % 4 == 0 && sp.d[d].s[o] < (int64_t(1) << 38);
        }
        for (int d = 0; d < sp.nd && ok; ++d) ok = sp.d[d].n < (int64_t(1) << 31);
        // 32 x 32 tiles are numbered in 32-bit arithmetic
        if (ok) {
            int64_t tiles = ((sp.d[0].n + 31) / 32) * ((sp.d[t].n + 31) / 32);
            for (int d = 1; d < sp.nd && ok; ++d)
                if (d != t) {
                    tiles *= sp.d[d].n;
                    ok = tiles < (int64_t(1) << 31);
                }
            ok = ok && tiles < (int64_t(1) << 31);
        }
        if (ok) {
            P.kernel = K_EW_TMA;
            P.tdim = t;
            P.vec = 4;
        }
    }
    return TL_OK;
}

}  // namespace tl
