// contract.cpp -- transposition and the general tensor-tensor product (Sec. 5.2,
// Table 3) as re-descriptions onto the mode-q kernels.
//
// transpose: C = A^tau is a copy from A, described in C's mode order (mode r
// of the description is A's mode tau_r with its extent and stride), so it runs
// on the entrywise kernels, which pick the tiled transpose when the fastest
// modes differ.
//
// ttt: the (q, phi, psi)-mode product splits the modes into three groups:
//   K   the q contracted mode pairs (a stride in A and one in B),
//   FA  A's r free modes            (a stride in A and one in C),
//   FB  B's s free modes            (a stride in B and one in C).
// One operand plays the tensor T of a mode-1 ttm / ttv, the other the matrix
// (or vector) V.  This needs K to collapse to a single dim jointly in T and V,
// and V's free group to collapse to a single dim jointly in V and C; T's free
// group may stay any number of dims (the ttm / ttv planners take them as the
// batch).  When the strides do not allow it, the operands are first copied to
// dense layouts that do (V only, then T too), and the result goes through a
// dense temporary when C's strides break V's free group.  The contraction
// itself therefore always runs on the tuned ttv / ttm kernels, including the
// tensor-core ttm for the TF32 / BF16 / split-BF16x3 precisions.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "plan.h"
#include "runtime.h"

namespace tl {
namespace {

// One mode of a group: its extent, its stride in the two operands that carry
// it, and where it sits in each operand (0-based mode numbers, -1 if absent).
struct GDim {
    int64_t n;
    int tmode, vmode, cmode;
};

struct Operand {
    uint32_t p = 0;
    int32_t dtype = TL_F32;
    int64_t n[kMaxDims];
    int64_t w[kMaxDims];
    void* data = nullptr;
    tl_tensor desc() const
    {
        tl_tensor t{};
        t.p = p;
        t.dtype = dtype;
        t.n = n;
        t.pi = nullptr;
        t.w = w;
        t.data = data;
        return t;
    }
};

Operand from_tensor(const Tensor& t)
{
    Operand o;
    o.p = t.p;
    o.dtype = t.dtype;
    for (uint32_t r = 0; r < t.p; ++r) {
        o.n[r] = t.n[r];
        o.w[r] = t.w[r];
    }
    o.data = t.data;
    return o;
}

// Collapses a group over two stride arrays; returns the number of dims left
// and, when it is at most one, the merged extent and strides.
int collapse_pair(const std::vector<GDim>& g, const int64_t* s0, int which0, const int64_t* s1,
                  int which1, int64_t& n, int64_t& a, int64_t& b)
{
    Space sp;
    sp.nops = 2;
    for (const GDim& d : g) {
        Dim& x = sp.d[sp.nd++];
        const int m0 = which0 == 0 ? d.tmode : which0 == 1 ? d.vmode : d.cmode;
        const int m1 = which1 == 0 ? d.tmode : which1 == 1 ? d.vmode : d.cmode;
        x.n = d.n;
        x.s[0] = s0[m0];
        x.s[1] = s1[m1];
        x.s[2] = 0;
    }
    collapse(sp, 0);
    n = 1;
    a = b = 1;
    if (sp.nd == 1) {
        n = sp.d[0].n;
        a = sp.d[0].s[0];
        b = sp.d[0].s[1];
    }
    return sp.nd;
}

// Dense strides for an operand whose modes are laid out in `order` (fastest
// first); returns the element count.
int64_t dense_in_order(Operand& o, const std::vector<int>& order)
{
    int64_t s = 1;
    for (int m : order) {
        o.w[m] = s;
        s *= o.n[m];
    }
    return s;
}

// Sorts a group's dims by one operand's strides (0 = T, 1 = V, 2 = C).
void sort_by(std::vector<GDim>& g, const Operand& o, int which)
{
    std::stable_sort(g.begin(), g.end(), [&](const GDim& x, const GDim& y) {
        const int mx = which == 0 ? x.tmode : which == 1 ? x.vmode : x.cmode;
        const int my = which == 0 ? y.tmode : which == 1 ? y.vmode : y.cmode;
        return o.w[mx] < o.w[my];
    });
}

// Copies src (as described) into buf, laid out by dst's (dense) strides.
int pack(const Operand& src, Operand& dst, void* buf, cudaStream_t st)
{
    dst.data = buf;
    tl_tensor s = src.desc(), d = dst.desc();
    return tl_entrywise(TL_COPY, &s, nullptr, 1.0, &d, st);
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" {

int tl_transpose(const tl_tensor* A_, const uint32_t* tau, const tl_tensor* C_, void* stream)
{
    NvtxRange nvtx_range("tl_transpose");
    Tensor A;
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    if (!tau || !C_ || C_->p != A.p) return TL_EINVAL;
    bool seen[kMaxDims] = {false};
    int64_t n[kMaxDims], w[kMaxDims];
    for (uint32_t r = 0; r < A.p; ++r) {
        if (tau[r] < 1 || tau[r] > A.p || seen[tau[r] - 1]) return TL_EINVAL;
        seen[tau[r] - 1] = true;
        n[r] = A.n[tau[r] - 1];
        w[r] = A.w[tau[r] - 1];
    }
    tl_tensor At{};
    At.p = A.p;
    At.dtype = A.dtype;
    At.n = n;
    At.pi = nullptr;
    At.w = w;
    At.data = A.data;
    // C's extents are checked against n by the entrywise planner
    return tl_entrywise(TL_COPY, &At, nullptr, 1.0, C_, stream);
}

int tl_ttt(const tl_tensor* A_, const uint32_t* phi, const tl_tensor* B_, const uint32_t* psi,
           uint32_t q, const tl_tensor* C_, int32_t precision, int32_t accumulate, void* stream)
{
    NvtxRange nvtx_range("tl_ttt");
    Tensor A, B;
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    rc = load_tensor(B_, false, B);
    if (rc) return rc;
    if (!phi || !psi || !C_ || A.dtype != B.dtype || q > A.p || q > B.p) return TL_EINVAL;
    const uint32_t r = A.p - q, s = B.p - q;
    bool sa[kMaxDims] = {false}, sb[kMaxDims] = {false};
    for (uint32_t k = 0; k < A.p; ++k) {
        if (phi[k] < 1 || phi[k] > A.p || sa[phi[k] - 1]) return TL_EINVAL;
        sa[phi[k] - 1] = true;
    }
    for (uint32_t k = 0; k < B.p; ++k) {
        if (psi[k] < 1 || psi[k] > B.p || sb[psi[k] - 1]) return TL_EINVAL;
        sb[psi[k] - 1] = true;
    }
    for (uint32_t k = 0; k < q; ++k)
        if (A.n[phi[r + k] - 1] != B.n[psi[s + k] - 1]) return TL_EINVAL;
    // C: order r + s; an order-0 result is one element (p = 0, or p = 1 with n = 1)
    Tensor C;
    if (r + s == 0) {
        if (!C_->data || C_->dtype != A.dtype) return TL_EINVAL;
        if (C_->p > 1 || (C_->p == 1 && (!C_->n || C_->n[0] != 1))) return TL_EINVAL;
        C.p = 1;
        C.dtype = A.dtype;
        C.n[0] = 1;
        C.w[0] = 1;
        C.data = C_->data;
    } else {
        rc = load_tensor(C_, true, C);
        if (rc) return rc;
        if (C.p != r + s || C.dtype != A.dtype) return TL_EINVAL;
        for (uint32_t k = 0; k < r; ++k)
            if (C.n[k] != A.n[phi[k] - 1]) return TL_EINVAL;
        for (uint32_t k = 0; k < s; ++k)
            if (C.n[r + k] != B.n[psi[k] - 1]) return TL_EINVAL;
    }
    if (precision < TL_P_DEFAULT || precision > TL_P_BF16X3) return TL_EINVAL;
    if (precision != TL_P_DEFAULT && (precision == TL_P_F64) != (A.dtype == TL_F64))
        return TL_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Orientation: T is the operand whose free group is the batch of the
    // mode-1 call; prefer one with free modes, then the larger.
    int64_t freeA = 1, freeB = 1;
    for (uint32_t k = 0; k < r; ++k) freeA *= A.n[phi[k] - 1];
    for (uint32_t k = 0; k < s; ++k) freeB *= B.n[psi[k] - 1];
    const bool t_is_a = (freeA > 1) != (freeB > 1) ? freeA > 1 : A.count() >= B.count();
    const Tensor& Tt = t_is_a ? A : B;
    const Tensor& Vt = t_is_a ? B : A;
    const uint32_t* tmap = t_is_a ? phi : psi;   // T's permutation tuple
    const uint32_t* vmap = t_is_a ? psi : phi;
    const uint32_t rt = t_is_a ? r : s, rv = t_is_a ? s : r;
    const uint32_t coff_t = t_is_a ? 0 : r, coff_v = t_is_a ? r : 0;   // first C mode of each free group

    std::vector<GDim> K, FT, FV;
    for (uint32_t k = 0; k < q; ++k)
        K.push_back({Tt.n[tmap[rt + k] - 1], (int)tmap[rt + k] - 1, (int)vmap[rv + k] - 1, -1});
    for (uint32_t k = 0; k < rt; ++k)
        FT.push_back({Tt.n[tmap[k] - 1], (int)tmap[k] - 1, -1, (int)(coff_t + k)});
    for (uint32_t k = 0; k < rv; ++k)
        FV.push_back({Vt.n[vmap[k] - 1], -1, (int)vmap[k] - 1, (int)(coff_v + k)});

    Operand T = from_tensor(Tt), V = from_tensor(Vt), Cc = from_tensor(C);
    Operand Cout = Cc;            // where the mode-1 call writes
    bool c_temp = false;
    int64_t nK, sTK, sVK, nV, sVV, sCV;
    int kdims = collapse_pair(K, T.w, 0, V.w, 1, nK, sTK, sVK);
    int vdims = collapse_pair(FV, V.w, 1, Cc.w, 2, nV, sVV, sCV);
    const size_t esz = A.elem();
    if (kdims > 1 || vdims > 1) {
        // level 1: V dense with K in T's stride order, then its free modes in C's
        std::vector<GDim> Ko = K, FVo = FV;
        sort_by(Ko, T, 0);
        sort_by(FVo, Cc, 2);
        int64_t tK, tmp0;
        const bool t_alone = collapse_pair(Ko, T.w, 0, T.w, 0, tK, tmp0, tmp0) <= 1;
        Operand Tp = T;
        if (!t_alone) {
            // level 2: T dense too, K first (in the order of the mode pairs),
            // then T's free modes in C's stride order
            Ko = K;
            std::vector<GDim> FTo = FT;
            sort_by(FTo, Cc, 2);
            std::vector<int> order;
            for (const GDim& d : Ko) order.push_back(d.tmode);
            for (const GDim& d : FTo) order.push_back(d.tmode);
            const int64_t cnt = dense_in_order(Tp, order);
            void* buf = workspace_slot(st, (size_t)cnt * esz, 3);
            if (!buf) return TL_ENOMEM;
            rc = pack(T, Tp, buf, st);
            if (rc) return rc;
        }
        Operand Vp = V;
        std::vector<int> order;
        for (const GDim& d : Ko) order.push_back(d.vmode);
        for (const GDim& d : FVo) order.push_back(d.vmode);
        const int64_t cnt = dense_in_order(Vp, order);
        void* buf = workspace_slot(st, (size_t)cnt * esz, 4);
        if (!buf) return TL_ENOMEM;
        rc = pack(V, Vp, buf, st);
        if (rc) return rc;
        T = Tp;
        V = Vp;
        kdims = collapse_pair(K, T.w, 0, V.w, 1, nK, sTK, sVK);
        vdims = collapse_pair(FV, V.w, 1, Cc.w, 2, nV, sVV, sCV);
        if (vdims > 1) {
            // C's strides break V's free group: write a dense temporary laid
            // out as [V's free modes in V's order, T's free modes] and copy
            std::vector<int> corder;
            for (const GDim& d : FVo) corder.push_back(d.cmode);
            for (const GDim& d : FT) corder.push_back(d.cmode);
            const int64_t cc = dense_in_order(Cout, corder);
            Cout.data = workspace_slot(st, (size_t)cc * esz, 5);
            if (!Cout.data) return TL_ENOMEM;
            c_temp = true;
            vdims = collapse_pair(FV, V.w, 1, Cout.w, 2, nV, sVV, sCV);
        }
        if (kdims > 1 || vdims > 1) return TL_EINVAL;   // unreachable by construction
    }
    if (nK == 1) sTK = sVK = 1;
    if (nV == 1) sVV = sCV = 1;

    // The mode-1 call: T' = (K, T's free modes), C' = (V's free group, T's free modes)
    int64_t tn[kMaxDims], tw[kMaxDims], cn[kMaxDims], cw[kMaxDims];
    uint32_t tp = 1;
    tn[0] = nK;
    tw[0] = sTK;
    cn[0] = nV;
    cw[0] = sCV;
    for (const GDim& d : FT) {
        if (d.n == 1) continue;
        tn[tp] = d.n;
        tw[tp] = T.w[d.tmode];
        cn[tp] = d.n;
        cw[tp] = Cout.w[d.cmode];
        ++tp;
    }
    if (tp == 1) {        // no free mode in T: a dummy extent-1 mode keeps order >= 2
        tn[1] = cn[1] = 1;
        tw[1] = cw[1] = 1;
        tp = 2;
    }
    tl_tensor Td{}, Cd{};
    Td.p = tp;
    Td.dtype = A.dtype;
    Td.n = tn;
    Td.w = tw;
    Td.data = T.data;
    const int acc_direct = c_temp ? 0 : accumulate;
    if (nV == 1) {
        // V's free modes are all of extent 1: a ttv of T with the vector V
        Cd.p = tp - 1;
        Cd.dtype = A.dtype;
        Cd.n = cn + 1;
        Cd.w = cw + 1;
        Cd.data = Cout.data;
        rc = tl_ttv(&Td, V.data, sVK, 1, &Cd, acc_direct, stream);
    } else {
        // a ttm of T with the matrix V(j, k) = V[j * sVV + k * sVK]; the
        // tensor-core path takes at most 512 rows per call
        const bool tc = precision == TL_P_TF32 || precision == TL_P_BF16 ||
                        precision == TL_P_BF16X3;
        const int64_t step = tc ? 512 : nV;
        Cd.p = tp;
        Cd.dtype = A.dtype;
        Cd.n = cn;
        Cd.w = cw;
        for (int64_t j0 = 0; j0 < nV && rc == TL_OK; j0 += step) {
            const int64_t Jb = std::min(step, nV - j0);
            cn[0] = Jb;
            Cd.data = static_cast<char*>(Cout.data) + (size_t)(j0 * sCV) * esz;
            const void* Vb = static_cast<const char*>(V.data) + (size_t)(j0 * sVV) * esz;
            rc = tl_ttm(&Td, Vb, Jb, sVV, sVK, 1, &Cd, precision, acc_direct, stream);
        }
    }
    if (rc || !c_temp) return rc;
    // copy (or add) the dense temporary into C, described in C's mode order
    tl_tensor Ct = Cc.desc(), Tmp = Cout.desc();
    if (accumulate) return tl_entrywise(TL_ADD, &Ct, &Tmp, 1.0, &Ct, stream);
    return tl_entrywise(TL_COPY, &Tmp, nullptr, 1.0, &Ct, stream);
}

}  // extern "C"
