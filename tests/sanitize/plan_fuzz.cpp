// plan_fuzz.cpp -- host-side fuzz check of the planner (descriptor
// validation, Eq. 14 strides, joint mode collapse) built with AddressSanitizer
// and UndefinedBehaviorSanitizer by tests/test_host_sanitizers.py.
//
// For random orders, extents, layout tuples and views it checks that the
// collapsed iteration spaces of ttv, ttm and entrywise plans enumerate exactly
// the offset tuples that the layout function (Sec. 3.2 Eq. 17) gives for every
// multi-index, computed here by brute force, and that invalid descriptors are
// rejected.  Exit status 0 on success; a mismatch prints the case and exits 1.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <tuple>
#include <vector>

#include "plan.h"

using namespace tl;

namespace {

std::mt19937_64 rng(20261204);

int64_t uni(int64_t lo, int64_t hi) { return std::uniform_int_distribution<int64_t>(lo, hi)(rng); }

struct Desc {
    std::vector<int64_t> n, w;
    std::vector<uint32_t> pi;
    tl_tensor t{};
    void fill(uint32_t p, int32_t dtype, void* data, bool with_w)
    {
        t.p = p;
        t.dtype = dtype;
        t.n = n.data();
        t.pi = pi.empty() ? nullptr : pi.data();
        t.w = with_w ? w.data() : nullptr;
        t.data = data;
    }
};

std::vector<uint32_t> random_perm(uint32_t p)
{
    std::vector<uint32_t> v(p);
    for (uint32_t r = 0; r < p; ++r) v[r] = r + 1;
    std::shuffle(v.begin(), v.end(), rng);
    return v;
}

// dense strides of layout pi (Eq. 14), written here independently
std::vector<int64_t> strides_of(const std::vector<int64_t>& n, const std::vector<uint32_t>& pi)
{
    std::vector<int64_t> w(n.size());
    int64_t s = 1;
    for (uint32_t r : pi) {
        w[r - 1] = s;
        s *= n[r - 1];
    }
    return w;
}

// a view of a dense parent: steps 1-3 along every mode, the parent's strides times the step
void random_view(std::vector<int64_t>& n, std::vector<int64_t>& w)
{
    for (size_t r = 0; r < n.size(); ++r) {
        const int64_t t = uni(1, 3);
        w[r] *= t;
    }
}

template <typename F>
void for_each_index(const std::vector<int64_t>& n, F f)
{
    std::vector<int64_t> i(n.size(), 0);
    for (int64_t x : n)
        if (x == 0) return;
    for (;;) {
        f(i);
        size_t r = 0;
        for (; r < n.size(); ++r) {
            if (++i[r] < n[r]) break;
            i[r] = 0;
        }
        if (r == n.size()) return;
    }
}

int64_t lam(const std::vector<int64_t>& w, const std::vector<int64_t>& i)
{
    int64_t s = 0;
    for (size_t r = 0; r < w.size(); ++r) s += w[r] * i[r];
    return s;
}

// every offset tuple the collapsed space enumerates
std::multiset<std::vector<int64_t>> enumerate(const Space& sp, int nops)
{
    std::multiset<std::vector<int64_t>> out;
    std::vector<int64_t> ext;
    for (int d = 0; d < sp.nd; ++d) ext.push_back(sp.d[d].n);
    for_each_index(ext, [&](const std::vector<int64_t>& i) {
        std::vector<int64_t> o(nops, 0);
        for (int d = 0; d < sp.nd; ++d)
            for (int k = 0; k < nops; ++k) o[k] += i[d] * sp.d[d].s[k];
        out.insert(o);
    });
    return out;
}

int failures = 0;

void fail(const char* what, int it)
{
    std::fprintf(stderr, "mismatch: %s (iteration %d)\n", what, it);
    ++failures;
}

}  // namespace

// The multiply-high division against plain division: small divisors, powers
// of two and random 32-bit divisors and dividends, including the extremes.
void check_fastdiv()
{
    std::vector<uint32_t> ds = {1, 2, 3, 5, 7, 10, 31, 32, 33, 63, 64, 65, 100, 127, 128, 1000,
                                65535, 65536, 65537, 0x7fffffffu, 0x80000000u, 0xffffffffu};
    for (int i = 0; i < 2000; ++i) ds.push_back((uint32_t)uni(1, 0xffffffffLL));
    for (uint32_t d : ds) {
        const FastDiv f = make_fastdiv(d);
        std::vector<uint32_t> ns = {0, 1, d - 1, d, d + 1, 0x7fffffffu, 0x80000000u, 0xfffffffeu,
                                    0xffffffffu};
        for (int i = 0; i < 200; ++i) ns.push_back((uint32_t)uni(0, 0xffffffffLL));
        for (uint32_t n : ns)
            if (fastdiv_host(n, f) != n / d) {
                std::fprintf(stderr, "fastdiv mismatch: %u / %u\n", n, d);
                ++failures;
                return;
            }
    }
}

int main(int argc, char** argv)
{
    const int iters = argc > 1 ? std::atoi(argv[1]) : 2000;
    check_fastdiv();
    static float dummy[1];
    for (int it = 0; it < iters && failures < 5; ++it) {
        const uint32_t p = (uint32_t)uni(1, 7);
        std::vector<int64_t> n(p);
        for (auto& x : n) x = uni(1, 5);
        Desc A, B, C;
        A.n = B.n = C.n = n;
        A.pi = random_perm(p);
        B.pi = random_perm(p);
        C.pi = random_perm(p);
        A.w = strides_of(n, A.pi);
        B.w = strides_of(n, B.pi);
        C.w = strides_of(n, C.pi);
        const bool view = uni(0, 1) == 1;
        if (view) random_view(A.n, A.w);
        A.fill(p, TL_F32, dummy, view);
        B.fill(p, TL_F32, dummy, false);
        C.fill(p, TL_F32, dummy, false);
        Tensor At, Bt, Ct;
        if (load_tensor(&A.t, false, At) || load_tensor(&B.t, false, Bt) ||
            load_tensor(&C.t, true, Ct)) {
            fail("valid descriptor rejected", it);
            continue;
        }
        // entrywise: (A, B, C) offsets of every multi-index
        {
            EwPlan P;
            if (plan_entrywise(TL_ADD, At, &Bt, Ct, P)) {
                fail("entrywise plan", it);
            } else {
                std::multiset<std::vector<int64_t>> ref;
                for_each_index(n, [&](const std::vector<int64_t>& i) {
                    ref.insert({lam(A.w, i), lam(B.w, i), lam(C.w, i)});
                });
                int64_t N = 1;
                for (auto x : n) N *= x;
                if (P.N != N || enumerate(P.sp, 3) != ref) fail("entrywise space", it);
            }
        }
        if (p < 2) continue;
        const uint32_t q = (uint32_t)uni(1, p);
        // ttv: (A offset at i_q = 0, C offset) for every output multi-index
        {
            std::vector<int64_t> nc;
            for (uint32_t r = 0; r < p; ++r)
                if (r != q - 1) nc.push_back(n[r]);
            Desc Cv;
            Cv.n = nc;
            Cv.pi = random_perm(p - 1);
            Cv.w = strides_of(nc, Cv.pi);
            Cv.fill(p - 1, TL_F32, dummy, false);
            Tensor Cvt;
            TtvPlan P;
            if (load_tensor(&Cv.t, true, Cvt) || plan_ttv(At, 1, q, Cvt, P, 152)) {
                fail("ttv plan", it);
            } else {
                std::multiset<std::vector<int64_t>> ref;
                for_each_index(n, [&](const std::vector<int64_t>& i) {
                    if (i[q - 1] != 0) return;
                    std::vector<int64_t> ic;
                    for (uint32_t r = 0; r < p; ++r)
                        if (r != q - 1) ic.push_back(i[r]);
                    ref.insert({lam(A.w, i), lam(Cv.w, ic)});
                });
                if (P.nq != n[q - 1] || (P.nq > 1 && P.saq != A.w[q - 1]) ||
                    enumerate(P.out, 2) != ref)
                    fail("ttv space", it);
            }
        }
        // ttm with J rows: (A offset at i_q = 0, C offset at j = 0) per row
        {
            const int64_t J = uni(1, 6);
            Desc Cm;
            Cm.n = n;
            Cm.n[q - 1] = J;
            Cm.pi = random_perm(p);
            Cm.w = strides_of(Cm.n, Cm.pi);
            Cm.fill(p, TL_F32, dummy, false);
            Tensor Cmt;
            TtmPlan P;
            if (load_tensor(&Cm.t, true, Cmt) ||
                plan_ttm(At, J, n[q - 1], 1, q, Cmt, TL_P_DEFAULT, P)) {
                fail("ttm plan", it);
            } else {
                std::multiset<std::vector<int64_t>> ref;
                for_each_index(n, [&](const std::vector<int64_t>& i) {
                    if (i[q - 1] != 0) return;
                    ref.insert({lam(A.w, i), lam(Cm.w, i)});
                });
                if (P.J != J || P.scq != Cm.w[q - 1] || enumerate(P.rows, 2) != ref)
                    fail("ttm space", it);
            }
        }
        // invalid descriptors are rejected, not read out of bounds
        {
            Desc X = A;
            X.pi = A.pi;
            if (p > 1) X.pi[0] = X.pi[1];
            X.fill(p, TL_F32, dummy, false);
            Tensor Xt;
            if (p > 1 && load_tensor(&X.t, false, Xt) != TL_EINVAL) fail("repeated pi accepted", it);
            Desc Y = C;
            Y.w = std::vector<int64_t>(p, 0);
            Y.fill(p, TL_F32, dummy, true);
            if (load_tensor(&Y.t, true, Xt) != TL_EINVAL) fail("zero stride accepted", it);
            tl_tensor Z = C.t;
            Z.p = 0;
            if (load_tensor(&Z, false, Xt) != TL_EINVAL) fail("order 0 accepted", it);
            Z.p = TL_MAX_ORDER + 1;
            if (load_tensor(&Z, false, Xt) != TL_EINVAL) fail("order > max accepted", it);
        }
    }
    if (failures) return 1;
    std::printf("ok %d\n", iters);
    return 0;
}
