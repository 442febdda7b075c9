// sequence.cu -- chained operations of Sec. 5.2 Table 3 on the device:
//   tl_ttvs  tensor times several vectors (times_vectors)
//   tl_ttms  tensor times several matrices (times_matrices, e.g. a Tucker
//            projection)
//   tl_hopm  the higher-order power method of the paper's last listing
// Each step runs through the single-call entry points (so it is planned and
// launched exactly like a direct call); intermediates stay on the device in
// a dedicated per-stream workspace slot, dense, in the layout the source
// tensor induces (its layout tuple with the contracted mode removed for ttv,
// unchanged for ttm), which keeps every step on a fast kernel.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "kernels.h"
#include "plan.h"
#include "runtime.h"

namespace tl {
namespace {

constexpr int kThreads = 256;

// u[i] = x[i] / nrm[0] in double, rounded to T; *lam = nrm[0].
template <typename T>
__global__ void __launch_bounds__(kThreads) normalize_kernel(const T* __restrict__ x, T* __restrict__ u,
                                                             int64_t n, const double* nrm, double* lam)
{
    const double l = *nrm;
    if (blockIdx.x == 0 && threadIdx.x == 0 && lam) *lam = l;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads)
        u[i] = (T)((double)x[i] / l);
}

// A dense tensor description with owned arrays.
struct Desc {
    uint32_t p = 0;
    int32_t dtype = TL_F32;
    std::vector<int64_t> n;
    std::vector<uint32_t> pi;
    void* data = nullptr;
    tl_tensor view() const
    {
        tl_tensor t{};
        t.p = p;
        t.dtype = dtype;
        t.n = n.data();
        t.pi = pi.data();
        t.w = nullptr;
        t.data = data;
        return t;
    }
};

// Layout tuple of A's strides (modes ordered by increasing stride).
std::vector<uint32_t> layout_of(const Tensor& A)
{
    std::vector<uint32_t> pi(A.p);
    for (uint32_t r = 0; r < A.p; ++r) pi[r] = r + 1;
    for (uint32_t i = 1; i < A.p; ++i) {
        uint32_t x = pi[i];
        int j = (int)i - 1;
        while (j >= 0 && A.w[x - 1] < A.w[pi[j] - 1]) {
            pi[j + 1] = pi[j];
            --j;
        }
        pi[j + 1] = x;
    }
    return pi;
}

// Removes mode m (1-based) from a layout tuple and renumbers.
std::vector<uint32_t> drop_mode(const std::vector<uint32_t>& pi, uint32_t m)
{
    std::vector<uint32_t> out;
    for (uint32_t r : pi)
        if (r != m) out.push_back(r > m ? r - 1 : r);
    return out;
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" {

int tl_ttvs(const tl_tensor* A_, const void* const* vecs, const uint32_t* modes, uint32_t count,
            const tl_tensor* C_, void* stream)
{
    NvtxRange nvtx_range("tl_ttvs");
    Tensor A, C;
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    rc = load_tensor(C_, true, C);
    if (rc) return rc;
    if (!vecs || !modes || count < 1 || count >= A.p) return TL_EINVAL;
    bool used[kMaxDims] = {false};
    for (uint32_t j = 0; j < count; ++j) {
        if (modes[j] < 1 || modes[j] > A.p || used[modes[j] - 1] || !vecs[j]) return TL_EINVAL;
        used[modes[j] - 1] = true;
    }
    // remaining modes must be C's modes, in order
    if (C.p != A.p - count || C.dtype != A.dtype) return TL_EINVAL;
    for (uint32_t r = 0, c = 0; r < A.p; ++r)
        if (!used[r] && C.n[c++] != A.n[r]) return TL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // sizes of the intermediates (steps 1..count-1) and the two buffers
    std::vector<int64_t> ext(A.n, A.n + A.p);
    std::vector<uint32_t> alive(A.p);
    for (uint32_t r = 0; r < A.p; ++r) alive[r] = r + 1;
    int64_t biggest = 0;
    {
        std::vector<int64_t> e = ext;
        std::vector<uint32_t> al = alive;
        for (int j = (int)count - 1; j >= 1; --j) {
            uint32_t q = 0;
            while (al[q] != modes[j]) ++q;
            e.erase(e.begin() + q);
            al.erase(al.begin() + q);
            int64_t c = 1;
            for (int64_t x : e) c *= x;
            if (c > biggest) biggest = c;
        }
    }
    uint8_t* buf = nullptr;
    if (count > 1) {
        buf = static_cast<uint8_t*>(workspace_slot(st, (size_t)2 * biggest * A.elem(), 1));
        if (!buf) return TL_ENOMEM;
    }
    // current tensor: starts as the caller's A (with its own strides)
    tl_tensor cur = *A_;
    Desc curd;                       // owns arrays once cur is an intermediate
    std::vector<uint32_t> pi_cur = layout_of(A);
    int ping = 0;
    for (int j = (int)count - 1; j >= 0; --j) {
        uint32_t q = 0;
        while (alive[q] != modes[j]) ++q;
        Desc nxt;
        nxt.dtype = A.dtype;
        nxt.n = ext;
        nxt.n.erase(nxt.n.begin() + q);
        nxt.p = (uint32_t)nxt.n.size();
        nxt.pi = drop_mode(pi_cur, q + 1);
        tl_tensor out;
        if (j == 0) {
            out = *C_;
        } else {
            nxt.data = buf + (size_t)ping * biggest * A.elem();
            out = nxt.view();
        }
        rc = tl_ttv(&cur, vecs[j], 1, q + 1, &out, 0, stream);
        if (rc) return rc;
        ext = nxt.n;
        alive.erase(alive.begin() + q);
        pi_cur = nxt.pi;
        curd = nxt;
        cur = curd.view();
        ping ^= 1;
    }
    return TL_OK;
}

int tl_ttms(const tl_tensor* A_, const void* const* mats, const int64_t* J, const uint32_t* modes,
            uint32_t count, const tl_tensor* C_, int32_t precision, void* stream)
{
    NvtxRange nvtx_range("tl_ttms");
    Tensor A, C;
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    rc = load_tensor(C_, true, C);
    if (rc) return rc;
    if (!mats || !J || !modes || count < 1 || count > A.p) return TL_EINVAL;
    bool used[kMaxDims] = {false};
    std::vector<int64_t> fin(A.n, A.n + A.p);
    for (uint32_t j = 0; j < count; ++j) {
        if (modes[j] < 1 || modes[j] > A.p || used[modes[j] - 1] || !mats[j] || J[j] < 1)
            return TL_EINVAL;
        used[modes[j] - 1] = true;
        fin[modes[j] - 1] = J[j];
    }
    if (C.p != A.p || C.dtype != A.dtype) return TL_EINVAL;
    for (uint32_t r = 0; r < A.p; ++r)
        if (C.n[r] != fin[r]) return TL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int64_t> ext(A.n, A.n + A.p);
    int64_t biggest = 0;
    {
        std::vector<int64_t> e = ext;
        for (int j = (int)count - 1; j >= 1; --j) {
            e[modes[j] - 1] = J[j];
            int64_t c = 1;
            for (int64_t x : e) c *= x;
            if (c > biggest) biggest = c;
        }
    }
    uint8_t* buf = nullptr;
    if (count > 1) {
        buf = static_cast<uint8_t*>(workspace_slot(st, (size_t)2 * biggest * A.elem(), 1));
        if (!buf) return TL_ENOMEM;
    }
    tl_tensor cur = *A_;
    Desc curd;
    const std::vector<uint32_t> pi = layout_of(A);
    int ping = 0;
    for (int j = (int)count - 1; j >= 0; --j) {
        const uint32_t m = modes[j];
        Desc nxt;
        nxt.dtype = A.dtype;
        nxt.n = ext;
        nxt.n[m - 1] = J[j];
        nxt.p = A.p;
        nxt.pi = pi;
        tl_tensor out;
        if (j == 0) {
            out = *C_;
        } else {
            nxt.data = buf + (size_t)ping * biggest * A.elem();
            out = nxt.view();
        }
        rc = tl_ttm(&cur, mats[j], J[j], ext[m - 1], 1, m, &out, precision, 0, stream);
        if (rc) return rc;
        ext = nxt.n;
        curd = nxt;
        cur = curd.view();
        ping ^= 1;
    }
    return TL_OK;
}

int tl_hopm(const tl_tensor* A_, void* const* u, double* lambda, uint32_t K, void* stream)
{
    NvtxRange nvtx_range("tl_hopm");
    Tensor A;
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    if (!u || !lambda || A.p < 2) return TL_EINVAL;
    for (uint32_t r = 0; r < A.p; ++r)
        if (!u[r]) return TL_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t nmax = 0;
    for (uint32_t r = 0; r < A.p; ++r) nmax = nmax > A.n[r] ? nmax : A.n[r];
    // slot 2: the unnormalised vector and the norm triple
    uint8_t* small = static_cast<uint8_t*>(workspace_slot(st, 64 + (size_t)nmax * 8, 2));
    if (!small) return TL_ENOMEM;
    double* nrm = reinterpret_cast<double*>(small);
    void* tmp = small + 64;
    std::vector<uint32_t> modes;
    std::vector<const void*> vecs;
    const int sms = device_sms();
    for (uint32_t k = 0; k < K; ++k) {
        for (uint32_t r = 1; r <= A.p; ++r) {
            modes.clear();
            vecs.clear();
            for (uint32_t m = 1; m <= A.p; ++m)
                if (m != r) {
                    modes.push_back(m);
                    vecs.push_back(u[m - 1]);
                }
            int64_t nr = A.n[r - 1];
            tl_tensor vt{};
            vt.p = 1;
            vt.dtype = A.dtype;
            vt.n = &nr;
            vt.data = tmp;
            rc = tl_ttvs(A_, vecs.data(), modes.data(), (uint32_t)modes.size(), &vt, stream);
            if (rc) return rc;
            rc = tl_norm(&vt, nrm, stream);
            if (rc) return rc;
            int grid = (int)((nr + kThreads - 1) / kThreads);
            if (grid > sms * 4) grid = sms * 4;
            if (grid < 1) grid = 1;
            if (A.dtype == TL_F64)
                normalize_kernel<double><<<grid, kThreads, 0, st>>>(
                    static_cast<const double*>(tmp), static_cast<double*>(u[r - 1]), nr, nrm,
                    lambda + (r - 1));
            else
                normalize_kernel<float><<<grid, kThreads, 0, st>>>(
                    static_cast<const float*>(tmp), static_cast<float*>(u[r - 1]), nr, nrm,
                    lambda + (r - 1));
            if (cudaGetLastError() != cudaSuccess) return TL_ECUDA;
            count_launches(1);
        }
    }
    return TL_OK;
}

}  // extern "C"
