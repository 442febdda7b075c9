// api.cpp -- the extern "C" entry points of tlgb.h: argument validation,
// planning, workspace management and kernel dispatch.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "kernels.h"
#include "plan.h"
#include "runtime.h"

namespace tl {

// ------------------------------------------------------------ device info ---

int device_sms()
{
    // per-device cache in a fixed table: the query path allocates nothing
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < kMaxDevices) {
        int v = cache[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < kMaxDevices) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

int smem_optin(const void* func, int bytes)
{
    struct Done {
        int dev;
        const void* func;
        int bytes;
    };
    static std::mutex mu;
    static std::vector<Done> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TL_ECUDA;
    std::lock_guard<std::mutex> lk(mu);
    for (const Done& d : done)
        if (d.dev == dev && d.func == func && d.bytes >= bytes) return TL_OK;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
        cudaSuccess) {
        cudaGetLastError();
        return TL_ECUDA;
    }
    done.push_back(Done{dev, func, bytes});
    return TL_OK;
}

// Readers of the per-file bounds-violation words of builds with
// TL_CHECK_BOUNDS (empty otherwise).
namespace {
std::mutex g_bounds_mu;
std::vector<int (*)(bool)> g_bounds_readers;
}  // namespace

int register_bounds_reader(int (*reader)(bool))
{
    std::lock_guard<std::mutex> lk(g_bounds_mu);
    g_bounds_readers.push_back(reader);
    return 0;
}

int bounds_status(bool clear)
{
    std::lock_guard<std::mutex> lk(g_bounds_mu);
    int rc = TL_OK;
    for (auto* f : g_bounds_readers) {
        const int r = f(clear);
        if (r != TL_OK && rc == TL_OK) rc = r;
    }
    return rc;
}

bool bounds_checked_build()
{
#ifdef TL_CHECK_BOUNDS
    return true;
#else
    return false;
#endif
}

static std::atomic<uint64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// -------------------------------------------------------------- workspace ---
// One buffer per (device, stream), grown on demand and kept until exit.

namespace {
struct WsKey {
    int dev;
    uintptr_t stream;
    int slot;
    bool operator<(const WsKey& o) const
    {
        if (dev != o.dev) return dev < o.dev;
        if (stream != o.stream) return stream < o.stream;
        return slot < o.slot;
    }
};
struct WsBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_ws_mu;
std::map<WsKey, WsBuf> g_ws;
}  // namespace

void* workspace(cudaStream_t st, size_t bytes) { return workspace_slot(st, bytes, 0); }

void* workspace_slot(cudaStream_t st, size_t bytes, int slot)
{
    if (bytes == 0) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    WsBuf& b = g_ws[WsKey{dev, reinterpret_cast<uintptr_t>(st), slot}];
    if (b.bytes >= bytes) return b.ptr;
    if (b.ptr) {
        // the old buffer may still be read by work queued on this stream
        if (cudaStreamSynchronize(st) != cudaSuccess) return nullptr;
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes < (size_t(1) << 20) ? (size_t(1) << 20) : bytes;
    void* p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    b.ptr = p;
    b.bytes = want;
    return p;
}

// ---------------------------------------------------------------- overlap ---

namespace {
struct Range {
    uintptr_t lo, hi;   // [lo, hi)
};
Range range_of(const Tensor& t)
{
    uintptr_t lo = reinterpret_cast<uintptr_t>(t.data);
    return Range{lo, lo + (uintptr_t)t.span() * t.elem()};
}
Range range_of(const void* p, int64_t span, size_t elem)
{
    uintptr_t lo = reinterpret_cast<uintptr_t>(p);
    return Range{lo, lo + (uintptr_t)span * elem};
}
bool overlaps(Range a, Range b) { return a.lo < b.hi && b.lo < a.hi; }
bool same_desc(const Tensor& a, const Tensor& b)
{
    if (a.data != b.data || a.p != b.p || a.dtype != b.dtype) return false;
    for (uint32_t r = 0; r < a.p; ++r)
        if (a.n[r] != b.n[r] || a.w[r] != b.w[r]) return false;
    return true;
}
}  // namespace

// ----------------------------------------------------------- shared paths ---

int prepare_ttv(const tl_tensor* A_, const void* b, int64_t incb, uint32_t q, const tl_tensor* C_,
                int num_sms, Tensor& A, Tensor& C, TtvPlan& P)
{
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    rc = load_tensor(C_, true, C);
    if (rc) return rc;
    if (!b) return TL_EINVAL;
    rc = plan_ttv(A, incb, q, C, P, num_sms);
    if (rc) return rc;
    Range rc_ = range_of(C);
    if (overlaps(rc_, range_of(A)) || overlaps(rc_, range_of(b, (P.nq - 1) * incb + 1, A.elem())))
        return TL_EINVAL;
    return TL_OK;
}

int prepare_ttm(const tl_tensor* A_, const void* B, int64_t J, int64_t ldb_row, int64_t ldb_col,
                uint32_t q, const tl_tensor* C_, int32_t precision, Tensor& A, Tensor& C,
                TtmPlan& P)
{
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    rc = load_tensor(C_, true, C);
    if (rc) return rc;
    if (!B || ldb_row < 0 || ldb_col < 0) return TL_EINVAL;
    rc = plan_ttm(A, J, ldb_row, ldb_col, q, C, precision, P);
    if (rc) return rc;
    Range rc_ = range_of(C);
    int64_t bspan = (J - 1) * ldb_row + (P.nq - 1) * ldb_col + 1;
    if (overlaps(rc_, range_of(A)) || overlaps(rc_, range_of(B, bspan, A.elem())))
        return TL_EINVAL;
    return TL_OK;
}

int prepare_entrywise(int32_t op, const tl_tensor* A_, const tl_tensor* B_, const tl_tensor* C_,
                      Tensor& A, Tensor& B, Tensor& C, bool& hasB, EwPlan& P)
{
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    rc = load_tensor(C_, true, C);
    if (rc) return rc;
    hasB = (B_ != nullptr);
    if (hasB) {
        rc = load_tensor(B_, false, B);
        if (rc) return rc;
    }
    rc = plan_entrywise(op, A, hasB ? &B : nullptr, C, P);
    if (rc) return rc;
    Range rc_ = range_of(C);
    if (overlaps(rc_, range_of(A)) && !same_desc(A, C)) return TL_EINVAL;
    if (hasB && overlaps(rc_, range_of(B)) && !same_desc(B, C)) return TL_EINVAL;
    return TL_OK;
}

int ttm_launches(const TtmPlan& P)
{
    return P.kernel == K_TTM_TC ? ttm_tc_launches(P) : ttm_simt_launches(P, device_sms());
}

int run_ttm(const TtmPlan& P, const void* A, const void* B, void* C, int accumulate, int sms,
            cudaStream_t st)
{
    if (P.kernel == K_TTM_TC) return launch_ttm_tc(P, A, B, C, accumulate, sms, st);
    void* ws = nullptr;
    const size_t wsb = ttm_simt_workspace_bytes(P, sms);
    if (wsb) {
        ws = workspace(st, wsb);
        if (!ws) return TL_ENOMEM;
    }
    return launch_ttm_simt(P, A, B, C, accumulate, ws, sms, st);
}

}  // namespace tl

using namespace tl;

extern "C" {

int tl_version(void) { return 100; }

int tl_bounds_checked(void) { return bounds_checked_build() ? 1 : 0; }

uint64_t tl_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int tl_selftest_wait_timeout(double limit_us, void* stream)
{
    int rc = selftest_wait_timeout(limit_us, static_cast<cudaStream_t>(stream));
    if (rc == TL_OK) count_launches(1);
    return rc;
}

int tl_device_status(void* stream)
{
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return TL_ECUDA;
    int a = ttm_tc_status(true);
    int b = ttv_status(true);
    int c = ew_status(true);
    int d = bounds_status(true);
    if (a == TL_ECUDA || b == TL_ECUDA || c == TL_ECUDA || d == TL_ECUDA) return TL_ECUDA;
    if (a == TL_ETIMEOUT || b == TL_ETIMEOUT || c == TL_ETIMEOUT) return TL_ETIMEOUT;
    return d;
}

const char* tl_strerror(int code)
{
    switch (code) {
    case TL_OK: return "ok";
    case TL_EINVAL: return "invalid argument";
    case TL_EUNSUPPORTED: return "unsupported dtype/precision combination";
    case TL_ENOMEM: return "out of memory or over the admission budget";
    case TL_ECUDA: return "CUDA error";
    case TL_ETIMEOUT: return "device wait timed out";
    case TL_ECANCELED: return "request cancelled";
    case TL_EBOUNDS: return "a mapped offset fell outside its operand (bounds-checked build)";
    case TL_PENDING: return "pending";
    default: return "unknown error";
    }
}

int tl_ttv(const tl_tensor* A_, const void* b, int64_t incb, uint32_t q, const tl_tensor* C_,
           int32_t accumulate, void* stream)
{
    NvtxRange nvtx_range("tl_ttv");
    Tensor A, C;
    TtvPlan P;
    int sms = device_sms();
    if (sms <= 0) return TL_ECUDA;
    int rc = prepare_ttv(A_, b, incb, q, C_, sms, A, C, P);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* ws = nullptr;
    size_t wb = ttv_workspace_bytes(P);
    if (wb) {
        ws = workspace(st, wb);
        if (!ws) return TL_ENOMEM;
    }
    rc = launch_ttv(P, A.data, b, C.data, ws, accumulate ? 1 : 0, sms, st);
    if (rc == TL_OK) count_launches(P.splits > 1 ? 2 : 1);
    return rc;
}

int tl_ttm(const tl_tensor* A_, const void* B, int64_t J, int64_t ldb_row, int64_t ldb_col,
           uint32_t q, const tl_tensor* C_, int32_t precision, int32_t accumulate, void* stream)
{
    NvtxRange nvtx_range("tl_ttm");
    Tensor A, C;
    TtmPlan P;
    int sms = device_sms();
    if (sms <= 0) return TL_ECUDA;
    int rc = prepare_ttm(A_, B, J, ldb_row, ldb_col, q, C_, precision, A, C, P);
    if (rc) return rc;
    rc = run_ttm(P, A.data, B, C.data, accumulate ? 1 : 0, sms, static_cast<cudaStream_t>(stream));
    if (rc == TL_OK) count_launches(ttm_launches(P));
    return rc;
}

int tl_entrywise(int32_t op, const tl_tensor* A_, const tl_tensor* B_, double alpha,
                 const tl_tensor* C_, void* stream)
{
    NvtxRange nvtx_range("tl_entrywise");
    Tensor A, B, C;
    EwPlan P;
    bool hasB = false;
    int sms = device_sms();
    if (sms <= 0) return TL_ECUDA;
    int rc = prepare_entrywise(op, A_, B_, C_, A, B, C, hasB, P);
    if (rc) return rc;
    rc = launch_entrywise(P, A.data, hasB ? B.data : nullptr, alpha, C.data, sms,
                          static_cast<cudaStream_t>(stream));
    if (rc == TL_OK && P.N > 0) count_launches(1);
    return rc;
}

static int norm_common(const Tensor& X, const Tensor* R, double* result, cudaStream_t st)
{
    Space sp;
    sp.nops = 2;
    for (uint32_t r = 0; r < X.p; ++r) {
        Dim& d = sp.d[sp.nd++];
        d.n = X.n[r];
        d.s[0] = X.w[r];
        d.s[1] = R ? R->w[r] : 0;
        d.s[2] = 0;
    }
    collapse(sp, 0);
    sp.limit[0] = X.span();
    sp.limit[1] = R ? R->span() : X.span();
    int nb = norm_partial_blocks(sp.count(), device_sms());
    double* partials = static_cast<double*>(workspace(st, sizeof(double) * 2 * (size_t)nb));
    if (!partials) return TL_ENOMEM;
    int rc = launch_norm(sp, X.dtype, X.data, R ? R->dtype : X.dtype, R ? R->data : nullptr,
                         partials, nb, result, st);
    if (rc == TL_OK) count_launches(2);
    return rc;
}

int tl_norm(const tl_tensor* A_, double* result, void* stream)
{
    NvtxRange nvtx_range("tl_norm");
    Tensor A;
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    if (!result) return TL_EINVAL;
    return norm_common(A, nullptr, result, static_cast<cudaStream_t>(stream));
}

int tl_rel_error(const tl_tensor* X_, const tl_tensor* R_, double* result, void* stream)
{
    NvtxRange nvtx_range("tl_rel_error");
    Tensor X, R;
    int rc = load_tensor(X_, false, X);
    if (rc) return rc;
    rc = load_tensor(R_, false, R);
    if (rc) return rc;
    if (!result || X.p != R.p) return TL_EINVAL;
    for (uint32_t r = 0; r < X.p; ++r)
        if (X.n[r] != R.n[r]) return TL_EINVAL;
    return norm_common(X, &R, result, static_cast<cudaStream_t>(stream));
}

static void append_space(std::string& s, const Space& sp)
{
    s += "[";
    for (int i = 0; i < sp.nd; ++i) {
        char b[128];
        std::snprintf(b, sizeof b, "%s[%lld", i ? "," : "", (long long)sp.d[i].n);
        s += b;
        for (int o = 0; o < sp.nops; ++o) {
            std::snprintf(b, sizeof b, ",%lld", (long long)sp.d[i].s[o]);
            s += b;
        }
        s += "]";
    }
    s += "]";
}

int tl_view(const tl_tensor* A_, const int64_t* f, const int64_t* t, const int64_t* l,
            tl_tensor* V, int64_t* n_out, int64_t* w_out)
{
    Tensor A;
    int rc = load_tensor(A_, false, A);
    if (rc) return rc;
    if (!f || !t || !l || !V || !n_out || !w_out) return TL_EINVAL;
    int64_t gamma = 0;
    for (uint32_t r = 0; r < A.p; ++r)
        if (t[r] < 1 || f[r] < 0 || f[r] > l[r] || l[r] >= A.n[r]) return TL_EINVAL;
    for (uint32_t r = 0; r < A.p; ++r) {
        n_out[r] = (l[r] - f[r]) / t[r] + 1;
        w_out[r] = A.w[r] * t[r];
        gamma += f[r] * A.w[r];
    }
    V->p = A.p;
    V->dtype = A.dtype;
    V->n = n_out;
    V->pi = nullptr;
    V->w = w_out;
    V->data = static_cast<char*>(A.data) + gamma * (int64_t)A.elem();
    return TL_OK;
}

int tl_plan_describe(int32_t op, const tl_tensor* A_, const tl_tensor* B_, uint32_t q, int64_t J,
                     int32_t precision, int32_t entry_op, const tl_tensor* C_, char* buf,
                     size_t buflen)
{
    const int kSms = 152;   // planning assumes a full GB300 when no GPU is queried
    std::string s;
    char b[512];
    int rc;
    if (op == TL_OP_TTV) {
        Tensor A, C;
        TtvPlan P;
        static const float dummy[1] = {0.f};
        rc = prepare_ttv(A_, dummy, 1, q, C_, kSms, A, C, P);
        if (rc) return rc;
        std::snprintf(b, sizeof b,
                      "{\"op\":\"ttv\",\"kernel\":\"%s\",\"nq\":%lld,\"saq\":%lld,\"nout\":%lld,"
                      "\"vec\":%d,\"lanes\":%d,\"splits\":%d,\"kchunk\":%lld,\"dims\":",
                      kernel_name(P.kernel), (long long)P.nq, (long long)P.saq,
                      (long long)P.nout, P.vec, P.lanes, P.splits, (long long)P.kchunk);
        s = b;
        append_space(s, P.out);
        s += "}";
    } else if (op == TL_OP_TTM) {
        Tensor A, C;
        TtmPlan P;
        static const float dummy[1] = {0.f};
        rc = prepare_ttm(A_, dummy, J, 0, 0, q, C_, precision, A, C, P);
        if (rc) return rc;
        const long long splits =
            P.kernel == K_TTM_SIMT ? (long long)ttm_simt_splits(P, 152, nullptr) : 1;
        std::snprintf(b, sizeof b,
                      "{\"op\":\"ttm\",\"kernel\":\"%s\",\"precision\":%d,\"nq\":%lld,"
                      "\"saq\":%lld,\"J\":%lld,\"scq\":%lld,\"M\":%lld,\"tc_variant\":%d,"
                      "\"splits\":%lld,",
                      kernel_name(P.kernel), P.precision, (long long)P.nq, (long long)P.saq,
                      (long long)P.J, (long long)P.scq, (long long)P.M, P.tc_variant, splits);
        s = b;
        if (P.kernel == K_TTM_TC) s += "\"tc\":" + ttm_tc_describe(P, C.data) + ",";
        if (ttm_skinny(P)) s += "\"skinny\":1,";
        else if (P.kernel == K_TTM_SIMT && P.dtype == TL_F32)
            s += "\"sgemm\":" + ttm_sgemm_describe(P, A.data, C.data, splits > 1) + ",";
        s += "\"dims\":";
        append_space(s, P.rows);
        s += "}";
    } else if (op == TL_OP_ENTRYWISE) {
        Tensor A, B, C;
        EwPlan P;
        bool hasB = false;
        rc = prepare_entrywise(entry_op, A_, B_, C_, A, B, C, hasB, P);
        if (rc) return rc;
        std::snprintf(b, sizeof b,
                      "{\"op\":\"entrywise\",\"kernel\":\"%s\",\"N\":%lld,\"vec\":%d,"
                      "\"tdim\":%d,\"dims\":",
                      kernel_name(P.kernel), (long long)P.N, P.vec, P.tdim);
        s = b;
        append_space(s, P.sp);
        s += "}";
    } else {
        return TL_EINVAL;
    }
    if (buf && buflen) {
        std::strncpy(buf, s.c_str(), buflen - 1);
        buf[buflen - 1] = '\0';
    }
    return TL_OK;
}

}  // extern "C"
