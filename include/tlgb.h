/*
 * tlgb.h -- C ABI of the GB300-native (sm_103a) tensor-times-vector,
 * tensor-times-matrix and entrywise library.
 *
 * The operations are those of Bassoy, "TLib: A Flexible C++ Tensor Framework
 * for Numerical Tensor Calculus" (arXiv 1711.10912):
 *   tl_ttv        mode-q tensor-times-vector, Sec. 5.2 Eq. 24
 *   tl_ttm        mode-q tensor-times-matrix, Sec. 5.2 Eq. 25
 *   tl_entrywise  layout-mixed entrywise ops, Sec. 5.1 Eqs. 22-23
 *   tl_norm       Frobenius norm, Sec. 5.2 Table 3
 * on dense or strided order-p tensors whose order p, extents n, layout tuple
 * pi and strides w (Sec. 3.1 Eqs. 12-14, Sec. 3.2 Eq. 17) are runtime values.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Modes q and layout tuples pi are 1-based, as in the paper's equations;
 *    multi-indices are 0-based with zero index offsets: `data` points at the
 *    element with multi-index (0,...,0) (a view's first element, Eq. 18).
 *  - Strides are in elements.  w == NULL derives the dense strides from pi by
 *    Eq. 14; pi == NULL means the first-order layout (1,...,p) (Eq. 12).
 *    Given strides must be >= 1; an output's strides must not make two of
 *    its elements share an address.
 *  - Extents n_r >= 1 (extent-1 modes are allowed and collapsed away).
 *  - Every data pointer is DEVICE memory owned by the caller; the library
 *    never frees it.  Descriptor arrays (n, pi, w) are host memory read
 *    during the call only.
 *  - Calls enqueue kernels on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and return without synchronising.  Argument errors are returned
 *    synchronously and enqueue nothing.
 *  - Outputs must not overlap any input (entrywise allows C == A or C == B
 *    when the two descriptors are identical).
 *  - Scratch memory: kernels that split a reduction across CTAs keep their
 *    partial sums in a per-(device, stream) workspace owned by the library.
 *    It is allocated (cudaMalloc) the first time a call on that stream needs
 *    more than it holds, and reused afterwards; make one call of each shape
 *    before capturing a stream into a CUDA graph.
 *
 * Return codes: TL_OK (0) or a negative TL_E* code; tl_strerror() names it.
 */
#ifndef TLGB_H
#define TLGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TL_OK            0
#define TL_EINVAL       -1   /* bad descriptor: p, q, pi not a permutation, shape mismatch */
#define TL_EUNSUPPORTED -2   /* dtype / precision combination not offered */
#define TL_ENOMEM       -3   /* admission or workspace allocation failed */
#define TL_ECUDA        -4   /* a CUDA launch or runtime call failed */
#define TL_ETIMEOUT     -5   /* a bounded device wait gave up */
#define TL_ECANCELED    -6   /* request cancelled or failed by the host */
#define TL_EBOUNDS      -7   /* bounds-checked builds only: a mapped offset left its operand */
#define TL_PENDING       1   /* tl_poll: the request has not completed yet */

#define TL_MAX_ORDER 16

/* element types of tensor data */
#define TL_F32 0
#define TL_F64 1

/* compute precision of tl_ttm */
#define TL_P_DEFAULT 0   /* the data type's own: FP32 or FP64 SIMT */
#define TL_P_F64     1   /* FP64 data, FP64 arithmetic */
#define TL_P_F32     2   /* FP32 data, FP32 FMA arithmetic */
#define TL_P_TF32    3   /* FP32 data, TF32 tensor-core products, FP32 accumulation */
#define TL_P_BF16    4   /* FP32 data rounded to BF16, FP32 accumulation */
#define TL_P_BF16X3  5   /* FP32 data split into BF16 hi+lo, hi*hi+hi*lo+lo*hi, FP32 accumulation */

/* entrywise operations (Sec. 5.1): C = A op B, COPY: C = A, SCALE: C = alpha*A */
#define TL_ADD   0
#define TL_SUB   1
#define TL_MUL   2
#define TL_DIV   3
#define TL_COPY  4
#define TL_SCALE 5

/*
 * Tensor descriptor: the (p, n, pi, w, data) description of Sec. 3.1-3.2.
 * n[0..p-1] extents; pi[0..p-1] 1-based layout tuple or NULL; w[0..p-1]
 * strides in elements or NULL; data = device address of element (0,...,0).
 */
typedef struct tl_tensor {
    uint32_t       p;
    int32_t        dtype;     /* TL_F32 or TL_F64 */
    const int64_t* n;
    const uint32_t* pi;
    const int64_t* w;
    void*          data;
} tl_tensor;

/*
 * tl_ttv -- mode-q tensor-times-vector, Sec. 5.2 Eq. 24:
 *   C(i_1..i_{q-1}, i_{q+1}..i_p) = sum_{k=0}^{n_q-1} A(i_1..k..i_p) * b(k)
 * A: order p >= 2, any layout/strides.  b: device vector of n_q elements of
 * A's dtype, element k at b[k*incb] (incb >= 1).  C: order p-1 with A's
 * extents without mode q, same dtype, any layout/strides.
 * accumulate = 0 overwrites C ('=' of Eq. 24); accumulate = 1 adds the sum
 * to C's current value (the initial value of the paper's inner product).
 * FP32 data accumulates in FP32, FP64 data in FP64.
 * Errors: TL_EINVAL (p < 2, q outside 1..p, bad pi/w/extents, C's shape or
 * dtype does not match), TL_ENOMEM (workspace), TL_ECUDA (launch).
 */
int tl_ttv(const tl_tensor* A, const void* b, int64_t incb, uint32_t q,
           const tl_tensor* C, int32_t accumulate, void* stream);

/*
 * tl_ttv_noalloc -- tl_ttv that allocates no device memory.  The paper has
 * no counterpart; this entry point is for callers that cannot let a library
 * call cudaMalloc: runtimes that own every byte of device memory through
 * their own allocator and budget (an allocation behind their back can fail
 * or break the budget), and latency-critical loops in which a cudaMalloc /
 * cudaFree, which can synchronise the device, is not acceptable.
 * Arguments, results and errors are those of tl_ttv, with these differences:
 *  - Scratch: when the planner splits the contraction across CTAs, the
 *    partial sums go to one static device array of
 *    TL_TTV_NOALLOC_SCRATCH_BYTES (4 MiB) that belongs to the library image:
 *    every GPU that loads the library holds it until the process exits.  A
 *    call whose partial sums would need more returns TL_ENOMEM and enqueues
 *    nothing; tl_ttv (which grows a workspace) handles such calls.
 *  - The first call on a device looks the array's device address up (once
 *    per device, with that device current); make that first call before any
 *    stream capture.
 *  - All calls on a device share the array, which keeps the last call's
 *    contents.  Every partial sum is written before it is read, so nothing
 *    needs clearing; but calls whose kernels overlap on the GPU (for example
 *    on two streams without an event between them) race on the array and
 *    must be serialised by the caller.
 */
#define TL_TTV_NOALLOC_SCRATCH_BYTES (4u << 20)
int tl_ttv_noalloc(const tl_tensor* A, const void* b, int64_t incb, uint32_t q,
                   const tl_tensor* C, int32_t accumulate, void* stream);

/*
 * tl_ttm -- mode-q tensor-times-matrix, Sec. 5.2 Eq. 25:
 *   C(i_1..j..i_p) = sum_{k=0}^{n_q-1} A(i_1..k..i_p) * B(j, k),  0 <= j < J
 * B: device J x n_q matrix of A's dtype, B(j,k) at B[j*ldb_row + k*ldb_col]
 * (row-major: ldb_row = n_q, ldb_col = 1).  C: A's extents with n_q
 * replaced by J, same dtype, any layout/strides.  precision selects the
 * arithmetic (TL_P_*); TF32, BF16 and BF16X3 need FP32 data and run on the
 * tcgen05 tensor cores when the shape is dense enough (else they fall back
 * to FP32 SIMT, which is at least as accurate).  accumulate as in tl_ttv.
 * Errors: TL_EINVAL, TL_EUNSUPPORTED (precision not valid for the dtype),
 * TL_ENOMEM, TL_ECUDA.
 */
int tl_ttm(const tl_tensor* A, const void* B, int64_t J, int64_t ldb_row, int64_t ldb_col,
           uint32_t q, const tl_tensor* C, int32_t precision, int32_t accumulate,
           void* stream);

/*
 * tl_entrywise -- Sec. 5.1 Eq. 23 (C(i) = A(i) op B(i)) and Eq. 22
 * (C(i) = alpha * A(i)) over every multi-index i of A's shape; A, B and C
 * may each have their own layout and strides (COPY with a different output
 * layout is the paper's relayout, Sec. 3.2).  B must be NULL for COPY and
 * SCALE and have A's shape and dtype otherwise.  alpha is used by SCALE only.
 * Errors: TL_EINVAL, TL_ECUDA.
 */
int tl_entrywise(int32_t op, const tl_tensor* A, const tl_tensor* B, double alpha,
                 const tl_tensor* C, void* stream);

/*
 * tl_ttvs -- tensor times several vectors (Sec. 5.2 Table 3, times_vectors):
 * vecs[j] (device, n_{modes[j]} contiguous elements of A's dtype) along the
 * distinct 1-based modes[j], applied from the last listed to the first (the
 * order the paper states, which keeps the remaining mode numbers valid); at
 * least one mode remains (count < p).  C: order p - count with A's remaining
 * extents in order, any layout.  Each step is a tl_ttv; intermediates are
 * dense, in the layout A's layout induces, in a per-stream workspace slot of
 * the library (allocated on first need, like the split-K workspace).
 * Errors: TL_EINVAL (repeated or out-of-range mode, count >= p, C's shape),
 * TL_ENOMEM, TL_ECUDA.
 */
int tl_ttvs(const tl_tensor* A, const void* const* vecs, const uint32_t* modes, uint32_t count,
            const tl_tensor* C, void* stream);

/*
 * tl_ttms -- tensor times several matrices (Sec. 5.2 Table 3,
 * times_matrices; e.g. a Tucker projection): mats[j] (device, J[j] x
 * n_{modes[j]}, row-major) along the distinct modes[j], last listed first.
 * C: A's extents with n_{modes[j]} replaced by J[j].  precision as tl_ttm,
 * for every step.  Intermediates as in tl_ttvs (A's layout).
 */
int tl_ttms(const tl_tensor* A, const void* const* mats, const int64_t* J, const uint32_t* modes,
            uint32_t count, const tl_tensor* C, int32_t precision, void* stream);

/*
 * tl_hopm -- the higher-order power method of the paper's last listing
 * (Sec. 5.2, best rank-1 approximation after De Lathauwer et al.): K sweeps;
 * in each, for r = 1..p: u_r <- A times every u except u_r (tl_ttvs with
 * mode r excluded), lambda_r <- ||u_r||_F (tl_norm, FP64), u_r <- u_r /
 * lambda_r.  u[r] (device, n_r contiguous elements of A's dtype) hold the
 * starting vectors and receive the results; lambda (device, p doubles)
 * receives the last sweep's norms.  Everything stays on the device.
 */
int tl_hopm(const tl_tensor* A, void* const* u, double* lambda, uint32_t K, void* stream);

/*
 * tl_transpose -- C = A^tau (Table 3, transpose): C(i^c) = A(i^a) with
 * i^c_r = i^a_{tau_r}, so C's extents are n^c_r = n^a_{tau_r}.  tau: p
 * 1-based entries, a permutation.  C: any layout or strides.  Runs as an
 * entrywise copy from A described in C's mode order (tiled transpose when
 * the fastest modes differ).  Errors: TL_EINVAL (tau not a permutation, C's
 * order or extents), as tl_entrywise otherwise.
 */
int tl_transpose(const tl_tensor* A, const uint32_t* tau, const tl_tensor* C, void* stream);

/*
 * tl_ttt -- the (q, phi, psi)-mode tensor-tensor product of Sec. 5.2 (Eqs. 26-27):
 * A of order q+r, B of order q+s, C of order r+s,
 *   C(i^c) = sum over the q contraction indices j of A(i^a) * B(i^b),
 *   i^a_{phi_k} = i^c_k (k <= r),  i^b_{psi_k} = i^c_{r+k} (k <= s),
 *   i^a_{phi_{r+k}} = i^b_{psi_{s+k}} = j_k (k <= q),
 * phi (q+r entries) and psi (q+s entries) 1-based permutations, with
 * n^a_{phi_{r+k}} = n^b_{psi_{s+k}}.  q = 0 is the outer product; r = s = 0
 * the inner product, whose C is one element (C->p = 0, or p = 1 with n = 1).
 * precision as tl_ttm (the tensor-core precisions apply when the product
 * runs as a ttm); accumulate != 0 adds to C.  Runs as one mode-1 ttv / ttm
 * over re-described operands; operands whose strides do not allow that are
 * first copied to dense layouts in per-stream workspace slots of the library,
 * and C is written through a dense temporary when its strides do not allow
 * it.  C must not overlap A or B.  Errors: TL_EINVAL (permutations, extents,
 * C's shape), TL_EUNSUPPORTED (precision vs dtype), TL_ENOMEM, TL_ECUDA.
 */
int tl_ttt(const tl_tensor* A, const uint32_t* phi, const tl_tensor* B, const uint32_t* psi,
           uint32_t q, const tl_tensor* C, int32_t precision, int32_t accumulate, void* stream);

/*
 * tl_norm -- Frobenius norm ||A||_F = sqrt(sum_i A(i)^2) (Table 3, norm),
 * accumulated in FP64 with a deterministic two-pass block reduction.
 * result: device pointer to three doubles, written asynchronously:
 * {||A||_F, ||A||_F, 0} (the layout of tl_rel_error's result).
 */
int tl_norm(const tl_tensor* A, double* result, void* stream);

/*
 * tl_rel_error -- ||X - R||_F / ||R||_F over two tensors of equal shape
 * (each in its own layout and dtype), in FP64 with the same deterministic
 * reduction; the error measure the library's parity checks report.
 * result: device pointer to three doubles {ratio, ||X-R||_F, ||R||_F}.
 */
int tl_rel_error(const tl_tensor* X, const tl_tensor* R, double* result, void* stream);

/* Name of a return code. */
const char* tl_strerror(int code);

/* Library version (major*10000 + minor*100 + patch). */
int tl_version(void);

/*
 * tl_bounds_checked -- 1 for the bounds-checked debug build of the library
 * (built with TL_CHECK_BOUNDS, libtlgb_checked.so), 0 for the product build.
 * In the checked build every offset that the kernels' index mappers produce
 * (the first element of each row, fiber or vector a thread touches, for
 * every operand) is compared with that operand's extent in memory, less the
 * accesses the plan adds along the contraction (A) or the output column (C
 * of ttm); an offset outside is recorded, replaced by 0 (the access stays
 * inside the operand) and reported by tl_device_status() as TL_EBOUNDS.
 * Kernels that address memory through TMA tensor maps (the tensor-core ttm,
 * the TMA entrywise tiles) are bounded by the maps' extents instead.
 */
int tl_bounds_checked(void);

/* Number of kernels this library has launched in this process (all devices,
   all streams), for launch accounting in benchmarks. */
uint64_t tl_launch_count(void);

/*
 * tl_device_status -- synchronises `stream`, then reports whether any
 * bounded device-side wait of the library's pipelined kernels gave up since
 * the last call: TL_ETIMEOUT (and the flag is cleared) or TL_OK; in the
 * bounds-checked build also TL_EBOUNDS (see tl_bounds_checked).  Such a
 * kernel does not hang: after about two seconds without progress it records
 * the timeout, drains its own copies, frees its tensor memory and returns,
 * leaving its output incomplete.
 */
int tl_device_status(void* stream);

/*
 * tl_selftest_wait_timeout -- launches one tiny kernel whose thread waits on
 * a barrier that nothing completes, with a limit of about `limit_us`
 * microseconds; the wait gives up, records the timeout exactly as the
 * pipelined kernels do and returns.  A following tl_device_status() reports
 * TL_ETIMEOUT.  Exercises the timeout path without hanging the GPU.
 */
int tl_selftest_wait_timeout(double limit_us, void* stream);

/*
 * tl_fma_peak_probe -- measurement helper with no counterpart in the paper:
 * enqueues one kernel that keeps every SM's FP32 FMA (dtype TL_F32) or FP64
 * DFMA (TL_F64) pipes busy with independent fused multiply-adds, `iters`
 * per chain (a positive multiple of 16), and writes the floating-point
 * operations it performs (2 per FMA) to *flops (host).  Timing it with
 * events on `stream` gives the device's measured FMA rate, the peak that
 * FP32 SIMT and FP64 operations are compared against.  sink: device pointer
 * to one element of the dtype (written only for a result no chain reaches,
 * so the arithmetic cannot be optimised away).  Changes no device setting.
 * Errors: TL_EINVAL (dtype, iters, null pointers), TL_ECUDA.
 */
int tl_fma_peak_probe(int32_t dtype, int64_t iters, void* sink, double* flops, void* stream);

/*
 * tl_view -- host-only: the descriptor of a view of A (Sec. 3.3): for every
 * mode r a range with first index f[r], step t[r] and last index l[r]
 * (inclusive), 0 <= f[r] <= l[r] < n_r and t[r] >= 1.  The view has extents
 * n'_r = (l_r - f_r) / t_r + 1 (Eq. 5), strides w'_r = w_r * t_r (Eq. 19,
 * with w the strides of the tensor the view refers to, so views of views
 * compose) and its first element at offset gamma = sum_r f_r w_r (Eq. 18).
 * Writes V = {A->p, A->dtype, n_out, NULL, w_out, A->data + gamma elements};
 * n_out and w_out are caller arrays of p entries that V points into.  Only
 * pointer arithmetic: the data are not touched.  Errors: TL_EINVAL.
 */
int tl_view(const tl_tensor* A, const int64_t* f, const int64_t* t, const int64_t* l,
            tl_tensor* V, int64_t* n_out, int64_t* w_out);

/*
 * tl_plan_describe -- host-only: validates the arguments of a ttv (op 0),
 * ttm (op 1) or entrywise (op 2) call exactly as the entry point would and
 * writes a one-line JSON description of the collapsed iteration space and
 * the kernel that would run into buf (NUL-terminated, truncated to buflen).
 * Touches no GPU.  For ttm, `J` and `precision` are used; `entry_op` is the
 * entrywise op.  Returns TL_OK or the error the entry point would return.
 */
int tl_plan_describe(int32_t op, const tl_tensor* A, const tl_tensor* B, uint32_t q,
                     int64_t J, int32_t precision, int32_t entry_op,
                     const tl_tensor* C, char* buf, size_t buflen);

/* ------------------------------------------------------------------------
 * Batched and served execution (no counterpart in the paper: these are the
 * systems layers around the three operations above).
 * ---------------------------------------------------------------------- */

#define TL_OP_TTV       0
#define TL_OP_TTM       1
#define TL_OP_ENTRYWISE 2

/*
 * One operation of a batch: kind selects which fields are used.
 *   TTV:       A, vec (b), incb, q, C, accumulate
 *   TTM:       A, vec (B), J, ldb_row, ldb_col, q, C, precision, accumulate
 *   ENTRYWISE: A, B (NULL-data for COPY/SCALE), C, entry_op, alpha
 * Tensor descriptors and their arrays are copied at submission; data
 * pointers must stay valid until the request completes.
 */
typedef struct tl_op {
    int32_t   kind;
    int32_t   entry_op;
    int32_t   precision;
    int32_t   accumulate;
    uint32_t  q;
    uint32_t  reserved;
    int64_t   J, ldb_row, ldb_col, incb;
    double    alpha;
    const void* vec;
    tl_tensor A, B, C;
} tl_op;

/*
 * Batched persistent launch: many operations of uneven order, extents and
 * layout in one launch.  tl_batch_create validates and plans every
 * operation (exactly as the single-call entry points would), cuts each into
 * work units and uploads one descriptor table; tl_batch_run enqueues one
 * persistent kernel that takes units from an atomic counter (operations it
 * does not take, such as tensor-core ttm, run through their own kernels).
 * flags: TL_BATCH_GRAPH captures the launch into a CUDA graph on the first
 * run and replays it afterwards; TL_BATCH_TUNE picks each shape class's
 * unit size and per-unit code by timing the candidates once (on `stream`,
 * at creation) and caching the choice in the file $TL_TUNE_CACHE (default
 * ~/.cache/tlgb_tune.txt).  tl_batch_create allocates the table and
 * synchronises `stream`; the data pointers of the operations must stay
 * valid for every run.  tl_batch_describe writes a JSON summary.
 */
typedef struct tl_batch tl_batch;
#define TL_BATCH_GRAPH 1
#define TL_BATCH_TUNE  2
int tl_batch_create(const struct tl_op* ops, size_t count, int32_t flags, void* stream,
                    tl_batch** out);
int tl_batch_run(tl_batch* batch, void* stream);
int tl_batch_destroy(tl_batch* batch);
int tl_batch_describe(const tl_batch* batch, char* buf, size_t buflen);

/*
 * Overrides the per-unit code of every operation of one kind in a batch
 * (for tuning experiments and tests): kind TL_OP_TTV with variant
 * TL_BV_TTV_COL (a thread per output), TL_BV_TTV_ROW4/8/32 (4, 8 or 32
 * lanes per output) or TL_BV_TTV_VEC (16 bytes of outputs per thread; applied
 * only where the outputs are contiguous in A and C, unit rounded up to whole
 * vectors), TL_OP_TTM with TL_BV_TTM_32 / TL_BV_TTM_64 (row tiles)
 * or TL_BV_TTM_SMALL (the matrix in shared memory, a row per thread; applied
 * only to operations with n_q <= 64 and J <= 64, or J <= 32 for FP64),
 * TL_OP_ENTRYWISE with TL_BV_EW.  `unit` is the outputs (rows for ttm) per
 * work unit, rounded up to whole row tiles for TL_BV_TTM_32 / 64.  Re-uploads the table (synchronising `stream`) and
 * drops a captured graph.
 */
#define TL_BV_TTV_COL   0
#define TL_BV_TTV_ROW4  1
#define TL_BV_TTV_ROW8  2
#define TL_BV_TTV_ROW32 3
#define TL_BV_TTM_32    4
#define TL_BV_TTM_64    5
#define TL_BV_EW        6
#define TL_BV_TTM_SMALL 7
#define TL_BV_TTV_VEC   8
int tl_batch_set_variant(tl_batch* batch, int32_t kind, int32_t variant, int64_t unit,
                         void* stream);

typedef struct tl_ctx tl_ctx;

/* Context flags */
#define TL_CTX_PERSISTENT 1   /* run batches through the persistent batched kernel */
#define TL_CTX_GRAPH      2   /* replay the persistent launch from a CUDA graph */

/*
 * tl_ctx_create -- a request context on the current device: `budget_bytes`
 * bounds the bytes of operands and outputs of requests admitted but not yet
 * completed (requests beyond it wait; a single request larger than the
 * budget is rejected with TL_ENOMEM), `streams` (>= 1) device streams carry
 * concurrent batches of small requests, at the highest stream priority; one
 * more stream, at the lowest priority, runs requests of 16 MB or more one at
 * a time (small requests queued behind one pass it).  Requests are admitted
 * in arrival order within each of the two classes, and a batch holds at most
 * 256 operations and 64 MB.  The context owns its streams, descriptor tables
 * and workspace and allocates them here.
 */
int tl_ctx_create(size_t budget_bytes, int32_t streams, int32_t flags, tl_ctx** out);
int tl_ctx_destroy(tl_ctx* ctx);

/*
 * tl_batch_submit -- validates `count` operations and enqueues them as one
 * request; returns at once with a ticket.  A request is admitted when the
 * budget allows and a stream is free, then launched as one batch (one
 * persistent launch, or one launch per operation without
 * TL_CTX_PERSISTENT).  Errors: TL_EINVAL (the index of the first bad
 * operation is not reported; use tl_plan_describe), TL_ENOMEM.
 */
int tl_batch_submit(tl_ctx* ctx, const tl_op* ops, size_t count, uint64_t* ticket);

/*
 * tl_poll -- non-blocking status of a ticket: *status = TL_PENDING, TL_OK or
 * a negative error; *latency_ms = submission-to-completion time once done.
 * A ticket is forgotten once its final status has been returned (by tl_poll
 * or tl_wait); asking again returns TL_EINVAL.
 */
int tl_poll(tl_ctx* ctx, uint64_t ticket, int32_t* status, double* latency_ms);

/* Blocks until the ticket completes (or timeout_ms passes: TL_ETIMEOUT). */
int tl_wait(tl_ctx* ctx, uint64_t ticket, double timeout_ms, int32_t* status,
            double* latency_ms);

/* Counters of a context: the most operand + output bytes ever admitted at
   once (never above the budget), batches launched and requests completed. */
int tl_ctx_stats(tl_ctx* ctx, size_t* max_inflight_bytes, uint64_t* batches,
                 uint64_t* completed);

/* Cancels a request that has not been launched yet (its status becomes
   TL_ECANCELED and TL_OK is returned); a launched request runs to completion
   (TL_PENDING is returned). */
int tl_cancel(tl_ctx* ctx, uint64_t ticket);

#ifdef __cplusplus
}
#endif

#endif /* TLGB_H */
