/*
 * tl_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * mode-q tensor-times-vector (ttv), mode-q tensor-times-matrix (ttm) and
 * entrywise operations of Bassoy, "TLib: A Flexible C++ Tensor Framework
 * for Numerical Tensor Calculus" (arXiv 1711.10912).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * CUDA path.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, helper, table
 * or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Conventions (paper notation):
 *   p        order of the tensor (Sec. 3)
 *   n[r]     extent of mode r (Sec. 3, Eq. 2); n[r] >= 1 is accepted
 *   pi[r]    layout tuple, 1-based permutation of 1..p (Sec. 3.1, Eqs. 12-13)
 *   w[r]     stride of mode r in elements (Sec. 3.1, Eq. 14)
 *   q        contraction mode, 1-based (Sec. 5.2, Eqs. 24-25)
 *   indices  i_r are 0-based with zero index offsets unless an offset tuple
 *            o is passed explicitly (Sec. 3.2, Eq. 17)
 * All arithmetic is IEEE double.  Sums run sequentially over ascending k,
 * the order of the innermost inner product of the paper's recursive ttv and
 * ttm (Sec. 5.2).  An optional Neumaier-compensated mode (Neumaier 1974,
 * "Rundungsfehleranalyse einiger Verfahren zur Summation endlicher
 * Summen") bounds the oracle's own rounding error on long sums.
 *
 * Multi-index sets are walked by an odometer with the first index varying
 * fastest (Sec. 3, Eq. 3; the paper's loops nest the first dimension
 * innermost).
 *
 * Every function returns 0 on success and a negative value on invalid
 * arguments; nothing here allocates memory except the small odometer
 * arrays on the stack (p <= ORC_MAX_ORDER).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define ORC_MAX_ORDER 16

enum { ORC_ADD = 0, ORC_SUB = 1, ORC_MUL = 2, ORC_DIV = 3, ORC_COPY = 4, ORC_SCALE = 5 };

/* ---------------------------------------------------------------------- */
/* Layout: Sec. 3.1                                                        */
/* ---------------------------------------------------------------------- */

/* Checks that pi is a permutation of 1..p (Sec. 3.1: Pi_p has p! members). */
static int is_permutation(uint32_t p, const uint32_t* pi)
{
    int seen[ORC_MAX_ORDER] = {0};
    for (uint32_t r = 0; r < p; ++r) {
        if (pi[r] < 1 || pi[r] > p) return 0;
        if (seen[pi[r] - 1]) return 0;
        seen[pi[r] - 1] = 1;
    }
    return 1;
}

/*
 * Stride tuple from layout tuple and shape, Sec. 3.1 Eq. 14:
 *   w_{pi_1} = 1,   w_{pi_r} = prod_{k=1}^{r-1} n_{pi_k}  (r > 1).
 * pi == NULL means the first-order layout pi_F = (1,...,p) (Eq. 12).
 */
int orc_strides(uint32_t p, const int64_t* n, const uint32_t* pi, int64_t* w)
{
    uint32_t piF[ORC_MAX_ORDER];
    if (p < 1 || p > ORC_MAX_ORDER) return -1;
    if (pi == NULL) {
        for (uint32_t r = 0; r < p; ++r) piF[r] = r + 1;
        pi = piF;
    }
    if (!is_permutation(p, pi)) return -2;
    for (uint32_t r = 0; r < p; ++r) {
        int64_t prod = 1;
        for (uint32_t k = 0; k + 1 <= r; ++k) prod *= n[pi[k] - 1];
        w[pi[r] - 1] = prod;
    }
    return 0;
}

/*
 * Non-hierarchical layout function, Sec. 3.2 Eq. 17:
 *   lambda(w, i, o) = sum_r w_r (i_r - o_r).
 * o == NULL means zero index offsets.
 */
int64_t orc_lambda(uint32_t p, const int64_t* w, const int64_t* i, const int64_t* o)
{
    int64_t j = 0;
    for (uint32_t r = 0; r < p; ++r) j += w[r] * (i[r] - (o ? o[r] : 0));
    return j;
}

/*
 * View of a tensor selected by index triplets (f_r, t_r, l_r), Sec. 3.3:
 *   extent        n'_r = floor((l_r - f_r) / t_r) + 1          (Eq. 5)
 *   first element gamma = lambda(w, f, o)                       (Eq. 18)
 *   view strides  w''_r = w_r * t_r                             (Eq. 19)
 * with w the strides of the referenced tensor (the reading in which the
 * step multiplies the referenced array's stride, Sec. 4.2 after Eq. 20).
 * f and l are members of the index set I_r = {o_r, ..., o_r + n_r - 1}
 * (Eq. 2); the garbled bound chain of Sec. 3 is read as
 * o_r <= f_r <= l_r < o_r + n_r (l inclusive), with t_r >= 1.
 * o == NULL means zero index offsets.
 */
int orc_view(uint32_t p, const int64_t* n, const int64_t* w, const int64_t* o,
             const int64_t* f, const int64_t* t, const int64_t* l,
             int64_t* nv, int64_t* wv, int64_t* gamma)
{
    if (p < 1 || p > ORC_MAX_ORDER) return -1;
    for (uint32_t r = 0; r < p; ++r) {
        int64_t lo = o ? o[r] : 0;
        if (t[r] < 1 || f[r] < lo || f[r] > l[r] || l[r] >= lo + n[r]) return -2;
        nv[r] = (l[r] - f[r]) / t[r] + 1;
        wv[r] = w[r] * t[r];
    }
    *gamma = orc_lambda(p, w, f, o);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Summation (ascending k, optional Neumaier compensation)                 */
/* ---------------------------------------------------------------------- */

typedef struct { double s, c; int comp; } acc_t;

static void acc_init(acc_t* a, double init, int comp) { a->s = init; a->c = 0.0; a->comp = comp; }

static void acc_add(acc_t* a, double t)
{
    if (!a->comp) { a->s += t; return; }
    double u = a->s + t;
    if (fabs(a->s) >= fabs(t)) a->c += (a->s - u) + t;
    else                       a->c += (t - u) + a->s;
    a->s = u;
}

static double acc_get(const acc_t* a) { return a->comp ? a->s + a->c : a->s; }

/* Advances a first-index-fastest odometer over extents ext[0..d-1].
   Returns 0 when the walk has wrapped around (finished). */
static int odometer_next(uint32_t d, const int64_t* ext, int64_t* idx)
{
    for (uint32_t r = 0; r < d; ++r) {
        if (++idx[r] < ext[r]) return 1;
        idx[r] = 0;
    }
    return 0;
}

static int any_zero(uint32_t d, const int64_t* ext)
{
    for (uint32_t r = 0; r < d; ++r) if (ext[r] < 1) return 1;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* ttv: Sec. 5.2 Eq. 24                                                    */
/* ---------------------------------------------------------------------- */

/*
 * C(i_1..i_{q-1}, i_{q+1}..i_p) = sum_{k=0}^{n_q-1} A(i_1..k..i_p) * b(k)
 *
 * The output is order p-1; its modes are A's modes without q, in order
 * (the reading of the garbled index tuple of Eq. 24 that makes C order
 * p-1, as the text before the equation states).  wC has p-1 entries.
 * accumulate != 0 starts each sum from the current C value, as the
 * paper's recursive listing does with its inner-product initial value;
 * accumulate == 0 follows the '=' of Eq. 24.
 */
static double ttv_point(uint32_t p, const int64_t* n, uint32_t q, const double* A,
                        const int64_t* wA, const double* b, int64_t incb,
                        int64_t* iA, double init, int comp)
{
    acc_t s;
    acc_init(&s, init, comp);
    for (int64_t k = 0; k < n[q - 1]; ++k) {
        iA[q - 1] = k;
        acc_add(&s, A[orc_lambda(p, wA, iA, NULL)] * b[k * incb]);
    }
    return acc_get(&s);
}

int orc_ttv(uint32_t p, const int64_t* n, uint32_t q,
            const double* A, const int64_t* wA,
            const double* b, int64_t incb,
            double* C, const int64_t* wC, int accumulate, int compensated)
{
    int64_t ext[ORC_MAX_ORDER], idx[ORC_MAX_ORDER] = {0}, iA[ORC_MAX_ORDER];
    if (p < 2 || p > ORC_MAX_ORDER || q < 1 || q > p) return -1;
    uint32_t d = p - 1;
    for (uint32_t r = 0, c = 0; r < p; ++r) if (r != q - 1) ext[c++] = n[r];
    if (any_zero(d, ext) || n[q - 1] < 1) return 0;
    do {
        for (uint32_t r = 0, c = 0; r < p; ++r) iA[r] = (r == q - 1) ? 0 : idx[c++];
        int64_t jc = orc_lambda(d, wC, idx, NULL);
        double init = accumulate ? C[jc] : 0.0;
        C[jc] = ttv_point(p, n, q, A, wA, b, incb, iA, init, compensated);
    } while (odometer_next(d, ext, idx));
    return 0;
}

/* Point evaluation of Eq. 24 at cnt output multi-indices (cnt x (p-1),
   row-major), without accumulation.  Used to check large outputs by sample. */
int orc_ttv_at(uint32_t p, const int64_t* n, uint32_t q,
               const double* A, const int64_t* wA,
               const double* b, int64_t incb,
               const int64_t* out_idx, int64_t cnt, double* out, int compensated)
{
    int64_t iA[ORC_MAX_ORDER];
    if (p < 2 || p > ORC_MAX_ORDER || q < 1 || q > p) return -1;
    for (int64_t e = 0; e < cnt; ++e) {
        const int64_t* oi = out_idx + e * (int64_t)(p - 1);
        for (uint32_t r = 0, c = 0; r < p; ++r) iA[r] = (r == q - 1) ? 0 : oi[c++];
        out[e] = ttv_point(p, n, q, A, wA, b, incb, iA, 0.0, compensated);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* ttm: Sec. 5.2 Eq. 25                                                    */
/* ---------------------------------------------------------------------- */

/*
 * C(i_1..i_{q-1}, j, i_{q+1}..i_p) = sum_{k=0}^{n_q-1} A(i_1..k..i_p) * B(j, k)
 *
 * B is J x n_q with B(j,k) at B[j*ldb_row + k*ldb_col]; C has A's shape
 * with extent J in mode q (the reading in which the second 'A' of the
 * sentence before Eq. 25 names the output C).  wC has p entries.
 */
static double ttm_point(uint32_t p, const int64_t* n, uint32_t q, const double* A,
                        const int64_t* wA, const double* B, int64_t j,
                        int64_t ldb_row, int64_t ldb_col, int64_t* iA,
                        double init, int comp)
{
    acc_t s;
    acc_init(&s, init, comp);
    for (int64_t k = 0; k < n[q - 1]; ++k) {
        iA[q - 1] = k;
        acc_add(&s, A[orc_lambda(p, wA, iA, NULL)] * B[j * ldb_row + k * ldb_col]);
    }
    return acc_get(&s);
}

int orc_ttm(uint32_t p, const int64_t* n, uint32_t q,
            const double* A, const int64_t* wA,
            const double* B, int64_t J, int64_t ldb_row, int64_t ldb_col,
            double* C, const int64_t* wC, int accumulate, int compensated)
{
    int64_t ext[ORC_MAX_ORDER], idx[ORC_MAX_ORDER] = {0}, iA[ORC_MAX_ORDER];
    if (p < 2 || p > ORC_MAX_ORDER || q < 1 || q > p || J < 0) return -1;
    for (uint32_t r = 0; r < p; ++r) ext[r] = (r == q - 1) ? J : n[r];
    if (any_zero(p, ext) || n[q - 1] < 1) return 0;
    do {
        for (uint32_t r = 0; r < p; ++r) iA[r] = idx[r];
        int64_t jc = orc_lambda(p, wC, idx, NULL);
        double init = accumulate ? C[jc] : 0.0;
        C[jc] = ttm_point(p, n, q, A, wA, B, idx[q - 1], ldb_row, ldb_col, iA, init, compensated);
    } while (odometer_next(p, ext, idx));
    return 0;
}

/* Point evaluation of Eq. 25 at cnt output multi-indices (cnt x p, row-major;
   entry q-1 of each multi-index is the row j of B). */
int orc_ttm_at(uint32_t p, const int64_t* n, uint32_t q,
               const double* A, const int64_t* wA,
               const double* B, int64_t ldb_row, int64_t ldb_col,
               const int64_t* out_idx, int64_t cnt, double* out, int compensated)
{
    int64_t iA[ORC_MAX_ORDER];
    if (p < 2 || p > ORC_MAX_ORDER || q < 1 || q > p) return -1;
    for (int64_t e = 0; e < cnt; ++e) {
        const int64_t* oi = out_idx + e * (int64_t)p;
        for (uint32_t r = 0; r < p; ++r) iA[r] = oi[r];
        out[e] = ttm_point(p, n, q, A, wA, B, oi[q - 1], ldb_row, ldb_col, iA, 0.0, compensated);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Entrywise: Sec. 5.1 Eqs. 22-23                                          */
/* ---------------------------------------------------------------------- */

static double apply_op(int op, double a, double b, double alpha)
{
    switch (op) {
    case ORC_ADD:   return a + b;
    case ORC_SUB:   return a - b;
    case ORC_MUL:   return a * b;
    case ORC_DIV:   return a / b;
    case ORC_COPY:  return a;
    default:        return alpha * a;   /* ORC_SCALE, Eq. 22 */
    }
}

/*
 * C(i) = A(i) (op) B(i) for every multi-index i of the shape n (Eq. 23);
 * op COPY gives C(i) = A(i) (a relayout when C's layout differs) and op
 * SCALE gives C(i) = alpha * A(i) (Eq. 22).  Each operand has its own
 * strides, so the three layouts may all differ.  B and wB are ignored
 * for COPY and SCALE.
 */
int orc_entrywise(int op, uint32_t p, const int64_t* n,
                  const double* A, const int64_t* wA,
                  const double* B, const int64_t* wB,
                  double alpha, double* C, const int64_t* wC)
{
    int64_t idx[ORC_MAX_ORDER] = {0};
    if (p < 1 || p > ORC_MAX_ORDER || op < ORC_ADD || op > ORC_SCALE) return -1;
    int unary = (op == ORC_COPY || op == ORC_SCALE);
    if (any_zero(p, n)) return 0;
    do {
        double a = A[orc_lambda(p, wA, idx, NULL)];
        double b = unary ? 0.0 : B[orc_lambda(p, wB, idx, NULL)];
        C[orc_lambda(p, wC, idx, NULL)] = apply_op(op, a, b, alpha);
    } while (odometer_next(p, n, idx));
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Transposition: Table 3 (transpose)                                      */
/* ---------------------------------------------------------------------- */

/*
 * C(i^c_1..i^c_p) = A(i^a_1..i^a_p) with i^c_r = i^a_{tau_r}, hence
 * n^c_r = n^a_{tau_r}; tau is a 1-based permutation of 1..p.  The odometer
 * walks C's multi-index; A's index is assembled from it by i^a_{tau_r} =
 * i^c_r.  wC has p entries (strides of C's modes).
 */
int orc_transpose(uint32_t p, const int64_t* nA, const double* A, const int64_t* wA,
                  const uint32_t* tau, double* C, const int64_t* wC)
{
    int64_t nc[ORC_MAX_ORDER], ic[ORC_MAX_ORDER] = {0}, ia[ORC_MAX_ORDER];
    if (p < 1 || p > ORC_MAX_ORDER || !is_permutation(p, tau)) return -1;
    for (uint32_t r = 0; r < p; ++r) nc[r] = nA[tau[r] - 1];
    if (any_zero(p, nc)) return 0;
    do {
        for (uint32_t r = 0; r < p; ++r) ia[tau[r] - 1] = ic[r];
        C[orc_lambda(p, wC, ic, NULL)] = A[orc_lambda(p, wA, ia, NULL)];
    } while (odometer_next(p, nc, ic));
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Tensor-tensor multiplication: Sec. 5.2 Eqs. 26-27 ((q, phi, psi)-mode)   */
/* ---------------------------------------------------------------------- */

/*
 * A has order q+r, B order q+s, C order r+s; phi (q+r entries) and psi
 * (q+s entries) are 1-based permutations.  With i^c the output index and
 * j the contraction index (q entries):
 *   i^a_{phi_k}     = i^c_k       (k = 1..r),   i^b_{psi_k}     = i^c_{r+k} (k = 1..s),
 *   i^a_{phi_{r+k}} = j_k         (k = 1..q),   i^b_{psi_{s+k}} = j_k       (k = 1..q),
 *   C(i^c) = sum_j A(i^a) * B(i^b),
 * and the extents must satisfy n^a_{phi_{r+k}} = n^b_{psi_{s+k}}.  q = 0 is
 * the outer product, r = s = 0 the inner product (C holds one element and
 * wC is not read).  The contraction index is walked by the odometer (first
 * contracted index fastest); accumulate and compensated as for ttv.
 */
int orc_ttt(uint32_t q, uint32_t r, uint32_t s,
            const int64_t* nA, const double* A, const int64_t* wA, const uint32_t* phi,
            const int64_t* nB, const double* B, const int64_t* wB, const uint32_t* psi,
            double* C, const int64_t* wC, int accumulate, int compensated)
{
    int64_t nc[ORC_MAX_ORDER], nj[ORC_MAX_ORDER];
    int64_t ic[ORC_MAX_ORDER] = {0}, j[ORC_MAX_ORDER], ia[ORC_MAX_ORDER], ib[ORC_MAX_ORDER];
    const uint32_t pa = q + r, pb = q + s, pc = r + s;
    if (pa < 1 || pb < 1 || pa > ORC_MAX_ORDER || pb > ORC_MAX_ORDER) return -1;
    if (!is_permutation(pa, phi) || !is_permutation(pb, psi)) return -1;
    for (uint32_t k = 0; k < q; ++k) {
        nj[k] = nA[phi[r + k] - 1];
        if (nB[psi[s + k] - 1] != nj[k]) return -2;
    }
    for (uint32_t k = 0; k < r; ++k) nc[k] = nA[phi[k] - 1];
    for (uint32_t k = 0; k < s; ++k) nc[r + k] = nB[psi[k] - 1];
    if (any_zero(pc, nc)) return 0;
    do {
        const int64_t co = pc ? orc_lambda(pc, wC, ic, NULL) : 0;
        acc_t acc;
        acc_init(&acc, accumulate ? C[co] : 0.0, compensated);
        for (uint32_t k = 0; k < r; ++k) ia[phi[k] - 1] = ic[k];
        for (uint32_t k = 0; k < s; ++k) ib[psi[k] - 1] = ic[r + k];
        if (!any_zero(q, nj)) {
            for (uint32_t k = 0; k < q; ++k) j[k] = 0;
            do {
                for (uint32_t k = 0; k < q; ++k) {
                    ia[phi[r + k] - 1] = j[k];
                    ib[psi[s + k] - 1] = j[k];
                }
                acc_add(&acc, A[orc_lambda(pa, wA, ia, NULL)] * B[orc_lambda(pb, wB, ib, NULL)]);
            } while (q > 0 && odometer_next(q, nj, j));
        }
        C[co] = acc_get(&acc);
    } while (pc > 0 && odometer_next(pc, nc, ic));
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Frobenius norm: Table 3 (norm)                                          */
/* ---------------------------------------------------------------------- */

/* ||A||_F = sqrt(sum_i A(i)^2), summed in the odometer order. */
double orc_norm(uint32_t p, const int64_t* n, const double* A, const int64_t* wA, int compensated)
{
    int64_t idx[ORC_MAX_ORDER] = {0};
    acc_t s;
    acc_init(&s, 0.0, compensated);
    if (p < 1 || p > ORC_MAX_ORDER || any_zero(p, n)) return 0.0;
    do {
        double a = A[orc_lambda(p, wA, idx, NULL)];
        acc_add(&s, a * a);
    } while (odometer_next(p, n, idx));
    return sqrt(acc_get(&s));
}

/* ||A - R||_F / ||R||_F over two identically shaped tensors with their own
   strides (the relative Frobenius error used for parity). */
double orc_rel_error(uint32_t p, const int64_t* n, const double* A, const int64_t* wA,
                     const double* R, const int64_t* wR)
{
    int64_t idx[ORC_MAX_ORDER] = {0};
    acc_t num, den;
    acc_init(&num, 0.0, 1);
    acc_init(&den, 0.0, 1);
    if (p < 1 || p > ORC_MAX_ORDER || any_zero(p, n)) return 0.0;
    do {
        double r = R[orc_lambda(p, wR, idx, NULL)];
        double e = A[orc_lambda(p, wA, idx, NULL)] - r;
        acc_add(&num, e * e);
        acc_add(&den, r * r);
    } while (odometer_next(p, n, idx));
    double d = acc_get(&den);
    return d > 0.0 ? sqrt(acc_get(&num) / d) : sqrt(acc_get(&num));
}

/* Version tag so a stale build is detectable. */
int orc_version(void) { return 2; }
