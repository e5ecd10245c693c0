/*
 * mpps.h -- C ABI of the GB300 (sm_103a) library for mixed-precision Paterson--Stockmeyer
 * evaluation of matrix polynomials (Liu, "Mixed-Precision Paterson--Stockmeyer Method for
 * Evaluating Polynomials of Matrices", arXiv 2312.17396).
 *
 * Problem (Section 2, Algorithm 2.1; Algorithm 4.1 for general coefficients): given
 * X in R^{n x n} and scalars b_0..b_m, compute p_m(X) = sum_i b_i X^i in the
 * Paterson--Stockmeyer form of eq. (1.1),
 *     p_m(X) = sum_{i=0}^{r} B_i (X^s)^i,  r = floor(m/s),
 *     B_i = sum_{j=0}^{s-1} b_{si+j} X^j  (i < r),   B_r = sum_{j=0}^{m-sr} b_{sr+j} X^j,
 * by Horner's rule in Y = X^s (eq. (2.4)), with the product of Horner step i done in the
 * precision u_i chosen by eq. (2.8) (Section 2, Algorithm 3.1 `fix_params` branch,
 * Algorithm 4.1) and the sums in FP64.
 *
 * Conventions shared by every entry point:
 *  - Matrices are real FP64, n x n, row-major and contiguous; a batch of `batch` matrices
 *    is contiguous with stride n*n elements.  Row-major is harmless: p(A^T) = p(A)^T.
 *  - Matrix pointers may be device pointers (cudaMalloc, torch CUDA tensors) or host
 *    pointers (pageable or pinned).  The library inspects each pointer.  When any matrix
 *    argument is on the host, the call copies it to the device, runs, copies the result
 *    back and synchronises the stream before returning.  When all are device pointers the
 *    call is asynchronous on `stream` except where noted.
 *  - `coeffs` is always a host array of m+1 doubles (b_0..b_m), read during the call.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *  - Workspace is allocated by the library with cudaMallocAsync on `stream` and released
 *    with cudaFreeAsync before the call returns (stream-ordered).
 *  - Every call returns a status; none aborts.  On failure mpps_last_error() returns a
 *    description (thread-local, valid until the next call on the same thread).  Invalid
 *    sizes or null pointers give MPPS_EINVAL before any GPU work is issued.
 *  - The caller owns all pointers passed in; the library keeps none after returning.
 */
#ifndef MPPS_H
#define MPPS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPPS_OK = 0,
    MPPS_EINVAL = 1,    /* invalid argument (size, pointer, policy) */
    MPPS_ENOMEM = 2,    /* device allocation failed */
    MPPS_ECUDA = 3,     /* a CUDA runtime/driver call or kernel launch failed */
    MPPS_ETIMEOUT = 4,  /* a bounded wait inside a kernel gave up (device error word set) */
    MPPS_ENOTSUP = 5,   /* not supported on this device / build */
    MPPS_ECHECK = 6     /* a check made on the GPU failed (e.g. a matrix needed more squarings
                           than policy.max_squarings; its result is NaN) */
} mpps_status;

/* Precision modes.  FIXED: every product in FP64 (Algorithm 2.1).  MIXED_PAPER: eq. (2.8)
 * with nu chosen as in Algorithm 3.1 and the format ladder of Section 4.1.1 extended to the
 * GPU formats.  MIXED_NS: as MIXED_PAPER but the Horner steps i <= fp64_floor_steps (the
 * products feeding B_0, B_1, ...) stay FP64. */
typedef enum { MPPS_FIXED_FP64 = 0, MPPS_MIXED_PAPER = 1, MPPS_MIXED_NS = 2 } mpps_mode;

/* Product formats, ordered from most to least precise.  The unit roundoff of each format's
 * rounded inputs: FP64 2^-53; BF16X3 (operands split into bf16 hi+lo, three products
 * hi*hi + hi*lo + lo*hi accumulated in FP32) 2^-16; TF32 2^-11; BF16 2^-8; FP8 (E4M3) 2^-4.
 * The BF16/TF32 operands are scaled by a power of two per matrix; FP8 ones by a power of two
 * per row of the left factor and per column of the right one, then by one per 32 entries
 * along the inner dimension (block scales applied by the tensor core), so that every block
 * keeps E4M3's 3 fraction bits.  All but FP64 accumulate in FP32 (unit 2^-24).
 * NONE marks a step with no product (B_r a scalar multiple of I, i.e. s divides m). */
typedef enum {
    MPPS_FMT_NONE = -1,
    MPPS_FMT_FP64 = 0,
    MPPS_FMT_BF16X3 = 1,
    MPPS_FMT_TF32 = 2,
    MPPS_FMT_BF16 = 3,
    MPPS_FMT_FP8 = 4
} mpps_format;

/* FP64 products emulated on the BF16 tensor cores with exact integer slices of 7 bits
 * (MPPS_FMT_F64E(k), 1 <= k <= MPPS_F64E_MAX_SLICES).  k <= 8: k slices per operand and the
 * slice pairs of order t + q <= k - 1, k(k+1)/2 BF16 products, error below 2^(2-7k) relative
 * to the row and column maxima of the operands (k = 8: FP64-level for products of moderate
 * length).  k = 9: the 8 slices with the pairs of order t + q <= 8 as well, 43 BF16 products,
 * error below 2^-55 (below an FP64 product's at every length). */
#define MPPS_F64E_MAX_SLICES 9
#define MPPS_FMT_F64E(k) (16 + (k))
#define MPPS_FMT_IS_F64E(f) ((f) > 16 && (f) <= 16 + MPPS_F64E_MAX_SLICES)
#define MPPS_F64E_SLICES(f) ((f) - 16)

#define MPPS_NUM_FORMATS 5
#define MPPS_MAX_R 64      /* largest r = floor(m/s) a report can describe */
#define MPPS_MAX_S 32      /* largest block size s */

typedef struct {
    int mode;               /* mpps_mode */
    double tol;             /* working precision u (u_0 of eq. (2.8)); <= 0 -> 2^-53 */
    double delta;           /* switch threshold delta of Algorithm 3.1; <= 0 -> 10 */
    int s;                  /* PS block size; 0 -> ceil(sqrt(m)) (Algorithm 2.1) */
    unsigned formats;       /* bit f allows format f; 0 -> all; FP64 is always allowed */
    int fp64_floor_steps;   /* MIXED_NS: steps i <= this stay FP64; < 0 -> 2 */
    int f64_slices;         /* 0: working-precision products on the FP64 pipe (DMMA);
                               k in 1..MPPS_F64E_MAX_SLICES: emulate them as MPPS_FMT_F64E(k),
                               and let mixed steps use F64E(k') for k' < k as well */
    int variable_s;         /* 1 (mixed modes, s = 0): the variable-s branch of Algorithm 3.1
                               (mpps_choose_s); 0: s = ceil(sqrt(m)) */
    int adjoint_recompute;  /* 1: the adjoints keep every ceil(sqrt(r))-th Horner iterate and
                               recompute the others (same products, same result); 0: keep all */
    int device_plan;        /* 1: the precision rule runs on the GPU (ps_eval, expm_taylor_ss):
                               no read-back of the norms; every format the rule may pick for a
                               step is launched and all but the chosen one return at once.
                               Same formats, scales and results as the host planner.  0: the
                               host plans after one read-back of the norms */
    int max_squarings;      /* expm with device_plan: k > 0 launches k squaring steps, each on
                               the matrices whose sigma exceeds its index (lists built on the
                               GPU), so the call reads nothing back and can be captured in a
                               CUDA graph; a matrix needing more than k squarings gets NaN and
                               MPPS_ECHECK is reported (at once, or by the next call that finds
                               the error word).  0: sigma is read back early in the call (the
                               GPU does not wait for it) and exactly max sigma steps run */
    int mixed_powers;       /* 1 (mixed modes, f64_slices = k > 0, host plan, fixed s >= 4):
                               the powers are formed as a tree: X^2..X^h by X^j = X^(j-1) X
                               (h = ceil(s/2)), Y = X^h X^(s-h), and the leaves X^(h+t) =
                               X^h X^t (t = 1..s-h-1), which feed only the block sums, each as
                               F64E(k') with k' <= k slices chosen by mpps_plan_powers (the
                               mixed precision inside the powers that Section 5 asks for).
                               0, or with device_plan, variable_s, the tape entries, a fixed
                               mode or s < 4: X_j = X_(j-1) X, every power in the working
                               precision */
} mpps_policy;

/* Per-matrix description of what a call did (filled when `rep` is non-NULL). */
typedef struct {
    int s, r, nu;                    /* block size, floor(m/s), first low-precision step */
    int sigma;                       /* squarings (expm only; 0 otherwise) */
    int fold;                        /* 1 when s divides m (step r has no product) */
    int fmt[MPPS_MAX_R + 1];         /* fmt[i]: format of the product P_i Y, i = 1..r */
    double u[MPPS_MAX_R + 1];        /* u[i]: precision asked for by eq. (2.8), i = 1..r */
    double normB[MPPS_MAX_R + 1];    /* ||B_i||_1, i = 0..r */
    double normY;                    /* ||X^s||_1 */
    double normX;                    /* ||X||_1 (after scaling, for expm) */
    int gemms[MPPS_NUM_FORMATS + 1]; /* products per format; [MPPS_NUM_FORMATS] = squarings */
    double cost_ratio;               /* eq. (3.8) with the digits of the chosen formats */
    int pow_fmt[MPPS_MAX_S + 1];     /* pow_fmt[j]: format of the product that formed X^j,
                                        j = 2..s (MPPS_FMT_NONE for j < 2 and past s) */
} mpps_report;

/* Fill *p with the defaults: MIXED_NS, tol 2^-53, delta 10, s 0, all formats, floor 2,
 * f64_slices 0 (working-precision products on the FP64 pipe), variable_s 0,
 * adjoint_recompute 0, device_plan 0, max_squarings 0, mixed_powers 0. */
void mpps_policy_default(mpps_policy* p);

/*
 * Host-only rule of the variable-s branch of Algorithm 3.1 (no GPU work).  Starting from
 * s0 = ceil(sqrt(m)), and only when ||X||_1 <= s0/e, s grows by one while
 *   ||Y||_1 > ||B_0||_1 ||X||_1^s   and   s < m   (and s < MPPS_MAX_S),
 * Y = X^s and B_0 = sum_{j<s} b_j X^j for the current s (||X||^s by repeated
 * multiplication).  normB0[k] and normY[k] are the norms for s = s0 + k, k < len.
 * Returns the chosen s (at most s0 + len - 1: the caller supplies norms as s grows), or -1
 * for m < 1, len < 1 or a NULL pointer.
 */
int mpps_choose_s(int m, double normX, const double* normB0, const double* normY, int len);

/*
 * Host-only precision planner (no GPU work): eq. (2.8) at nu = 1,
 *   u_i = max(tol, ||B_0|| tol / (||B_i|| ||Y||^i)),  i = 1..r  (||Y||^i by repeated
 *   multiplication; a zero denominator gives u_i = +inf),
 * nu = min{i : u_i >= delta*tol} (r+1 if none) and u_1..u_{nu-1} = tol (Algorithm 3.1,
 * Algorithm 4.1); format_i = the cheapest allowed format whose unit roundoff is <= u_i and,
 * for FP32-accumulated formats, n 2^-24 <= u_i (Section 4.1.1's rule max{u* <= u_i}).
 * normB: r+1 values ||B_0||..||B_r|| with r = floor(m/s); normY = ||X^s||_1.
 * Writes s, r, nu, fold, fmt, u, normB, normY and cost_ratio of *out.
 * Returns MPPS_EINVAL for m < 0, n <= 0, r > MPPS_MAX_R, s > MPPS_MAX_S or a NULL pointer.
 */
mpps_status mpps_plan(int m, int n, const double* normB, double normY, const mpps_policy* policy,
                      mpps_report* out);

/*
 * Host-only rule for the leaves of the power tree of policy.mixed_powers (no GPU work).
 * With h = ceil(s/2) the leaves are X^j, j = h+1..s-1, formed as X^h X^(j-h); they feed only
 * the block sums B_i = sum_j b_{si+j} X^j, so a leaf's error dX^j reaches p(X) through
 * sum_i |b_{si+j}| ||Y||^i ||dX^j||, and an emulated product with k' slices errs by about
 * u_F64E(k') ||X^h|| ||X^(j-h)||.  In the manner of eq. (2.8), with the norms of the chain
 * powers (the leaves not yet formed) and the L leaves sharing the budget:
 *   u_j = ||B_0||_low tol / (L ||X^h|| ||X^(j-h)|| sum_{i >= 0, si+j <= m} |b_{si+j}| ||Y||^i),
 *   ||B_0||_low = max(0, ||B_0||_partial - sum_j |b_j| ||X^h|| ||X^(j-h)||),
 * and leaf j takes the fewest slices k' (4 <= k' <= f64_slices) with u_F64E(k') <= u_j
 * (u_F64E(k') = 2^(2-7k') for k' <= 8, 2^-55 for k' = 9).
 *   coeffs   : b_0..b_m.
 *   normXpow : s values ||X^1||_1..||X^s||_1 (the leaves' entries are not read).
 *   normBpart: r+1 values ||B_i||_1 (r = floor(m/s)) of the blocks without their leaf terms.
 *   fmt_out  : s+1 entries: MPPS_FMT_F64E(k') for the leaves, MPPS_FMT_F64E(f64_slices) for
 *              X^2..X^h and Y, MPPS_FMT_NONE for j < 2.
 *   normB_out: r+1 values for the block rule (mpps_plan): ||B_0||_low, and for i >= 1 the
 *              partial norm plus the bound of the block's leaf terms (upper bounds).
 * Returns MPPS_EINVAL for bad sizes or NULL pointers, MPPS_ENOTSUP when the policy forms
 * no tree (mixed_powers 0, a fixed mode, f64_slices 0, or s < 4).
 */
mpps_status mpps_plan_powers(int m, int s, const double* coeffs, const double* normXpow,
                             const double* normBpart, const mpps_policy* policy, int* fmt_out,
                             double* normB_out);

/*
 * p_m(A) for a batch of matrices (Algorithm 2.1 / Algorithm 4.1).
 *   coeffs : host, m+1 doubles b_0..b_m.            m >= 0.
 *   A      : batch x n x n input (host or device), not modified.
 *   out    : batch x n x n result (host or device); may not alias A.
 *   policy : NULL -> defaults (mpps_policy_default).
 *   rep    : NULL, or `batch` reports (host memory).
 * Steps: powers X^2..X^s in FP64; ||B_i||_1 and ||Y||_1 in FP64; the host planner; Horner
 * products in the planned formats with the block sums fused into their epilogues.  The
 * norms are read back to the host once per call, so the call synchronises `stream` once.
 */
mpps_status ps_eval(const double* coeffs, int m, const double* A, int n, int batch,
                    const mpps_policy* policy, double* out, mpps_report* rep, void* stream);

/*
 * exp(A) by the degree-m Taylor polynomial with scaling and squaring, eq. (3.6):
 * sigma = max(0, ceil(log2 ||A||_1)) so that ||2^-sigma A||_1 <= 1, X = 2^-sigma A (exact),
 * P = p_m(X) evaluated as in ps_eval with b_i = 1/i!, then sigma squarings in FP64.
 *   m      : Taylor degree (0 -> 30).
 *   Others as in ps_eval.  Synchronises `stream` once (norms for sigma and the planner).
 */
mpps_status expm_taylor_ss(const double* A, int n, int batch, int m, const mpps_policy* policy,
                           double* out, mpps_report* rep, void* stream);

/*
 * One item of an uneven batch: its own order n and Taylor degree m (0 -> 30).
 * A and out are device pointers to n x n row-major FP64 matrices (out may not alias A).
 */
typedef struct {
    const double* A;
    double* out;
    int n;
    int m;
} mpps_group_item;

/*
 * exp(A) for `count` matrices of different orders and degrees (scaling and squaring as in
 * expm_taylor_ss, one sigma per matrix).  Matrices are bucketed by (n rounded up to a
 * multiple of 32, m); each bucket is zero-padded block-diagonally -- exact, since
 * p(diag(A, 0)) = diag(p(A), b_0 I) and ||diag(A, 0)||_1 = ||A||_1 -- and evaluated as one
 * batch with the precision rule on the GPU (as with policy.device_plan), per-matrix plans
 * and operand scales; the n x n results are scattered back.  The buckets run on up to 8
 * library streams that fork from `stream` and join it again, so small buckets overlap.
 *   items : host array of `count` descriptors (device matrix pointers).
 *   rep   : NULL, or `count` reports (host), in item order (norms include the padding's
 *           b_{is} I part of each block).
 * With policy.max_squarings = 0 the call reads every sigma back once, early (one host wait,
 * before the heavy work is enqueued); with max_squarings = k > 0 it reads nothing back and
 * can be captured in a CUDA graph (see mpps_policy).  A report synchronises per bucket.
 */
mpps_status expm_taylor_ss_grouped(const mpps_group_item* items, int count,
                                   const mpps_policy* policy, mpps_report* rep, void* stream);

/*
 * One item of an uneven batch of polynomial evaluations: its own order n, degree m and
 * coefficients b_0..b_m (host array, read during the call).  A and out are device pointers to
 * n x n row-major FP64 matrices (out may not alias A).
 */
typedef struct {
    const double* A;
    double* out;
    int n;
    int m;
    const double* coeffs;
} mpps_poly_item;

/*
 * p(A) for `count` matrices of different orders, degrees and coefficients (Algorithm 2.1 /
 * Algorithm 4.1 per matrix, the precision rule of eq. (2.8) per matrix): bucketed by (n
 * rounded up to a multiple of 32, m, coefficients) and zero-padded as in
 * expm_taylor_ss_grouped (p(diag(A, 0)) = diag(p(A), b_0 I)), each bucket planned on the GPU
 * and the buckets run on forked streams.  No read-back unless `rep` is given; capturable in
 * a CUDA graph.  items: host array of `count` descriptors; rep: NULL or `count` reports.
 */
mpps_status ps_eval_grouped(const mpps_poly_item* items, int count, const mpps_policy* policy,
                            mpps_report* rep, void* stream);

/*
 * Gradient of f(A) = <G, p_m(A)> = sum_ij G_ij p_m(A)_ij with respect to A, i.e. the
 * Frechet derivative L_p(A^T, G) (the paper states no adjoint; this is the derivative of
 * the PS evaluation of Algorithm 2.1 / 4.1, computed by reverse mode through its steps):
 *   forward: the powers X_2..X_s and the Horner iterates P_r..P_1 under `policy` (eq. (2.8));
 *   reverse: Pbar_0 = G; for i = 1..r: Ybar += P_i^T Pbar_{i-1}, Pbar_i = Pbar_{i-1} Y^T,
 *            Xbar_j += b_{(i-1)s+j} Pbar_{i-1};  then Xbar_s += Ybar and the power chain
 *            Xbar_{j-1} += Xbar_j X^T, Xbar_1 += X_{j-1}^T Xbar_j (j = s..2); gradA = Xbar_1.
 * The two products of reverse step i run in the format the forward rule of each matrix picks
 * for u_i / d, d = m / min(1, ||X||_1) (the high-order blocks weigh up to m/||X|| times more
 * in the gradient than in p(X)), the batch taking the most precise; the power chain runs in
 * the working precision.  FIXED_FP64 keeps every product in the working precision.
 * Equivalent to ps_eval_forward_tape into a private tape followed by ps_eval_adjoint_tape.
 *   coeffs : host, m+1 doubles.   A, G : batch x n x n (host or device).
 *   policy : NULL -> defaults; f64_slices selects the working-precision products (0 = FP64
 *            pipe, k = MPPS_FMT_F64E(k)); adjoint_recompute keeps ceil(sqrt(r)) iterates.
 *   gradA  : batch x n x n output (host or device).
 * Synchronises `stream` (the forward plans on the host; the reverse pass reads the tape's
 * header).
 */
mpps_status ps_eval_adjoint(const double* coeffs, int m, const double* A, const double* G,
                            int n, int batch, const mpps_policy* policy, double* gradA,
                            void* stream);

/* Element type of the matrices of the tape entry points: FP64, or FP32 storage (evaluated
 * in FP64: inputs widened exactly, results rounded to nearest FP32). */
#define MPPS_STORAGE_F64 0
#define MPPS_STORAGE_F32 1

/* Host planner of the reverse pass (no GPU work): mpps_plan with every u_i of eq. (2.8)
 * divided by d = m / min(1, normX) before nu and the formats are chosen (see
 * ps_eval_adjoint).  normX = ||X||_1.  Errors as mpps_plan. */
mpps_status mpps_plan_adjoint(int m, int n, const double* normB, double normY, double normX,
                              const mpps_policy* policy, mpps_report* out);

/* Bytes of the tape of ps_eval_forward_tape for this call shape and policy (s and
 * adjoint_recompute fix its layout): the power table, the kept Horner iterates and a header
 * with the formats of both passes.  0 for invalid arguments (see mpps_last_error). */
size_t ps_eval_tape_bytes(int m, int n, int batch, const mpps_policy* policy);

/*
 * p_m(A) as in ps_eval, keeping what the reverse pass needs in `tape` (caller-owned device
 * memory of at least ps_eval_tape_bytes(m, n, batch, policy) bytes): the powers, the Horner
 * iterates (all, or with adjoint_recompute every ceil(sqrt(r))-th and the top one) and the
 * planned formats.  policy.variable_s is ignored (s = policy.s or ceil(sqrt(m))).
 *   A, out  : batch x n x n device matrices of `storage` (MPPS_STORAGE_F64 or _F32).
 * Synchronises `stream` once (the planner reads the block norms).
 */
mpps_status ps_eval_forward_tape(const double* coeffs, int m, const void* A, int storage, int n,
                                 int batch, const mpps_policy* policy, void* out, void* tape,
                                 size_t tape_bytes, void* stream);

/*
 * Gradient of <G, p_m(A)> from the tape of an earlier ps_eval_forward_tape call with the
 * same coeffs, m, storage, n, batch and policy (checked against the tape's header:
 * MPPS_EINVAL if they differ).  The tape is read (in recompute mode its rolling slots are
 * overwritten, so a tape serves one reverse pass at a time).  G, gradA: batch x n x n device
 * matrices of `storage`.  Synchronises `stream` (reads the tape's header).
 */
mpps_status ps_eval_adjoint_tape(const double* coeffs, int m, const void* tape, size_t tape_bytes,
                                 const void* G, int storage, int n, int batch,
                                 const mpps_policy* policy, void* gradA, void* stream);

/* ps_eval_adjoint for FP32-stored matrices (device pointers only): A and G widened exactly,
 * both passes in FP64 under `policy`, the gradient rounded to FP32. */
mpps_status ps_eval_adjoint_f32(const double* coeffs, int m, const float* A, const float* G,
                                int n, int batch, const mpps_policy* policy, float* gradA,
                                void* stream);

/*
 * exp(A) by the [13/13] Pade approximant r = q^-1 p with scaling and squaring (the Pade
 * numerator and denominator of Section 4.1 evaluated from one power chain, then a linear
 * solve): sigma = smallest integer >= 0 with 2^-sigma ||A||_1 <= theta_13 = 5.3719...
 * (the bound of the [13/13] approximant's backward error by the working precision),
 * X = 2^-sigma A, V = sum_k c_{2k} X^{2k} and W = sum_k c_{2k+1} X^{2k} (degree-6 polynomials
 * in X^2, each by the PS evaluation of ps_eval under `policy`), U = X W, p = V + U,
 * q = p(-X) = V - U, R = q^-1 p by lu_solve (below), then sigma squarings.  The
 * products X^2, X W, those of the solve and the squarings run in the working precision of
 * `policy` (f64_slices: FP64 pipe or emulated).
 *   A, out : batch x n x n (host or device); out may not alias A.
 * Synchronises `stream`.  MPPS_ECHECK when q(X) has a zero pivot (not for the exact q on
 * the scaled argument, whose zeros lie outside |x| <= theta_13).
 */
mpps_status expm_pade13(const double* A, int n, int batch, const mpps_policy* policy, double* out,
                        void* stream);

/*
 * R = Q^-1 P for each of `batch` systems: the q(X)^-1 p(X) solve of the Pade approximant
 * (Section 4.1), by LU factorisation with partial pivoting (row interchanges chosen by the
 * first largest magnitude in the pivot column), blocked in 64 x 64 tiles: every panel is
 * factored on the FP64 pipe by one thread-block cluster, every block update and the block
 * forward and back substitutions run as tile products in the working precision of
 * `policy` (f64_slices = 0: FP64 pipe; k > 0: emulated FP64 with k slices; the other policy
 * fields are not used), the diagonal blocks through their inverses.
 *   Q, P, R : batch x n x n row-major (host or device); R may alias P or Q.
 * Synchronises `stream`.  MPPS_ECHECK when a pivot is exactly zero (Q singular in the
 * arithmetic of the factorisation); R then holds non-finite values.
 */
mpps_status lu_solve(const double* Q, const double* P, int n, int batch, const mpps_policy* policy,
                     double* R, void* stream);

/*
 * Gradient of f(A) = <G, r(A)> for the scaling-and-squaring approximant of exp,
 * r(A) = p_m(2^-sigma A)^(2^sigma) of eq. (3.6) with b_i = 1/i! and sigma = max(0,
 * ceil(log2 ||A||_1)) per matrix (the paper states no adjoint; this is reverse mode through
 * the squarings, then through the PS evaluation as in ps_eval_adjoint):
 *   S_0 = p_m(X), X = 2^-sigma A;  S_{k+1} = S_k^2;
 *   Sbar_sigma = G;  Sbar_k = Sbar_{k+1} S_k^T + S_k^T Sbar_{k+1};
 *   gradA = 2^-sigma L_p(X^T, Sbar_0).
 * The squarings S_0..S_{sigma-1} are stored (sigma n^2 doubles per matrix), and the
 * polynomial's powers and iterates on a tape as in ps_eval_forward_tape.
 *   A, G   : batch x n x n (host or device).     m : Taylor degree (0 -> 30).
 *   policy : NULL -> defaults.  The polynomial and its reverse pass follow the policy as in
 *            ps_eval_adjoint; the squarings and their reverse pass run in its working
 *            precision (f64_slices: 0 = FP64 pipe, k = emulated).
 *   gradA  : batch x n x n output (host or device).
 * Synchronises `stream` (sigma is read back; the forward polynomial plans on the host).
 */
mpps_status expm_taylor_ss_adjoint(const double* A, const double* G, int n, int batch, int m,
                                   const mpps_policy* policy, double* gradA, void* stream);

/*
 * C = A B for a batch of n x n FP64 matrices, the product computed in `format`
 * (an mpps_format other than NONE, or MPPS_FMT_F64E(k)): the building block of every step
 * above.  MPPS_FMT_F64E(k) splits the rows of A and the columns of B into k exact bf16
 * slices and sums the slice products exactly on the tensor cores.  For the
 * low-precision formats each operand is scaled by a power of two chosen from its largest
 * entry, rounded to the format, multiplied on the tensor cores with FP32 accumulation,
 * and the result scaled back in FP64.  Asynchronous for device pointers.
 */
mpps_status mpps_matmul(const double* A, const double* B, double* C, int n, int batch,
                        int format, void* stream);

/*
 * C = A^T B, otherwise as mpps_matmul (the transposed products of the reverse passes, exposed
 * with the same formats).  The emulated formats slice A's columns directly as the rows of the
 * left operand (no transpose is formed; the same slices as those of the rows of A^T, so the
 * result equals mpps_matmul of A^T and B bit for bit); the other formats transpose A first.
 */
mpps_status mpps_matmul_ta(const double* A, const double* B, double* C, int n, int batch,
                           int format, void* stream);

/*
 * mpps_matmul_noalloc -- mpps_matmul for callers that may not allocate device memory.
 * (The paper has no counterpart: this is a deployment variant of the product above.)
 * Some callers cannot let a library allocate: code running beside a framework whose
 * caching allocator has already reserved the device memory (a cudaMalloc would fail or
 * fragment that pool), latency-bound loops that must not call the allocator because it
 * can synchronise the device and take unbounded time, and plug-ins that are handed their
 * buffers and are not allowed to own device memory.  This entry point calls no cudaMalloc,
 * cudaFree or other allocating routine: the scratch the tensor-core product needs (rounded
 * operand copies, their power-of-two scales or FP8 block-scale codes, an error word) lives in
 * one fixed device array of
 * MPPS_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the library
 * holds until the process exits.
 *   A, B, C : device pointers only (host pointers give MPPS_EINVAL); batch x n x n FP64,
 *             row-major; C may not alias A or B.  format: MPPS_FMT_FP64 .. MPPS_FMT_FP8
 *             (the emulated MPPS_FMT_F64E(k) products are not offered here).
 *   Sizes whose scratch exceeds MPPS_NOALLOC_SCRATCH_BYTES give MPPS_EINVAL (the limit
 *   fits one 2048 x 2048 product in any format; FP64 products use no scratch).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress
 * with that device current); make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's contents, so calls that overlap on the
 * GPU (different streams, or different host threads) race: serialise them.  Synchronises
 * `stream` before returning (it reads the kernel's error word).
 */
#define MPPS_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
mpps_status mpps_matmul_noalloc(const double* A, const double* B, double* C, int n, int batch,
                                int format, void* stream);

/* Benchmark instrumentation (off by default).  When enabled, every kernel launch of the
 * library is bracketed by two CUDA events recorded on the launch stream and tagged with a
 * kernel class: MPPS_PROF_GEMM_F64 (FP64-pipe products), MPPS_PROF_GEMM_TC (low-precision
 * tensor-core products), MPPS_PROF_ELEMENTWISE (block sums, norms, conversions, copies),
 * MPPS_PROF_GEMM_F64E (emulated FP64 products), MPPS_PROF_SLICE (the exact bf16 slicing of
 * the emulated products' operands, with its column maxima).  mpps_profile_read waits for the
 * recorded events and returns, for one class since the last reset, the number of launches,
 * their summed durations (ms) and their summed executed flops (products: 2 n^3 per matrix
 * times the number of tensor-core products issued; total_work may be NULL).  Do not enable
 * it while a stream is being captured into a CUDA graph. */
#define MPPS_PROF_GEMM_F64 0
#define MPPS_PROF_GEMM_TC 1
#define MPPS_PROF_ELEMENTWISE 2
#define MPPS_PROF_GEMM_F64E 3
#define MPPS_PROF_SLICE 4
#define MPPS_PROF_NUM_CLASSES 5
void mpps_profile_enable(int on);
void mpps_profile_reset(void);
mpps_status mpps_profile_read(int kernel_class, long long* launches, double* total_ms,
                              double* total_work);

/* Self-test of the failure path of the library's bounded waits (no counterpart in the
 * paper): launches one CTA that waits on an mbarrier nothing arrives on; the wait gives up
 * after limit_us microseconds, sets an error word and the kernel returns normally, so the
 * call returns MPPS_ETIMEOUT and the CUDA context stays usable.  limit_us in 1..2000000. */
mpps_status mpps_selftest_bounded_wait(int limit_us, void* stream);

/* The library keeps its device workspaces (the power table, the slice planes, the
 * rounded operand copies) in a private stream-ordered memory pool per device that does not
 * give freed memory back between calls, so that repeated calls of one size allocate at no
 * cost.  mpps_release_workspace waits for every device that has such a pool
 * (cudaDeviceSynchronize) and returns the pool's unused memory to the driver.  Returns
 * MPPS_ECUDA if a synchronisation or the trim fails. */
mpps_status mpps_release_workspace(void);

/*
 * Measured choice of product schedules.  Two products have more than one valid schedule:
 * the emulated FP64 product with 7..9 slices (whole output tiles per CTA, or the K range of
 * tiles split between CTAs) and the tensor-core low-precision product (128 x 64 or
 * 128 x 128 tiles).  By default a rule measured on GB300 chooses.  With tuning on, the first
 * launch of each (kind, n, batch, variant) times every candidate on its own operands (CUDA
 * events on the call's stream; the call then waits for those launches), keeps the fastest
 * for the rest of the process and leaves that candidate's output.  Launches whose epilogue
 * accumulates into their own output are not tuned.  Host-only calls.
 *   mpps_autotune_enable : 1 = on, 0 = off (initially MPPS_AUTOTUNE=1 in the environment).
 *   mpps_autotune_clear  : forget every measured choice.
 *   mpps_autotune_entries: the table: kind (0 = emulated-product split, 1 = tensor-core tile
 *                          width), n, batch, variant (slice count or format), choice (index
 *                          of the fastest candidate) and the mean time of each of up to 4
 *                          candidates in ms (ms[4 i + c]); fills at most `cap` rows (any
 *                          pointer may be NULL) and returns the number of entries.
 */
void mpps_autotune_enable(int on);
void mpps_autotune_clear(void);
int mpps_autotune_entries(int* kind, int* n, int* batch, int* variant, int* choice, float* ms,
                          int cap);

/* Description of the last failure on this thread ("" if none). */
const char* mpps_last_error(void);

/* Library version string. */
const char* mpps_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MPPS_H */
