/*
 * mpps_oracle.c -- CPU oracle for Paterson--Stockmeyer (PS) evaluation of matrix
 * polynomials, written from Liu, "Mixed-Precision Paterson--Stockmeyer Method for
 * Evaluating Polynomials of Matrices" (arXiv 2312.17396).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls
 * this file; it shares no code, header, table or helper with the CUDA path.  Only the
 * test-suite, the smoke check and the timed CPU baseline of the benchmark use it.
 *
 * What it computes (all plain, unblocked loops, so that each routine can be read
 * against the paper):
 *   - Algorithm 2.1 (fixed-precision PS) literally, in double-double ("twice the digits
 *     of the working precision", which is how Section 3.4 builds its reference
 *     solutions) and in plain double, with a counter of matrix products;
 *   - textbook Horner and evaluation through explicit powers (the s=1 and s=m special
 *     cases of eq. (1.1)), for cross-checks;
 *   - Taylor exp with scaling and squaring, eq. (3.6): p_m(2^-sigma A)^(2^sigma);
 *   - p(X)^k V for a block of columns V, by Horner on vectors, so that sampled columns
 *     of a large result can be checked one by one;
 *   - the adjoint of A -> <G, p(A)>, i.e. the Frechet derivative L_p(A^T, G) written as
 *     its defining double sum  sum_k c_k sum_{j<k} (A^T)^j G (A^T)^(k-1-j);
 *   - the 1-norm (max column sum), the error measure of Section 3.4.
 *
 * Double-double arithmetic uses published error-free transformations: Knuth's TwoSum,
 * Dekker's Fast2Sum, the FMA-based TwoProd, and the double-word algorithms of Joldes,
 * Muller and Popescu, "Tight and rigorous error bounds for basic building blocks of
 * double-word arithmetic", ACM TOMS 44(2), 2017 (AccurateDWPlusDW, DWTimesDW3).  This
 * file must be compiled without -ffast-math and with -ffp-contract=off.
 *
 * Layout: every matrix is n x n, row-major, contiguous.  A double-double matrix is two
 * arrays (hi, lo) of the same layout.  Parallelism (OpenMP) is only over independent
 * output rows, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double hi, lo; } dd;

/* ---- error-free transformations and double-word arithmetic ---------------------- */
static inline dd two_sum(double a, double b) {            /* Knuth TwoSum */
    double s = a + b, bb = s - a;
    dd r = { s, (a - (s - bb)) + (b - bb) };
    return r;
}
static inline dd fast_two_sum(double a, double b) {       /* Dekker Fast2Sum, |a|>=|b| */
    double s = a + b;
    dd r = { s, b - (s - a) };
    return r;
}
static inline dd two_prod(double a, double b) {           /* exact product via FMA */
    double p = a * b;
    dd r = { p, fma(a, b, -p) };
    return r;
}
static inline dd dd_add(dd x, dd y) {                      /* AccurateDWPlusDW */
    dd s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
    double c = s.lo + t.hi;
    dd v = fast_two_sum(s.hi, c);
    double w = t.lo + v.lo;
    return fast_two_sum(v.hi, w);
}
static inline dd dd_mul(dd x, dd y) {                      /* DWTimesDW3 */
    dd c = two_prod(x.hi, y.hi);
    double tl0 = x.lo * y.lo;
    double tl1 = fma(x.hi, y.lo, tl0);
    double cl2 = fma(x.lo, y.hi, tl1);
    double cl3 = c.lo + cl2;
    return fast_two_sum(c.hi, cl3);
}
static inline dd dd_from(double a) { dd r = { a, 0.0 }; return r; }
static inline dd dd_neg(dd a) { dd r = { -a.hi, -a.lo }; return r; }

/* ---- dd matrices ---------------------------------------------------------------- */
typedef struct { int n; dd* v; } ddmat;

static ddmat ddm_alloc(int n) {
    ddmat M; M.n = n; M.v = (dd*)calloc((size_t)n * n + 1, sizeof(dd)); return M;
}
static void ddm_free(ddmat* M) { free(M->v); M->v = NULL; }
static void ddm_zero(ddmat M) { memset(M.v, 0, sizeof(dd) * (size_t)M.n * M.n); }
static void ddm_copy(ddmat D, ddmat S) { memcpy(D.v, S.v, sizeof(dd) * (size_t)S.n * S.n); }
static void ddm_identity(ddmat M) {
    ddm_zero(M);
    for (int i = 0; i < M.n; ++i) M.v[(size_t)i * M.n + i] = dd_from(1.0);
}
/* C = A*B, plain triple loop (i, k, j order) with dd accumulation. C must not alias. */
static void ddm_mul(ddmat C, ddmat A, ddmat B) {
    int n = A.n;
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        dd* c = C.v + (size_t)i * n;
        for (int j = 0; j < n; ++j) c[j] = dd_from(0.0);
        for (int k = 0; k < n; ++k) {
            dd a = A.v[(size_t)i * n + k];
            if (a.hi == 0.0 && a.lo == 0.0) continue;
            const dd* b = B.v + (size_t)k * n;
            for (int j = 0; j < n; ++j) c[j] = dd_add(c[j], dd_mul(a, b[j]));
        }
    }
}
/* M += c * S */
static void ddm_axpy(ddmat M, dd c, ddmat S) {
    size_t N = (size_t)M.n * M.n;
    for (size_t t = 0; t < N; ++t) M.v[t] = dd_add(M.v[t], dd_mul(c, S.v[t]));
}
static void ddm_add_diag(ddmat M, dd c) {
    for (int i = 0; i < M.n; ++i) M.v[(size_t)i * M.n + i] = dd_add(M.v[(size_t)i * M.n + i], c);
}
static void ddm_load(ddmat M, const double* X) {
    size_t N = (size_t)M.n * M.n;
    for (size_t t = 0; t < N; ++t) M.v[t] = dd_from(X[t]);
}
static void ddm_store(ddmat M, double* hi, double* lo) {
    size_t N = (size_t)M.n * M.n;
    for (size_t t = 0; t < N; ++t) { hi[t] = M.v[t].hi; if (lo) lo[t] = M.v[t].lo; }
}

static int ceil_sqrt(int m) {
    int s = (int)floor(sqrt((double)m));
    while (s * s < m) ++s;
    while (s > 1 && (s - 1) * (s - 1) >= m) --s;
    return s;
}

/*
 * Algorithm 2.1 (Section 2), literally, in double-double.
 *   s <- ceil(sqrt(m)) unless s_in > 0;  r <- floor(m/s);
 *   X_0 = I, X_i = X_{i-1} X for i = 1..s;
 *   P = sum_{j=0}^{m-sr} b_{sr+j} X_j;
 *   for i = r-1 down to 0:  P = sum_{j=0}^{s-1} b_{si+j} X_j + X_s P.
 * X_1 = X_0 X = X is a copy, not counted; the counter reports the s-1 products forming
 * X_2..X_s and the r products X_s P, i.e. s-1+r as in Section 3.4.
 * coef_hi/coef_lo: the m+1 coefficients b_0..b_m as double-double.
 * Returns 0 on success, -1 on bad arguments.
 */
int orc_ps_dd(const double* coef_hi, const double* coef_lo, int m, int s_in,
              const double* X, int n, double* P_hi, double* P_lo, long* mults) {
    if (m < 0 || n <= 0 || !coef_hi || !X || !P_hi) return -1;
    long count = 0;
    if (m == 0) {
        ddmat P = ddm_alloc(n); ddm_zero(P);
        dd b0 = { coef_hi[0], coef_lo ? coef_lo[0] : 0.0 };
        ddm_add_diag(P, b0); ddm_store(P, P_hi, P_lo); ddm_free(&P);
        if (mults) *mults = 0;
        return 0;
    }
    int s = s_in > 0 ? s_in : ceil_sqrt(m);
    int r = m / s;
    ddmat* Xp = (ddmat*)malloc(sizeof(ddmat) * (size_t)(s + 1));
    for (int i = 0; i <= s; ++i) Xp[i] = ddm_alloc(n);
    ddm_identity(Xp[0]);
    ddm_load(Xp[1], X);
    for (int i = 2; i <= s; ++i) { ddm_mul(Xp[i], Xp[i - 1], Xp[1]); ++count; }

    ddmat P = ddm_alloc(n), T = ddm_alloc(n);
    ddm_zero(P);
    for (int j = 0; j <= m - s * r; ++j) {
        dd b = { coef_hi[s * r + j], coef_lo ? coef_lo[s * r + j] : 0.0 };
        ddm_axpy(P, b, Xp[j]);
    }
    for (int i = r - 1; i >= 0; --i) {
        ddm_mul(T, Xp[s], P); ++count;          /* X_s P */
        for (int j = 0; j < s; ++j) {           /* + sum_j b_{si+j} X_j */
            dd b = { coef_hi[s * i + j], coef_lo ? coef_lo[s * i + j] : 0.0 };
            ddm_axpy(T, b, Xp[j]);
        }
        ddm_copy(P, T);
    }
    ddm_store(P, P_hi, P_lo);
    ddm_free(&P); ddm_free(&T);
    for (int i = 0; i <= s; ++i) ddm_free(&Xp[i]);
    free(Xp);
    if (mults) *mults = count;
    return 0;
}

/* Textbook Horner in double-double: P = b_m I; for k = m-1..0: P = P X + b_k I.
 * This is eq. (1.1) with s = 1 (the special case discussed after Theorem 2.1). */
int orc_horner_dd(const double* coef_hi, const double* coef_lo, int m,
                  const double* X, int n, double* P_hi, double* P_lo, long* mults) {
    if (m < 0 || n <= 0) return -1;
    ddmat Xm = ddm_alloc(n), P = ddm_alloc(n), T = ddm_alloc(n);
    ddm_load(Xm, X);
    ddm_zero(P);
    dd bm = { coef_hi[m], coef_lo ? coef_lo[m] : 0.0 };
    ddm_add_diag(P, bm);
    long count = 0;
    for (int k = m - 1; k >= 0; --k) {
        ddm_mul(T, P, Xm); ++count;
        dd b = { coef_hi[k], coef_lo ? coef_lo[k] : 0.0 };
        ddm_add_diag(T, b);
        ddm_copy(P, T);
    }
    ddm_store(P, P_hi, P_lo);
    ddm_free(&Xm); ddm_free(&P); ddm_free(&T);
    if (mults) *mults = count;
    return 0;
}

/* Explicit powers in double-double: P = sum_k b_k X^k with X^k = X^{k-1} X
 * (eq. (1.1) with s = m). */
int orc_powers_dd(const double* coef_hi, const double* coef_lo, int m,
                  const double* X, int n, double* P_hi, double* P_lo) {
    if (m < 0 || n <= 0) return -1;
    ddmat Xm = ddm_alloc(n), K = ddm_alloc(n), T = ddm_alloc(n), P = ddm_alloc(n);
    ddm_load(Xm, X);
    ddm_identity(K);
    ddm_zero(P);
    for (int k = 0; k <= m; ++k) {
        if (k > 0) { ddm_mul(T, K, Xm); ddm_copy(K, T); }
        dd b = { coef_hi[k], coef_lo ? coef_lo[k] : 0.0 };
        ddm_axpy(P, b, K);
    }
    ddm_store(P, P_hi, P_lo);
    ddm_free(&Xm); ddm_free(&K); ddm_free(&T); ddm_free(&P);
    return 0;
}

/* Scaling and squaring, eq. (3.6), in double-double: X = 2^-sigma A (exact in binary),
 * P = p(X) by Algorithm 2.1, then sigma squarings P <- P P. */
int orc_expm_ss_dd(const double* coef_hi, const double* coef_lo, int m, int s_in,
                   const double* A, int n, int sigma, double* E_hi, double* E_lo) {
    if (n <= 0 || sigma < 0) return -1;
    size_t N = (size_t)n * n;
    double* X = (double*)malloc(sizeof(double) * N);
    double* ph = (double*)malloc(sizeof(double) * N);
    double* pl = (double*)malloc(sizeof(double) * N);
    for (size_t t = 0; t < N; ++t) X[t] = ldexp(A[t], -sigma);
    int rc = orc_ps_dd(coef_hi, coef_lo, m, s_in, X, n, ph, pl, NULL);
    if (rc == 0) {
        ddmat P = ddm_alloc(n), T = ddm_alloc(n);
        for (size_t t = 0; t < N; ++t) { P.v[t].hi = ph[t]; P.v[t].lo = pl[t]; }
        for (int k = 0; k < sigma; ++k) { ddm_mul(T, P, P); ddm_copy(P, T); }
        ddm_store(P, E_hi, E_lo);
        ddm_free(&P); ddm_free(&T);
    }
    free(X); free(ph); free(pl);
    return rc;
}

/*
 * W = p(X)^reps V for an n x k block V (row-major n x k), by Horner on vectors:
 * W <- b_m V; for j = m-1..0: W <- X W + b_j V.  Repeated `reps` times (reps = 2^sigma
 * gives columns of p(X)^(2^sigma), the scaling-and-squaring result of eq. (3.6)).
 * X is given in double (the matrix the polynomial is evaluated at), V in double.
 */
int orc_ps_apply_dd(const double* coef_hi, const double* coef_lo, int m,
                    const double* X, int n, const double* V, int k, long reps,
                    double* W_hi, double* W_lo) {
    if (m < 0 || n <= 0 || k <= 0 || reps < 0) return -1;
    size_t NK = (size_t)n * k;
    dd* cur = (dd*)malloc(sizeof(dd) * NK);
    dd* acc = (dd*)malloc(sizeof(dd) * NK);
    dd* tmp = (dd*)malloc(sizeof(dd) * NK);
    for (size_t t = 0; t < NK; ++t) cur[t] = dd_from(V[t]);
    for (long rep = 0; rep < reps; ++rep) {
        dd bm = { coef_hi[m], coef_lo ? coef_lo[m] : 0.0 };
        for (size_t t = 0; t < NK; ++t) acc[t] = dd_mul(bm, cur[t]);
        for (int j = m - 1; j >= 0; --j) {
            #pragma omp parallel for schedule(static)
            for (int i = 0; i < n; ++i) {
                dd* w = tmp + (size_t)i * k;
                for (int c = 0; c < k; ++c) w[c] = dd_from(0.0);
                for (int l = 0; l < n; ++l) {
                    double x = X[(size_t)i * n + l];
                    if (x == 0.0) continue;
                    dd xd = dd_from(x);
                    const dd* a = acc + (size_t)l * k;
                    for (int c = 0; c < k; ++c) w[c] = dd_add(w[c], dd_mul(xd, a[c]));
                }
            }
            dd bj = { coef_hi[j], coef_lo ? coef_lo[j] : 0.0 };
            for (size_t t = 0; t < NK; ++t) acc[t] = dd_add(tmp[t], dd_mul(bj, cur[t]));
        }
        memcpy(cur, acc, sizeof(dd) * NK);
    }
    for (size_t t = 0; t < NK; ++t) { W_hi[t] = cur[t].hi; if (W_lo) W_lo[t] = cur[t].lo; }
    free(cur); free(acc); free(tmp);
    return 0;
}

/*
 * Gradient of f(A) = <G, p(A)> = sum_ij G_ij p(A)_ij with respect to A:
 *   grad = L_p(A^T, G) = sum_{k=1}^m c_k sum_{j=0}^{k-1} (A^T)^j G (A^T)^(k-1-j),
 * the Frechet derivative of p at A^T in direction G (the paper states no adjoint; this is
 * the definition of the derivative of a matrix polynomial).  Written as the double sum,
 * with the powers Q_j = (A^T)^j formed once by repeated multiplication.  Double-double.
 */
/* D = sum_k c_k sum_{j<k} (A^T)^j Gm (A^T)^(k-1-j) for a double-double Gm. */
static void adjoint_sum_dd(const double* coef_hi, const double* coef_lo, int m,
                           const double* A, ddmat Gm, ddmat D) {
    int n = Gm.n;
    int nq = m > 0 ? m : 1;
    ddmat* Q = (ddmat*)malloc(sizeof(ddmat) * (size_t)nq);
    for (int j = 0; j < nq; ++j) Q[j] = ddm_alloc(n);
    ddmat At = ddm_alloc(n), T = ddm_alloc(n), U = ddm_alloc(n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) At.v[(size_t)i * n + j] = dd_from(A[(size_t)j * n + i]);
    ddm_identity(Q[0]);
    for (int j = 1; j < nq; ++j) ddm_mul(Q[j], Q[j - 1], At);
    ddm_zero(D);
    for (int k = 1; k <= m; ++k) {
        dd c = { coef_hi[k], coef_lo ? coef_lo[k] : 0.0 };
        for (int j = 0; j <= k - 1; ++j) {
            ddm_mul(T, Q[j], Gm);
            ddm_mul(U, T, Q[k - 1 - j]);
            ddm_axpy(D, c, U);
        }
    }
    for (int j = 0; j < nq; ++j) ddm_free(&Q[j]);
    free(Q);
    ddm_free(&At); ddm_free(&T); ddm_free(&U);
}

int orc_adjoint_dd(const double* coef_hi, const double* coef_lo, int m,
                   const double* A, const double* G, int n, double* D_hi, double* D_lo) {
    if (m < 0 || n <= 0) return -1;
    ddmat Gm = ddm_alloc(n), D = ddm_alloc(n);
    ddm_load(Gm, G);
    adjoint_sum_dd(coef_hi, coef_lo, m, A, Gm, D);
    ddm_store(D, D_hi, D_lo);
    ddm_free(&Gm); ddm_free(&D);
    return 0;
}

/*
 * Gradient of A -> <G, r(A)> for the scaling-and-squaring approximant of eq. (3.6),
 * r(A) = p(X)^(2^sigma), X = 2^-sigma A, sigma given: the chain rule through each step.
 *   S_0 = p(X), S_{k+1} = S_k S_k                      (k < sigma)
 *   d<G, S_sigma> : Sbar_sigma = G,  Sbar_k = Sbar_{k+1} S_k^T + S_k^T Sbar_{k+1}
 *   Xbar = sum_k c_k sum_{j<k} (X^T)^j Sbar_0 (X^T)^(k-1-j),   Abar = 2^-sigma Xbar.
 * All in double-double; S_0 from Algorithm 2.1 (orc_ps_dd).
 */
int orc_expm_ss_adjoint_dd(const double* coef_hi, const double* coef_lo, int m,
                           const double* A, const double* G, int n, int sigma,
                           double* D_hi, double* D_lo) {
    if (m < 0 || n <= 0 || sigma < 0) return -1;
    size_t N = (size_t)n * n;
    double* X = (double*)malloc(sizeof(double) * N);
    double* ph = (double*)malloc(sizeof(double) * N);
    double* pl = (double*)malloc(sizeof(double) * N);
    for (size_t t = 0; t < N; ++t) X[t] = ldexp(A[t], -sigma);
    int rc = orc_ps_dd(coef_hi, coef_lo, m, 0, X, n, ph, pl, NULL);
    if (rc == 0) {
        int ns = sigma > 0 ? sigma : 1;
        ddmat* S = (ddmat*)malloc(sizeof(ddmat) * (size_t)ns);
        for (int k = 0; k < ns; ++k) S[k] = ddm_alloc(n);
        for (size_t t = 0; t < N; ++t) { S[0].v[t].hi = ph[t]; S[0].v[t].lo = pl[t]; }
        for (int k = 1; k < sigma; ++k) ddm_mul(S[k], S[k - 1], S[k - 1]);
        ddmat Sb = ddm_alloc(n), St = ddm_alloc(n), T1 = ddm_alloc(n), T2 = ddm_alloc(n),
              D = ddm_alloc(n);
        ddm_load(Sb, G);
        for (int k = sigma - 1; k >= 0; --k) {
            for (int i = 0; i < n; ++i)          /* St = S_k^T */
                for (int j = 0; j < n; ++j) St.v[(size_t)i * n + j] = S[k].v[(size_t)j * n + i];
            ddm_mul(T1, Sb, St);
            ddm_mul(T2, St, Sb);
            for (size_t t = 0; t < N; ++t) Sb.v[t] = dd_add(T1.v[t], T2.v[t]);
        }
        adjoint_sum_dd(coef_hi, coef_lo, m, X, Sb, D);
        for (size_t t = 0; t < N; ++t) {   /* exact power-of-two scaling of both words */
            D_hi[t] = ldexp(D.v[t].hi, -sigma);
            D_lo[t] = ldexp(D.v[t].lo, -sigma);
        }
        for (int k = 0; k < ns; ++k) ddm_free(&S[k]);
        free(S);
        ddm_free(&Sb); ddm_free(&St); ddm_free(&T1); ddm_free(&T2); ddm_free(&D);
    }
    free(X); free(ph); free(pl);
    return rc;
}

/* Product of two double-double matrices (hi/lo pairs), C = A B; used by the tests to
 * check group properties such as exp(A) exp(-A) = I at double-double accuracy. */
int orc_matmul_dd(const double* A_hi, const double* A_lo, const double* B_hi,
                  const double* B_lo, int n, double* C_hi, double* C_lo) {
    if (n <= 0) return -1;
    ddmat A = ddm_alloc(n), B = ddm_alloc(n), C = ddm_alloc(n);
    size_t N = (size_t)n * n;
    for (size_t t = 0; t < N; ++t) {
        A.v[t].hi = A_hi[t]; A.v[t].lo = A_lo ? A_lo[t] : 0.0;
        B.v[t].hi = B_hi[t]; B.v[t].lo = B_lo ? B_lo[t] : 0.0;
    }
    ddm_mul(C, A, B);
    ddm_store(C, C_hi, C_lo);
    ddm_free(&A); ddm_free(&B); ddm_free(&C);
    return 0;
}

/* ---- plain double versions: the timed CPU baseline ------------------------------ */

static void dm_mul(double* C, const double* A, const double* B, int n) {
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double* c = C + (size_t)i * n;
        for (int j = 0; j < n; ++j) c[j] = 0.0;
        for (int k = 0; k < n; ++k) {
            double a = A[(size_t)i * n + k];
            const double* b = B + (size_t)k * n;
            for (int j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

/* Algorithm 2.1 in plain double, same steps and counter as orc_ps_dd. */
int orc_ps_d(const double* coef, int m, int s_in, const double* X, int n, double* P_out,
             long* mults) {
    if (m < 0 || n <= 0) return -1;
    size_t N = (size_t)n * n;
    long count = 0;
    if (m == 0) {
        memset(P_out, 0, sizeof(double) * N);
        for (int i = 0; i < n; ++i) P_out[(size_t)i * n + i] = coef[0];
        if (mults) *mults = 0;
        return 0;
    }
    int s = s_in > 0 ? s_in : ceil_sqrt(m);
    int r = m / s;
    double** Xp = (double**)malloc(sizeof(double*) * (size_t)(s + 1));
    for (int i = 0; i <= s; ++i) Xp[i] = (double*)calloc(N, sizeof(double));
    for (int i = 0; i < n; ++i) Xp[0][(size_t)i * n + i] = 1.0;
    memcpy(Xp[1], X, sizeof(double) * N);
    for (int i = 2; i <= s; ++i) { dm_mul(Xp[i], Xp[i - 1], Xp[1], n); ++count; }
    double* P = (double*)calloc(N, sizeof(double));
    double* T = (double*)malloc(sizeof(double) * N);
    for (int j = 0; j <= m - s * r; ++j)
        for (size_t t = 0; t < N; ++t) P[t] += coef[s * r + j] * Xp[j][t];
    for (int i = r - 1; i >= 0; --i) {
        dm_mul(T, Xp[s], P, n); ++count;
        for (int j = 0; j < s; ++j)
            for (size_t t = 0; t < N; ++t) T[t] += coef[s * i + j] * Xp[j][t];
        memcpy(P, T, sizeof(double) * N);
    }
    memcpy(P_out, P, sizeof(double) * N);
    free(P); free(T);
    for (int i = 0; i <= s; ++i) free(Xp[i]);
    free(Xp);
    if (mults) *mults = count;
    return 0;
}

/* Scaling and squaring in plain double (eq. (3.6)); the timed CPU baseline for the
 * matrix exponential. */
int orc_expm_ss_d(const double* coef, int m, int s_in, const double* A, int n, int sigma,
                  double* E) {
    if (n <= 0 || sigma < 0) return -1;
    size_t N = (size_t)n * n;
    double* X = (double*)malloc(sizeof(double) * N);
    double* T = (double*)malloc(sizeof(double) * N);
    for (size_t t = 0; t < N; ++t) X[t] = ldexp(A[t], -sigma);
    int rc = orc_ps_d(coef, m, s_in, X, n, E, NULL);
    for (int k = 0; rc == 0 && k < sigma; ++k) { dm_mul(T, E, E, n); memcpy(E, T, sizeof(double) * N); }
    free(X); free(T);
    return rc;
}

/* 1-norm: max_j sum_i |M_ij| (the norm of the error measure in Section 3.4). */
double orc_norm1(const double* M, int rows, int cols) {
    double best = 0.0;
    for (int j = 0; j < cols; ++j) {
        double sum = 0.0;
        for (int i = 0; i < rows; ++i) sum += fabs(M[(size_t)i * cols + j]);
        if (sum > best) best = sum;
    }
    return best;
}

/* Number of OpenMP threads the oracle runs with (1 when built without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
