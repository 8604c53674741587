/*
 * simplex_oracle.c -- plain FP64 revised simplex on the CPU.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this file.  It shares no code with
 * the CUDA path and is deliberately slow and literal: explicit dense B^-1,
 * plain loops, sums in increasing index order, no BLAS.  It is compiled with
 * -ffp-contract=off so that x86 and Arm hosts produce the same bits.
 *
 * Parallel build (-fopenmp, liboracle_omp.so): the loops over independent
 * output elements -- PRICE over columns j, FTRAN and the Step 8 update over
 * rows i, the Gauss-Jordan elimination over rows, bbar and y after a
 * reinversion -- are shared among threads.  Every element is still summed by
 * one thread in the same increasing index order, so both builds give the
 * same bits; every decision (CHUZC, CHUZR, tabu, follow mode) stays serial.
 *
 * Problem: max c^T x  s.t.  A x <= b, x >= 0, b >= 0 (A is m x n, row-major).
 * Section 2.1 states the method for min C^T X, AX = b with A = (A', I_m);
 * the max form is the same problem with C' = -c.  Variables 0..n-1 are the
 * structural x_j, variables n..n+m-1 are the slacks (column e_i of I_m).
 *
 * Notation (max form):  y = c_B^T B^-1  (the paper's W up to sign),
 * d_j = c_j - y^T a_j (the paper's z_j - c_j of Step 3 for C = -c),
 * alpha = B^-1 a_q (the paper's Y_k of Step 5), bbar = B^-1 b (Step 2).
 *
 * One iteration follows Steps 3-8 of Section 2.1:
 *   Step 3  PRICE    d_j for every nonbasic j (slack n+i has d = -y_i).
 *   Step 4  CHUZC    optimal if max_j d_j <= tol_d over all nonbasic j;
 *                    otherwise q = argmax d_j over nonbasic, non-tabu j with
 *                    d_j > tol_d, exact ties to the smallest j.  If every
 *                    improving j is tabu, the tabu list is ignored for this
 *                    iteration (aspiration).
 *   Step 5  FTRAN    alpha = B^-1 a_q; unbounded if no alpha_i > tol_piv.
 *   Step 6  CHUZR    theta_i = bbar_i / alpha_i over alpha_i > tol_piv;
 *                    tie set T = {theta_i <= theta_min + tol_tie*max(1,|theta_min|)};
 *                    r = the element of T with the largest alpha_i, exact
 *                    ties to the smallest basic variable index.  (Sections
 *                    2.2 and 3.4 ask for the leaving element with the most
 *                    noticeable objective improvement; every tied row gives
 *                    the same improvement theta*d_q, so the largest pivot is
 *                    taken as the deciding criterion.)
 *           TABU     if |T| > 1 (no unique leaving element, Sections 2.2/3.4)
 *                    or the pivot is degenerate (theta <= tol_tie), the
 *                    leaving variable may not enter during the next
 *                    `tabu_tenure` iterations.
 *   Step 7           basis[r] <- q.
 *   Step 8  UPDATE   tableau pivot on [ -y | z ; B^-1 | bbar ]: row r is
 *                    divided by alpha_r, then every other row i gets the new
 *                    row r times -alpha_i added (row 0 uses d_q).
 * Reinversion: every `reinvert_every` iterations B^-1 is rebuilt from the
 * basis columns by Gauss-Jordan elimination with partial pivoting, and bbar,
 * y and z are recomputed from it.  (The paper only updates; periodic
 * reinversion is an addition of this design.)
 * Lexicographic rule (ratio_rule 2; the textbook anti-cycling rule the
 * paper's tabu rule is compared with, Sections 2.2 and 3.4): among the tie set
 * T the leaving row is the one whose row of B^-1 divided by alpha_i is
 * lexicographically smallest, columns compared in increasing order; two
 * entries count as equal when they differ by at most tol_tie times the
 * larger of 1 and their magnitudes (an exact zero of the update and its
 * reinverted counterpart must not decide).  Rows of a nonsingular B^-1 are
 * independent, so the rule always decides.  Callers switch the tabu list
 * and the safety net off with it.
 * Cycling safety net: after `bland_after` consecutive degenerate pivots both
 * rules become Bland's (entering: smallest improving index, tabu ignored;
 * leaving: smallest basic variable index in the tie set) until the next
 * non-degenerate pivot.
 *
 * Follow mode: given another solver's pivot sequence, the oracle makes its
 * own decision at every iteration and, where the other solver chose
 * differently, accepts that choice only if, in the oracle's own arithmetic, it
 * is tied with the oracle's choice to within `tie_cmp` (relative).  An
 * accepted choice is then adopted and the oracle continues from it, so the
 * whole foreign sequence is checked pivot by pivot.  With `follow_relaxed`
 * the entering choice only has to be an improving, eligible column (for
 * solvers that screen the pricing in lower precision); the leaving row is
 * still checked against the ratio test.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_RUNNING 0
#define OR_OPTIMAL 1
#define OR_UNBOUNDED 2
#define OR_ITER_LIMIT 3
#define OR_SINGULAR 4
#define OR_MISMATCH 5
#define OR_NOMEM 6

/* trace flags */
#define TF_DEGENERATE 1
#define TF_TABU_PUSH 2
#define TF_ASPIRATION 4
#define TF_BLAND 8
#define TF_ADOPT_Q 16
#define TF_ADOPT_R 32
#define TF_TIE_SET 64

typedef struct {
    int32_t reinvert_every; /* 0 = never */
    int32_t tabu_tenure;    /* 0 = tabu rule off */
    int32_t max_iters;
    int32_t bland_after;    /* 0 = no Bland fallback */
    int32_t ratio_rule;     /* 0 = largest alpha in the tie set, 1 = smallest basic index,
                               2 = lexicographic (rows of B^-1 / alpha_i) */
    int32_t follow_relaxed; /* follow mode: accept any improving eligible entering column */
    double tol_d, tol_piv, tol_tie;
    double tie_cmp;         /* follow mode: relative tie window (1e-12) */
} oracle_opts;

typedef struct {
    int32_t status, iterations, reinversions, degenerate;
    int32_t tabu_pushes, bland_fallbacks, aspirations, adopted;
    int32_t mismatch_at, mismatch_kind;
    double objective;
} oracle_result;

typedef struct {
    int32_t* q;
    int32_t* r;
    double* theta;
    double* dq;
    int32_t* flags;
    double* margin_q; /* (d_q - best other eligible d) / max(1,|d_q|) */
    double* margin_r; /* min relative separation of r from the other rows */
    int32_t cap;
} oracle_trace;

static double dmax(double a, double b) { return a > b ? a : b; }

/* Threads of the parallel build (nt > 0 sets them); 1 in the serial build. */
int oracle_threads(int nt) {
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}

/* Column j of [A | I_m] as a dense m-vector. */
static void column(int m, int n, const double* A, int j, double* out) {
    if (j < n) {
        for (int i = 0; i < m; ++i) out[i] = A[(size_t)i * n + j];
    } else {
        for (int i = 0; i < m; ++i) out[i] = 0.0;
        out[j - n] = 1.0;
    }
}

/*
 * Gauss-Jordan inverse with partial pivoting on the augmented matrix [M | I].
 * M is k x k row-major; the inverse is written to `inv` (k x k row-major).
 * Row operations whose multiplier is exactly zero are skipped (they change
 * nothing).  Returns 0, or -1 if a pivot column is entirely zero.
 */
int oracle_gj_inverse(int k, const double* M, double* inv) {
    size_t w = 2 * (size_t)k;
    double* G = (double*)malloc(sizeof(double) * (size_t)k * w);
    if (!G) return -2;
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) G[i * w + j] = M[(size_t)i * k + j];
        for (int j = 0; j < k; ++j) G[i * w + k + j] = (i == j) ? 1.0 : 0.0;
    }
    for (int j = 0; j < k; ++j) {
        int p = j;
        double best = fabs(G[j * w + j]);
        for (int i = j + 1; i < k; ++i) {
            double v = fabs(G[i * w + j]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) { free(G); return -1; }
        if (p != j) {
            for (size_t t = 0; t < w; ++t) {
                double tmp = G[j * w + t]; G[j * w + t] = G[p * w + t]; G[p * w + t] = tmp;
            }
        }
        double piv = G[j * w + j];
        for (size_t t = 0; t < w; ++t) G[j * w + t] /= piv;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < k; ++i) {
            if (i == j) continue;
            double f = G[i * w + j];
            if (f == 0.0) continue;
            for (size_t t = 0; t < w; ++t) G[i * w + t] -= f * G[j * w + t];
        }
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) inv[(size_t)i * k + j] = G[i * w + k + j];
    free(G);
    return 0;
}

/* d_j = c_j - sum_i y_i a_ij for every structural j (summed in increasing i),
   d_{n+i} = -y_i for the slacks; basic variables are reported as well. */
void oracle_reduced_costs(int m, int n, const double* A, const double* c, const double* y, double* d) {
    double* dot = (double*)calloc((size_t)n, sizeof(double));
#ifdef _OPENMP
    /* each thread owns a block of columns and adds its rows in increasing i */
#pragma omp parallel for schedule(static)
    for (int j0 = 0; j0 < n; j0 += 512) {
        const int j1 = j0 + 512 < n ? j0 + 512 : n;
        for (int i = 0; i < m; ++i) {
            const double* Ai = A + (size_t)i * n;
            double yi = y[i];
            for (int j = j0; j < j1; ++j) dot[j] += yi * Ai[j];
        }
    }
#else
    for (int i = 0; i < m; ++i) {
        const double* Ai = A + (size_t)i * n;
        double yi = y[i];
        for (int j = 0; j < n; ++j) dot[j] += yi * Ai[j];
    }
#endif
    for (int j = 0; j < n; ++j) d[j] = c[j] - dot[j];
    for (int i = 0; i < m; ++i) d[n + i] = -y[i];
    free(dot);
}

static double cost(int n, const double* c, int j) { return j < n ? c[j] : 0.0; }

/* Lexicographic comparison of rows i and r of B^-1, each divided by its
 * alpha: -1 if row i comes first, +1 if row r does, 0 if every column is equal
 * within tau (relative to the larger of 1 and the two magnitudes). */
static int lex_cmp(const double* Binv, int m, const double* alpha, int i, int r, double tau) {
    const double* bi = Binv + (size_t)i * m;
    const double* br = Binv + (size_t)r * m;
    for (int c = 0; c < m; ++c) {
        double vi = bi[c] / alpha[i], vr = br[c] / alpha[r];
        double sc = dmax(1.0, dmax(fabs(vi), fabs(vr)));
        if (fabs(vi - vr) <= tau * sc) continue;
        return vi < vr ? -1 : 1;
    }
    return 0;
}

/* Rebuild B^-1, bbar, y and z from the basis. */
static int reinvert(int m, int n, const double* A, const double* b, const double* c,
                    const int32_t* basis, double* Binv, double* bbar, double* y, double* z) {
    double* B = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* col = (double*)malloc(sizeof(double) * (size_t)m);
    if (!B || !col) { free(B); free(col); return -2; }
    for (int p = 0; p < m; ++p) {
        column(m, n, A, basis[p], col);
        for (int i = 0; i < m; ++i) B[(size_t)i * m + p] = col[i];
    }
    int rc = oracle_gj_inverse(m, B, Binv);
    free(B);
    free(col);
    if (rc) return rc;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += Binv[(size_t)i * m + k] * b[k];
        bbar[i] = s;
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < m; ++k) {
        double s = 0.0;
        for (int p = 0; p < m; ++p) s += cost(n, c, basis[p]) * Binv[(size_t)p * m + k];
        y[k] = s;
    }
    double zz = 0.0;
    for (int p = 0; p < m; ++p) zz += cost(n, c, basis[p]) * bbar[p];
    *z = zz;
    return 0;
}

/*
 * Solve.  Optional inputs: start_basis (m indices; NULL = slack basis),
 * follow_q/follow_r (another solver's choices; follow_q[t] = -1 means it
 * stopped at iteration t with status follow_status).  Optional outputs may be
 * NULL: x (n), y_out (m), basis_out (m), binv_out (m*m), bbar_out (m), trace.
 */
/* ---- checking another solver's pivots (follow mode) and the separation
 * margins of the trace.  None of this changes the method's own decisions. */

/* How far the entering choice q stands from the best other candidate of the
   same rule: (d_q - second) / max(1, |d_q|). */
static double entering_margin(int N, const double* d, const int32_t* pos, const int32_t* tabu_until, int it,
                              int aspiration, int q) {
    double second = -INFINITY;
    for (int j = 0; j < N; ++j)
        if (j != q && pos[j] < 0 && (aspiration || tabu_until[j] <= it) && d[j] > second) second = d[j];
    return (d[q] - second) / dmax(1.0, fabs(d[q]));
}

/* The smallest relative separation of the leaving row r from every other row
   with alpha_i > tol_piv: by alpha within the tie set (none under the
   lexicographic rule), by ratio outside it. */
static double leaving_margin(int m, const oracle_opts* o, const double* alpha, const double* theta, double tmin,
                             double thr, int r) {
    double margin = INFINITY;
    for (int i = 0; i < m; ++i) {
        if (i == r || !(alpha[i] > o->tol_piv)) continue;
        double sep;
        if (theta[i] <= thr && o->ratio_rule == 2) sep = INFINITY;
        else if (theta[i] <= thr) sep = (alpha[r] - alpha[i]) / dmax(1.0, alpha[r]);
        else sep = (theta[i] - thr) / dmax(1.0, fabs(tmin));
        if (sep < margin) margin = sep;
    }
    return margin;
}

/* The other solver's entering choice fq at this iteration (fq < 0: it
   stopped), against the oracle's own (*opt, *q).  A different choice is
   accepted when, in the oracle's arithmetic, it is tied with the oracle's
   within tie_cmp (or, with follow_relaxed, is any improving eligible column);
   it is then adopted (*opt, *q, *flags |= TF_ADOPT_Q).  Returns 0 on a
   mismatch. */
static int follow_entering(const oracle_opts* o, int N, const double* d, const int32_t* pos,
                           const int32_t* tabu_until, int it, int bland, double dmax_all, int fq,
                           int follow_status, int* opt, int* q, int* flags, int32_t* adopted) {
    const double eps = o->tie_cmp;
    if (fq < 0 || *opt) {
        if (fq < 0 && *opt && follow_status == OR_OPTIMAL) return 1;
        /* borderline optimality: max d within the tie window of tol_d */
        int border = fabs(dmax_all - o->tol_d) <= eps * dmax(1.0, fabs(o->tol_d));
        if (fq < 0 && follow_status == OR_OPTIMAL && border) {
            *opt = 1;
            (*adopted)++;
            return 1;
        }
        if (fq >= 0 && *opt && border && fq < N && pos[fq] < 0) {
            *opt = 0;
            *q = fq;
            *flags |= TF_ADOPT_Q;
            (*adopted)++;
            return 1;
        }
        /* the other solver stopped for another reason: the leaving step decides */
        return fq < 0 && !*opt && follow_status != OR_OPTIMAL;
    }
    if (fq == *q) return 1;
    int ok = fq < N && pos[fq] < 0;
    if (ok && bland) {
        for (int j = 0; j < fq && ok; ++j)
            if (pos[j] < 0 && d[j] > o->tol_d + eps * dmax(1.0, o->tol_d)) ok = 0;
        if (d[fq] < o->tol_d - eps * dmax(1.0, o->tol_d)) ok = 0;
    } else if (ok) {
        int asp = (*flags & TF_ASPIRATION) != 0;
        if (!asp && tabu_until[fq] > it) ok = 0;
        if (o->follow_relaxed) {
            /* any improving column is a valid simplex pivot */
            if (!(d[fq] > o->tol_d - eps * dmax(1.0, o->tol_d))) ok = 0;
        } else if (d[fq] < d[*q] - eps * dmax(1.0, fabs(d[*q]))) {
            ok = 0;
        }
    }
    if (!ok) return 0;
    *q = fq;
    *flags |= TF_ADOPT_Q;
    (*adopted)++;
    return 1;
}

/* The other solver's leaving row fr (fr < 0: unbounded) against the oracle's
   own r, for the same entering column.  A different row is accepted when it
   is in the tie set within tie_cmp and tied with r by the ratio rule (or r
   itself is at the tie set's edge); it is then adopted (*r, theta[fr],
   *flags |= TF_ADOPT_R).  Returns 0 on a mismatch. */
static int follow_leaving(const oracle_opts* o, int m, const double* Binv, const double* bbar, const double* alpha,
                          double* theta, double tmin, double thr, int bland, int fr, int* r, int* flags,
                          int32_t* adopted) {
    const double eps = o->tie_cmp;
    if (fr < 0 || *r < 0) {
        if (fr < 0 && *r < 0) return 1;
        double amax = -INFINITY;
        for (int i = 0; i < m; ++i) amax = dmax(amax, alpha[i]);
        int border = fabs(amax - o->tol_piv) <= eps * dmax(1.0, o->tol_piv);
        if (!border) return 0;
        *r = fr;
        if (fr >= 0) {
            theta[fr] = bbar[fr] / alpha[fr];
            *flags |= TF_ADOPT_R;
        }
        (*adopted)++;
        return 1;
    }
    if (fr == *r) return 1;
    int ok = fr < m && alpha[fr] > o->tol_piv - eps * dmax(1.0, o->tol_piv);
    if (ok) {
        double th = bbar[fr] / alpha[fr];
        double sc = dmax(1.0, fabs(tmin));
        if (th > thr + eps * sc) ok = 0;
        /* the oracle's row r must itself be near the tie-set edge, or fr must
           carry a pivot tied with alpha_r */
        int r_border = theta[*r] >= thr - eps * sc;
        int a_tie = alpha[fr] >= alpha[*r] - eps * dmax(1.0, alpha[*r]);
        if (o->ratio_rule == 1 || bland) a_tie = 1;
        /* lexicographic: fr may not come after r beyond the follow tolerance */
        if (o->ratio_rule == 2) a_tie = lex_cmp(Binv, m, alpha, fr, *r, eps) <= 0;
        if (!(a_tie || r_border)) ok = 0;
        if (ok) theta[fr] = th;
    }
    if (!ok) return 0;
    *r = fr;
    *flags |= TF_ADOPT_R;
    (*adopted)++;
    return 1;
}

int oracle_solve(int m, int n, const double* A, const double* b, const double* c,
                 const oracle_opts* o, const int32_t* start_basis,
                 const int32_t* follow_q, const int32_t* follow_r, int32_t follow_len, int32_t follow_status,
                 oracle_trace* tr, double* x, double* y_out, int32_t* basis_out,
                 double* binv_out, double* bbar_out, oracle_result* res) {
    const int N = n + m;
    memset(res, 0, sizeof(*res));
    res->mismatch_at = -1;
    double* Binv = (double*)calloc((size_t)m * m, sizeof(double));
    double* bbar = (double*)malloc(sizeof(double) * m);
    double* y = (double*)calloc((size_t)m, sizeof(double));
    double* d = (double*)malloc(sizeof(double) * N);
    double* aq = (double*)malloc(sizeof(double) * m);
    double* alpha = (double*)malloc(sizeof(double) * m);
    double* theta = (double*)malloc(sizeof(double) * m);
    double* rho = (double*)malloc(sizeof(double) * m);
    int32_t* basis = (int32_t*)malloc(sizeof(int32_t) * m);
    int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* tabu_until = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    if (!Binv || !bbar || !y || !d || !aq || !alpha || !theta || !rho || !basis || !pos || !tabu_until) {
        res->status = OR_NOMEM;
        goto done;
    }
    for (int j = 0; j < N; ++j) pos[j] = -1;
    double z = 0.0;
    int it = 0;
    if (start_basis) {
        for (int p = 0; p < m; ++p) { basis[p] = start_basis[p]; pos[basis[p]] = p; }
        int rc = reinvert(m, n, A, b, c, basis, Binv, bbar, y, &z);
        if (rc) { res->status = OR_SINGULAR; goto done; }
        res->reinversions++;
    } else {
        /* Step 1 with B = I_m (slack basis): B^-1 = I, bbar = b, y = 0, z = 0. */
        for (int p = 0; p < m; ++p) {
            basis[p] = n + p;
            pos[n + p] = p;
            Binv[(size_t)p * m + p] = 1.0;
            bbar[p] = b[p];
        }
    }
    int degen_run = 0, bland = 0;

    for (;;) {
        if (it >= o->max_iters) { res->status = OR_ITER_LIMIT; break; }
        int flags = bland ? TF_BLAND : 0;

        /* Step 3: PRICE. */
        oracle_reduced_costs(m, n, A, c, y, d);

        /* Step 4: optimality test over every nonbasic variable. */
        double dmax_all = -INFINITY;
        for (int j = 0; j < N; ++j)
            if (pos[j] < 0 && d[j] > dmax_all) dmax_all = d[j];
        int opt = !(dmax_all > o->tol_d);

        int q = -1;
        double margin_q = INFINITY;
        if (!opt) {
            if (bland) {
                for (int j = 0; j < N; ++j)
                    if (pos[j] < 0 && d[j] > o->tol_d) { q = j; break; }
            } else {
                for (int j = 0; j < N; ++j)
                    if (pos[j] < 0 && tabu_until[j] <= it && d[j] > o->tol_d && (q < 0 || d[j] > d[q])) q = j;
                if (q < 0) {
                    flags |= TF_ASPIRATION;
                    res->aspirations++;
                    for (int j = 0; j < N; ++j)
                        if (pos[j] < 0 && d[j] > o->tol_d && (q < 0 || d[j] > d[q])) q = j;
                }
                margin_q = entering_margin(N, d, pos, tabu_until, it, (flags & TF_ASPIRATION) != 0, q);
            }
        }

        /* Follow mode: the other solver's entering choice, adopted when tied. */
        if (it < follow_len && !follow_entering(o, N, d, pos, tabu_until, it, bland, dmax_all, follow_q[it],
                                                follow_status, &opt, &q, &flags, &res->adopted)) {
            res->status = OR_MISMATCH;
            res->mismatch_at = it;
            res->mismatch_kind = 1;
            break;
        }
        if (opt) { res->status = OR_OPTIMAL; break; }
        double dq = d[q];

        /* Step 5: FTRAN alpha = B^-1 a_q. */
        column(m, n, A, q, aq);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            const double* Bi = Binv + (size_t)i * m;
            if (q < n) {
                for (int k = 0; k < m; ++k) s += Bi[k] * aq[k];
            } else {
                s = Bi[q - n];
            }
            alpha[i] = s;
        }

        /* Step 6: CHUZR ratio test with the tie set. */
        double tmin = INFINITY;
        int nR = 0;
        for (int i = 0; i < m; ++i) {
            if (alpha[i] > o->tol_piv) {
                theta[i] = bbar[i] / alpha[i];
                if (theta[i] < tmin) tmin = theta[i];
                nR++;
            }
        }
        int r = -1;
        int tcount = 0;
        double thr = 0.0;
        if (nR > 0) {
            thr = tmin + o->tol_tie * dmax(1.0, fabs(tmin));
            for (int i = 0; i < m; ++i) {
                if (!(alpha[i] > o->tol_piv) || !(theta[i] <= thr)) continue;
                tcount++;
                if (r < 0) { r = i; continue; }
                if (o->ratio_rule == 1 || bland) {
                    if (basis[i] < basis[r]) r = i;
                } else if (o->ratio_rule == 2) {
                    int cmp = lex_cmp(Binv, m, alpha, i, r, o->tol_tie);
                    if (cmp < 0 || (cmp == 0 && basis[i] < basis[r])) r = i;
                } else if (alpha[i] > alpha[r] || (alpha[i] == alpha[r] && basis[i] < basis[r])) {
                    r = i;
                }
            }
        }
        const double margin_r = r >= 0 ? leaving_margin(m, o, alpha, theta, tmin, thr, r) : INFINITY;

        /* Follow mode: the other solver's leaving row, adopted when tied. */
        if (it < follow_len && follow_q[it] >= 0 &&
            !follow_leaving(o, m, Binv, bbar, alpha, theta, tmin, thr, bland, follow_r[it], &r, &flags,
                            &res->adopted)) {
            res->status = OR_MISMATCH;
            res->mismatch_at = it;
            res->mismatch_kind = 2;
            break;
        }
        if (r < 0) { res->status = OR_UNBOUNDED; break; }
        if (tcount > 1) flags |= TF_TIE_SET;

        double th = theta[r]; /* step length: bbar_r / alpha_r */
        double ar = alpha[r];
        int degenerate = th <= o->tol_tie;
        if (degenerate) { flags |= TF_DEGENERATE; res->degenerate++; }
        if (o->tabu_tenure > 0 && (tcount > 1 || degenerate)) {
            tabu_until[basis[r]] = it + 1 + o->tabu_tenure;
            flags |= TF_TABU_PUSH;
            res->tabu_pushes++;
        }

        if (tr && it < tr->cap) {
            tr->q[it] = q;
            tr->r[it] = r;
            tr->theta[it] = th;
            tr->dq[it] = dq;
            tr->flags[it] = flags;
            if (tr->margin_q) tr->margin_q[it] = margin_q;
            if (tr->margin_r) tr->margin_r[it] = margin_r;
        }

        /* Step 8: tableau pivot.  Row r divided by alpha_r, then row i gets
           -alpha_i times the new row r; row 0 ([-y | z]) uses d_q. */
        double* Br = Binv + (size_t)r * m;
        for (int k = 0; k < m; ++k) rho[k] = Br[k] / ar; /* new row r */
        for (int k = 0; k < m; ++k) Br[k] = rho[k];
        double bnew_r = bbar[r] / ar;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < m; ++i) {
            if (i == r) continue;
            double ai = alpha[i];
            if (ai == 0.0) continue;
            double* Bi = Binv + (size_t)i * m;
            for (int k = 0; k < m; ++k) Bi[k] -= ai * rho[k];
            bbar[i] -= ai * bnew_r;
        }
        bbar[r] = bnew_r;
        for (int k = 0; k < m; ++k) y[k] += dq * rho[k];
        z += dq * bnew_r;

        /* Step 7: basis exchange. */
        pos[basis[r]] = -1;
        basis[r] = q;
        pos[q] = r;
        it++;

        /* degenerate-run bookkeeping for the Bland safety net */
        if (degenerate) degen_run++; else degen_run = 0;
        if (bland && !degenerate) bland = 0;
        if (!bland && o->bland_after > 0 && degen_run >= o->bland_after) {
            bland = 1;
            res->bland_fallbacks++;
        }

        if (o->reinvert_every > 0 && it % o->reinvert_every == 0) {
            int rc = reinvert(m, n, A, b, c, basis, Binv, bbar, y, &z);
            if (rc) { res->status = OR_SINGULAR; break; }
            res->reinversions++;
        }
    }
    res->iterations = it;
    res->objective = z;
    if (x) {
        for (int j = 0; j < n; ++j) x[j] = 0.0;
        for (int p = 0; p < m; ++p)
            if (basis[p] < n) x[basis[p]] = bbar[p];
    }
    if (y_out) memcpy(y_out, y, sizeof(double) * m);
    if (basis_out) memcpy(basis_out, basis, sizeof(int32_t) * m);
    if (binv_out) memcpy(binv_out, Binv, sizeof(double) * (size_t)m * m);
    if (bbar_out) memcpy(bbar_out, bbar, sizeof(double) * m);
done:
    free(Binv); free(bbar); free(y); free(d); free(aq); free(alpha); free(theta); free(rho);
    free(basis); free(pos); free(tabu_until);
    return res->status;
}
