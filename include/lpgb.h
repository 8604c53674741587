/*
 * lpgb.h -- C ABI of the GB300 dense revised simplex solver.
 *
 * Solves   max c^T x   s.t.   A x <= b,  x >= 0
 * with the revised simplex method of Section 2.1 (Steps 1-8): slack columns
 * A = (A', I_m) form the starting basis, Dantzig pricing (Step 3/4), the ratio
 * test (Step 6), and the explicit-inverse tableau pivot (Step 8, Figure 1),
 * with the tabu anti-cycling rule of Sections 2.2 and 3.4.  When some b_i < 0
 * the slack basis is infeasible and a solve starts with Phase I (the
 * two-phase method of Section 3.4, one artificial variable).  Every step runs
 * in the library's own CUDA kernels (sm_103a); there is no CPU fallback.
 *
 * Conventions
 *  - m = number of constraints (rows of A), n = number of structural
 *    variables.  Variable j < n is x_j; variable n+i is the slack of row i.
 *  - A is dense, row-major, m x n, FP64 (the paper's d_A[i*n+j], Section 3.2).
 *  - Every pointer argument is a HOST pointer unless the argument says
 *    otherwise.  Host buffers are read or written synchronously; the caller
 *    keeps ownership of every buffer it passes.
 *  - Return codes: LP_OK (0) or a negative LP_ERR_*.  A solve that ends
 *    optimal, unbounded or at the iteration limit returns LP_OK and reports
 *    the outcome in lp_result.status (LP_INFEASIBLE too).
 *  - A handle owns all of its device memory.  One handle must not be used
 *    from two host threads at once; different handles are independent.
 */
#ifndef LPGB_H
#define LPGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define LP_OK 0
#define LP_ERR_INVALID_ARG (-1) /* bad size, NULL pointer, NaN/Inf, b_i < 0 */
#define LP_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define LP_ERR_OOM (-3)         /* device allocation failed */
#define LP_ERR_SINGULAR (-4)    /* reinversion met a zero pivot column */
#define LP_ERR_TIMEOUT (-5)     /* a bounded device wait gave up */
#define LP_ERR_STATE (-6)       /* call not valid in the handle's state */
#define LP_ERR_DEVICE (-7)      /* a kernel reported an internal error */

/* ---- solve outcome (lp_result.status) ----------------------------------- */
#define LP_RUNNING 0
#define LP_OPTIMAL 1            /* Step 4: every reduced cost <= tol_d */
#define LP_UNBOUNDED 2          /* Step 5: no alpha_i > tol_piv */
#define LP_ITER_LIMIT 3
#define LP_INFEASIBLE 4         /* Phase I (b with negative entries): no x >= 0 with Ax <= b */

/* ---- trace flags (lp_get_trace) ----------------------------------------- */
#define LP_TF_DEGENERATE 1      /* step length theta <= tol_tie */
#define LP_TF_TABU_PUSH 2       /* the leaving variable became tabu */
#define LP_TF_ASPIRATION 4      /* every improving candidate was tabu */
#define LP_TF_BLAND 8           /* Bland safety net active */
#define LP_TF_TIE_SET 64        /* the ratio test had more than one tied row */
#define LP_TF_GUIDED 128        /* the entering variable came from lp_set_priority */

/* lp_options.anticycling. */
#define LP_ANTICYCLING_TABU 0           /* CHUZC masks tabu variables, the tie set's largest alpha
                                           leaves, Bland safety net after bland_after degenerate
                                           pivots (the method) */
#define LP_ANTICYCLING_LEXICOGRAPHIC 1  /* no tabu list and no safety net; the tie set's row whose
                                           row of B^-1 / alpha_i is lexicographically smallest
                                           leaves (entries within tol_tie relative count as equal;
                                           then the smaller basic index); runs on the
                                           slack-structured and captured-graph engines */

/* lp_options.engine: how the pivots of price_mode 0 run. */
#define LP_ENGINE_DENSE 0       /* persistent cooperative kernel on the m x m B^-1, graph_iters
                                   pivots per launch: PRICE reads all of A, UPDATE all of B^-1 */
#define LP_ENGINE_GRAPH 1       /* captured CUDA graphs of three kernels per pivot */
#define LP_ENGINE_STRUCTURED 2  /* persistent kernel on the slack-structured B^-1: only the k
                                   rows whose slack is nonbasic carry nonzero y and non-unit
                                   B^-1 columns, so PRICE reads k rows of A and UPDATE/FTRAN
                                   k columns of B^-1 (exactly the same pivots up to the
                                   order of summation; extra device memory: 8 ld (n + m) bytes) */

/* lp_result.engine_reason: the first condition, checked in this order, that kept
   lp_create from running the engine lp_options.engine asked for. */
#define LP_ENGINE_REASON_NONE 0            /* the asked engine runs */
#define LP_ENGINE_REASON_PRICE_MODE 1      /* price_mode 1 runs on captured graphs; price_mode 2
                                              on the dense persistent engine */
#define LP_ENGINE_REASON_LEXICOGRAPHIC 2   /* LP_ENGINE_DENSE: the lexicographic rule runs on
                                              captured graphs there */
#define LP_ENGINE_REASON_NO_COOPERATIVE 3  /* the device refuses cooperative launches, or has
                                              more than 1024 SMs */
#define LP_ENGINE_REASON_SIZE 4            /* LP_ENGINE_STRUCTURED: more than 256 rows per SM,
                                              or its 28 ld bytes of shared memory exceed the
                                              device's per-block limit (m above about 5600 on
                                              152 SMs) */
#define LP_ENGINE_REASON_OCCUPANCY 5       /* the persistent kernel does not fit one CTA per SM */
#define LP_ENGINE_REASON_OUT_OF_CORE 6     /* tableau_budget_mb: B^-1 streams through the device in row
                                              blocks (Case 2), on the captured-graph engine's kernels */

typedef struct lp_handle lp_handle;

/*
 * Options.  lp_default_options() fills the method's settings:
 * reinvert_every 64, tabu_tenure 7, bland_after 50, max_iters 50,000,000,
 * price_mode 0, topk 16, trace_cap 0, graph_iters 64, kernel_timing 0,
 * engine LP_ENGINE_STRUCTURED (LP_ENGINE_DENSE where it does not fit),
 * anticycling LP_ANTICYCLING_TABU, reinvert_refine 1, reinvert_tc 1,
 * tol_d 1e-9, tol_piv 1e-9, tol_tie 1e-12, cuda_stream NULL.
 */
typedef struct lp_options {
    int32_t reinvert_every; /* rebuild B^-1 from the basis every k pivots (0: never) */
    int32_t tabu_tenure;    /* iterations a tabu variable may not enter (0: rule off) */
    int32_t max_iters;      /* iteration limit */
    int32_t bland_after;    /* consecutive degenerate pivots before Bland's rule (0: off) */
    int32_t price_mode;     /* 0: FP64 PRICE; 1: BF16 screen, the screened best columns
                               re-priced in FP64, full FP64 PRICE whenever none improves
                               (captured-graph engine); 2: FP64 PRICE over a compressed
                               sparse column copy of A, built on the device (dense
                               engines; extra device memory 12 m n bytes) */
    int32_t topk;           /* price_mode 1: columns re-priced per screening block (1 or 2;
                               larger values act as 2); batches: candidates per LP (1..8) */
    int32_t trace_cap;      /* record (q, r, theta, d_q, flags) of the first trace_cap pivots */
    int32_t graph_iters;    /* pivots per captured CUDA graph launch */
    int32_t kernel_timing;  /* s >= 1: time the PRICE and UPDATE launches of every s-th
                               pivot of each captured graph with CUDA events (1 = all);
                               timed pivots run without launch overlap */
    int32_t engine;         /* LP_ENGINE_*: how the pivots of price_mode 0 run (captured
                               CUDA graphs wherever the device refuses a cooperative launch) */
    int32_t anticycling;    /* LP_ANTICYCLING_*: the tabu rule of Sections 2.2/3.4 (default) or
                               the lexicographic rule it is compared with */
    int32_t reinvert_refine; /* 1 (default): a periodic reinversion refines the updated inverse
                               by one Newton-Schulz step, Y + Y (I - B11 Y), when
                               ||I - B11 Y||_inf <= refine_tol (else, and with 0, B11 is
                               eliminated afresh by Gauss-Jordan); needs 3 k^2 <= m^2 */
    int32_t reinvert_tc;    /* 1 (default): the reinversion's slack-row product -A[S, J] B11^-1
                               runs on the BF16 tensor cores from exact 7-bit slices of its
                               FP64 operands, combined in 64-bit fixed point (k <= 1024;
                               extra device memory about 16 m min(m, 1024) bytes); 0: FP64 FMAs */
    double tol_d;           /* optimality tolerance on the reduced costs */
    double tol_piv;         /* smallest admissible pivot alpha_r */
    double tol_tie;         /* relative width of the ratio-test tie set */
    double refine_tol;      /* reinvert_refine: largest ||I - B11 Y||_inf that is refined (default
                               and maximum 2^-26, so that one step leaves the residual below
                               2^-52; 0 refines only an exact inverse) */
    double tableau_budget_mb; /* device memory granted to the explicit inverse (the tableau of
                               Step 8), in MB (1e6 bytes); 0 (default): no limit.  When the
                               m x ld FP64 inverse exceeds it (Case 2 of Section 3), B^-1
                               lives in pinned host memory and streams through two device
                               buffers of budget/2 each in blocks of consecutive rows, every
                               pivot (the captured-graph engine's kernels; the block updated
                               last stays on the device for the next pivot, row r is fetched
                               once).  The reinversion's scratch is not counted.  Not with
                               LP_ANTICYCLING_LEXICOGRAPHIC. */
    void* cuda_stream;      /* cudaStream_t to run on; NULL: the handle's own stream */
} lp_options;

/* Outcome and counters of one lp_solve call. */
typedef struct lp_result {
    int32_t status;          /* LP_OPTIMAL, LP_UNBOUNDED, LP_ITER_LIMIT or LP_INFEASIBLE */
    int32_t iterations;      /* pivots performed (cumulative over the handle) */
    int32_t reinversions;    /* reinversions performed */
    int32_t degenerate;      /* pivots with theta <= tol_tie */
    int32_t tabu_pushes;     /* times the tabu rule fired */
    int32_t bland_fallbacks; /* times the Bland safety net switched on */
    int32_t aspirations;     /* iterations where every improving candidate was tabu */
    int32_t tc_reinversions; /* reinversions whose slack-row product ran on the tensor cores */
    double objective;        /* c^T x at the final basis */
    double seconds;          /* device time of the solve (CUDA events) */
    double reinvert_seconds; /* device time spent in reinversion */
    double bytes_moved;      /* algorithmic HBM bytes of PRICE and UPDATE/FTRAN */
    double price_seconds;    /* kernel_timing: summed device time of PRICE launches */
    double update_seconds;   /* kernel_timing: summed device time of UPDATE launches */
    double price_bytes;      /* algorithmic bytes of the timed PRICE launches */
    double update_bytes;     /* algorithmic bytes of the timed UPDATE launches */
    int32_t price_launches;  /* kernel_timing: PRICE launches timed */
    int32_t update_launches; /* kernel_timing: UPDATE launches timed */
    int64_t kernel_launches; /* all kernels this call launched (graph nodes included) */
    int32_t warm_repairs;    /* lp_set_basis_repair: repair pivots performed; lp_set_crash: crash
                                pivots performed */
    int32_t warm_fallback;   /* 1: the proposal was unusable, the solve started from the slack basis */
    int32_t screen_passes;   /* price_mode 1: BF16 screen + re-price passes (cumulative) */
    int32_t full_passes;     /* price_mode 1: full FP64 PRICE passes (cumulative) */
    double reinvert_gj_seconds;       /* part of reinvert_seconds: elimination of B11 */
    double reinvert_assemble_seconds; /* part: B^-1 rows, bbar, duals */
    double chain_seconds;    /* kernel_timing, persistent engine: device time of its launches */
    double chain_bytes;      /* algorithmic PRICE + UPDATE bytes of those launches */
    int32_t chain_launches;  /* persistent launches timed */
    int32_t persistent;      /* 1: the pivots ran in the dense persistent kernel, 2: in the
                                slack-structured one, 0: in captured graphs */
    int32_t phase1_iterations; /* b with negative entries: pivots of the Phase I problem */
    int32_t phase1_exchanged;  /* 1: the artificial ended basic at zero and was exchanged */
    int32_t refined_reinversions; /* reinversions done by refinement (reinvert_refine) */
    int32_t engine_reason;   /* LP_ENGINE_REASON_*: why `persistent` is not the engine that
                                lp_options.engine asked for (0: it is) */
    double refine_residual_max;   /* largest ||I - B11 Y||_inf of the updated inverse found by the
                                     refinement checks of this solve (drift of the updates) */
    int32_t ooc_blocks;      /* tableau_budget_mb: row blocks B^-1 streams in (0: resident) */
    int32_t ooc_block_rows;  /* rows per block */
    double ooc_bytes;        /* host <-> device bytes of the streamed blocks in this solve */
} lp_result;

/*
 * lp_selftest_barrier_timeout -- checks the bounded wait of the persistent
 * engine's grid barrier (no counterpart in the paper): a cooperative grid of
 * `blocks` CTAs (1..64) waits at a barrier that expects one CTA more than it
 * has.  Every CTA gives up after its spin limit (about 2 s), so the call
 * returns LP_ERR_TIMEOUT and the context stays usable; LP_OK would mean the
 * wait ended without the barrier completing, LP_ERR_CUDA a refused launch.
 * Synchronizes `cuda_stream` (NULL = default stream).
 */
int lp_selftest_barrier_timeout(int32_t blocks, void* cuda_stream);

/* Fills *opt with the defaults listed above. */
void lp_default_options(lp_options* opt);

/*
 * lp_create -- copies the problem to the GPU and prepares the slack basis
 * (Step 1 with B = I_m, Section 2.1; the whole tableau stays resident in
 * device memory, Case 1 of Section 3).
 *  out              receives the new handle (set to NULL on error)
 *  m, n             constraints and structural variables, both >= 1
 *  A_rowmajor       m x n FP64, row-major
 *  b, c             m and n FP64 values.  If some b_i < 0, every lp_solve
 *                   that starts from the slack basis first solves the Phase I
 *                   problem  max -x0  s.t.  A x - x0 e <= b,  x, x0 >= 0
 *                   (e_i = 1 where b_i < 0) on a second, internal handle with
 *                   the same options, from the slack basis with x0 in the row
 *                   of the most negative b_i.  An optimum below
 *                   -1e-9 max(1, max|b_i|) ends the solve with LP_INFEASIBLE;
 *                   otherwise its final basis (x0 exchanged for the nonbasic
 *                   slack s with the largest |B^-1[p][s]| if it is still basic
 *                   at zero in row p) is the Phase II start.
 *  inputs_on_device 0: A, b, c are host pointers; 1: device pointers, which
 *                   must stay valid until lp_create returns.  Device inputs
 *                   are read on the handle's stream (lp_options.cuda_stream,
 *                   else a non-blocking stream of the handle's own), which
 *                   does not wait for other streams: the caller finishes
 *                   (or orders before that stream) the work that writes them.
 *                   Host inputs are read before lp_create returns.  A host A
 *                   in pinned or registered memory is read in place by the
 *                   device and checked for NaN/Inf there, as device inputs
 *                   are; a pageable one is checked on the host (by several
 *                   threads when large) before any device work, then copied.
 *  opt              options, or NULL for the defaults
 * Errors: LP_ERR_INVALID_ARG (sizes, NULL, NaN/Inf), LP_ERR_OOM,
 * LP_ERR_CUDA.  The handle is on the current CUDA device.
 */
int lp_create(lp_handle** out, int32_t m, int32_t n, const double* A_rowmajor,
              const double* b, const double* c, int32_t inputs_on_device,
              const lp_options* opt);

/*
 * lp_set_basis -- warm start: the next lp_solve starts from this basis
 * instead of the slack basis.  basis_m holds m distinct variable indices in
 * [0, n+m) (host pointer).  B^-1 is rebuilt from the basis columns when the
 * solve starts; a basis that is not primal feasible (some bbar_i < 0) is
 * rejected at that point with LP_ERR_INVALID_ARG, a singular one with
 * LP_ERR_SINGULAR.
 */
int lp_set_basis(lp_handle* h, const int32_t* basis_m);

/*
 * lp_update_problem -- replaces A, b, c of a handle with a new problem of the
 * same m and n (same conventions as lp_create) and returns to the slack basis,
 * reusing every device buffer and the captured graph.  For families of LPs
 * (for example the perturbed instances a learned warm start is trained on).
 * Device inputs are read on the handle's stream, as for lp_create.
 */
int lp_update_problem(lp_handle* h, const double* A_rowmajor, const double* b, const double* c,
                      int32_t inputs_on_device);

/*
 * lp_set_priority -- guided entering rule for warm starts (price_mode 0 only;
 * LP_ERR_STATE otherwise).  vars (host) lists `count` distinct variables (a
 * predicted set).  While any listed variable is nonbasic, not tabu and
 * improving (d_j > tol_d), CHUZC enters the listed one with the largest d_j
 * (Dantzig's rule restricted to the list); otherwise the normal rule applies,
 * so the solve first works on the predicted columns.  Every pivot is still
 * an ordinary ratio-test pivot, so primal feasibility is never lost and the
 * optimum is certified by the usual test.  count = 0 clears the list; the
 * list survives lp_reset and lp_update_problem.
 */
int lp_set_priority(lp_handle* h, const int32_t* vars, int32_t count);

/*
 * lp_set_basis_repair -- warm start from a proposed basis that may be primal
 * infeasible (the paper has no warm start; this is the repair of the learned
 * warm start).  When the next lp_solve starts, B^-1 is rebuilt from the
 * proposal (basis_m: m distinct variables, host pointer).  While some basic
 * value is negative, the most negative position p leaves and the nonbasic
 * slack with the most negative B^-1[p][s] enters -- an ordinary tableau pivot
 * that makes position p positive and keeps B nonsingular -- for at most
 * max_repairs pivots (counted as iterations).  A singular proposal, or one
 * still infeasible after max_repairs, is dropped and the solve starts from the
 * slack basis (lp_result.warm_fallback = 1).  The primal simplex then runs to
 * the optimum as usual.
 */
int lp_set_basis_repair(lp_handle* h, const int32_t* basis_m, int32_t max_repairs);

/*
 * lp_set_crash -- warm start by a crash from the slack basis (the paper has no
 * warm start; the learned warm start's use of a predicted set).  When the next
 * lp_solve starts, the `count` structurals in vars (host; distinct, in [0, n),
 * count <= m) enter one by one in the order given, each by an ordinary pivot:
 * FTRAN of its column and the ratio test of Step 6 with the method's tie rule,
 * so the basis stays primal feasible.  A variable is passed over when it is
 * basic already, when its column has no alpha_i > tol_piv, or when the ratio
 * test would make a structural leave (the crash replaces slacks only).  The
 * plain method then runs to the optimum; lp_result.warm_repairs counts the
 * crash pivots (they are iterations).  One solve consumes the list; lp_set_basis,
 * lp_set_basis_repair and lp_reset clear it, and it clears a pending
 * lp_set_basis.  LP_ERR_STATE when b has a negative entry (Phase I) or B^-1 is
 * out of core (tableau_budget_mb).
 */
int lp_set_crash(lp_handle* h, const int32_t* vars, int32_t count);

/* lp_reset -- return to the slack basis and clear all counters. */
int lp_reset(lp_handle* h);

/*
 * lp_solve -- runs simplex iterations (Steps 3-8) until optimal, unbounded or
 * the iteration limit, on the handle's stream; returns when the device is done.
 * After it returns, lp_get_* read the final state.  Errors: LP_ERR_CUDA,
 * LP_ERR_SINGULAR, LP_ERR_DEVICE, LP_ERR_INVALID_ARG (infeasible warm basis).
 */
int lp_solve(lp_handle* h, lp_result* out);

/*
 * lp_get_solution -- x (n values), duals y = c_B^T B^-1 (m values; y_i >= 0 at
 * an optimum), objective.  Any output pointer may be NULL.  LP_ERR_STATE
 * before the first lp_solve and after a solve that ended LP_INFEASIBLE.
 */
int lp_get_solution(const lp_handle* h, double* x_n, double* y_m, double* objective);

/* lp_get_basis -- the m basic variable indices, in basis-position order. */
int lp_get_basis(const lp_handle* h, int32_t* basis_m);

/*
 * lp_get_state -- inspection of the explicit inverse (Figure 1 tableau):
 * binv (m*m, row-major, row p belongs to basis position p) and bbar (m).
 * Either pointer may be NULL.
 */
int lp_get_state(const lp_handle* h, double* binv, double* bbar);

/*
 * lp_get_trace -- the recorded pivots (needs trace_cap > 0): entering
 * variable q, leaving basis position r, step length theta, reduced cost d_q
 * and LP_TF_* flags of pivot t in element t.  Copies min(cap, recorded)
 * entries and stores that number in *count.  Any array may be NULL.
 */
int lp_get_trace(const lp_handle* h, int32_t* q, int32_t* r, double* theta,
                 double* dq, int32_t* flags, int32_t cap, int32_t* count);

/*
 * lp_price_static -- reduced costs and Dantzig's entering choice for callers
 * that cannot allocate memory.  The paper has no counterpart: this entry point
 * exists for callers such as code that runs inside a CUDA graph it is
 * capturing itself, or a runtime whose device memory is fixed up front, where
 * a cudaMalloc (even one hidden inside a library) is not allowed.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Computes d_j = c_j - y^T a_j for every nonbasic structural j and
 * d_{n+i} = -y_i for every nonbasic slack i, and writes the largest d_j > tol_d
 * (exact ties to the smallest j) to *q_out with its value in *dq_out;
 * *q_out = -1 when no d_j exceeds tol_d (the basis is optimal).  The tabu
 * rule is not applied.
 *
 * All pointers are DEVICE pointers owned by the caller:
 *  A_colmajor  n columns of lda doubles (column j at A_colmajor + j*lda),
 *              16-byte aligned; only the first m entries of a column are read
 *  lda         >= m and even
 *  c (n), y (m), pos (n+m: pos[j] >= 0 marks a basic variable)
 *  q_out (1 int32), dq_out (1 double)
 *  cuda_stream cudaStream_t (NULL: the legacy default stream); the call only
 *              enqueues work and returns
 * Limits: 1 <= m <= LP_PRICE_STATIC_MAX_M (y is staged in shared memory),
 * n >= 1; larger sizes return LP_ERR_INVALID_ARG without touching the GPU.
 *
 * Scratch: 17 KB of partial results live in a file-scope device array that
 * every GPU loading this library holds until the process exits.  All calls
 * share it and it keeps the last call's contents (the counter that must start
 * at zero is cleared by every call), so calls whose kernels overlap on the GPU
 * race with each other: serialise them, e.g. on one stream.  The first call
 * on a device looks up the array's device address and sets the kernel's
 * shared-memory limit; make that first call before any stream capture.  The
 * address is kept per device context: the first call after the device's
 * context was replaced (cudaDeviceReset) repeats that set-up.
 */
#define LP_PRICE_STATIC_MAX_M 12288
int lp_price_static(int32_t m, int32_t n, const double* A_colmajor, int32_t lda,
                    const double* c, const double* y, const int32_t* pos, double tol_d,
                    int32_t* q_out, double* dq_out, void* cuda_stream);

/*
 * lp_tc_gemm -- D = A B^T on the tensor cores (tcgen05.mma, FP32 accumulation
 * in tensor memory; operand tiles staged by TMA).  The building block of the
 * reinversion's FP64 products, which are formed from exact 7-bit slices of
 * their operands (no counterpart in the paper, whose reinversion-free method
 * needs no such product), and of the warm-start network.  Exposed so that the
 * primitive can be checked on its own.
 *
 * All pointers are DEVICE pointers owned by the caller:
 *  A  M x K, row-major with row stride lda elements (lda >= K, lda % 8 == 0)
 *  B  N x K, row-major with row stride ldb elements (ldb >= K, ldb % 8 == 0)
 *     (16-bit elements: bf16 != 0 selects BF16, else FP16; 16-byte aligned)
 *  D  M x N FP32, row stride ldd >= N
 * Runs on cuda_stream (NULL: legacy default stream) and waits for it.
 * Returns LP_OK, LP_ERR_INVALID_ARG (shape, stride or alignment), LP_ERR_CUDA,
 * or LP_ERR_TIMEOUT (a bounded wait inside the kernel gave up).
 */
int lp_tc_gemm(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B, int32_t ldb,
               float* D, int32_t ldd, int32_t bf16, void* cuda_stream);

/* ---- batches of small LPs ------------------------------------------------ */

/*
 * A batch holds many independent small LPs that are solved in persistent
 * launches: one CTA solves one LP at a time (Steps 1-8 of Section 2.1 with the
 * tabu rule of Sections 2.2/3.4 and reinversion every reinvert_every pivots),
 * taking LPs from an atomic work queue per size bucket (m <= 64, 128, 192,
 * 256).  For batches price_mode defaults to 1: a BF16 screen of the columns,
 * the top `topk` (at most 8 here) re-priced in FP64, and the full FP64 PRICE
 * whenever no candidate improves, so optimality is always certified in FP64.
 */
typedef struct lp_batch lp_batch;

#define LP_BATCH_MAX_M 256
#define LP_BATCH_MAX_N 512

typedef struct lp_batch_result {
    int32_t solved;          /* LPs that ended optimal */
    int32_t unbounded;
    int32_t iter_limit;
    int32_t failed;          /* LPs whose reinversion met a singular basis */
    int64_t iterations;      /* pivots summed over the batch */
    double seconds;          /* device time of the solve (CUDA events) */
    double fp64_flops;       /* algorithmic FP64 flops: FTRAN + update + re-pricing */
} lp_batch_result;

/*
 * lp_batch_create -- copies `count` LPs to the GPU.  m[k], n[k] (host arrays)
 * give the sizes (1 <= m <= LP_BATCH_MAX_M, 1 <= n <= LP_BATCH_MAX_N).  A holds
 * every A_k row-major, one after another; b every b_k (all >= 0) and c every
 * c_k, likewise concatenated.  inputs_on_device selects host (0) or device (1)
 * pointers for A, b, c.  opt: NULL for the defaults (price_mode 1, topk 8);
 * trace_cap > 0 records each LP's first trace_cap pivots.
 */
int lp_batch_create(lp_batch** out, int32_t count, const int32_t* m, const int32_t* n,
                    const double* A, const double* b, const double* c,
                    int32_t inputs_on_device, const lp_options* opt);

/* lp_batch_solve -- solves every LP of the batch from its slack basis. */
int lp_batch_solve(lp_batch* h, lp_batch_result* out);

/*
 * lp_batch_get -- per-LP results into host arrays (any may be NULL): status
 * and iterations (count each), objective (count), x (sum of n_k, concatenated)
 * and duals y (sum of m_k, concatenated).  LP_ERR_STATE before a solve.
 */
int lp_batch_get(const lp_batch* h, int32_t* status, int32_t* iterations, double* objective,
                 double* x, double* y);

/* lp_batch_get_trace -- entering variable q and leaving position r of LP k's
   first min(cap, recorded) pivots (needs trace_cap > 0). */
int lp_batch_get_trace(const lp_batch* h, int32_t k, int32_t* q, int32_t* r, int32_t cap,
                       int32_t* count);

/*
 * Autotuner.  table[2*b] = threads per CTA (128, 256 or 512) and
 * table[2*b+1] = 1 to keep B^-1 in shared memory (only where it fits) or 0
 * for an L2-resident global slot, for size buckets b = 0..3.
 * lp_batch_tune times every valid configuration of every non-empty bucket on
 * the batch itself (`trials` solves each), keeps the fastest, and writes the
 * table if it is not NULL; lp_batch_set_tuning installs a saved table.
 */
int lp_batch_tune(lp_batch* h, int32_t* table, int32_t trials);
int lp_batch_set_tuning(lp_batch* h, const int32_t* table);

/* lp_batch_destroy -- frees the batch (NULL is ignored). */
void lp_batch_destroy(lp_batch* h);

/* ---- learned warm start: the network ------------------------------------ */

/*
 * A 3-layer perceptron in -> hidden -> hidden -> out with ReLU, trained with
 * binary cross-entropy on logits, L = (1/B) sum_b sum_o [softplus(z) - t z],
 * and Adam (beta 0.9 / 0.999, eps 1e-8).  The GEMMs run on the tensor cores
 * with FP16 operands and FP32 accumulation; FP32 master weights and Adam
 * moments are kept on the device.  Parameters are packed W1 (in x hidden,
 * row-major), b1, W2 (hidden x hidden), b2, W3 (hidden x out), b3.  X and T
 * are DEVICE pointers to FP32 row-major [batch x in] and [batch x out];
 * params and grads are HOST pointers; the handle runs on cuda_stream.  The
 * paper has no learned component: this is the warm start of this design.
 */
typedef struct lp_mlp lp_mlp;
int lp_mlp_create(lp_mlp** out, int32_t in_dim, int32_t hidden, int32_t out_dim,
                  int32_t max_batch, void* cuda_stream);
int64_t lp_mlp_num_params(const lp_mlp* h);
int lp_mlp_set_params(lp_mlp* h, const float* params);        /* also resets Adam */
int lp_mlp_get_params(const lp_mlp* h, float* params);
/* logits: DEVICE pointer [batch x out]; enqueued on the handle's stream */
int lp_mlp_forward(lp_mlp* h, const float* X, int32_t batch, float* logits);
/* loss and the gradient of every parameter (host), without an update */
int lp_mlp_gradients(lp_mlp* h, const float* X, const float* T, int32_t batch,
                     float* grads, float* loss);
/* one Adam step with learning rate lr; *loss (host, may be NULL) is the batch loss */
int lp_mlp_train_step(lp_mlp* h, const float* X, const float* T, int32_t batch, float lr,
                      float* loss);
void lp_mlp_destroy(lp_mlp* h);

/* ---- learned warm start: LP families ------------------------------------- */

/*
 * lp_family_perturb -- one instance of the family of a base LP (A0, b0, c0):
 * every entry of A, b and c is the base entry times an independent N(1, sigma^2)
 * draw (Box-Muller on SplitMix64 in counter mode under `key`, pairs of draws in
 * the order A row-major, then b, then c).  All pointers are DEVICE pointers
 * (A0, A: m x n row-major); nothing is allocated; enqueued on cuda_stream.
 */
int lp_family_perturb(int32_t m, int32_t n, const double* A0, const double* b0, const double* c0,
                      uint64_t key, double sigma, double* A, double* b, double* c, void* cuda_stream);

/*
 * lp_family_features -- the 2(m+n) network inputs of an instance (DEVICE
 * float32 out): (b/b0 - 1)/sigma (m), (c/c0 - 1)/sigma (n), then the row (m)
 * and column (n) means of A/A0 over the nonzero entries of A0, minus 1, times
 * sqrt(count)/sigma.  Device pointers; nothing is allocated.
 */
int lp_family_features(int32_t m, int32_t n, const double* A0, const double* b0, const double* c0,
                       const double* A, const double* b, const double* c, double sigma,
                       float* features, void* cuda_stream);

/*
 * lp_family_propose -- the network's proposed basis from its n+m scores
 * (DEVICE float32 `scores`, higher = more likely basic; structurals first,
 * then slacks).  The structurals with score > threshold, in the order (score
 * descending, index ascending), at most m of them, are J_0 .. J_{k-1}; the k
 * slack rows of lowest score (ties: lower row) give up their positions, the
 * t-th of them to J_t; every other row keeps its slack.  Outputs (DEVICE
 * int32): basis (m entries, a valid proposal for lp_set_basis_repair) and
 * work (m + 1 entries: J in its first min(k, m) entries, the number of
 * structurals with score > threshold, before the cap at m, in work[m]).  Nothing is
 * allocated; enqueued on cuda_stream.  Errors: LP_ERR_INVALID_ARG (sizes,
 * NULL), LP_ERR_CUDA.
 */
int lp_family_propose(int32_t m, int32_t n, const float* scores, float threshold, int32_t* basis,
                      int32_t* work, void* cuda_stream);

/* lp_destroy -- frees the handle and its device memory (NULL is ignored). */
void lp_destroy(lp_handle* h);

/* lp_strerror -- a static description of a return code. */
const char* lp_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LPGB_H */
