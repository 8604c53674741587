// lpgb_internal.cuh -- device data layout and kernel declarations of the
// dense revised simplex solver (Section 2.1, Steps 1-8; tabu rule of Sections
// 2.2 and 3.4; tableau of Figure 1 held resident in device memory, Case 1 of
// Section 3).
//
// Device layout (HBM):
//   A_cm   n columns of ld doubles (column-major, ld = m rounded up to 64,
//          padding rows zero): PRICE streams whole columns, FTRAN stages one.
//   binv   m rows of ld doubles (row-major explicit B^-1, padding zero).
//   bbar, theta: m doubles.   y, rho: ld doubles (padding zero).
//   alpha  two buffers of ld doubles (current / next pivot column).
//   basis  m int32 (basis position -> variable); pos n+m int32 (variable ->
//          position or -1); tabu_until n+m int32.
//   ctrl   one Ctrl block: every decision of the iteration lives on the
//          device, so a captured graph of many iterations needs no host
//          round trip.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace lpgb {

constexpr int kLdAlign = 64;          // doubles; one warp-wide double2 sweep
constexpr int kWarp = 32;

// internal status values (beyond the public LP_* outcomes)
constexpr int kRunning = 0;
constexpr int kOptimal = 1;
constexpr int kUnbounded = 2;
constexpr int kIterLimit = 3;
constexpr int kReinvert = 10;          // host must rebuild B^-1 before continuing
constexpr int kRebuildStopped = 11;    // a rebuild to be redone by elimination (or one that failed):
                                       // a launch queued behind it does nothing

// device error codes (Ctrl::err)
constexpr int kErrNone = 0;
constexpr int kErrSingular = 1;
constexpr int kErrBadIndex = 2;
constexpr int kErrInfeasibleStart = 3;
constexpr int kErrTimeout = 4;         // a bounded device wait ran out

// trace flags (same values as LP_TF_*)
constexpr int kTfDegenerate = 1;
constexpr int kTfTabuPush = 2;
constexpr int kTfAspiration = 4;
constexpr int kTfBland = 8;
constexpr int kTfTieSet = 64;

struct Params {
    int32_t m, n, ld;
    int32_t reinvert_every, tabu_tenure, max_iters, bland_after, trace_cap;
    double tol_d, tol_piv, tol_tie;
    double b_scale;        // max(1, max_i b_i): scale of the feasibility check
    int32_t price_mode;    // 0: FP64 PRICE; 1: BF16 screen + FP64 re-price of the top k
    int32_t topk;          // candidates re-priced in FP64 (price_mode 1), <= kMaxTopk
    int32_t lex;           // 1: lexicographic leaving rule (no tabu list, no safety net)
    int32_t prio;          // 1: a priority list is set (lp_set_priority; guided entering rule)
    double nnz;            // price_mode 2: nonzeros of A
    int32_t screen;        // slack-structured engine: PRICE through the exact FP32 screen
    int32_t reinvert_tc;   // slack-row product of the reinversion on the tensor cores
};

constexpr int kMaxTopk = 32;

struct Ctrl {
    int32_t status;        // kRunning / kOptimal / kUnbounded / kIterLimit / kReinvert
    int32_t it;            // pivots done
    int32_t q;             // entering variable of the pending pivot
    int32_t r;             // leaving basis position of the pending pivot
    int32_t tcount;        // size of the ratio-test tie set
    int32_t abuf;          // which alpha buffer is current
    int32_t pending;       // 1: the B^-1 update of the last pivot is still to be applied
    int32_t flags;         // trace flags gathered during the iteration
    int32_t degen_run;     // consecutive degenerate pivots
    int32_t bland;         // Bland safety net active
    int32_t n_degenerate, n_tabu, n_bland, n_asp;
    int32_t n_reinv;
    int32_t err;           // kErr*
    int32_t ticket_price;  // last-block tickets (reset by the last block)
    int32_t ticket_update;
    int32_t k_struct;      // reinversion: number of structural basic columns
    int32_t ticket_pivot;
    int32_t nsb;           // structural variables in the basis
    int32_t k_live;        // slack-structured engine: rows whose slack is nonbasic (live slots)
    int32_t repair;        // warm-start repair: 1 running, 2 feasible, 3 cannot repair, 4 limit reached
    int32_t need_full;     // price_mode 1: the screen found no improving candidate
    int32_t n_full;        // price_mode 1: full FP64 PRICE passes
    int32_t n_lp;          // price_mode 1: screen + re-price passes
    int32_t ticket_lp;     // last-block tickets of the screen and re-price kernels
    int32_t ticket_rp;
    int32_t n_price;       // PRICE launches that did work
    int32_t n_update;      // UPDATE launches that did work
    int32_t map_par;       // slack-structured engine: which slot map is current
    int32_t screen_off;    // slack-structured engine: A outside the FP32 screen's range
    double bytes_price;    // algorithmic HBM bytes moved by PRICE
    double bytes_update;   // algorithmic HBM bytes moved by UPDATE/FTRAN
    double dq;             // d_q of the pending pivot
    double theta;          // step length bbar_r / alpha_r
    double alpha_r;        // pivot element
    double z;              // objective c_B^T bbar
    double refine_res;     // reinversion by refinement: ||I - B11 Y0||_inf of the stored inverse
    double repair_tol;     // warm-start repair: basic values below -repair_tol are repaired
    int32_t repair_limit;  // warm-start repair: no repair pivot once it reaches this count
    int32_t crash;         // warm-start crash: 1 running, 2 done
    int32_t crash_t;       // next position in the crash list
    int32_t crash_n;       // entries of the crash list
    int32_t refine_rej;    // reinversion by refinement: the residual was above the tolerance (the
                           // rebuild is discarded and redone by elimination)
    int32_t ticket_reinv;  // last-block ticket of k_reinv_finish (reset by the last block)
};

// Per-CTA ratio-test record of k_iterate: the CTA's smallest ratio, and its
// best row and tie count under the tie threshold of that ratio.
struct RowPart {
    double tmin, a, th;
    int32_t var, row, cnt, pad_;
};

// The same two records packed for 16-byte loads (k_iterate_s, where every CTA
// reads every CTA's record after a grid barrier).
// Values to be ordered are stored as order-preserving 64-bit integer images.
struct alignas(16) PriceRec {
    long long d_all, d_nt;
    int32_t j_all, j_nt, j_min, j_pr;
    long long d_min, d_pr;
    int32_t k_pr, pad_[3];
};
struct alignas(16) RowRec {
    long long tmin, thr;   // smallest ratio and its tie threshold
    double a, th;          // best row: pivot element and ratio
    int32_t var, row, cnt, pad_;
};

// Candidate triple of CHUZC (per block partial).
struct PriceCand {
    double d_all; int32_t j_all;   // best nonbasic (optimality test, aspiration)
    int32_t j_min;                 // smallest improving index (Bland)
    double d_nt;  int32_t j_nt;    // best nonbasic non-tabu
    int32_t k_pr;                  // priority rank of j_pr (guided entering rule)
    double d_min;                  // d of j_min
    double d_pr;  int32_t j_pr;    // improving non-tabu column with the best priority
    int32_t pad_;
};

constexpr int32_t kNoRank = 0x7fffffff;
constexpr int kTfGuided = 128;

// BF16 screen partial of one block: its best two columns by approximate d,
// and its best exact slack.
struct LpCand {
    float d0; int32_t j0;
    float d1; int32_t j1;
    double ds; int32_t js; int32_t pad_;
};

struct TraceBuf {
    int32_t* q; int32_t* r; double* theta; double* dq; int32_t* flags;
};

struct DevState {
    Params p;
    const double* A_cm;
    const uint16_t* A_lp;    // price_mode 1: BF16 copy of A_cm (same layout)
    float* y32;              // FP32 copy of y (ld), for the BF16 screen
    LpCand* lp_part;         // per-block screen partials
    const int64_t* csc_ptr;  // price_mode 2: n+1 column starts of the sparse copy of A
    const int32_t* csc_row;  // its row indices (increasing within a column)
    const double* csc_val;   // its values
    int32_t* cand;           // kMaxTopk candidate columns (-1 = none)
    double* cand_d;          // their exact reduced costs
    const double* c;
    const double* b;
    double* binv;            // out of core (Case 2): pinned host memory, read and written by
                             // kernels over the host link only outside the per-pivot blocks
    const double* prow;      // out of core: row r of the updated B^-1 for k_pivot (else null)
    double* bbar;
    double* y;
    double* rho;
    double* alpha;      // 2 * ld
    double* theta;      // m
    int32_t* basis;
    int32_t* pos;
    int32_t* tabu_until;
    int32_t* rank;           // n+m: entering priority (kNoRank = none), lp_set_priority
    Ctrl* ctrl;
    PriceCand* price_part;
    double* upd_part;   // per-block theta minima
    RowPart* row_part;  // k_iterate: per-CTA ratio-test record
    int32_t* row_var;   // m: basic variable of each row as seen by the last FTRAN (k_iterate)
    int32_t* lex_rows;  // m: rows of the ratio-test tie set (lexicographic rule)
    int32_t* crash_list;  // m: the structurals a warm-start crash enters, in order (lp_set_crash)
    uint32_t* gbar;     // k_iterate grid barrier: arrivals, released epoch
    // slack-structured engine (k_iterate_s): the constraint rows in slot order,
    // the rows whose slack is nonbasic in slots [0, k_live)
    double* A_p;        // n columns of ld doubles: A with its rows in slot order
    float* A_p32;       // its FP32 copy (the PRICE screen)
    float* c32lo;       // c rounded down and up to FP32 (the PRICE screen)
    float* c32hi;
    double* bp;         // m rows of ld doubles: B^-1 columns of the live slots
    double* yp;         // 2*ld: y in slot order (zero outside the live slots), two copies by map_par
    int32_t* slot_row;  // 2*m: slot -> row, two copies (current, next) by map_par
    int32_t* row_slot;  // 2*m: row -> slot, same two copies
    int32_t* uslot;     // m: basis position -> slot of its basic slack, or -1
    PriceRec* price_rec;  // per-CTA CHUZC partials of k_iterate_s
    RowRec* row_rec;      // per-CTA ratio-test records of k_iterate_s
    TraceBuf trace;
    // reinversion scratch
    int32_t* rv_struct_pos;  // k structural basis positions (increasing)
    int32_t* rv_rows;        // k rows whose slack is nonbasic (increasing)
    int32_t* rv_row_index;   // m: row -> index in rv_rows, or -1
    int32_t* rv_slack_pos;   // m-k rows whose slack is basic (increasing row)
    int32_t* rv_b_of_pos;    // m: basis position -> structural index b, or -1
    int32_t* rv_g_of_row;    // m: row -> index in rv_slack_pos, or -1
    int32_t* rv_J;           // k: structural variable of index b
    double* rv_cJ;           // k: its cost
    double* rv_W;            // m*m: dense B11^-1 (k x k) then -A[S,J] B11^-1 ((m-k) x k)
    int32_t* rv_pivrow;      // k: pivot row chosen for column t (GJ)
    int32_t* rv_rowdone;     // k: row already used as pivot
    __nv_bfloat16* oz_xs;    // reinvert_tc: 7-bit slices of A[S, J] (8 rows per slack row), or null
    __nv_bfloat16* oz_ys;    // reinvert_tc: slices of B11^-1 (8 rows per column)
    int32_t* oz_ex;          // reinvert_tc: row exponents of A[S, J] (m)
    int32_t* oz_ey;          // reinvert_tc: column exponents of B11^-1 (m)
    double* rv_M;            // k*k column-major workspace (B11 then its GJ form)
    double* rv_f;            // 2*k published pivot columns
};

// Order-preserving integer image of a double: on GB300 every FP64 instruction
// (compares and min/max included) holds the slow FP64 pipe as long as an FMA,
// while integer compares do not.  dkey(a) > dkey(b) exactly when a > b, and
// -0 and +0 share one key (no NaN is ever compared).
__device__ __forceinline__ long long dkey(double d) {
    long long b = __double_as_longlong(d);
    if ((b & 0x7fffffffffffffffLL) == 0) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double kdouble(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

// ---- launch geometry -----------------------------------------------------
// Programmatic dependent launch: wait for the previous kernel of the stream
// (its completion and memory), then let the next kernel's CTAs be scheduled.
// Both are no-ops for a kernel launched without the programmatic attribute.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch `kernel` on `st`, with programmatic stream serialization when pdl.
template <typename... Args>
inline cudaError_t launch_k(void (*kernel)(Args...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

struct Geometry {
    int sms;
    int price_blocks, price_threads;
    int price_lp_blocks;  // BF16 screening kernel (price_mode 1)
    int update_blocks, update_threads;
    int pivot_blocks, pivot_threads;
    int pdl;  // graph kernels use programmatic dependent launch
};

// ---- kernels (kernels_iter.cu) ----------------------------------------------
void launch_init_slack(const DevState& s, cudaStream_t st);
// pdl: launch with programmatic stream serialization (the kernel may start
// while the previous kernel of the stream finishes; it waits for that kernel's
// completion and memory in griddepcontrol.wait before touching any state).
void launch_pivot(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl = false);
void launch_price(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl = false);  // the whole PRICE + CHUZC of the mode
void launch_to_bf16(const double* src, uint16_t* dst, size_t count, cudaStream_t st);
void launch_update(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl = false);
// Up to `iters` pivots in one cooperative launch of `blocks` CTAs (price_mode 0).
cudaError_t launch_iterate(const DevState& s, int blocks, int iters, cudaStream_t st);
int occupancy_iterate(int ld);
// The same on the slack-structured form of B^-1 (kernels_struct.cu).
cudaError_t launch_iterate_s(const DevState& s, int blocks, int iters, cudaStream_t st);
int occupancy_iterate_s(int ld);
bool struct_engine_fits(int m, int ld, int ctas);  // shared-memory and per-CTA row limits
// Dense state -> structured state: slot map check (rebuilt when force or
// inconsistent, then A_p regathered), live B^-1 columns and y, start at PRICE.
void launch_struct_enter(const DevState& s, int force, int32_t* relayout, cudaStream_t st, bool compact);
void launch_struct_scatter_y(const DevState& s, cudaStream_t st);  // yp -> y (row order)
void launch_struct_init_maps(const DevState& s, cudaStream_t st);
// Bounded-wait self-test: a grid barrier that cannot complete (lp_selftest_barrier_timeout).
int barrier_selftest(int blocks, cudaStream_t st);
size_t price_smem_bytes(int ld);
size_t update_smem_bytes(int ld);
void configure_iter_kernels(int ld);

// ---- sparse copy of A (kernels_sparse.cu) ----------------------------------------
// cnt: n int32 scratch; ptr: n+1 column starts (ptr[n] = nonzeros).
void launch_csc_count(const double* A_cm, int m, int n, int ld, int32_t* cnt, int64_t* ptr, cudaStream_t st);
void launch_csc_fill(const double* A_cm, int m, int n, int ld, const int64_t* ptr, int32_t* row, double* val,
                     cudaStream_t st);

// ---- reinversion (kernels_reinv.cu) -------------------------------------------
// k_expect >= 0: the structural count the host expects (err = kErrBadIndex otherwise)
void launch_reinv_classify(const DevState& s, int k_expect, cudaStream_t st);
void launch_reinv_gj(const DevState& s, int k, const Geometry& g, cudaStream_t st);
int reinv_gj_launches(int k);
int launch_reinv_assemble(const DevState& s, int k, const Geometry& g, cudaStream_t st, int from_gj, bool dense_rows);
bool refine_fits(int k, int m);
// Case 2 out-of-core blocks of B^-1 (ooc.cu)
void launch_ooc_update(const DevState& s, const Geometry& g, double* win, int i0, int i1, cudaStream_t st);
void launch_ooc_chuzr(const DevState& s, cudaStream_t st);
void launch_ooc_fetch_row(const DevState& s, const double* host_binv, const double* win, int w0, int w1,
                          double* prow, cudaStream_t st);
int configure_ooc_kernels(int ld);
// sliced FP64 products on the tensor cores (ozaki.cu)
bool oz_fits(int k);
size_t oz_scratch_x_elems(int m);
size_t oz_scratch_y_elems(int m);
cudaError_t oz_slack_product(const double* A_cm, int ld, const int32_t* J, const int32_t* S, const double* W,
                             int k, int nslack, double* C, __nv_bfloat16* xs, __nv_bfloat16* ys, int32_t* ex,
                             int32_t* ey, int32_t* err, cudaStream_t st);
cudaError_t oz_refine_residual_product(const double* B11_cm, const double* Y0, int k, double* P,
                                       __nv_bfloat16* xs, __nv_bfloat16* ys, int32_t* ex, int32_t* ey,
                                       int32_t* err, cudaStream_t st);
cudaError_t oz_refine_update_product(const double* Y0, const double* R, int k, double* P, __nv_bfloat16* xs,
                                     __nv_bfloat16* ys, int32_t* ex, int32_t* ey, int32_t* err, cudaStream_t st);
int launch_refine_residual(const DevState& s, int k, int from_struct, int k_live, int par, cudaStream_t st);
int launch_refine_apply(const DevState& s, int k, cudaStream_t st);
// refine_tol >= 0: the rebuild came from a refinement, accepted when its residual is <= refine_tol
void launch_reinv_finish(const DevState& s, int k, const Geometry& g, cudaStream_t st, int check_feasible,
                         double refine_tol);
int occupancy_price(int ld);
int occupancy_price_lp(int ld);
int occupancy_update(int ld);

// ---- setup (kernels_setup.cu) ---------------------------------------------------
void launch_transpose_pad(const double* A_rm, int m, int n, int ld, double* A_cm, cudaStream_t st);
void launch_build_aux(const double* A_cm, int ld, int m, int n, const double* b, double* A_aux, double* c_aux,
                      cudaStream_t st);
void launch_validate(const double* A_cm, const double* b, const double* c, int m, int n, int ld,
                     int32_t* flag, cudaStream_t st);
void launch_load_basis(const DevState& s, cudaStream_t st);
void launch_crash_begin(const DevState& s, int count, cudaStream_t st);
void launch_crash_steps(const DevState& s, const Geometry& g, int steps, cudaStream_t st);
void launch_repair_begin(const DevState& s, double tol, int limit_it, cudaStream_t st);
void launch_repair_steps(const DevState& s, const Geometry& g, int steps, cudaStream_t st);

// t 2^s as the nearest binary64 (ties to even), t != 0, built from the
// IEEE-754 binary64 format with integer instructions only (on this chip every
// FP64 instruction holds a scheduler's FP64 pipe for ~64 cycles); results
// below 2^-1022 flush to zero, above the range become infinite.
__device__ __forceinline__ double ll_scaled(long long t, int s) {
    const unsigned long long sign = t < 0 ? (1ull << 63) : 0ull;
    const unsigned long long u = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
    const int msb = 63 - __clzll((long long)u);
    int e = msb + s;  // weight of the leading bit
    unsigned long long mant;
    if (msb > 52) {
        const int sh = msb - 52;
        const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        mant = u >> sh;
        if (rem > half || (rem == half && (mant & 1ull))) {
            ++mant;
            if (mant == (1ull << 53)) { mant >>= 1; ++e; }
        }
    } else {
        mant = u << (52 - msb);
    }
    const int be = e + 1023;
    if (be >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    if (be <= 0) return __longlong_as_double((long long)sign);
    return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace lpgb
