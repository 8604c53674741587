// solver.cu -- host driver and C ABI (include/lpgb.h).
//
// A handle keeps the whole tableau resident in device memory (Case 1 of
// Section 3; the out-of-core Case 2 is not needed within GB300 memory).  The
// iteration loop runs as a captured CUDA graph of `graph_iters` iterations
// (each = pivot bookkeeping, PRICE+CHUZC, UPDATE+FTRAN+CHUZR); the host only
// reads the 160-byte control block after each graph launch, and rebuilds B^-1
// when the device asks for it.
#include "lpgb_internal.cuh"
#include "../../include/lpgb.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

using namespace lpgb;

struct lp_handle {
    int device = 0;
    int m = 0, n = 0, ld = 0;
    lp_options opt{};
    Params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevState ds{};
    Geometry geo{};
    Ctrl* h_ctrl = nullptr;          // pinned mirror of the control block
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t rgraph = nullptr;  // kRepairBatch warm-start repair steps (captured on first use)
    cudaGraphExec_t cgraph = nullptr;  // kRepairBatch warm-start crash steps (captured on first use)
    std::vector<void*> allocs;
    char* pool_base = nullptr;  // the chunk small buffers are carved from (dalloc)
    size_t pool_used = 0;
    int32_t* flag = nullptr;         // device validation flag
    bool solved = false;
    bool primed = false;             // q and r of the next pivot are on the device
    bool neg_b = false;               // some b_i < 0: every solve from the slack basis starts with Phase I
    bool infeasible = false;          // the last solve found no feasible point (Phase I)
    std::vector<double> h_b;          // b on the host (Phase I start row)
    bool warm_pending = false;
    int warm_repair_max = -1;         // >= 0: lp_set_basis_repair
    std::vector<int32_t> warm_basis;
    std::vector<int32_t> crash;       // lp_set_crash: structurals to enter first (consumed by the next solve)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, er0 = nullptr, er1 = nullptr, erg = nullptr, era = nullptr;
    double reinv_gj_s = 0.0, reinv_asm_s = 0.0;
    int32_t reinv_refined = 0;       // reinversions of this solve done by refinement
    int32_t reinv_tc = 0;            // reinversions of this solve whose slack rows ran on the tensor cores
    double refine_res_max = 0.0;     // largest residual the refinement checks of this solve found
    std::vector<cudaEvent_t> tev;    // kernel_timing: 3 events per timed iteration of the graph
    bool persist = false;            // pivots run in k_iterate (cooperative, one CTA per SM)
    int persist_blocks = 0;
    cudaEvent_t evc0 = nullptr, evc1 = nullptr;  // kernel_timing around k_iterate launches
    bool structured = false;         // pivots run in k_iterate_s (LP_ENGINE_STRUCTURED)
    int engine_reason = LP_ENGINE_REASON_NONE;  // why the engine that runs is not the one asked for
    // Case 2 (tableau_budget_mb exceeded): B^-1 in pinned host memory, streamed in row blocks
    bool ooc = false;
    int ooc_rows = 0, ooc_w = 0;        // rows per block, blocks
    double* ooc_host = nullptr;         // B^-1 (m x ld), pinned host memory
    double* ooc_buf[2] = {};            // device block buffers (ooc_rows x ld)
    double* ooc_prow = nullptr;         // device copy of row r for the next pivot
    int ooc_res = -1, ooc_res_buf = 0;  // block left on the device by the last pass (-1: none), its buffer
    bool ooc_primed = false;
    double ooc_bytes = 0.0;             // host <-> device block bytes of this solve
    cudaStream_t ooc_h2d = nullptr, ooc_d2h = nullptr;
    cudaEvent_t ooc_ev_h2d[2] = {}, ooc_ev_upd[2] = {}, ooc_ev_d2h[2] = {};
    bool s_ready = false;            // the structured state (bp, yp, slot maps) is current; the dense
                                     // B^-1 and y are stale while it is
    bool s_force = true;             // rebuild the slot map and A_p on the next entry
    int32_t* s_relayout = nullptr;   // device flag: the entry rebuilt the slot map
    int32_t* csc_cnt = nullptr;      // price_mode 2: per-column nonzero counts (scratch)
    double chain_s = 0.0, chain_b = 0.0;
    int chain_n = 0;
    double reinvert_seconds = 0.0;
    // per-solve accumulators
    double price_s = 0.0, update_s = 0.0, price_b = 0.0, update_b = 0.0;
    int32_t price_n = 0, update_n = 0;
    int64_t launches = 0;
};

namespace {

int cuda_fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return LP_ERR_OOM;
    return LP_ERR_CUDA;
}

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// Device buffers of the handle.  Buffers of at most kPoolMax bytes are carved,
// 256-byte aligned as cudaMalloc's, from shared chunks of kPoolChunk bytes;
// larger ones get an allocation of their own.  A handle makes a dozen
// cudaMalloc calls (and its destruction as many cudaFree calls) instead of
// dozens.  Everything is freed with the handle (free_all).
constexpr size_t kPoolMax = size_t(1) << 20, kPoolChunk = size_t(16) << 20, kPoolAlign = 256;
template <typename T>
int dalloc(lp_handle* h, T** ptr, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void* p = nullptr;
    if (bytes <= kPoolMax) {
        const size_t need = (bytes + kPoolAlign - 1) & ~(kPoolAlign - 1);
        if (!h->pool_base || h->pool_used + need > kPoolChunk) {
            cudaError_t e = cudaMalloc(&p, kPoolChunk);
            if (e != cudaSuccess) return cuda_fail(e);
            h->allocs.push_back(p);
            h->pool_base = static_cast<char*>(p);
            h->pool_used = 0;
        }
        p = h->pool_base + h->pool_used;
        h->pool_used += need;
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_fail(e);
        h->allocs.push_back(p);
    }
    *ptr = static_cast<T*>(p);
    return LP_OK;
}

#define TRY(x)                  \
    do {                        \
        int rc_ = (x);          \
        if (rc_ != LP_OK) return rc_; \
    } while (0)

int device_err_code(int err) {
    switch (err) {
        case kErrNone: return LP_OK;
        case kErrSingular: return LP_ERR_SINGULAR;
        case kErrInfeasibleStart: return LP_ERR_INVALID_ARG;
        case kErrTimeout: return LP_ERR_TIMEOUT;
        default: return LP_ERR_DEVICE;
    }
}

int read_ctrl(lp_handle* h) {
    CK(cudaMemcpyAsync(h->h_ctrl, h->ds.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

void free_all(lp_handle* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->rgraph) cudaGraphExecDestroy(h->rgraph);
    if (h->cgraph) cudaGraphExecDestroy(h->cgraph);
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    h->pool_base = nullptr;
    h->pool_used = 0;
    if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->er0) cudaEventDestroy(h->er0);
    if (h->er1) cudaEventDestroy(h->er1);
    if (h->erg) cudaEventDestroy(h->erg);
    if (h->era) cudaEventDestroy(h->era);
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    h->tev.clear();
    if (h->evc0) cudaEventDestroy(h->evc0);
    if (h->evc1) cudaEventDestroy(h->evc1);
    h->evc0 = h->evc1 = nullptr;
    if (h->ooc_host) cudaFreeHost(h->ooc_host);
    h->ooc_host = nullptr;
    for (int b = 0; b < 2; ++b) {
        if (h->ooc_ev_h2d[b]) cudaEventDestroy(h->ooc_ev_h2d[b]);
        if (h->ooc_ev_upd[b]) cudaEventDestroy(h->ooc_ev_upd[b]);
        if (h->ooc_ev_d2h[b]) cudaEventDestroy(h->ooc_ev_d2h[b]);
    }
    if (h->ooc_h2d) cudaStreamDestroy(h->ooc_h2d);
    if (h->ooc_d2h) cudaStreamDestroy(h->ooc_d2h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

int setup_geometry(lp_handle* h) {
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, h->device));
    Geometry& g = h->geo;
    g.sms = prop.multiProcessorCount;
    configure_iter_kernels(h->ld);
    const int occ_p = std::max(1, occupancy_price(h->ld));
    g.price_threads = 1024;
    g.update_threads = 1024;
    g.pivot_threads = 64;
    // PRICE: columns dealt round-robin to one 1024-thread block per SM (the
    // block's warps spread its column groups evenly over the SM's four
    // schedulers).
    g.price_blocks = std::max(1, std::min(g.sms * std::min(occ_p, 1), h->n));
    // BF16 screen: sms * min(occupancy, 2) blocks, a whole number per SM
    int lb = g.sms * 2;
    if (h->opt.price_mode == 1) lb = g.sms * std::min(2, std::max(1, occupancy_price_lp(h->ld)));
    g.price_lp_blocks = std::max(1, std::min(lb, std::max(1, (h->n + 1) / 2)));
    // UPDATE: rows dealt round-robin to one block per SM, one row per warp
    // (one block per SM keeps the staging of rho and a_q to one copy per SM).
    int ub = std::min(g.sms, h->m);
    g.update_blocks = std::max(1, ub);
    // pivot bookkeeping: O(m) vector work, one element per thread spread over the SMs
    g.pivot_blocks = std::max(1, std::min(2 * g.sms, (h->ld + 63) / 64));
    return LP_OK;
}

// Kernel timing samples every `stride`-th iteration of the graph: events sit
// around that iteration's kernels, and a kernel that follows an event is
// launched without the programmatic attribute.
int timing_stride(const lp_handle* h) { return h->opt.kernel_timing > 0 ? h->opt.kernel_timing : 0; }

int capture_graph_once(lp_handle* h, bool pdl) {
    cudaGraph_t graph = nullptr;
    const int G = h->opt.graph_iters;
    const int stride = timing_stride(h);
    int slot = 0;
    bool after_event = true;  // the graph's first kernel follows no kernel of the graph
    auto mark = [&](int which, bool timed) {
        if (!timed) return;
        cudaEventRecordWithFlags(h->tev[3 * (size_t)slot + which], h->stream, cudaEventRecordExternal);
        after_event = true;
    };
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int t = 0; t < G; ++t) {
        const bool timed = stride > 0 && t % stride == 0;
        launch_pivot(h->ds, h->geo, h->stream, pdl && !after_event);
        after_event = false;
        mark(0, timed);
        launch_price(h->ds, h->geo, h->stream, pdl && !after_event);
        after_event = false;
        mark(1, timed);
        launch_update(h->ds, h->geo, h->stream, pdl && !after_event);
        after_event = false;
        mark(2, timed);
        if (timed) ++slot;
    }
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e);
    return LP_OK;
}

constexpr int kRepairBatch = 16;  // warm-start repair pivots enqueued per read of the outcome

// kRepairBatch warm-start repair steps; their limit and tolerance are read
// from Ctrl, so one capture serves every solve of the handle.
int capture_repair_graph(lp_handle* h) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    launch_repair_steps(h->ds, h->geo, kRepairBatch, h->stream);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(&h->rgraph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e);
    return LP_OK;
}

// kRepairBatch warm-start crash steps (kernels_setup.cu); they read their
// state from Ctrl and the crash list, so one capture serves every solve.
int capture_crash_graph(lp_handle* h) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    launch_crash_steps(h->ds, h->geo, kRepairBatch, h->stream);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(&h->cgraph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e);
    return LP_OK;
}

int capture_graph(lp_handle* h) {
    const int G = h->opt.graph_iters;
    const int stride = timing_stride(h);
    if (stride > 0) {
        h->tev.resize(3 * (size_t)((G + stride - 1) / stride), nullptr);
        for (auto& e : h->tev) CK(cudaEventCreate(&e));
    }
    h->geo.pdl = 1;
    if (capture_graph_once(h, true) == LP_OK) return LP_OK;
    // programmatic edges refused by this driver: plain stream order
    (void)cudaGetLastError();
    h->geo.pdl = 0;
    return capture_graph_once(h, false);
}

// ---- Case 2: B^-1 in host memory, streamed through the device in row blocks ----
// The block left on the device by the last pass goes back to host memory (on
// the solve's stream, after every block copy of the pass).
int ooc_flush(lp_handle* h) {
    if (!h->ooc || h->ooc_res < 0) return LP_OK;
    const int i0 = h->ooc_res * h->ooc_rows, i1 = std::min(h->m, i0 + h->ooc_rows);
    CK(cudaStreamWaitEvent(h->stream, h->ooc_ev_d2h[0], 0));
    CK(cudaStreamWaitEvent(h->stream, h->ooc_ev_d2h[1], 0));
    CK(cudaMemcpyAsync(h->ooc_host + (size_t)i0 * h->ld, h->ooc_buf[h->ooc_res_buf],
                       sizeof(double) * (size_t)(i1 - i0) * h->ld, cudaMemcpyDeviceToHost, h->stream));
    h->ooc_bytes += 8.0 * (double)(i1 - i0) * h->ld;
    h->ooc_res = -1;
    return LP_OK;
}

// One pass over every block: copy in (one cudaMemcpyAsync per block, except the
// block the last pass left on the device), Step 8 of the pending pivot fused
// with the next FTRAN and the ratios, copy out (except the block visited last,
// which stays); then the ratio test over all rows and the fetch of row r.
// Blocks are visited from the end where the resident block is, so the order
// alternates between passes.
int ooc_pass(lp_handle* h) {
    const int W = h->ooc_w, R = h->ooc_rows, m = h->m, ld = h->ld;
    const bool desc = h->ooc_res == W - 1 && W > 1;
    int prev = -1;
    for (int t = 0; t < W; ++t) {
        const int w = desc ? W - 1 - t : t;
        const int i0 = w * R, i1 = std::min(m, i0 + R);
        const size_t bytes = sizeof(double) * (size_t)(i1 - i0) * ld;
        int bi;
        if (t == 0 && h->ooc_res == w) {
            bi = h->ooc_res_buf;
        } else {
            bi = prev < 0 ? 0 : prev ^ 1;
            // every earlier copy-out is complete (the host rows of this block
            // are current) and so is the last use of this buffer
            CK(cudaStreamWaitEvent(h->ooc_h2d, h->ooc_ev_d2h[0], 0));
            CK(cudaStreamWaitEvent(h->ooc_h2d, h->ooc_ev_d2h[1], 0));
            CK(cudaStreamWaitEvent(h->ooc_h2d, h->ooc_ev_upd[bi], 0));
            CK(cudaMemcpyAsync(h->ooc_buf[bi], h->ooc_host + (size_t)i0 * ld, bytes, cudaMemcpyHostToDevice,
                               h->ooc_h2d));
            CK(cudaEventRecord(h->ooc_ev_h2d[bi], h->ooc_h2d));
            CK(cudaStreamWaitEvent(h->stream, h->ooc_ev_h2d[bi], 0));
            h->ooc_bytes += (double)bytes;
        }
        launch_ooc_update(h->ds, h->geo, h->ooc_buf[bi], i0, i1, h->stream);
        CK(cudaGetLastError());
        CK(cudaEventRecord(h->ooc_ev_upd[bi], h->stream));
        h->launches += 1;
        if (t < W - 1) {
            CK(cudaStreamWaitEvent(h->ooc_d2h, h->ooc_ev_upd[bi], 0));
            CK(cudaMemcpyAsync(h->ooc_host + (size_t)i0 * ld, h->ooc_buf[bi], bytes, cudaMemcpyDeviceToHost,
                               h->ooc_d2h));
            CK(cudaEventRecord(h->ooc_ev_d2h[bi], h->ooc_d2h));
            h->ooc_bytes += (double)bytes;
        } else {
            h->ooc_res = w;
            h->ooc_res_buf = bi;
        }
        prev = bi;
    }
    // the host copy is current before row r is read from it
    CK(cudaStreamWaitEvent(h->stream, h->ooc_ev_d2h[0], 0));
    CK(cudaStreamWaitEvent(h->stream, h->ooc_ev_d2h[1], 0));
    launch_ooc_chuzr(h->ds, h->stream);
    const int r0 = h->ooc_res * R, r1 = std::min(m, r0 + R);
    launch_ooc_fetch_row(h->ds, h->ooc_host, h->ooc_buf[h->ooc_res_buf], r0, r1, h->ooc_prow, h->stream);
    CK(cudaGetLastError());
    h->launches += 2;
    return LP_OK;
}

// One iteration of Case 2: the pending pivot's bookkeeping (row r from the
// device copy), PRICE + CHUZC, and a pass over the blocks.  The first
// iteration after a reset or a reinversion only prices and passes.
int ooc_iteration(lp_handle* h) {
    if (h->ooc_primed) {
        DevState so = h->ds;
        so.prow = h->ooc_prow;
        launch_pivot(so, h->geo, h->stream, false);
        h->launches += 1;
    }
    launch_price(h->ds, h->geo, h->stream, false);
    CK(cudaGetLastError());
    h->launches += 1;
    TRY(ooc_pass(h));
    h->ooc_primed = true;
    return LP_OK;
}

// Largest admissible refine_tol, ||I - B11 Y0||_inf of the stored inverse that
// a reinversion refines (one Newton-Schulz step then leaves a residual below
// 2^-52, at the rounding level); above it the basis is eliminated afresh.
constexpr double kRefineTolMax = 1.0 / 67108864.0;  // 2^-26

// What a queued rebuild needs when it is settled.
struct ReinvQueued {
    bool try_refine = false;  // B11^-1 by refinement, verdict on the device
    bool compact = false;     // no dense B^-1: the structured engine follows
    int tc = 0;               // the slack rows ran on the tensor cores
    int k_host = 0;           // the structural count the host assumed
};

// Rebuild B^-1, bbar, y, z from the current basis: queues the kernels (a
// refinement without reading the control block, elimination after one read of
// the structural count).  `refine`: the stored inverse is that of the current
// basis (a periodic reinversion, the last update applied), so B11^-1 may come
// from one refinement step of it.  `to_struct`: the next consumer is the
// slack-structured engine, which then receives its live columns straight from
// B11^-1 and the slack rows (the dense B^-1 is not written).
//
// A refinement takes k from the last read (the classification checks it) and
// its residual test on the device (k_reinv_finish); a residual above the
// tolerance is seen when the rebuild is settled, and the rebuild is then
// redone by elimination.  Until then the finishing kernel leaves the status at
// kRebuildStopped, so that a launch queued behind the rebuild does nothing.
int reinvert_queue(lp_handle* h, int check_feasible, bool refine, bool to_struct, ReinvQueued* q) {
    q->compact = to_struct && h->structured;
    TRY(ooc_flush(h));  // the rebuild reads and writes B^-1 in host memory
    h->ooc_primed = false;
    q->k_host = h->h_ctrl->nsb;
    q->try_refine = refine && h->opt.reinvert_refine && h->h_ctrl->pending == 0 && refine_fits(q->k_host, h->m);
    CK(cudaEventRecord(h->er0, h->stream));
    launch_reinv_classify(h->ds, q->try_refine ? q->k_host : -1, h->stream);
    int k = q->k_host;
    if (!q->try_refine) {
        TRY(read_ctrl(h));
        if (h->h_ctrl->err != kErrNone) return device_err_code(h->h_ctrl->err);
        k = h->h_ctrl->k_struct;
    }
    CK(cudaEventRecord(h->erg, h->stream));
    if (q->try_refine) {
        const bool from_struct = h->structured && h->s_ready;
        h->launches += launch_refine_residual(h->ds, k, from_struct ? 1 : 0, h->h_ctrl->k_live, h->h_ctrl->map_par,
                                              h->stream);
        h->launches += launch_refine_apply(h->ds, k, h->stream);
    } else {
        launch_reinv_gj(h->ds, k, h->geo, h->stream);
        h->launches += reinv_gj_launches(k);
    }
    // classification, B11^-1 of an elimination, the slack rows, the dense rows, the finish
    h->launches += 1 + (k > 0 && !q->try_refine ? 1 : 0) + (k > 0 && h->ds.p.m > k ? 1 : 0) + (q->compact ? 0 : 1) + 1;
    CK(cudaEventRecord(h->era, h->stream));
    q->tc = launch_reinv_assemble(h->ds, k, h->geo, h->stream, q->try_refine ? 0 : 1, !q->compact);
    if (q->tc) h->launches += 2;  // exponents and slices of both operands (the GEMM replaces k_slack_gemm)
    launch_reinv_finish(h->ds, k, h->geo, h->stream, check_feasible, q->try_refine ? h->opt.refine_tol : -1.0);
    CK(cudaGetLastError());
    CK(cudaEventRecord(h->er1, h->stream));
    h->primed = false;
    return LP_OK;
}

// After a read of the control block behind a queued rebuild: its time, its
// counters and the verdict.  *redo: the rebuild must be done again by
// elimination (the refinement's residual was above the tolerance, or the basis
// held another structural count than the host's; that error flag is cleared).
int reinvert_settle(lp_handle* h, const ReinvQueued& q, bool* redo) {
    *redo = false;
    float ms = 0.f, mg = 0.f, ma = 0.f;
    CK(cudaEventElapsedTime(&ms, h->er0, h->er1));
    CK(cudaEventElapsedTime(&mg, h->erg, h->era));
    CK(cudaEventElapsedTime(&ma, h->era, h->er1));
    h->reinvert_seconds += ms * 1e-3;
    h->reinv_gj_s += mg * 1e-3;
    h->reinv_asm_s += ma * 1e-3;
    const Ctrl& C = *h->h_ctrl;
    if (q.try_refine && C.err == kErrBadIndex && C.k_struct != q.k_host) {
        // every kernel after the classification stopped: nothing was rebuilt
        CK(cudaMemsetAsync(&h->ds.ctrl->err, 0, sizeof(int32_t), h->stream));
        *redo = true;
        return LP_OK;
    }
    if (C.err != kErrNone) return device_err_code(C.err);
    if (q.try_refine) {
        h->refine_res_max = std::max(h->refine_res_max, C.refine_res);
        if (C.refine_rej) {
            *redo = true;
            return LP_OK;
        }
        h->reinv_refined++;
    }
    if (q.tc) h->reinv_tc++;
    return LP_OK;
}

// The structured engine's entry from a compact rebuild.
int struct_enter_compact(lp_handle* h) {
    launch_struct_enter(h->ds, h->s_force ? 1 : 0, h->s_relayout, h->stream, true);
    CK(cudaGetLastError());
    h->launches += 3;
    h->s_force = false;
    h->s_ready = true;
    return LP_OK;
}

// The rebuild, read and settled.
int reinvert(lp_handle* h, int check_feasible, bool refine, bool to_struct = false) {
    ReinvQueued q;
    TRY(reinvert_queue(h, check_feasible, refine, to_struct, &q));
    TRY(read_ctrl(h));
    h->s_ready = false;
    bool redo = false;
    TRY(reinvert_settle(h, q, &redo));
    if (redo) return reinvert(h, check_feasible, false, to_struct);
    if (q.compact) TRY(struct_enter_compact(h));
    return LP_OK;
}

int reset_state(lp_handle* h) {
    h->ooc_res = -1;  // B^-1 = I is written to host memory; no block is on the device
    h->ooc_primed = false;
    launch_init_slack(h->ds, h->stream);
    CK(cudaGetLastError());
    h->primed = false;
    h->s_ready = false;
    h->s_force = true;  // canonical slot order: a solve from the slack basis repeats bit for bit
    h->solved = false;
    h->reinvert_seconds = 0.0;
    return LP_OK;
}

// x[0 .. n) holds no NaN or infinity: a double is finite unless its 11
// exponent bits are all ones; branch-free over each chunk, and large arrays
// split over up to 16 host threads.
bool finite_all(const double* x, size_t n) {
    const auto chunk = [x](size_t i0, size_t i1) {
        uint64_t bad = 0;
        for (size_t i = i0; i < i1; ++i) {
            uint64_t u;
            std::memcpy(&u, x + i, sizeof(u));
            bad |= (uint64_t)(((u >> 52) & 0x7ffu) == 0x7ffu);
        }
        return bad == 0;
    };
    constexpr size_t kPar = size_t(1) << 22;
    const unsigned nt = std::min(16u, std::thread::hardware_concurrency());
    if (n < kPar || nt < 2) return chunk(0, n);
    const size_t per = (n + nt - 1) / nt;
    std::vector<char> ok(nt, 1);
    std::vector<std::thread> th;
    try {
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&chunk, &ok, per, n, t] {
                const size_t i0 = std::min(n, (size_t)t * per), i1 = std::min(n, i0 + per);
                ok[t] = chunk(i0, i1) ? 1 : 0;
            });
    } catch (...) {
        for (auto& t : th) t.join();
        return chunk(0, n);  // no threads to be had: one pass
    }
    for (auto& t : th) t.join();
    for (char v : ok)
        if (!v) return false;
    return true;
}

// The device address of a host array the device can read directly (pinned
// or registered host memory), else nullptr.
const void* host_device_view(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Rows p0 .. p0+np-1 of B^-1 (indexed by constraint row) into out[np][m],
// from the dense inverse or, while the structured engine's state is current,
// from its live columns and the unit columns of the basic slacks.
int binv_rows(const lp_handle* h, int p0, int np, double* out) {
    const int m = h->m;
    if (!(h->structured && h->s_ready)) {
        CK(cudaMemcpy2D(out, sizeof(double) * m, h->ds.binv + (size_t)p0 * h->ld, sizeof(double) * h->ld,
                        sizeof(double) * m, np, h->ooc ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost));
        return LP_OK;
    }
    Ctrl c;
    CK(cudaMemcpy(&c, h->ds.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    const int k = c.k_live, par = c.map_par;
    std::vector<double> live((size_t)np * std::max(k, 1));
    std::vector<int32_t> rs((size_t)m), bv((size_t)np);
    if (k > 0)
        CK(cudaMemcpy2D(live.data(), sizeof(double) * k, h->ds.bp + (size_t)p0 * h->ld, sizeof(double) * h->ld,
                        sizeof(double) * k, np, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rs.data(), h->ds.row_slot + (size_t)par * m, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(bv.data(), h->ds.basis + p0, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    for (int p = 0; p < np; ++p)
        for (int i = 0; i < m; ++i)
            out[(size_t)p * m + i] = rs[i] < k ? live[(size_t)p * k + rs[i]] : (bv[p] == h->n + i ? 1.0 : 0.0);
    return LP_OK;
}

// Phase I (Section 3.4: artificial variables and the two-phase method), with
// the textbook single artificial x0: maximise -x0 over [A | -e] x' <= b, where
// e marks the rows with b_i < 0, from the slack basis with x0 in the row of
// the most negative b_i (feasible: x0 = -min b).  The auxiliary LP runs on a
// second handle with the same kernels and options.  On an optimum of 0 the
// final basis becomes the Phase II start of `h` (an artificial left basic at
// zero is exchanged for the nonbasic slack with the largest |B^-1[p][s]|, the
// pivot of that exchange); below -1e-9 max(1, max|b|) the LP is infeasible.
// *status: LP_OPTIMAL (start staged), LP_INFEASIBLE, or the auxiliary solve's
// own status (iteration limit).
int run_phase1(lp_handle* h, int* iters, int* status, int* exchanged) {
    const int m = h->m, n = h->n;
    *iters = 0;
    *exchanged = 0;
    double* A_aux = nullptr;
    double* c_aux = nullptr;
    CK(cudaMalloc(&A_aux, sizeof(double) * (size_t)m * (n + 1)));
    if (cudaMalloc(&c_aux, sizeof(double) * (size_t)(n + 1)) != cudaSuccess) {
        cudaFree(A_aux);
        return LP_ERR_OOM;
    }
    launch_build_aux(h->ds.A_cm, h->ld, m, n, h->ds.b, A_aux, c_aux, h->stream);
    lp_options o = h->opt;
    o.cuda_stream = h->stream;
    o.trace_cap = 0;
    o.kernel_timing = 0;
    lp_handle* aux = nullptr;
    int rc = lp_create(&aux, m, n + 1, A_aux, h->ds.b, c_aux, 1, &o);  // copies, synchronises
    cudaFree(A_aux);
    cudaFree(c_aux);
    if (rc != LP_OK) return rc;
    int istar = 0;
    for (int i = 1; i < m; ++i)
        if (h->h_b[i] < h->h_b[istar]) istar = i;
    std::vector<int32_t> basis(m);
    for (int i = 0; i < m; ++i) basis[i] = n + 1 + i;
    basis[istar] = n;
    lp_result r1;
    rc = lp_set_basis(aux, basis.data());
    if (rc == LP_OK) rc = lp_solve(aux, &r1);
    if (rc == LP_OK) {
        *iters = r1.iterations;
        if (r1.status != LP_OPTIMAL) {
            *status = r1.status;
        } else if (r1.objective < -1e-9 * h->p.b_scale) {
            *status = LP_INFEASIBLE;
        } else {
            rc = lp_get_basis(aux, basis.data());
            int p = -1;
            for (int i = 0; i < m && rc == LP_OK; ++i)
                if (basis[i] == n) p = i;
            if (rc == LP_OK && p >= 0) {
                std::vector<double> row(m);
                std::vector<char> in_basis((size_t)n + 1 + m, 0);
                for (int i = 0; i < m; ++i) in_basis[basis[i]] = 1;
                if (binv_rows(aux, p, 1, row.data()) != LP_OK) {
                    rc = LP_ERR_CUDA;
                } else {
                    double best = -1.0;
                    int s = -1;
                    for (int i = 0; i < m; ++i) {
                        if (in_basis[(size_t)n + 1 + i]) continue;
                        const double v = std::fabs(row[i]);
                        if (v > best) { best = v; s = i; }
                    }
                    if (s < 0 || !(best > 1e-12)) rc = LP_ERR_SINGULAR;
                    else { basis[p] = n + 1 + s; *exchanged = 1; }
                }
            }
            if (rc == LP_OK) {
                h->warm_basis.resize(m);
                for (int i = 0; i < m; ++i) h->warm_basis[i] = basis[i] < n ? basis[i] : basis[i] - 1;
                h->warm_pending = true;
                h->warm_repair_max = -1;
                *status = LP_OPTIMAL;
            }
        }
    }
    lp_destroy(aux);
    return rc;
}

}  // namespace

extern "C" {

int lp_selftest_barrier_timeout(int32_t blocks, void* cuda_stream) {
    if (blocks < 1 || blocks > 64) return LP_ERR_INVALID_ARG;
    return barrier_selftest(blocks, static_cast<cudaStream_t>(cuda_stream));
}

void lp_default_options(lp_options* o) {
    if (!o) return;
    o->reinvert_every = 64;
    o->tabu_tenure = 7;
    o->max_iters = 50000000;
    o->bland_after = 50;
    o->price_mode = 0;
    o->topk = 16;
    o->trace_cap = 0;
    o->graph_iters = 64;
    o->kernel_timing = 0;
    o->engine = LP_ENGINE_STRUCTURED;
    o->anticycling = LP_ANTICYCLING_TABU;
    o->reinvert_refine = 1;
    o->reinvert_tc = 1;
    o->tol_d = 1e-9;
    o->tol_piv = 1e-9;
    o->tol_tie = 1e-12;
    o->refine_tol = kRefineTolMax;
    o->cuda_stream = nullptr;
}

const char* lp_strerror(int code) {
    switch (code) {
        case LP_OK: return "ok";
        case LP_ERR_INVALID_ARG: return "invalid argument";
        case LP_ERR_CUDA: return "CUDA runtime error";
        case LP_ERR_OOM: return "out of device memory";
        case LP_ERR_SINGULAR: return "singular basis during reinversion";
        case LP_ERR_TIMEOUT: return "bounded device wait timed out";
        case LP_ERR_STATE: return "call not valid in the handle's state";
        case LP_ERR_DEVICE: return "device-side internal error";
        default: return "unknown error";
    }
}

// Copies A (row-major -> padded column-major), b (padded) and c to the device,
// validates them and refreshes the BF16 copy and the feasibility scale.
static int upload_problem(lp_handle* h, const double* A, const double* b, const double* c, int32_t on_device) {
    const int m = h->m, n = h->n, ld = h->ld;
    DevState& s = h->ds;
    Params& P = h->p;
    double* A_cm = const_cast<double*>(s.A_cm);
    double* bb = const_cast<double*>(s.b);
    double* cc = const_cast<double*>(s.c);
    int32_t* flag = h->flag;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double* A_src = A;
    double* staging = nullptr;
    const void* view = on_device ? nullptr : host_device_view(A);
    if (view) {
        A_src = static_cast<const double*>(view);  // pinned host memory: the transpose reads it in place
    } else if (!on_device) {
        CK(cudaMalloc(&staging, (size_t)m * n * sizeof(double)));
        cudaError_t e = cudaMemcpyAsync(staging, A, (size_t)m * n * sizeof(double), kind, h->stream);
        if (e != cudaSuccess) { cudaFree(staging); return cuda_fail(e); }
        A_src = staging;
    }
    launch_transpose_pad(A_src, m, n, ld, A_cm, h->stream);
    CK(cudaMemsetAsync(bb, 0, (size_t)ld * sizeof(double), h->stream));
    CK(cudaMemcpyAsync(bb, b, (size_t)m * sizeof(double), kind, h->stream));
    CK(cudaMemcpyAsync(cc, c, (size_t)n * sizeof(double), kind, h->stream));
    CK(cudaMemsetAsync(flag, 0, sizeof(int32_t), h->stream));
    launch_validate(A_cm, bb, cc, m, n, ld, flag, h->stream);
    if (P.price_mode == 1) launch_to_bf16(A_cm, const_cast<uint16_t*>(s.A_lp), (size_t)n * ld, h->stream);
    if (P.price_mode == 2) {
        // sparse copy of A: counts and column starts, then the nonzeros
        launch_csc_count(A_cm, m, n, ld, h->csc_cnt, const_cast<int64_t*>(s.csc_ptr), h->stream);
        launch_csc_fill(A_cm, m, n, ld, s.csc_ptr, const_cast<int32_t*>(s.csc_row), const_cast<double*>(s.csc_val),
                        h->stream);
        int64_t nnz = 0;
        CK(cudaMemcpyAsync(&nnz, s.csc_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        P.nnz = (double)nnz;
        s.p = P;
    }
    int32_t hflag = 0;
    CK(cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (staging) CK(cudaFree(staging));
    if (hflag & 7) return LP_ERR_INVALID_ARG;
    h->neg_b = (hflag & 8) != 0;
    // b scale for the feasibility check of warm starts
    {
        h->h_b.resize(m);
        CK(cudaMemcpy(h->h_b.data(), bb, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost));
        double sc = 1.0;
        for (double v : h->h_b) sc = std::max(sc, std::fabs(v));
        P.b_scale = sc;
        s.p = P;
    }
    return LP_OK;
}

static int create_impl(lp_handle* h, int32_t m, int32_t n, const double* A, const double* b,
                       const double* c, int32_t on_device) {
    CK(cudaGetDevice(&h->device));
    h->m = m;
    h->n = n;
    h->ld = (m + kLdAlign - 1) / kLdAlign * kLdAlign;
    const int ld = h->ld;
    if ((size_t)ld * sizeof(double) * 2 > 200 * 1024) return LP_ERR_INVALID_ARG;  // smem staging limit

    if (h->opt.cuda_stream) {
        h->stream = static_cast<cudaStream_t>(h->opt.cuda_stream);
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));
    CK(cudaEventCreate(&h->er0));
    CK(cudaEventCreate(&h->er1));
    CK(cudaEventCreate(&h->erg));
    CK(cudaEventCreate(&h->era));
    CK(cudaMallocHost(&h->h_ctrl, sizeof(Ctrl)));

    DevState& s = h->ds;
    Params& P = h->p;
    P.m = m; P.n = n; P.ld = ld;
    P.reinvert_every = h->opt.reinvert_every;
    P.tabu_tenure = h->opt.tabu_tenure;
    P.max_iters = h->opt.max_iters;
    P.bland_after = h->opt.bland_after;
    P.trace_cap = std::max(0, h->opt.trace_cap);
    P.tol_d = h->opt.tol_d;
    P.tol_piv = h->opt.tol_piv;
    P.tol_tie = h->opt.tol_tie;
    P.price_mode = h->opt.price_mode;
    P.topk = h->opt.topk;
    P.lex = h->opt.anticycling == LP_ANTICYCLING_LEXICOGRAPHIC ? 1 : 0;
    P.prio = 0;
    P.reinvert_tc = h->opt.reinvert_tc;
    if (P.lex) {
        // the lexicographic rule needs neither the tabu list nor the safety net
        P.tabu_tenure = 0;
        P.bland_after = 0;
    }
    s.p = P;

    double *A_cm, *cc, *bb, *binv, *bbar, *y, *rho, *alpha, *theta, *upd_part, *rv_M, *rv_f;
    int32_t *basis, *pos, *tabu, *rv_sp, *rv_rows, *rv_ri, *rv_piv, *rv_done, *rv_slack, *flag;
    Ctrl* ctrl;
    PriceCand* price_part;
    TRY(dalloc(h, &A_cm, (size_t)n * ld));
    TRY(dalloc(h, &cc, (size_t)n));
    TRY(dalloc(h, &bb, (size_t)ld));
    // Case 2 of Section 3: the explicit inverse does not fit the memory granted to it
    const double tab_bytes = 8.0 * (double)m * (double)ld;
    if (h->opt.tableau_budget_mb > 0.0 && tab_bytes > 1e6 * h->opt.tableau_budget_mb) {
        const double row_bytes = 8.0 * (double)ld;
        h->ooc = true;
        h->ooc_rows = (int)std::max(1.0, std::floor(0.5e6 * h->opt.tableau_budget_mb / row_bytes));
        h->ooc_rows = std::min(h->ooc_rows, m);
        h->ooc_w = (m + h->ooc_rows - 1) / h->ooc_rows;
        if (P.lex) return LP_ERR_INVALID_ARG;  // its tie-break reads rows of B^-1 that are not on the device
        CK(cudaMallocHost(&h->ooc_host, sizeof(double) * (size_t)m * ld));
        binv = h->ooc_host;  // device-accessible (unified addressing): init and reinversion write it directly
        TRY(dalloc(h, &h->ooc_buf[0], (size_t)h->ooc_rows * ld));
        TRY(dalloc(h, &h->ooc_buf[1], (size_t)h->ooc_rows * ld));
        TRY(dalloc(h, &h->ooc_prow, (size_t)ld));
        CK(cudaStreamCreateWithFlags(&h->ooc_h2d, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->ooc_d2h, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            CK(cudaEventCreateWithFlags(&h->ooc_ev_h2d[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->ooc_ev_upd[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->ooc_ev_d2h[b], cudaEventDisableTiming));
        }
        if (configure_ooc_kernels(ld) != 0) return LP_ERR_CUDA;
    } else {
        TRY(dalloc(h, &binv, (size_t)m * ld));
    }
    TRY(dalloc(h, &bbar, (size_t)m));
    TRY(dalloc(h, &y, (size_t)ld));
    TRY(dalloc(h, &rho, (size_t)ld));
    TRY(dalloc(h, &alpha, 2 * (size_t)ld));
    TRY(dalloc(h, &theta, (size_t)m));
    TRY(dalloc(h, &basis, (size_t)m));
    TRY(dalloc(h, &pos, (size_t)(n + m)));
    TRY(dalloc(h, &tabu, (size_t)(n + m)));
    TRY(dalloc(h, &ctrl, 1));
    CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), h->stream));
    TRY(dalloc(h, &flag, 1));
    h->flag = flag;
    TRY(dalloc(h, &s.rank, (size_t)(n + m)));
    TRY(dalloc(h, &rv_sp, (size_t)m));
    TRY(dalloc(h, &rv_rows, (size_t)m));
    TRY(dalloc(h, &rv_ri, (size_t)m));
    TRY(dalloc(h, &rv_piv, (size_t)m));
    TRY(dalloc(h, &rv_done, (size_t)m));
    TRY(dalloc(h, &rv_slack, (size_t)m));
    TRY(dalloc(h, &rv_M, (size_t)m * m));
    TRY(dalloc(h, &s.rv_W, (size_t)m * m));
    TRY(dalloc(h, &s.rv_b_of_pos, (size_t)m));
    TRY(dalloc(h, &s.rv_g_of_row, (size_t)m));
    TRY(dalloc(h, &s.rv_J, (size_t)m));
    TRY(dalloc(h, &s.rv_cJ, (size_t)m));
    TRY(dalloc(h, &rv_f, 2 * (size_t)m));
    TRY(dalloc(h, &s.y32, (size_t)ld));
    TRY(dalloc(h, &s.cand, (size_t)kMaxTopk + 1));
    TRY(dalloc(h, &s.cand_d, (size_t)kMaxTopk + 1));
    if (P.reinvert_tc && m > 1) {
        // digit slices of the slack-row product (k <= 1024 structural columns)
        TRY(dalloc(h, &s.oz_xs, oz_scratch_x_elems(m)));
        TRY(dalloc(h, &s.oz_ys, oz_scratch_y_elems(m)));
        TRY(dalloc(h, &s.oz_ex, (size_t)m));
        TRY(dalloc(h, &s.oz_ey, (size_t)m));
    }
    if (P.price_mode == 2) {
        // capacity for a fully dense A, so the captured graphs' pointers never change
        int64_t* ptr = nullptr;
        int32_t* row = nullptr;
        double* val = nullptr;
        TRY(dalloc(h, &ptr, (size_t)n + 1));
        TRY(dalloc(h, &row, (size_t)m * n));
        TRY(dalloc(h, &val, (size_t)m * n));
        TRY(dalloc(h, &h->csc_cnt, (size_t)n));
        s.csc_ptr = ptr;
        s.csc_row = row;
        s.csc_val = val;
    }
    if (P.price_mode == 1) {
        uint16_t* lp = nullptr;
        TRY(dalloc(h, &lp, (size_t)n * ld));
        s.A_lp = lp;
    }
    TRY(setup_geometry(h));
    // per-block partials: every grid, including k_iterate's one CTA per SM
    const int parts = std::max(std::max(h->geo.price_blocks, h->geo.price_lp_blocks),
                               std::max(h->geo.update_blocks, h->geo.sms));
    TRY(dalloc(h, &price_part, (size_t)parts));
    TRY(dalloc(h, &s.lp_part, (size_t)parts));
    TRY(dalloc(h, &upd_part, (size_t)parts));
    TRY(dalloc(h, &s.row_var, (size_t)m));
    TRY(dalloc(h, &s.lex_rows, (size_t)m));
    TRY(dalloc(h, &s.crash_list, (size_t)m));
    TRY(dalloc(h, &s.row_part, (size_t)parts));
    TRY(dalloc(h, &s.gbar, 2));
    if (P.trace_cap > 0) {
        TRY(dalloc(h, &s.trace.q, (size_t)P.trace_cap));
        TRY(dalloc(h, &s.trace.r, (size_t)P.trace_cap));
        TRY(dalloc(h, &s.trace.theta, (size_t)P.trace_cap));
        TRY(dalloc(h, &s.trace.dq, (size_t)P.trace_cap));
        TRY(dalloc(h, &s.trace.flags, (size_t)P.trace_cap));
    }
    s.A_cm = A_cm; s.c = cc; s.b = bb; s.binv = binv; s.bbar = bbar; s.y = y; s.rho = rho;
    s.alpha = alpha; s.theta = theta; s.basis = basis; s.pos = pos; s.tabu_until = tabu;
    s.ctrl = ctrl; s.price_part = price_part; s.upd_part = upd_part;
    s.rv_struct_pos = rv_sp; s.rv_rows = rv_rows; s.rv_row_index = rv_ri; s.rv_slack_pos = rv_slack;
    s.rv_pivrow = rv_piv; s.rv_rowdone = rv_done; s.rv_M = rv_M; s.rv_f = rv_f;

    {
        std::vector<int32_t> none((size_t)n + m, kNoRank);
        CK(cudaMemcpy(s.rank, none.data(), sizeof(int32_t) * none.size(), cudaMemcpyHostToDevice));
    }
    TRY(upload_problem(h, A, b, c, on_device));
    TRY(reset_state(h));
    // Persistent engines.  The slack-structured one when asked for (the
    // default) and it fits: price_mode 0, a device that runs cooperative
    // launches with one 1024-thread CTA on every SM.  Otherwise the dense one,
    // unless captured graphs are asked for or the mode needs them (the BF16
    // screen; the lexicographic tie-break, which the dense engine lacks).
    {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
        // (the ratio tests hold one CTA record per thread: at most 1024 CTAs)
        const bool want_s = h->opt.engine == LP_ENGINE_STRUCTURED;
        const bool fits_s = want_s && h->opt.price_mode == 0 && coop && h->geo.sms <= 1024 &&
                            struct_engine_fits(h->m, h->ld, h->geo.sms);
        const bool occ_s = fits_s && occupancy_iterate_s(h->ld) >= 1;
        // the first condition that keeps the asked engine from running
        if (h->ooc) {
            h->engine_reason = LP_ENGINE_REASON_OUT_OF_CORE;
        } else if (h->opt.engine != LP_ENGINE_GRAPH) {
            if (h->opt.price_mode == 1) h->engine_reason = LP_ENGINE_REASON_PRICE_MODE;
            else if (P.lex && !want_s) h->engine_reason = LP_ENGINE_REASON_LEXICOGRAPHIC;
            else if (!coop || h->geo.sms > 1024) h->engine_reason = LP_ENGINE_REASON_NO_COOPERATIVE;
            else if (want_s && h->opt.price_mode != 0) h->engine_reason = LP_ENGINE_REASON_PRICE_MODE;
            else if (want_s && !fits_s) h->engine_reason = LP_ENGINE_REASON_SIZE;
            else if (want_s && !occ_s) h->engine_reason = LP_ENGINE_REASON_OCCUPANCY;
        }
        if (occ_s && !h->ooc) {
            const int m = h->m, n = h->n, ld = h->ld;
            TRY(dalloc(h, &s.A_p, (size_t)n * ld));
            TRY(dalloc(h, &s.A_p32, (size_t)n * ld));
            TRY(dalloc(h, &s.c32lo, (size_t)n));
            TRY(dalloc(h, &s.c32hi, (size_t)n));
            h->p.screen = 1;
            s.p.screen = 1;
            TRY(dalloc(h, &s.bp, (size_t)m * ld));
            TRY(dalloc(h, &s.yp, 2 * (size_t)ld));
            TRY(dalloc(h, &s.slot_row, 2 * (size_t)m));
            TRY(dalloc(h, &s.row_slot, 2 * (size_t)m));
            TRY(dalloc(h, &s.uslot, (size_t)m));
            TRY(dalloc(h, &h->s_relayout, 1));
            TRY(dalloc(h, &s.price_rec, (size_t)h->geo.sms));
            TRY(dalloc(h, &s.row_rec, (size_t)h->geo.sms));
            CK(cudaMemsetAsync(s.bp, 0, sizeof(double) * (size_t)m * ld, h->stream));
            CK(cudaMemsetAsync(s.yp, 0, sizeof(double) * 2 * (size_t)ld, h->stream));
            launch_struct_init_maps(s, h->stream);
            CK(cudaGetLastError());
            h->structured = true;
            h->persist_blocks = h->geo.sms;
            h->s_force = true;
        } else if (!h->ooc && h->opt.engine != LP_ENGINE_GRAPH && h->opt.price_mode != 1 && !P.lex && coop &&
                   h->geo.sms <= 1024 && occupancy_iterate(h->ld) >= 1) {
            h->persist = true;
            h->persist_blocks = h->geo.sms;  // the partial arrays hold at least sms entries
        } else if (!h->ooc && h->opt.engine != LP_ENGINE_GRAPH && h->engine_reason == LP_ENGINE_REASON_NONE) {
            h->engine_reason = LP_ENGINE_REASON_OCCUPANCY;
        }
        if ((h->persist || h->structured) && h->opt.kernel_timing > 0) {
            CK(cudaEventCreate(&h->evc0));
            CK(cudaEventCreate(&h->evc1));
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_create(lp_handle** out, int32_t m, int32_t n, const double* A, const double* b, const double* c,
              int32_t on_device, const lp_options* opt) {
    if (!out) return LP_ERR_INVALID_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || !A || !b || !c) return LP_ERR_INVALID_ARG;
    if ((int64_t)n + m > (int64_t)1 << 30) return LP_ERR_INVALID_ARG;
    lp_options o;
    lp_default_options(&o);
    if (opt) o = *opt;
    if (o.graph_iters < 1 || o.graph_iters > 4096 || o.engine < 0 || o.engine > LP_ENGINE_STRUCTURED || o.anticycling < 0 || o.anticycling > 1 || o.reinvert_refine < 0 || o.reinvert_refine > 1 || o.reinvert_tc < 0 || o.reinvert_tc > 1 || o.max_iters < 0 || o.reinvert_every < 0 || o.tabu_tenure < 0 || o.kernel_timing < 0 ||
        o.bland_after < 0 || o.price_mode < 0 || o.price_mode > 2 || o.topk < 1 || o.topk > kMaxTopk || !(o.tol_d >= 0) || !(o.tol_piv > 0) || !(o.tol_tie >= 0) || !(o.refine_tol >= 0 && o.refine_tol <= kRefineTolMax))
        return LP_ERR_INVALID_ARG;
    if (!on_device) {
        // (a pinned A is checked on the device after its upload, like device inputs)
        if ((!host_device_view(A) && !finite_all(A, (size_t)m * n)) || !finite_all(c, n) || !finite_all(b, m))
            return LP_ERR_INVALID_ARG;
    }
    lp_handle* h = new (std::nothrow) lp_handle();
    if (!h) return LP_ERR_OOM;
    h->opt = o;
    int rc = create_impl(h, m, n, A, b, c, on_device);
    if (rc != LP_OK) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return LP_OK;
}

int lp_set_basis_repair(lp_handle* h, const int32_t* basis, int32_t max_repairs) {
    if (max_repairs < 0) return LP_ERR_INVALID_ARG;
    int rc = lp_set_basis(h, basis);
    if (rc == LP_OK) h->warm_repair_max = max_repairs;
    return rc;
}

int lp_set_crash(lp_handle* h, const int32_t* vars, int32_t count) {
    if (!h || count < 0 || count > h->m || (count > 0 && !vars)) return LP_ERR_INVALID_ARG;
    if (h->neg_b || h->ooc) return LP_ERR_STATE;  // needs a feasible slack basis and B^-1 on the device
    std::vector<char> seen((size_t)h->n, 0);
    for (int t = 0; t < count; ++t) {
        const int v = vars[t];
        if (v < 0 || v >= h->n || seen[v]) return LP_ERR_INVALID_ARG;
        seen[v] = 1;
    }
    h->crash.assign(vars, vars + count);
    h->warm_pending = false;
    return LP_OK;
}

int lp_set_basis(lp_handle* h, const int32_t* basis) {
    if (!h || !basis) return LP_ERR_INVALID_ARG;
    h->warm_repair_max = -1;
    h->crash.clear();
    std::vector<char> seen((size_t)h->n + h->m, 0);
    for (int p = 0; p < h->m; ++p) {
        const int v = basis[p];
        if (v < 0 || v >= h->n + h->m || seen[v]) return LP_ERR_INVALID_ARG;
        seen[v] = 1;
    }
    h->warm_basis.assign(basis, basis + h->m);
    h->warm_pending = true;
    return LP_OK;
}

int lp_update_problem(lp_handle* h, const double* A, const double* b, const double* c, int32_t on_device) {
    if (!h || !A || !b || !c) return LP_ERR_INVALID_ARG;
    if (!on_device) {
        if ((!host_device_view(A) && !finite_all(A, (size_t)h->m * h->n)) || !finite_all(c, h->n) ||
            !finite_all(b, h->m))
            return LP_ERR_INVALID_ARG;
    }
    h->warm_pending = false;
    TRY(upload_problem(h, A, b, c, on_device));
    h->s_force = true;
    TRY(reset_state(h));
    CK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_set_priority(lp_handle* h, const int32_t* vars, int32_t count) {
    if (!h || count < 0 || (count > 0 && !vars)) return LP_ERR_INVALID_ARG;
    if (h->opt.price_mode != 0) return LP_ERR_STATE;
    const int N = h->n + h->m;
    if (count > N) return LP_ERR_INVALID_ARG;
    std::vector<int32_t> rank((size_t)N, kNoRank);
    for (int t = 0; t < count; ++t) {
        const int v = vars[t];
        if (v < 0 || v >= N || rank[v] != kNoRank) return LP_ERR_INVALID_ARG;
        rank[v] = t;
    }
    CK(cudaMemcpyAsync(h->ds.rank, rank.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->p.prio = count > 0 ? 1 : 0;  // the persistent kernels skip the priority reductions without a list
    h->ds.p.prio = h->p.prio;
    return LP_OK;
}

int lp_reset(lp_handle* h) {
    if (!h) return LP_ERR_INVALID_ARG;
    h->warm_pending = false;
    h->crash.clear();
    TRY(reset_state(h));
    CK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_solve(lp_handle* h, lp_result* out) {
    if (!h) return LP_ERR_INVALID_ARG;
    CK(cudaEventRecord(h->ev0, h->stream));
    h->reinvert_seconds = 0.0;
    h->reinv_gj_s = h->reinv_asm_s = 0.0;
    h->reinv_refined = 0;
    h->reinv_tc = 0;
    h->refine_res_max = 0.0;
    h->ooc_bytes = 0.0;
    h->price_s = h->update_s = h->price_b = h->update_b = 0.0;
    h->price_n = h->update_n = 0;
    h->chain_s = h->chain_b = 0.0;
    h->chain_n = 0;
    h->launches = 0;
    h->infeasible = false;
    int warm_repairs = 0, warm_fallback = 0;
    int phase1_iters = 0, phase1_status = 0, phase1_exch = 0;
    if (h->neg_b && !h->warm_pending) {
        TRY(run_phase1(h, &phase1_iters, &phase1_status, &phase1_exch));
        if (phase1_status != LP_OPTIMAL) {
            // no feasible start: the LP is infeasible, or Phase I hit its iteration limit
            CK(cudaEventRecord(h->ev1, h->stream));
            CK(cudaEventSynchronize(h->ev1));
            float ms1 = 0.f;
            CK(cudaEventElapsedTime(&ms1, h->ev0, h->ev1));
            h->solved = true;
            h->infeasible = phase1_status == LP_INFEASIBLE;
            if (out) {
                memset(out, 0, sizeof(*out));
                out->status = phase1_status;
                out->seconds = ms1 * 1e-3;
                out->phase1_iterations = phase1_iters;
                out->persistent = h->structured ? 2 : (h->persist ? 1 : 0);
                out->engine_reason = h->engine_reason;
            }
            return LP_OK;
        }
    }
    if (h->warm_pending) {
        TRY(reset_state(h));
        CK(cudaMemcpyAsync(h->ds.basis, h->warm_basis.data(), sizeof(int32_t) * h->m,
                           cudaMemcpyHostToDevice, h->stream));
        launch_load_basis(h->ds, h->stream);
        CK(cudaGetLastError());
        h->warm_pending = false;
        if (h->warm_repair_max < 0) {
            TRY(reinvert(h, 1, false));
        } else {
            int rc = reinvert(h, 0, false);
            bool ok = rc == LP_OK;
            if (rc != LP_OK && rc != LP_ERR_SINGULAR) return rc;
            if (ok) {
                // repair pivots in batches (a captured graph of kRepairBatch
                // steps), the outcome read once per batch
                TRY(read_ctrl(h));
                const int it0 = h->h_ctrl->it;
                const int limit = it0 + h->warm_repair_max;
                launch_repair_begin(h->ds, 1e-9 * h->p.b_scale, limit, h->stream);
                h->launches += 1;
                if (!h->rgraph) TRY(capture_repair_graph(h));
                for (;;) {
                    CK(cudaGraphLaunch(h->rgraph, h->stream));
                    h->launches += 4 * kRepairBatch;
                    TRY(read_ctrl(h));
                    const Ctrl& C = *h->h_ctrl;
                    if (C.err != kErrNone) return device_err_code(C.err);
                    if (C.repair == 2) break;                       // feasible
                    if (C.repair >= 3) { ok = false; break; }       // no slack can repair, or the cap
                    if (C.status == kReinvert) TRY(reinvert(h, 0, true));
                    else if (C.status != kRunning) break;
                }
                warm_repairs = h->h_ctrl->it - it0;
            }
            if (!ok) {
                warm_fallback = 1;
                TRY(reset_state(h));
            }
            h->primed = false;
        }
    }
    if (h->neg_b || h->ooc) h->crash.clear();  // (lp_update_problem may have brought a negative b)
    if (!h->crash.empty()) {
        // crash from the slack basis: the listed structurals enter by ordinary
        // ratio-test pivots, in batches of a captured graph, the outcome read
        // once per batch
        const int cn = (int)h->crash.size();
        TRY(reset_state(h));
        CK(cudaMemcpyAsync(h->ds.crash_list, h->crash.data(), sizeof(int32_t) * cn, cudaMemcpyHostToDevice,
                           h->stream));
        h->crash.clear();
        TRY(read_ctrl(h));
        const int it0 = h->h_ctrl->it;
        launch_crash_begin(h->ds, cn, h->stream);
        h->launches += 1;
        if (!h->cgraph) TRY(capture_crash_graph(h));
        for (;;) {
            CK(cudaGraphLaunch(h->cgraph, h->stream));
            h->launches += 4 * kRepairBatch;
            TRY(read_ctrl(h));
            const Ctrl& C = *h->h_ctrl;
            if (C.err != kErrNone) return device_err_code(C.err);
            if (C.crash == 2 && C.pending == 0) break;
            if (C.status == kReinvert) TRY(reinvert(h, 0, true));
            else if (C.status != kRunning) break;
        }
        warm_repairs = h->h_ctrl->it - it0;
        h->primed = false;
    }
    TRY(read_ctrl(h));
    // A periodic rebuild for the structured engine is queued with its entry and
    // the next launch behind it, and settled at the read after that launch.
    ReinvQueued rq;
    bool queued = false;
    for (;;) {
        const Ctrl& C = *h->h_ctrl;
        if (queued) {
            queued = false;
            bool redo = false;
            TRY(reinvert_settle(h, rq, &redo));
            if (redo) {
                TRY(reinvert(h, 0, false, true));
                continue;
            }
        }
        if (C.err != kErrNone) return device_err_code(C.err);
        if (C.status == kReinvert) {
            if (h->structured && h->s_ready && !h->ooc) {
                TRY(reinvert_queue(h, 0, true, true, &rq));
                TRY(struct_enter_compact(h));
                queued = true;  // the launch below runs behind the rebuild
            } else {
                TRY(reinvert(h, 0, true, true));
                continue;
            }
        } else if (C.status != kRunning) {
            break;
        }
        if (h->ooc) {
            TRY(ooc_iteration(h));
            TRY(read_ctrl(h));
            continue;
        }
        if (h->structured) {
            if (!h->s_ready) {
                // enter the structured form from the dense state (rebuilt B^-1 or slack basis)
                launch_struct_enter(h->ds, h->s_force ? 1 : 0, h->s_relayout, h->stream, false);
                CK(cudaGetLastError());
                h->launches += 3;
                h->s_force = false;
                h->s_ready = true;
            }
            const Ctrl before = C;
            if (h->evc0) CK(cudaEventRecord(h->evc0, h->stream));
            // one step more than graph_iters: the first step after an entry only
            // prices and runs the ratio test, so a reinversion period fits one launch
            const cudaError_t e = launch_iterate_s(h->ds, h->persist_blocks, h->opt.graph_iters + 1, h->stream);
            if (e == cudaSuccess) {
                h->launches += 1;
                if (h->evc1) CK(cudaEventRecord(h->evc1, h->stream));
                TRY(read_ctrl(h));
                if (h->evc1) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, h->evc0, h->evc1));
                    const Ctrl& A = *h->h_ctrl;
                    h->chain_s += ms * 1e-3;
                    h->chain_b += (A.bytes_price - before.bytes_price) + (A.bytes_update - before.bytes_update);
                    h->chain_n++;
                }
                continue;
            }
            // the cooperative launch was refused: rebuild the dense state and
            // continue on the dense engines
            (void)cudaGetLastError();
            if (queued) {
                queued = false;
                TRY(read_ctrl(h));
                bool redo = false;
                TRY(reinvert_settle(h, rq, &redo));
            }
            h->structured = false;
            TRY(reinvert(h, 0, false));
            continue;
        }
        if (!h->primed) {
            launch_price(h->ds, h->geo, h->stream);
            launch_update(h->ds, h->geo, h->stream);
            CK(cudaGetLastError());
            h->launches += 2;
            h->primed = true;
        }
        const Ctrl before = C;
        if (h->persist) {
            if (h->evc0) CK(cudaEventRecord(h->evc0, h->stream));
            const cudaError_t e = launch_iterate(h->ds, h->persist_blocks, h->opt.graph_iters, h->stream);
            if (e == cudaSuccess) {
                h->launches += 1;
                if (h->evc1) CK(cudaEventRecord(h->evc1, h->stream));
                TRY(read_ctrl(h));
                if (h->evc1) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, h->evc0, h->evc1));
                    const Ctrl& A = *h->h_ctrl;
                    h->chain_s += ms * 1e-3;
                    h->chain_b += (A.bytes_price - before.bytes_price) + (A.bytes_update - before.bytes_update);
                    h->chain_n++;
                }
                continue;
            }
            // the cooperative launch was refused: captured graphs from here on
            (void)cudaGetLastError();
            h->persist = false;
        }
        if (!h->graph) TRY(capture_graph(h));  // on the first use of the captured-graph engine
        CK(cudaGraphLaunch(h->graph, h->stream));
        h->launches += 3 * (int64_t)h->opt.graph_iters;
        TRY(read_ctrl(h));
        if (!h->tev.empty()) {
            // kernels that did work occupy the first slots of the graph
            const Ctrl& A = *h->h_ctrl;
            // a PRICE slot did work when the FP64 pass or (price_mode 1) the screen ran
            const int np = std::min((A.n_price - before.n_price) + (A.n_lp - before.n_lp) -
                                        (A.n_full - before.n_full),
                                    h->opt.graph_iters);
            const int nu = std::min(A.n_update - before.n_update, h->opt.graph_iters);
            // timed iterations are 0, stride, 2*stride, ...: slot i times iteration i*stride
            const int stride = timing_stride(h);
            const int tp = (np + stride - 1) / stride, tu = (nu + stride - 1) / stride;
            for (int i = 0; i < tp; ++i) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, h->tev[3 * i], h->tev[3 * i + 1]) == cudaSuccess) h->price_s += ms * 1e-3;
            }
            for (int i = 0; i < tu; ++i) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, h->tev[3 * i + 1], h->tev[3 * i + 2]) == cudaSuccess) h->update_s += ms * 1e-3;
            }
            h->price_n += tp;
            h->update_n += tu;
            // bytes of the timed launches: this graph's bytes in proportion
            if (np > 0) h->price_b += (A.bytes_price - before.bytes_price) * tp / np;
            if (nu > 0) h->update_b += (A.bytes_update - before.bytes_update) * tu / nu;
        }
    }
    if (h->structured && h->s_ready) {
        // the duals of the solution, in row order
        launch_struct_scatter_y(h->ds, h->stream);
        CK(cudaGetLastError());
        h->launches += 1;
    }
    TRY(ooc_flush(h));  // B^-1 whole in host memory for lp_get_state and the next solve
    CK(cudaEventRecord(h->ev1, h->stream));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->solved = true;
    if (out) {
        const Ctrl& C = *h->h_ctrl;
        memset(out, 0, sizeof(*out));
        out->status = C.status;
        out->iterations = C.it;
        out->reinversions = C.n_reinv;
        out->degenerate = C.n_degenerate;
        out->tabu_pushes = C.n_tabu;
        out->bland_fallbacks = C.n_bland;
        out->aspirations = C.n_asp;
        out->objective = C.z;
        out->seconds = ms * 1e-3;
        out->reinvert_seconds = h->reinvert_seconds;
        out->bytes_moved = C.bytes_price + C.bytes_update;
        out->price_seconds = h->price_s;
        out->update_seconds = h->update_s;
        out->price_bytes = h->price_b;
        out->update_bytes = h->update_b;
        out->price_launches = h->price_n;
        out->update_launches = h->update_n;
        out->kernel_launches = h->launches;
        out->warm_repairs = warm_repairs;
        out->warm_fallback = warm_fallback;
        out->screen_passes = C.n_lp;
        out->full_passes = C.n_full;
        out->reinvert_gj_seconds = h->reinv_gj_s;
        out->reinvert_assemble_seconds = h->reinv_asm_s;
        out->chain_seconds = h->chain_s;
        out->chain_bytes = h->chain_b;
        out->chain_launches = h->chain_n;
        out->persistent = h->structured ? 2 : (h->persist ? 1 : 0);
                out->engine_reason = h->engine_reason;
        out->phase1_iterations = phase1_iters;
        out->phase1_exchanged = phase1_exch;
        out->refined_reinversions = h->reinv_refined;
        out->tc_reinversions = h->reinv_tc;
        out->ooc_blocks = h->ooc ? h->ooc_w : 0;
        out->ooc_block_rows = h->ooc ? h->ooc_rows : 0;
        out->ooc_bytes = h->ooc_bytes;
        out->refine_residual_max = h->refine_res_max;
    }
    return LP_OK;
}

int lp_get_solution(const lp_handle* h, double* x, double* y, double* objective) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (!h->solved || h->infeasible) return LP_ERR_STATE;
    const int m = h->m, n = h->n;
    std::vector<int32_t> basis(m);
    std::vector<double> bbar(m);
    CK(cudaMemcpyAsync(basis.data(), h->ds.basis, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(bbar.data(), h->ds.bbar, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    if (y) CK(cudaMemcpyAsync(y, h->ds.y, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (x) {
        for (int j = 0; j < n; ++j) x[j] = 0.0;
        for (int p = 0; p < m; ++p)
            if (basis[p] < n) x[basis[p]] = bbar[p];
    }
    if (objective) *objective = h->h_ctrl->z;
    return LP_OK;
}

int lp_get_basis(const lp_handle* h, int32_t* basis) {
    if (!h || !basis) return LP_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(basis, h->ds.basis, sizeof(int32_t) * h->m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_get_state(const lp_handle* h, double* binv, double* bbar) {
    if (!h) return LP_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    if (binv) TRY(binv_rows(h, 0, h->m, binv));
    if (bbar) CK(cudaMemcpyAsync(bbar, h->ds.bbar, sizeof(double) * h->m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_get_trace(const lp_handle* h, int32_t* q, int32_t* r, double* theta, double* dq, int32_t* flags,
                 int32_t cap, int32_t* count) {
    if (!h || cap < 0) return LP_ERR_INVALID_ARG;
    int avail = std::min(h->h_ctrl->it, h->p.trace_cap);
    int k = std::min(avail, cap);
    if (count) *count = k;
    if (k == 0) return LP_OK;
    const TraceBuf& t = h->ds.trace;
    if (q) CK(cudaMemcpyAsync(q, t.q, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, h->stream));
    if (r) CK(cudaMemcpyAsync(r, t.r, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, h->stream));
    if (theta) CK(cudaMemcpyAsync(theta, t.theta, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    if (dq) CK(cudaMemcpyAsync(dq, t.dq, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    if (flags) CK(cudaMemcpyAsync(flags, t.flags, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

void lp_destroy(lp_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"
