// C ABI of libsa and its host runtime: device-resident reference, per-context
// workspaces, the batched and plain execution forms, and the serving loop.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "admission.h"
#include "kernels.h"

using namespace sa;

// ---------------------------------------------------------------------------
// errors

namespace {

// rectangle jobs from which their height walks run over the rectangle list instead of
// one thread per job of the batch (about two waves of warps of the walk kernel)
constexpr uint32_t kListWalkMin = 16384;

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CU(expr)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            cudaGetLastError();                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? SA_ENOMEM : SA_ECUDA,         \
                        "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),         \
                        __FILE__, __LINE__);                                            \
        }                                                                               \
    } while (0)

#define TRY(expr)                     \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != SA_OK) return rc_; \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes, const char* what) {
        if (bytes <= cap && p) return SA_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t nb = std::max<size_t>(bytes + bytes / 8, 1 << 16);
        cudaError_t e = cudaMalloc(&p, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(SA_ENOMEM, "cudaMalloc of %zu bytes for %s failed: %s", nb, what,
                        cudaGetErrorString(e));
        }
        cap = nb;
        return SA_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// layout of the plan block (device, mirrored to pinned host memory)
struct PlanBlock {
    PlanStats st;
    uint32_t hist[kNumKeys];
    uint32_t key_off[kNumKeys + 1];
    uint32_t cursor[kNumKeys];
    uint32_t cfg_begin[kNumCfg + 1];
    uint32_t _pad;
    uint64_t totals[4];
    uint32_t cls_count[kNumCls];   // jobs per direction-pass class (kCls*)
    uint32_t ovf_count[kNumCfg];   // jobs the 16-bit pass sent to the 32-bit rerun, per bucket
    uint32_t rect_begin[kNumCfg + 1];  // each bucket's first job in the rectangle-pass list
};

// Device buffers of one computation at a time (grown on demand, reused).
struct Workspace {
    DevBuf jobs, reads, out, cigar;          // inputs/outputs of the host-buffer entry points
    DevBuf key, order, rpack, state, rect, tb, count, coff, sizes, offs, bsum;
    DevBuf colbest, tmp_ops, arena, plan, counters, blists, band, ovf, lkeys, rsort;
    PlanBlock* h_plan = nullptr;             // pinned mirror of the plan block
    // the score segment (order, packing, score passes, overflow rerun) as a CUDA
    // graph, replayed while a call's launches would be identical (same key)
    cudaGraphExec_t seg_exec = nullptr;
    uint64_t seg_key = 0;
    uint64_t seg_seen = 0;         // the previous call's key: a graph is captured on its second sight
    // side streams, forked from and joined back into the call's stream: one per
    // length bucket for the score passes ([0, kNumCfg)), one per band class
    // ([0, kNumBand)) and one per bucket for the rectangle passes, which run beside
    // the band classes ([kNumBand, kNumBand + kNumCfg))
    static constexpr int kNumSide = kNumBand + kNumCfg;
    cudaStream_t side[kNumSide] = {};
    cudaEvent_t fork = nullptr, join[kNumSide] = {};
    bool side_ok = false;
    cudaEvent_t ev[16] = {};
    bool ev_ok = false;
    DevBuf* all_[25] = {};
    DevBuf* const* bufs(size_t* n) {
        all_[0] = &jobs; all_[1] = &reads; all_[2] = &out; all_[3] = &cigar; all_[4] = &key;
        all_[5] = &order; all_[6] = &rpack; all_[7] = &state; all_[8] = &rect; all_[9] = &tb;
        all_[10] = &count; all_[11] = &coff; all_[12] = &sizes; all_[13] = &offs; all_[14] = &bsum;
        all_[15] = &colbest; all_[16] = &lkeys; all_[17] = &tmp_ops; all_[18] = &arena;
        all_[19] = &plan; all_[20] = &counters; all_[21] = &blists; all_[22] = &band; all_[23] = &ovf;
        all_[24] = &rsort;
        *n = 25;
        return all_;
    }
    // device bytes the workspace holds
    uint64_t bytes() {
        size_t n = 0;
        DevBuf* const* b = bufs(&n);
        uint64_t t = 0;
        for (size_t k = 0; k < n; k++) t += b[k]->cap;
        return t;
    }
    void release() {
        size_t n = 0;
        DevBuf* const* all = bufs(&n);
        for (size_t k = 0; k < n; k++) all[k]->release();
        if (h_plan) cudaFreeHost(h_plan);
        h_plan = nullptr;
        if (seg_exec) cudaGraphExecDestroy(seg_exec);
        seg_exec = nullptr;
        seg_key = 0;
        seg_seen = 0;
        if (side_ok) {
            for (int k = 0; k < kNumSide; k++) {
                cudaStreamDestroy(side[k]);
                cudaEventDestroy(join[k]);
            }
            cudaEventDestroy(fork);
        }
        side_ok = false;
        if (ev_ok)
            for (auto& e : ev) cudaEventDestroy(e);
        ev_ok = false;
    }
};

// What a computation needs: the reference, its plan and a workspace of its own.
struct Ctx {
    const uint32_t* d_words;
    uint64_t len;
    int num_sms;
    Workspace* ws;
    sa_stats* last;
    const Plan* plan;
    const uint8_t* d_plan_cfg;    // device copy of plan->cfg
    // the default plan on fewer lane-group configurations, for batches below
    // kFinePlanJobs (or null: always d_plan_cfg).  Each non-empty configuration
    // is one persistent launch of each pass, run in turn; below about a million
    // jobs the finer row steps split the batch into launches of less than a
    // wave each, whose tails cost more than the padding rows they save.
    const uint8_t* d_plan_coarse = nullptr;
};
constexpr uint32_t kFinePlanJobs = 1u << 20;

// Every read length on the smallest of the configurations with K = 4, 7, 10, ...,
// 28 (8 lanes) or 32 (8 lanes, n <= 256) or the 32-lane ones: the earlier set
// of 14 configurations.
void coarse_plan(Plan* p) {
    default_plan(p);
    for (int n = 1; n <= (int)SA_MAX_READ; n++) {
        int c = p->cfg[n];
        while (cfg_L(c) == 8 && cfg_K(c) != 32 && (cfg_K(c) - 4) % 3 != 0) c++;
        p->cfg[n] = (uint8_t)c;
    }
}

}  // namespace

struct sa_reference {
    int device = 0;
    uint64_t len = 0;
    uint32_t* d_words = nullptr;
    int num_sms = 0;
    cudaStream_t own = nullptr;
    std::mutex mu;
    Workspace ws;
    sa_stats last{};
    Plan plan;
    uint8_t* d_plan_cfg = nullptr;
    uint8_t* d_plan_coarse = nullptr;  // the coarse default plan (small batches)
    bool plan_default = true;          // no plan installed: small batches use d_plan_coarse
    Ctx ctx() {
        return Ctx{d_words, len, num_sms, &ws, &last, &plan, d_plan_cfg, plan_default ? d_plan_coarse : nullptr};
    }
};

// ---------------------------------------------------------------------------
// the computation

namespace {

int check_params(const sa_params* p, Score* sc) {
    TRY(sa::check_scoring(p, sc));
    if (p->width != 0 && p->width != 16 && p->width != 32) return fail(SA_EINVAL, "width must be 0, 16 or 32");
    if (p->form != SA_FORM_BATCHED && p->form != SA_FORM_PLAIN) return fail(SA_EINVAL, "unknown form");
    if (p->arena_mb < 0) return fail(SA_EINVAL, "arena_mb must be >= 0");
    return SA_OK;
}

// The 16-bit packed score pass serves LOCAL alignment of schemes with
// match + B < 1024, B = max(gap open + extend, mismatch): it holds 32 (H + B) in a
// signed 16-bit half, exact below its overflow threshold H + B = 1024 - match (see
// fill16.cuh); jobs that reach the threshold are flagged and recomputed by the
// 32-bit pass, and other schemes run the 32-bit pass.
bool use16(const sa_params* P) {
    if (P->mode != SA_LOCAL || P->width == 32 || P->form == SA_FORM_PLAIN) return false;
    const sa_scoring& s = P->sc;
    const int64_t B = std::max<int64_t>((int64_t)s.gap_open + s.gap_extend, s.mismatch);
    return s.match + B < 1024;
}

int ensure_side(Workspace& ws) {
    if (ws.side_ok) return SA_OK;
    for (int k = 0; k < Workspace::kNumSide; k++) {
        CU(cudaStreamCreateWithFlags(&ws.side[k], cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&ws.join[k], cudaEventDisableTiming));
    }
    CU(cudaEventCreateWithFlags(&ws.fork, cudaEventDisableTiming));
    ws.side_ok = true;
    return SA_OK;
}

int ensure_events(Workspace& ws) {
    if (ws.ev_ok) return SA_OK;
    for (auto& e : ws.ev) CU(cudaEventCreate(&e));
    ws.ev_ok = true;
    return SA_OK;
}

struct Timer {
    Workspace& ws;
    cudaStream_t st;
    bool on;
    int next = 0;
    Timer(Workspace& w, cudaStream_t s, bool enabled) : ws(w), st(s), on(enabled) {}
    int mark() {
        if (!on || next >= 16) return -1;
        cudaEventRecord(ws.ev[next], st);
        return next++;
    }
    // the index a mark recorded inside a replayed graph takes (nothing recorded here)
    int reserve() {
        if (!on || next >= 16) return -1;
        return next++;
    }
    void mark_at(int k) {
        if (k >= 0) cudaEventRecord(ws.ev[k], st);
    }
    float ms(int a, int b) {
        if (!on || a < 0 || b < 0) return 0.f;
        float t = 0.f;
        cudaEventSynchronize(ws.ev[b]);
        cudaEventElapsedTime(&t, ws.ev[a], ws.ev[b]);
        return t;
    }
};

constexpr uint32_t kPlainBatch = 65536;     // jobs per launch of the plain form

// SA_TRACE=1 in the environment: synchronise after each phase and log it to
// stderr with its host time (debugging aid; off by default).
struct Trace {
    bool on;
    cudaStream_t st;
    std::chrono::steady_clock::time_point t0;
    explicit Trace(cudaStream_t s) : on(getenv("SA_TRACE") != nullptr), st(s),
                                     t0(std::chrono::steady_clock::now()) {}
    void operator()(const char* what) {
        if (!on) return;
        const cudaError_t e = cudaStreamSynchronize(st);
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        fprintf(stderr, "[sa] %9.3f ms  %s  (%s)\n", ms, what, cudaGetErrorString(e));
        fflush(stderr);
    }
};
constexpr int kBlock = 128;

// NVTX ranges on the host timeline of a call: one for the call and one per
// phase (a profiler shows them above the phase's launches; free without one)
struct NvtxPhases {
    bool open = false;
    explicit NvtxPhases(const char* call) { nvtxRangePushA(call); }
    void next(const char* phase) {
        if (open) nvtxRangePop();
        nvtxRangePushA(phase);
        open = true;
    }
    ~NvtxPhases() {
        if (open) nvtxRangePop();
        nvtxRangePop();
    }
};

int check_bad_read(PlanBlock* dp, PlanBlock* hp, cudaStream_t st) {
    CU(cudaMemcpyAsync(&hp->st.bad_read, &dp->st.bad_read, 4, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hp->st.bad_read != 0xffffffffu)
        return fail(SA_EINVAL, "job %u: read has a base other than A, C, G, T", hp->st.bad_read);
    return SA_OK;
}

// The whole computation on device buffers.  If grow_cigar is given, the ops
// go to that (grown) buffer instead of d_cigar; cigar_cap still bounds them.
int run_device(Ctx& X, const sa_params* P, const Score& sc, const sa_job* d_jobs, uint32_t n_jobs,
               const char* d_reads, uint64_t reads_len, sa_result* d_out, uint32_t* d_cigar,
               uint64_t cigar_cap, uint64_t* cigar_used, DevBuf* grow_cigar, cudaStream_t st) {
    Workspace& ws = *X.ws;
    sa_stats stats{};
    stats.jobs = n_jobs;
    if (cigar_used) *cigar_used = 0;
    if (n_jobs == 0) {
        *X.last = stats;
        return SA_OK;
    }
    const bool plain = P->form == SA_FORM_PLAIN;
    const bool want_cigar = P->want_cigar != 0;
    const int mode = P->mode;
    const int32_t min_score = P->min_score;
    if (P->profile) TRY(ensure_events(ws));
    Timer tm(ws, st, P->profile != 0);
    Trace trace(st);
    NvtxPhases nvtx("sa_align_batch");
    nvtx.next("plan");
    const int t0 = tm.mark();
    uint32_t launches = 0;

    // --- plan: validation, buckets, statistics
    TRY(ws.plan.ensure(sizeof(PlanBlock), "plan"));
    if (!ws.h_plan) CU(cudaMallocHost((void**)&ws.h_plan, sizeof(PlanBlock)));
    PlanBlock* dp = ws.plan.as<PlanBlock>();
    PlanBlock* hp = ws.h_plan;
    CU(cudaMemsetAsync(dp, 0, sizeof(PlanBlock), st));
    CU(cudaMemsetAsync(&dp->st.bad_job, 0xff, sizeof(uint32_t) * 2, st));
    CU(cudaMemsetAsync(&dp->st.bad_walk, 0xff, 2 * sizeof(uint32_t), st));   // bad_walk, dbg_site
    TRY(ws.key.ensure((size_t)n_jobs * sizeof(uint16_t), "keys"));
    TRY(ws.counters.ensure(256 * sizeof(uint32_t), "counters"));
    CU(cudaMemsetAsync(ws.counters.p, 0, 256 * sizeof(uint32_t), st));
    int counter_next = 0;
    const uint8_t* plan_tab = (X.d_plan_coarse && n_jobs < kFinePlanJobs) ? X.d_plan_coarse : X.d_plan_cfg;
    launch_plan(d_jobs, n_jobs, reads_len, (int64_t)X.len, plan_tab, ws.key.as<uint16_t>(), dp->hist,
                &dp->st, st);
    launches++;
    CU(cudaGetLastError());
    trace("plan");
    CU(cudaMemcpyAsync(hp, dp, offsetof(PlanBlock, key_off), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hp->st.bad_job != 0xffffffffu)
        return fail(SA_EINVAL, "job %u is invalid (read length 1..%u, window 1..%u inside the reference, "
                    "read inside the reads buffer, flags SA_RC only)", hp->st.bad_job, SA_MAX_READ, SA_MAX_WINDOW);
    const uint32_t max_n = hp->st.max_n, max_m = hp->st.max_m;
    stats.cells = hp->st.cells;
    uint32_t cfg_count[kNumCfg], cfg_begin[kNumCfg + 1];
    {
        uint32_t acc = 0;
        for (int c = 0; c < kNumCfg; c++) {
            cfg_begin[c] = acc;
            uint32_t s = 0;
            for (int k = 0; k < kNumSizeCls; k++) s += hp->hist[c * kNumSizeCls + k];
            cfg_count[c] = s;
            acc += s;
        }
        cfg_begin[kNumCfg] = acc;
    }
    const int plain_cfg = cfg_for_rows((int)max_n);

    // --- buffers
    const uint32_t rw = (max_n + 15) / 16;
    TRY(ws.order.ensure((size_t)n_jobs * 4, "order"));
    TRY(ws.rpack.ensure((size_t)n_jobs * rw * 4, "packed reads"));
    TRY(ws.state.ensure((size_t)n_jobs * sizeof(JobState), "job state"));
    TRY(ws.rect.ensure((size_t)n_jobs * sizeof(Rect), "rectangles"));
    TRY(ws.tb.ensure((size_t)n_jobs * sizeof(TbOut), "traceback"));
    TRY(ws.count.ensure((size_t)n_jobs * 4, "cigar counts"));
    TRY(ws.coff.ensure((size_t)n_jobs * 8, "cigar offsets"));
    TRY(ws.sizes.ensure((size_t)n_jobs * 8, "rect sizes"));
    TRY(ws.offs.ensure((size_t)n_jobs * 8, "rect offsets"));
    TRY(ws.bsum.ensure(scan_bsum_len(n_jobs) * 8, "scan"));
    const uint32_t tmp_stride = 2 * max_n + 3;
    if (want_cigar) TRY(ws.tmp_ops.ensure((size_t)n_jobs * tmp_stride * 4, "cigar scratch"));
    CU(cudaMemcpyAsync(dp->cfg_begin, cfg_begin, sizeof(cfg_begin), cudaMemcpyHostToDevice, st));

    // persistent grids: resident 128-thread blocks per SM of each kernel
    auto grid_for = [&](int cfg, int kind) {
        int bps = fill_max_blocks_per_sm(cfg, kind, mode);
        if (bps < 1) bps = 1;
        return X.num_sms * bps;
    };
    // 16-bit pairs per length bucket: when asked for (width 16 in the parameters or
    // the plan), or by default when no job of the bucket can reach the 16-bit
    // threshold (a * rows + B < 1024 - a)
    bool w16[kNumCfg] = {};
    bool any16 = false;
    for (int c = 0; c < kNumCfg; c++) {
        const int64_t rows = (int64_t)cfg_L(c) * cfg_K(c);
        const int64_t B = std::max<int64_t>((int64_t)P->sc.gap_open + P->sc.gap_extend, P->sc.mismatch);
        const bool safe = (int64_t)P->sc.match * (rows + 1) + B < 1024;
        const int pw = X.plan ? X.plan->width[c] : 0;
        const bool want16 = P->width == 16 || (P->width == 0 && (pw == 16 || (pw == 0 && safe)));
        w16[c] = !plain && cfg_count[c] && use16(P) && want16;
        any16 = any16 || w16[c];
    }
    // column slots and lane keys for the lane groups / warps the launches below use
    // (a persistent grid, capped by the items there are).  When the buckets' score
    // passes together fit about two waves of the GPU, they run concurrently (one
    // side stream each; a small batch is otherwise a chain of latency-bound
    // launches) and each bucket gets its own range (cb_group0 / lk_warp0); large
    // batches run them in turn on one range.  The reruns reuse the first range.
    int max_groups = 1, max_grid = 1;
    uint64_t cb_group0[kNumCfg] = {}, lk_warp0[kNumCfg] = {}, groups_total = 0, warps16_total = 0;
    auto blocks_for = [&](int c, int kind, uint64_t jobs, uint32_t jobs_per_warp) {
        const uint64_t warps = (jobs + jobs_per_warp - 1) / jobs_per_warp;
        return (int)std::min<uint64_t>(grid_for(c, kind), (warps + 3) / 4);
    };
    int n_buckets = 0;
    uint64_t blocks_sum = 0;
    for (int c = 0; c < kNumCfg; c++) {
        if (plain || !cfg_count[c]) continue;
        n_buckets++;
        const uint32_t G = 32 / cfg_L(c);
        blocks_sum += w16[c] ? blocks_for(c, kFillScore16, cfg_count[c], 2 * G)
                             : blocks_for(c, kFillScore, cfg_count[c], G);
        max_grid = std::max(max_grid, grid_for(c, w16[c] ? kFillScore16 : kFillScore));
    }
    const bool fork_buckets = !plain && !trace.on && n_buckets > 1 && blocks_sum <= 2ull * max_grid;
    // Large batches run the buckets' score passes in turn on two alternating
    // streams, each with its own scratch range: a persistent launch's blocks leave
    // the SMs one by one as its work runs out, and the next bucket's launch on the
    // other stream takes them, so one bucket's tail overlaps the next one's start.
    const bool pipe_buckets = !plain && !trace.on && !fork_buckets && n_buckets > 1;
    int bucket_lane[kNumCfg] = {};
    {
        int k = 0;
        for (int c = 0; c < kNumCfg; c++)
            if (cfg_count[c]) bucket_lane[c] = pipe_buckets ? (k++ & 1) : 0;
    }
    for (int c = 0; c < kNumCfg; c++) {
        if (plain ? c != plain_cfg : !cfg_count[c]) continue;
        const uint32_t G = 32 / cfg_L(c);
        const uint64_t count = plain ? std::min<uint64_t>(n_jobs, kPlainBatch) : cfg_count[c];
        int blocks = 0, b_score = 0;
        if (plain) {
            blocks = b_score = blocks_for(c, kFillPlain, count, G);
        } else {
            blocks = blocks_for(c, kFillScore, count, G);      // 32-bit pass or the rerun
            b_score = blocks;
            if (w16[c]) {
                b_score = blocks_for(c, kFillScore16, count, 2 * G);
                blocks = std::max(blocks, b_score);
                const uint64_t w16_warps = (uint64_t)b_score * (kBlock / 32);
                lk_warp0[c] = fork_buckets ? warps16_total : 0;
                warps16_total = fork_buckets ? warps16_total + w16_warps : std::max(warps16_total, w16_warps);
            }
        }
        cb_group0[c] = fork_buckets ? groups_total : 0;
        if (fork_buckets) groups_total += (uint64_t)b_score * (kBlock / 32) * G;
        max_groups = std::max(max_groups, blocks * (kBlock / 32) * (int)G);
    }
    groups_total = std::max<uint64_t>(groups_total, (uint64_t)max_groups);
    if (pipe_buckets) {
        // lane 1's ranges follow lane 0's
        for (int c = 0; c < kNumCfg; c++) {
            cb_group0[c] = bucket_lane[c] ? (uint64_t)max_groups : 0;
            lk_warp0[c] = bucket_lane[c] ? warps16_total : 0;
        }
        groups_total = 2 * (uint64_t)max_groups;
        warps16_total *= 2;
    }
    TRY(ws.colbest.ensure(groups_total * cb_words(max_m) * 4, "column maxima"));
    if (any16) TRY(ws.lkeys.ensure(std::max<uint64_t>(warps16_total, 1) * lane_key_words(max_m) * 4, "lane keys"));
    if (fork_buckets || pipe_buckets) TRY(ensure_side(ws));

    FillArgs base{};
    base.ref = X.d_words;
    base.ref_len = (int64_t)X.len;
    base.jobs = d_jobs;
    base.rpack = ws.rpack.as<uint32_t>();
    base.rw = rw;
    base.order = ws.order.as<uint32_t>();
    base.sc = sc;
    base.state = ws.state.as<JobState>();
    base.colbest = ws.colbest.as<int32_t>();
    base.cb_stride = cb_words(max_m);
    base.lane_keys = any16 ? ws.lkeys.as<uint32_t>() : nullptr;
    base.lk_stride = lane_key_words(max_m);
    base.n_state = n_jobs;
    base.cb_cap = ws.colbest.cap / 4;
    base.lk_cap = any16 ? ws.lkeys.cap / 4 : 0;
    base.dbg = &dp->st.dbg_site;
    base.rect = ws.rect.as<Rect>();
    base.wave = 0;
    uint32_t* counters = ws.counters.as<uint32_t>();
    auto next_counter = [&]() { return counters + (counter_next++ % 256); };

    int t1 = -1, tfill1 = -1, tfill16 = -1, trect1 = -1, ttb1 = -1;
    if (plain) {
        launch_iota(ws.order.as<uint32_t>(), n_jobs, st);
        launch_pack_reads(d_jobs, n_jobs, reinterpret_cast<const uint8_t*>(d_reads),
                          ws.rpack.as<uint32_t>(), rw, &dp->st.bad_read, st);
        launches += 2;
        CU(cudaGetLastError());
        trace("order + pack reads");
        t1 = tm.mark();
    }
    if (!plain) {
        nvtx.next("score segment");
        if (any16) TRY(ws.ovf.ensure((size_t)n_jobs * 4, "overflow list"));
        // the score segment: stage (order, packed reads), one persistent score-pass
        // launch per non-empty length bucket (16-bit pairs where chosen), then the
        // 32-bit rerun of the jobs whose maximum reached the 16-bit threshold.  Its
        // launches depend only on `key` below, so without phase timing it is
        // captured once as a CUDA graph and replayed while the key stays the same.
        const int counter_base = counter_next;
        int seg_counters = 0;          // item counters the segment's launches take
        for (int c = 0; c < kNumCfg; c++) {
            if (!cfg_count[c]) continue;
            stats.fill_launches++;
            if (w16[c]) stats.jobs16 += cfg_count[c];
            launches += 1 + (w16[c] ? 1 : 0);
            seg_counters += 1 + (w16[c] ? 1 : 0);
        }
        launches += 3 + (any16 ? 1 : 0);
        t1 = tm.reserve();
        tfill16 = any16 ? tm.reserve() : -1;
        tfill1 = tm.reserve();
        auto issue_segment = [&]() -> int {
        launch_plan_order(ws.key.as<uint16_t>(), n_jobs, dp->hist, dp->key_off, dp->cursor,
                          ws.order.as<uint32_t>(), st);
        launch_pack_reads(d_jobs, n_jobs, reinterpret_cast<const uint8_t*>(d_reads),
                          ws.rpack.as<uint32_t>(), rw, &dp->st.bad_read, st);
        CU(cudaGetLastError());
        trace("order + pack reads");
        tm.mark_at(t1);
        if (fork_buckets || pipe_buckets) CU(cudaEventRecord(ws.fork, st));
        if (pipe_buckets) CU(cudaStreamWaitEvent(ws.side[0], ws.fork, 0));
        for (int c = 0; c < kNumCfg; c++) {
            if (!cfg_count[c]) continue;
            FillLaunch fl{};
            fl.args = base;
            fl.args.pos_begin = cfg_begin[c];
            fl.args.pos_count = cfg_count[c];
            fl.args.item_counter = next_counter();
            // this bucket's own column-slot and lane-key ranges
            fl.args.colbest = base.colbest + cb_group0[c] * base.cb_stride;
            fl.args.cb_cap = base.cb_cap - cb_group0[c] * base.cb_stride;
            if (w16[c]) {
                fl.args.lane_keys = base.lane_keys + lk_warp0[c] * base.lk_stride;
                fl.args.lk_cap = base.lk_cap - lk_warp0[c] * base.lk_stride;
            }
            fl.kind = w16[c] ? kFillScore16 : kFillScore;
            fl.block = kBlock;
            const uint32_t per_warp = (32 / cfg_L(c)) * (w16[c] ? 2 : 1);
            const uint64_t warps_needed = (cfg_count[c] + per_warp - 1) / per_warp;
            fl.grid = (int)std::min<uint64_t>(grid_for(c, fl.kind), (warps_needed + 3) / 4);
            fl.stream = fork_buckets ? ws.side[c] : (bucket_lane[c] ? ws.side[0] : st);
            if (fork_buckets) CU(cudaStreamWaitEvent(ws.side[c], ws.fork, 0));
            launch_fill_cfg(c, fl);
            if (fork_buckets) CU(cudaEventRecord(ws.join[c], ws.side[c]));
            if (trace.on) { char b[64]; snprintf(b, sizeof b, "score pass cfg %d (%u jobs)", c, cfg_count[c]); trace(b); }
        }
        if (fork_buckets)
            for (int c = 0; c < kNumCfg; c++)
                if (cfg_count[c]) CU(cudaStreamWaitEvent(st, ws.join[c], 0));
        if (pipe_buckets) {
            CU(cudaEventRecord(ws.join[0], ws.side[0]));
            CU(cudaStreamWaitEvent(st, ws.join[0], 0));
        }
        CU(cudaGetLastError());
        if (any16) {
            tm.mark_at(tfill16);
            launch_collect_overflow(ws.order.as<uint32_t>(), n_jobs, ws.state.as<JobState>(), dp->cfg_begin,
                                    ws.ovf.as<uint32_t>(), dp->ovf_count, st);
            for (int c = 0; c < kNumCfg; c++) {
                if (!w16[c]) continue;
                FillLaunch fl{};
                fl.args = base;
                fl.args.order = ws.ovf.as<uint32_t>();
                fl.args.pos_begin = cfg_begin[c];
                fl.args.pos_count = 0;
                fl.args.count_ptr = &dp->ovf_count[c];
                fl.args.item_counter = next_counter();
                fl.kind = kFillScore;
                fl.block = kBlock;
                const uint32_t G = 32 / cfg_L(c);
                const uint64_t warps_needed = (cfg_count[c] + G - 1) / G;
                fl.grid = (int)std::min<uint64_t>(grid_for(c, kFillScore), (warps_needed + 3) / 4);
                fl.stream = st;
                launch_fill_cfg(c, fl);
            }
            CU(cudaGetLastError());
            trace("overflow rerun");
        }
        tm.mark_at(tfill1);
        return SA_OK;
        };
        // everything the segment's launches depend on
        uint64_t key = 1469598103934665603ull;
        auto mix = [&](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
        const void* ptrs[] = {d_jobs, d_reads, X.d_words, ws.key.p, ws.order.p, ws.rpack.p, ws.state.p,
                              ws.colbest.p, ws.lkeys.p, ws.ovf.p, ws.counters.p, dp, (const void*)st};
        for (const void* q : ptrs) mix((uint64_t)(uintptr_t)q);
        mix(n_jobs); mix(reads_len); mix(X.len); mix(max_n); mix(max_m); mix((uint64_t)mode);
        mix((uint64_t)(uint32_t)sc.a); mix((uint64_t)(uint32_t)sc.b); mix((uint64_t)(uint32_t)sc.GO);
        mix((uint64_t)(uint32_t)sc.GE);
        for (int c = 0; c < kNumCfg; c++) { mix(cfg_count[c]); mix(w16[c]); }
        mix(tm.on ? 1 : 0);
        if (trace.on || tm.on) {
            // phase timing and tracing run the launches directly (their event
            // records and synchronisations are not graph nodes)
            TRY(issue_segment());
        } else if (ws.seg_exec && ws.seg_key == key) {
            CU(cudaGraphLaunch(ws.seg_exec, st));
            stats.graph_replays++;
        } else if (ws.seg_seen != key) {
            // a key seen once (a one-off batch shape, as in serving) runs directly:
            // capturing and instantiating would cost more than it saves
            ws.seg_seen = key;
            TRY(issue_segment());
        } else {
            if (ws.seg_exec) cudaGraphExecDestroy(ws.seg_exec);
            ws.seg_exec = nullptr;
            ws.seg_key = 0;
            CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const int rc = issue_segment();
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (rc != SA_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            CU(ce);
            const cudaError_t ie = cudaGraphInstantiate(&ws.seg_exec, g, 0);
            cudaGraphDestroy(g);
            CU(ie);
            ws.seg_key = key;
            CU(cudaGraphLaunch(ws.seg_exec, st));
        }
        counter_next = counter_base + seg_counters;

        if (want_cigar) {
            // --- reduced traceback: banded direction pass for most jobs, the
            // wavefront rectangle pass (in arena waves) for wide bands, then the walk
            // band lists, then the compacted list of the rectangle pass's jobs
            TRY(ws.blists.ensure((size_t)n_jobs * (kNumBand + 2) * 4, "band lists"));
            uint32_t* lists[kNumBand];
            for (int k = 0; k < kNumBand; k++) lists[k] = ws.blists.as<uint32_t>() + (size_t)k * n_jobs;
            uint32_t* rect_list = ws.blists.as<uint32_t>() + (size_t)kNumBand * n_jobs;
            uint32_t* rect_list_pos = ws.blists.as<uint32_t>() + (size_t)(kNumBand + 1) * n_jobs;
            nvtx.next("traceback classes");
            // the results' count array serves as the rectangle flags here (the results
            // phase rewrites it)
            uint32_t* rect_flag = ws.count.as<uint32_t>();
            // byte heights instead of nibbles (band and rectangle passes) when LOCAL
            // scores stay below 255
            const bool heights = mode == SA_LOCAL && (int64_t)sc.a * max_n <= 254;
            launch_rect_plan(d_jobs, ws.order.as<uint32_t>(), n_jobs, dp->cfg_begin, ws.state.as<JobState>(), sc,
                             min_score, 1, ws.rect.as<Rect>(), ws.sizes.as<uint64_t>(), lists,
                             dp->cls_count, rect_flag, heights ? 1 : 0, X.d_words, ws.rpack.as<uint32_t>(), rw,
                             st);
            launch_scan_u64(ws.sizes.as<uint64_t>(), n_jobs, ws.offs.as<uint64_t>(),
                            ws.bsum.as<uint64_t>(), &dp->totals[0], st);
            TRY(ws.rsort.ensure(rect_sort_bytes(), "rectangle sort"));
            launch_rect_list(ws.order.as<uint32_t>(), n_jobs, rect_flag, ws.rect.as<Rect>(), ws.rsort.p,
                             ws.bsum.as<uint64_t>(), &dp->totals[2], rect_list, rect_list_pos, dp->rect_begin, st);
            launches += 10;
            CU(cudaGetLastError());
            trace("rect plan + scan");
            CU(cudaMemcpyAsync(&hp->totals[0], &dp->totals[0], 8, cudaMemcpyDeviceToHost, st));
            CU(cudaMemcpyAsync(hp->rect_begin, dp->rect_begin, sizeof(hp->rect_begin), cudaMemcpyDeviceToHost, st));
            CU(cudaMemcpyAsync(hp->cls_count, dp->cls_count, sizeof(hp->cls_count), cudaMemcpyDeviceToHost, st));
            CU(cudaMemcpyAsync(hp->ovf_count, dp->ovf_count, sizeof(hp->ovf_count), cudaMemcpyDeviceToHost, st));
            TRY(check_bad_read(dp, hp, st));
            const uint64_t total_words = hp->totals[0];
            uint32_t nb[kNumBand];
            for (int k = 0; k < kNumBand; k++) nb[k] = hp->cls_count[band_cls(k)];
            stats.diag_jobs = hp->cls_count[kClsDiag];
            stats.band_jobs = nb[0] + nb[1] + nb[2] + nb[3];
            stats.rect_jobs = hp->cls_count[kClsRect];
            for (int c = 0; c < kNumCfg; c++) stats.overflow_reruns += w16[c] ? hp->ovf_count[c] : 0u;
            // band regions: 32 jobs of a class share a region of max_n rows x B/8 words x 32 lanes
            BandLayout bl{};
            uint64_t band_words = 0;
            for (int k = 0; k < kNumBand; k++) {
                bl.warp_stride[k] = (uint64_t)max_n * (band_width_of(k) / (heights ? 4 : 8)) * 32;
                bl.base[k] = band_words;
                band_words += (uint64_t)((nb[k] + 31) / 32) * bl.warp_stride[k];
            }
            TRY(ws.band.ensure(std::max<uint64_t>(band_words, 1) * 4, "band arena"));
            bl.arena = ws.band.as<uint32_t>();
            // the band classes run on side streams, concurrently with each other and
            // with the rectangle pass (independent jobs); joined before the results
            nvtx.next("band and rectangle passes, walks");
            const bool fork = !trace.on && (nb[0] || nb[1] || nb[2] || nb[3]);
            if (fork) {
                TRY(ensure_side(ws));
                CU(cudaEventRecord(ws.fork, st));
            }
            for (int k = 0; k < kNumBand; k++) {
                BandArgs ba{};
                ba.ref = X.d_words;
                ba.ref_len = (int64_t)X.len;
                ba.jobs = d_jobs;
                ba.rpack = ws.rpack.as<uint32_t>();
                ba.rw = rw;
                ba.rect = ws.rect.as<Rect>();
                ba.list = lists[k];
                ba.count = nb[k];
                ba.arena = ws.band.as<uint32_t>() + bl.base[k];
                ba.warp_stride = bl.warp_stride[k];
                ba.sc = sc;
                ba.state = ws.state.as<JobState>();
                ba.tmp_ops = ws.tmp_ops.as<uint32_t>();
                ba.tmp_stride = tmp_stride;
                ba.tb = ws.tb.as<TbOut>();
                ba.err_job = &dp->st.bad_walk;
                ba.region_cap = (uint64_t)((nb[k] + 31) / 32) * bl.warp_stride[k];
                ba.n_state = n_jobs;
                ba.dbg = &dp->st.dbg_site;
                if (ba.count) {
                    if (fork) CU(cudaStreamWaitEvent(ws.side[k], ws.fork, 0));
                    launches += launch_band(band_cls(k), ba, heights, fork ? ws.side[k] : st);
                    if (fork) CU(cudaEventRecord(ws.join[k], ws.side[k]));
                }
            }
            CU(cudaGetLastError());
            trace("band passes");
            // largest item: G jobs of the largest rectangle (bounded by the whole window)
            uint64_t item_max = 0;
            for (int c = 0; c < kNumCfg; c++)
                if (cfg_count[c])
                    item_max = std::max<uint64_t>(item_max, (uint64_t)(32 / cfg_L(c)) *
                                                      rect_words(cfg_L(c), cfg_K(c), (int)max_m, heights));
            size_t free_b = 0, tot_b = 0;
            CU(cudaMemGetInfo(&free_b, &tot_b));
            uint64_t avail = (uint64_t)((double)(free_b + ws.arena.cap) * 0.6) / 4;
            if (P->arena_mb > 0) avail = std::min<uint64_t>(avail, ((uint64_t)P->arena_mb << 20) / 4);
            uint64_t arena_words = total_words ? total_words : 1;
            uint64_t wave_words = 0;   // 0: everything in one wave
            if (arena_words > avail) {
                arena_words = std::max<uint64_t>(avail, 2 * item_max);
                wave_words = arena_words - item_max;
            }
            TRY(ws.arena.ensure(arena_words * 4, "direction arena"));
            launch_rect_assign(ws.order.as<uint32_t>(), rect_list_pos, hp->rect_begin[kNumCfg],
                               ws.offs.as<uint64_t>(), wave_words, ws.rect.as<Rect>(), &dp->st.max_wave, st);
            launches++;
            const uint32_t waves = wave_words ? (uint32_t)((total_words + wave_words - 1) / wave_words) : 1;
            stats.waves = total_words ? waves : 0;
            // small batches: the buckets' rectangle passes run concurrently too (each
            // writes only its jobs' arena ranges); a wave's fork re-records ws.fork,
            // whose earlier waits were already taken
            for (uint32_t wv = 0; wv < waves; wv++) {
                // several buckets with rectangle jobs: their passes run concurrently on
                // the buckets' side streams (a large batch's few long rectangles a bucket
                // leave most of the GPU idle in each launch)
                int rect_buckets = 0;
                for (int c = 0; c < kNumCfg; c++) rect_buckets += hp->rect_begin[c + 1] > hp->rect_begin[c];
                const bool rect_fork = (fork_buckets || rect_buckets > 1) && !trace.on && total_words;
                if (rect_fork) TRY(ensure_side(ws));
                if (rect_fork) CU(cudaEventRecord(ws.fork, st));
                for (int c = 0; c < kNumCfg && total_words; c++) {
                    const uint32_t r0 = hp->rect_begin[c], rn = hp->rect_begin[c + 1] - r0;
                    if (!rn) continue;           // no job of this bucket needs the rectangle
                    FillLaunch fl{};
                    fl.args = base;
                    fl.args.order = rect_list;
                    fl.args.pos_begin = r0;
                    fl.args.pos_count = rn;
                    fl.args.item_counter = next_counter();
                    fl.args.arena = ws.arena.as<uint32_t>();
                    fl.args.arena_cap = ws.arena.cap / 4;
                    fl.args.wave = (int)wv;
                    // byte heights: two jobs a lane group in 16-bit halves when the bucket
                    // has more of them than two full waves of the pair kernel's lane
                    // groups (fewer long rectangles: one job a group, more groups)
                    const bool pairs = heights &&
                        (uint64_t)rn >= 2ull * grid_for(c, kFillRectH16) * (kBlock / 32) * (32 / cfg_L(c)) * 2;
                    fl.kind = pairs ? kFillRectH16 : (heights ? kFillRectH : kFillRect);
                    if (pairs && wv == 0) stats.rect_pairs += rn;
                    fl.block = kBlock;
                    const uint32_t G = (32 / cfg_L(c)) * (pairs ? 2 : 1);
                    const uint64_t warps_needed = (rn + G - 1) / G;
                    fl.grid = (int)std::min<uint64_t>(grid_for(c, fl.kind), (warps_needed + 3) / 4);
                    fl.stream = rect_fork ? ws.side[kNumBand + c] : st;
                    if (rect_fork) CU(cudaStreamWaitEvent(fl.stream, ws.fork, 0));
                    launch_fill_cfg(c, fl);
                    if (rect_fork) CU(cudaEventRecord(ws.join[kNumBand + c], fl.stream));
                    launches++;
                    if (trace.on) { char b[64]; snprintf(b, sizeof b, "rect pass cfg %d wave %u", c, wv); trace(b); }
                }
                if (rect_fork)
                    for (int c = 0; c < kNumCfg; c++)
                        if (hp->rect_begin[c + 1] > hp->rect_begin[c])
                            CU(cudaStreamWaitEvent(st, ws.join[kNumBand + c], 0));
                if (wv == 0) trect1 = tm.mark();
                HeightWalk hwk{heights ? 1 : 0, X.d_words, ws.rpack.as<uint32_t>(), rw, sc};
                const uint32_t n_rect = hp->rect_begin[kNumCfg];
                if (heights && n_rect >= kListWalkMin) {
                    // many rectangle jobs: the height walks one thread per rectangle-list
                    // entry (every lane walks, fewer warps); the rest (gapless jobs) once,
                    // with the first wave.  Few of them walk faster one a warp, in
                    // parallel (low-similarity batch, 286k walks: 3.47 -> 3.2 ms; uneven
                    // batch, 1.8k walks packed: 0.45 -> 0.86 ms)
                    if (wv == 0) {
                        launch_traceback(d_jobs, 0, n_jobs, ws.state.as<JobState>(), ws.rect.as<Rect>(),
                                         ws.arena.as<uint32_t>(), bl, 0, mode, 0, -1, min_score,
                                         ws.tmp_ops.as<uint32_t>(), tmp_stride, ws.tb.as<TbOut>(),
                                         &dp->st.bad_walk, hwk, st, nullptr, 1);
                        launches++;
                    }
                    launch_traceback(d_jobs, 0, n_rect, ws.state.as<JobState>(), ws.rect.as<Rect>(),
                                     ws.arena.as<uint32_t>(), bl, (int)wv, mode, 0, -1, min_score,
                                     ws.tmp_ops.as<uint32_t>(), tmp_stride, ws.tb.as<TbOut>(), &dp->st.bad_walk,
                                     hwk, st, rect_list, 2);
                } else {
                    launch_traceback(d_jobs, 0, n_jobs, ws.state.as<JobState>(), ws.rect.as<Rect>(),
                                     ws.arena.as<uint32_t>(), bl, (int)wv, mode, 0, -1, min_score,
                                     ws.tmp_ops.as<uint32_t>(), tmp_stride, ws.tb.as<TbOut>(), &dp->st.bad_walk,
                                     hwk, st);
                }
                launches++;
                CU(cudaGetLastError());
                trace("traceback");
            }
            if (fork)
                for (int k = 0; k < kNumBand; k++)
                    if (nb[k]) CU(cudaStreamWaitEvent(st, ws.join[k], 0));
            ttb1 = tm.mark();
        } else {
            CU(cudaMemcpyAsync(hp->ovf_count, dp->ovf_count, sizeof(hp->ovf_count), cudaMemcpyDeviceToHost, st));
            TRY(check_bad_read(dp, hp, st));
            for (int c = 0; c < kNumCfg; c++) stats.overflow_reruns += w16[c] ? hp->ovf_count[c] : 0u;
        }
    } else {
        // --- plain form: fixed-size batches in job order, one configuration for the
        // longest read, whole-window direction bits, one fill + one traceback each
        nvtx.next("plain form: fill and traceback batches");
        const int c = plain_cfg;
        const int L = cfg_L(c), K = cfg_K(c);
        const uint32_t G = 32 / L;
        const uint64_t stride = dir_words(L, K, (int)max_m);
        const uint32_t B = std::min(n_jobs, kPlainBatch);
        TRY(ws.arena.ensure((size_t)B * stride * 4, "direction arena"));
        for (uint32_t j0 = 0; j0 < n_jobs; j0 += B) {
            const uint32_t nb = std::min(B, n_jobs - j0);
            launch_plain_rect(d_jobs, j0, nb, stride, ws.rect.as<Rect>(), st);
            FillLaunch fl{};
            fl.args = base;
            fl.args.pos_begin = j0;
            fl.args.pos_count = nb;
            fl.args.item_counter = next_counter();
            fl.args.arena = ws.arena.as<uint32_t>();
            fl.args.arena_cap = ws.arena.cap / 4;
            fl.args.plain = 1;
            fl.kind = kFillPlain;
            fl.block = kBlock;
            const uint64_t warps_needed = (nb + G - 1) / G;
            fl.grid = (int)std::min<uint64_t>(grid_for(c, kFillPlain), (warps_needed + 3) / 4);
            fl.stream = st;
            launch_fill_cfg(c, fl);
            stats.fill_launches++;
            launches += 2;
            if (want_cigar) {
                launch_traceback(d_jobs, j0, nb, ws.state.as<JobState>(), ws.rect.as<Rect>(),
                                 ws.arena.as<uint32_t>(), BandLayout{}, 0, mode, 1, c, min_score,
                                 ws.tmp_ops.as<uint32_t>(), tmp_stride, ws.tb.as<TbOut>(), &dp->st.bad_walk,
                                 HeightWalk{}, st);
                launches++;
            }
            CU(cudaGetLastError());
        }
        tfill1 = tm.mark();
        TRY(check_bad_read(dp, hp, st));
    }

    // --- results
    nvtx.next("results");
    const int tfin0 = tm.mark();
    launch_cigar_count(d_jobs, n_jobs, ws.state.as<JobState>(), ws.tb.as<TbOut>(), mode,
                       want_cigar ? 1 : 0, min_score, ws.count.as<uint32_t>(), st);
    launch_scan_u32(ws.count.as<uint32_t>(), n_jobs, ws.coff.as<uint64_t>(), ws.bsum.as<uint64_t>(),
                    &dp->totals[1], st);
    launches += 4;
    CU(cudaGetLastError());
    trace("cigar count + scan");
    CU(cudaMemcpyAsync(&hp->totals[1], &dp->totals[1], 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&hp->st.bad_walk, &dp->st.bad_walk, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hp->st.dbg_site != 0xffffffffu)
        return fail(SA_ECUDA, "internal error: a kernel store was out of range (bounds-checked build, "
                    "store site %u)", hp->st.dbg_site);
    if (hp->st.bad_walk != 0xffffffffu)
        return fail(SA_ECUDA, "internal error: the traceback of job %u left its direction-bit rectangle",
                    hp->st.bad_walk);
    const uint64_t ops_total = hp->totals[1];
    if (cigar_used) *cigar_used = ops_total;
    if (ops_total > cigar_cap)
        return fail(SA_EOVERFLOW, "CIGAR buffer holds %llu ops, %llu needed",
                    (unsigned long long)cigar_cap, (unsigned long long)ops_total);
    if (ops_total > 0xffffffffull)
        return fail(SA_EOVERFLOW, "more than 2^32 CIGAR ops in one call; split the batch");
    uint32_t* dst = d_cigar;
    if (grow_cigar) {
        TRY(grow_cigar->ensure(ops_total * 4 + 4, "cigar"));
        dst = grow_cigar->as<uint32_t>();
    } else if (ops_total && !dst) {
        return fail(SA_EOVERFLOW, "no CIGAR buffer, %llu ops needed", (unsigned long long)ops_total);
    }
    launch_finalize(d_jobs, n_jobs, ws.state.as<JobState>(), ws.tb.as<TbOut>(),
                    ws.count.as<uint32_t>(), ws.coff.as<uint64_t>(), ws.tmp_ops.as<uint32_t>(),
                    tmp_stride, mode, want_cigar ? 1 : 0, min_score, d_out, dst, st);
    launches++;
    CU(cudaGetLastError());
    trace("finalize");
    const int tfin1 = tm.mark();
    CU(cudaStreamSynchronize(st));
    stats.kernel_launches = launches;
    if (P->profile) {
        stats.ms_stage = tm.ms(t0, t1);
        stats.ms_fill = tm.ms(t1, tfill16 >= 0 ? tfill16 : tfill1);
        stats.ms_rerun = tfill16 >= 0 ? tm.ms(tfill16, tfill1) : 0.f;
        // classification and the rectangle pass (the band passes run alongside on
        // side streams); then the rectangle walks and the join with the band passes
        stats.ms_rect = tm.ms(tfill1, trect1);
        stats.ms_traceback = tm.ms(trect1, ttb1);
        stats.ms_finalize = tm.ms(tfin0, tfin1);
        stats.ms_total = tm.ms(t0, tfin1);
    }
    *X.last = stats;
    return SA_OK;
}

// Host-buffer form on top of run_device: copy in, compute, copy out.
int run_host(Ctx& X, const sa_params* P, const Score& sc, const sa_job* jobs, uint32_t n_jobs,
             const char* reads, uint64_t reads_len, sa_result* out, uint32_t* cigar,
             uint64_t cigar_cap, uint64_t* cigar_used, cudaStream_t st) {
    Workspace& ws = *X.ws;
    if (cigar_used) *cigar_used = 0;
    if (n_jobs == 0) return SA_OK;
    TRY(ws.jobs.ensure((size_t)n_jobs * sizeof(sa_job), "jobs"));
    TRY(ws.reads.ensure(reads_len + 16, "reads"));
    TRY(ws.out.ensure((size_t)n_jobs * sizeof(sa_result), "results"));
    CU(cudaMemcpyAsync(ws.jobs.p, jobs, (size_t)n_jobs * sizeof(sa_job), cudaMemcpyHostToDevice, st));
    if (reads_len) CU(cudaMemcpyAsync(ws.reads.p, reads, reads_len, cudaMemcpyHostToDevice, st));
    uint64_t used = 0;
    const int rc = run_device(X, P, sc, ws.jobs.as<sa_job>(), n_jobs, ws.reads.as<char>(), reads_len,
                              ws.out.as<sa_result>(), nullptr, cigar_cap, &used, &ws.cigar, st);
    if (cigar_used) *cigar_used = used;
    if (rc != SA_OK) return rc;
    if (used && !cigar) return fail(SA_EOVERFLOW, "cigar is NULL, %llu ops needed", (unsigned long long)used);
    CU(cudaMemcpyAsync(out, ws.out.p, (size_t)n_jobs * sizeof(sa_result), cudaMemcpyDeviceToHost, st));
    if (used) CU(cudaMemcpyAsync(cigar, ws.cigar.p, used * 4, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return SA_OK;
}

cudaStream_t pick_stream(sa_reference* R, void* s) {
    return s ? static_cast<cudaStream_t>(s) : R->own;
}

}  // namespace

// ---------------------------------------------------------------------------
// serving

namespace {

struct Request {
    uint64_t ticket = 0;
    std::vector<sa_job> jobs;
    std::vector<char> reads;
    uint64_t est_bytes = 0;
    int rc = SA_PENDING;
    std::string err;
    std::vector<sa_result> out;
    std::vector<uint32_t> cigar;
};

}  // namespace

struct sa_server {
    sa_reference* ref = nullptr;
    sa_params params{};
    Score sc{};
    uint64_t budget = 0;
    uint64_t in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    sa_server_stats counters{};        // guarded by mu
    struct Slot {
        Workspace ws;
        sa_stats last{};
        cudaStream_t stream = nullptr;
        std::thread th;
        uint64_t held = 0;             // device bytes its workspace holds (guarded by mu)
    };
    std::vector<std::unique_ptr<Slot>> slots;
};

namespace {

// Device memory one request needs while it runs: per-job workspace (job, result,
// state, rectangle, plan and scan entries, packed read, CIGAR scratch of 2n+3
// ops), the band regions at their widest (64 diagonals: 8 words a row), and the
// wavefront-rectangle arena, which runs in waves and is charged at most 4 GB.
uint64_t estimate_bytes(const sa_job* jobs, uint32_t n, uint64_t reads_len) {
    uint64_t b = reads_len + (uint64_t)n * (sizeof(sa_job) + sizeof(sa_result) + 256);
    uint64_t rect = 0;
    for (uint32_t k = 0; k < n; k++) {
        const uint32_t rn = std::max(std::min(jobs[k].read_len, SA_MAX_READ), 1u);
        const uint32_t m = std::min(jobs[k].win_len, SA_MAX_WINDOW);
        const int c = cfg_for_rows((int)rn);
        b += (uint64_t)4 * ((rn + 15) / 16) + (uint64_t)4 * (2 * rn + 3) + (uint64_t)32 * rn;
        rect += 4 * dir_words(cfg_L(c), cfg_K(c), (int)m);
    }
    return b + std::min<uint64_t>(rect, 4ull << 30);
}

// Pinned host staging buffer of a server slot (grown on demand).
struct PinnedBuf {
    void* p = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes) {
        if (bytes <= cap && p) return true;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t nb = std::max<size_t>(bytes + bytes / 2, 1 << 16);
        if (cudaHostAlloc(&p, nb, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        cap = nb;
        return true;
    }
    ~PinnedBuf() {
        if (p) cudaFreeHost(p);
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Jobs of one coalesced device batch at most.
constexpr uint64_t kCoalesceJobs = 1ull << 20;

// Runs the requests of `batch` as one device batch: jobs concatenated (read
// offsets rebased) in pinned staging, results and CIGAR ops split back per
// request.  The CIGAR staging is sized by the ops actually produced.
// Runs fn(k) for k in [0, n) on up to `threads` host threads (the calling one
// included); the staging copies of a large coalesced batch are memory-bandwidth
// bound and one thread leaves most of the host's bandwidth idle.
template <typename F>
void parallel_for(size_t n, unsigned threads, F&& fn) {
    threads = (unsigned)std::min<size_t>(threads, n);
    if (threads <= 1) {
        for (size_t k = 0; k < n; k++) fn(k);
        return;
    }
    std::atomic<size_t> next{0};
    std::atomic<bool> failed{false};
    auto worker = [&] {
        try {
            for (size_t k = next++; k < n; k = next++) fn(k);
        } catch (...) {
            failed = true;                 // reported to the caller after the join
            next = n;
        }
    };
    std::vector<std::thread> pool;
    pool.reserve(threads - 1);
    for (unsigned t = 1; t < threads; t++) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    if (failed) throw std::bad_alloc();
}

unsigned staging_threads(uint64_t bytes) {
    if (bytes < (16ull << 20)) return 1;                       // small batches: one thread
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    return std::min(8u, std::max(1u, hw / 2));
}

int run_batch(sa_server* S, sa_server::Slot* slot, std::vector<std::shared_ptr<Request>>& batch,
              PinnedBuf& hjobs, PinnedBuf& hreads, PinnedBuf& hout, PinnedBuf& hcig) {
    uint64_t nj = 0, nr = 0, cap = 0;
    for (auto& rq : batch) {
        nj += rq->jobs.size();
        nr += rq->reads.size();
        for (const sa_job& j : rq->jobs) cap += 2ull * j.read_len + 3;   // 2n+3 ops bound every job
    }
    if (!hjobs.ensure(nj * sizeof(sa_job)) || !hreads.ensure(nr + 16) || !hout.ensure(nj * sizeof(sa_result)))
        return fail(SA_ENOMEM, "pinned staging allocation failed");
    sa_job* J = hjobs.as<sa_job>();
    char* Rd = hreads.as<char>();
    // each request's jobs and reads go to their own ranges of the staging buffers
    std::vector<uint64_t> job0(batch.size()), read0(batch.size());
    {
        uint64_t jo = 0, ro = 0;
        for (size_t k = 0; k < batch.size(); k++) {
            job0[k] = jo;
            read0[k] = ro;
            jo += batch[k]->jobs.size();
            ro += batch[k]->reads.size();
        }
    }
    const unsigned nthreads = staging_threads(nj * sizeof(sa_job) + nr);
    parallel_for(batch.size(), nthreads, [&](size_t k) {
        const Request& rq = *batch[k];
        sa_job* dst = J + job0[k];
        for (size_t q = 0; q < rq.jobs.size(); q++) {
            dst[q] = rq.jobs[q];
            dst[q].read_off += read0[k];
        }
        if (!rq.reads.empty()) std::memcpy(Rd + read0[k], rq.reads.data(), rq.reads.size());
    });
    Workspace& ws = slot->ws;
    const cudaStream_t st = slot->stream;
    Ctx X{S->ref->d_words, S->ref->len, S->ref->num_sms, &ws, &slot->last, &S->ref->plan,
          S->ref->d_plan_cfg, S->ref->plan_default ? S->ref->d_plan_coarse : nullptr};
    uint64_t used = 0;
    if (nj) {
        TRY(ws.jobs.ensure(nj * sizeof(sa_job), "jobs"));
        TRY(ws.reads.ensure(nr + 16, "reads"));
        TRY(ws.out.ensure(nj * sizeof(sa_result), "results"));
        CU(cudaMemcpyAsync(ws.jobs.p, J, nj * sizeof(sa_job), cudaMemcpyHostToDevice, st));
        if (nr) CU(cudaMemcpyAsync(ws.reads.p, Rd, nr, cudaMemcpyHostToDevice, st));
        TRY(run_device(X, &S->params, S->sc, ws.jobs.as<sa_job>(), (uint32_t)nj, ws.reads.as<char>(), nr,
                       ws.out.as<sa_result>(), nullptr, cap, &used, &ws.cigar, st));
        if (!hcig.ensure(std::max<uint64_t>(used, 1) * 4)) return fail(SA_ENOMEM, "pinned staging allocation failed");
        CU(cudaMemcpyAsync(hout.p, ws.out.p, nj * sizeof(sa_result), cudaMemcpyDeviceToHost, st));
        if (used) CU(cudaMemcpyAsync(hcig.p, ws.cigar.p, used * 4, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
    }
    const sa_result* O = hout.as<sa_result>();
    const uint32_t* C = hcig.as<uint32_t>();
    parallel_for(batch.size(), staging_threads(nj * sizeof(sa_result) + used * 4), [&](size_t k) {
        Request& rq = *batch[k];
        const uint64_t b = job0[k], n = rq.jobs.size();
        rq.out.assign(O + b, O + b + n);
        uint64_t c0 = 0, c1 = 0;
        if (n) {
            c0 = O[b].cigar_off;
            c1 = (uint64_t)O[b + n - 1].cigar_off + O[b + n - 1].cigar_len;
        }
        rq.cigar.assign(C + c0, C + c1);
        for (sa_result& r : rq.out) r.cigar_off -= (uint32_t)c0;
    });
    return SA_OK;
}

void slot_main(sa_server* S, sa_server::Slot* slot) {
    cudaSetDevice(S->ref->device);
    PinnedBuf hjobs, hreads, hout, hcig;
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        uint64_t est = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // FIFO admission (admission.h): the head request starts when the memory
            // it needs fits; the requests queued behind it join its device batch
            // while they fit.  The memory is re-read for every decision, and a head
            // request that does not fit looks again every few milliseconds (device
            // memory can come free outside the server, with no notification).
            bool stalled = false;      // the head request waited for memory
            size_t take = 0;
            auto view = [](const std::shared_ptr<Request>& q) {
                return std::make_pair((uint64_t)q->jobs.size(), q->est_bytes);
            };
            for (;;) {
                if (S->stop) return;
                if (S->queue.empty()) {
                    S->cv_work.wait(lk);
                    continue;
                }
                size_t fr = 0, tot = 0;
                if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
                    cudaGetLastError();
                    fr = 0;
                }
                uint64_t held = 0;
                for (auto& sl : S->slots) held += sl->held;
                const uint64_t cap = admission_cap(S->budget, (uint64_t)fr, held);
                take = admit_front(S->queue, view, S->in_use, cap, kCoalesceJobs, &est);
                if (take) break;
                stalled = true;
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
            }
            if (stalled) S->counters.admission_stalls++;
            uint64_t nj = 0;
            for (size_t k = 0; k < take; k++) {
                nj += S->queue.front()->jobs.size();
                batch.push_back(S->queue.front());
                S->queue.pop_front();
            }
            S->in_use += est;
            S->counters.batches++;
            S->counters.coalesced += batch.size() - 1;
            S->counters.jobs += nj;
        }
        int rc;
        try {
            rc = run_batch(S, slot, batch, hjobs, hreads, hout, hcig);
        } catch (...) {
            rc = fail(SA_ENOMEM, "host memory exhausted while staging a batch");
        }
        std::vector<int> rcs(batch.size(), rc);
        std::vector<std::string> msgs(batch.size(), rc == SA_OK ? std::string() : std::string(g_err));
        if (rc != SA_OK && batch.size() > 1) {
            // one request's error (an invalid job) must not fail its batch mates
            for (size_t k = 0; k < batch.size(); k++) {
                std::vector<std::shared_ptr<Request>> one{batch[k]};
                try {
                    rcs[k] = run_batch(S, slot, one, hjobs, hreads, hout, hcig);
                } catch (...) {
                    rcs[k] = fail(SA_ENOMEM, "host memory exhausted while staging a request");
                }
                msgs[k] = rcs[k] == SA_OK ? std::string() : std::string(g_err);
            }
        }
        const uint64_t held_now = slot->ws.bytes();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= est;
            slot->held = held_now;
            for (size_t k = 0; k < batch.size(); k++) {
                Request& rq = *batch[k];
                rq.err = msgs[k];
                rq.rc = rcs[k];
                if (rcs[k] == SA_OK) S->counters.completed++;
                else S->counters.failed++;
                rq.jobs.clear();
                rq.jobs.shrink_to_fit();
                rq.reads.clear();
                rq.reads.shrink_to_fit();
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char* sa_last_error(void) { return g_err; }

void sa_default_params(sa_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->sc.match = 1;
    p->sc.mismatch = 2;
    p->sc.gap_open = 2;
    p->sc.gap_extend = 1;
    p->mode = SA_LOCAL;
    p->want_cigar = 1;
    p->width = 0;
    p->min_score = INT32_MIN;
    p->form = SA_FORM_BATCHED;
    p->profile = 0;
}

int sa_create_reference(const char* acgt, uint64_t len, int device, sa_reference** out) {
    try {
        g_err[0] = 0;
        if (!out) return fail(SA_EINVAL, "out is NULL");
        *out = nullptr;
        if (!acgt) return fail(SA_EINVAL, "acgt is NULL");
        if (len == 0) return fail(SA_EINVAL, "empty reference");
        int ndev = 0;
        CU(cudaGetDeviceCount(&ndev));
        if (device < 0 || device >= ndev) return fail(SA_EINVAL, "device %d not present (%d devices)", device, ndev);
        CU(cudaSetDevice(device));
        std::unique_ptr<sa_reference> R(new (std::nothrow) sa_reference());
        if (!R) return fail(SA_ENOMEM, "host allocation failed");
        R->device = device;
        R->len = len;
        CU(cudaDeviceGetAttribute(&R->num_sms, cudaDevAttrMultiProcessorCount, device));
        CU(cudaStreamCreateWithFlags(&R->own, cudaStreamNonBlocking));
        const uint64_t words = (len + 15) / 16 + kRefFrontPad + kRefTailPad;
        CU(cudaMalloc(&R->d_words, words * 4));
        default_plan(&R->plan);
        CU(cudaMalloc(&R->d_plan_cfg, sizeof(R->plan.cfg)));
        CU(cudaMemcpy(R->d_plan_cfg, R->plan.cfg, sizeof(R->plan.cfg), cudaMemcpyHostToDevice));
        {
            Plan coarse;
            coarse_plan(&coarse);
            CU(cudaMalloc(&R->d_plan_coarse, sizeof(coarse.cfg)));
            CU(cudaMemcpy(R->d_plan_coarse, coarse.cfg, sizeof(coarse.cfg), cudaMemcpyHostToDevice));
        }
        CU(cudaMemsetAsync(R->d_words, 0, words * 4, R->own));
        const uint64_t chunk = 256ull << 20;  // multiple of 16
        uint8_t* stage = nullptr;
        unsigned long long* bad = nullptr;
        int rc = SA_OK;
        unsigned long long hbad = ~0ull;
        if (cudaMalloc(&stage, std::min<uint64_t>(chunk, len)) != cudaSuccess ||
            cudaMalloc(&bad, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(SA_ENOMEM, "staging allocation failed");
        }
        if (rc == SA_OK) {
            cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), R->own);
            for (uint64_t off = 0; off < len && rc == SA_OK; off += chunk) {
                const uint64_t sz = std::min(chunk, len - off);
                if (cudaMemcpyAsync(stage, acgt + off, sz, cudaMemcpyHostToDevice, R->own) != cudaSuccess)
                    rc = fail(SA_ECUDA, "reference upload failed");
                launch_pack_ref(stage, sz, off, R->d_words + kRefFrontPad, bad, R->own);
            }
            cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, R->own);
            const cudaError_t e = cudaStreamSynchronize(R->own);
            if (rc == SA_OK && e != cudaSuccess) rc = fail(SA_ECUDA, "reference packing failed: %s", cudaGetErrorString(e));
        }
        if (stage) cudaFree(stage);
        if (bad) cudaFree(bad);
        if (rc == SA_OK && hbad != ~0ull) rc = fail(SA_EINVAL, "reference position %llu is not A, C, G or T", hbad);
        if (rc != SA_OK) {
            cudaFree(R->d_words);
            cudaStreamDestroy(R->own);
            return rc;
        }
        *out = R.release();
        return SA_OK;
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

int sa_destroy_reference(sa_reference* R) {
    if (!R) return fail(SA_EINVAL, "reference is NULL");
    try {
        cudaSetDevice(R->device);
        {
            std::lock_guard<std::mutex> lk(R->mu);
            cudaStreamSynchronize(R->own);
            R->ws.release();
            cudaFree(R->d_words);
            cudaFree(R->d_plan_cfg);
            cudaFree(R->d_plan_coarse);
            cudaStreamDestroy(R->own);
        }
        delete R;
        return SA_OK;
    } catch (...) {
        return fail(SA_ECUDA, "unexpected host exception");
    }
}

uint64_t sa_reference_length(const sa_reference* R) { return R ? R->len : 0; }

int sa_last_stats(const sa_reference* R, sa_stats* out) {
    if (!R || !out) return fail(SA_EINVAL, "NULL argument");
    *out = R->last;
    return SA_OK;
}

int sa_align_batch_dev(sa_reference* R, const sa_params* P, const sa_job* d_jobs, uint32_t n_jobs,
                       const char* d_reads, uint64_t reads_len, sa_result* d_out, uint32_t* d_cigar,
                       uint64_t cigar_cap, uint64_t* cigar_used, void* stream) {
    try {
        g_err[0] = 0;
        if (!R) return fail(SA_EINVAL, "reference is NULL");
        Score sc;
        TRY(check_params(P, &sc));
        if (n_jobs && (!d_jobs || !d_out)) return fail(SA_EINVAL, "NULL job or result buffer");
        if (n_jobs && !d_reads) return fail(SA_EINVAL, "reads is NULL");
        std::lock_guard<std::mutex> lk(R->mu);
        CU(cudaSetDevice(R->device));
        Ctx X = R->ctx();
        return run_device(X, P, sc, d_jobs, n_jobs, d_reads, reads_len, d_out, d_cigar, cigar_cap,
                          cigar_used, nullptr, pick_stream(R, stream));
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

int sa_align_batch(sa_reference* R, const sa_params* P, const sa_job* jobs, uint32_t n_jobs,
                   const char* reads, uint64_t reads_len, sa_result* out, uint32_t* cigar,
                   uint64_t cigar_cap, uint64_t* cigar_used, void* stream) {
    try {
        g_err[0] = 0;
        if (!R) return fail(SA_EINVAL, "reference is NULL");
        Score sc;
        TRY(check_params(P, &sc));
        if (n_jobs && (!jobs || !out)) return fail(SA_EINVAL, "NULL job or result buffer");
        if (n_jobs && !reads) return fail(SA_EINVAL, "reads is NULL");
        std::lock_guard<std::mutex> lk(R->mu);
        CU(cudaSetDevice(R->device));
        Ctx X = R->ctx();
        return run_host(X, P, sc, jobs, n_jobs, reads, reads_len, out, cigar, cigar_cap, cigar_used,
                        pick_stream(R, stream));
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

// ---------------------------------------------------------------------------
// tuned plan

namespace {

constexpr uint32_t kPlanMagic = 0x4C504153u;   // "SAPL"
constexpr uint32_t kPlanVersion = 2u;   // 2: 33 configurations
constexpr uint64_t kPlanBytes = 8 + sizeof(Plan::cfg) + sizeof(Plan::width);

int upload_plan(sa_reference* R) {
    CU(cudaMemcpy(R->d_plan_cfg, R->plan.cfg, sizeof(R->plan.cfg), cudaMemcpyHostToDevice));
    return SA_OK;
}

// Score-pass time (ms) of `jobs` under `trial`, second of two runs.
int time_trial(sa_reference* R, const sa_params* P, const Score& sc, const Plan& trial, uint8_t* d_cfg,
               const sa_job* jobs, uint32_t n, const char* reads, uint64_t reads_len, float* ms) {
    CU(cudaMemcpy(d_cfg, trial.cfg, sizeof(trial.cfg), cudaMemcpyHostToDevice));
    sa_params q = *P;
    q.want_cigar = 0;
    q.profile = 1;
    q.width = 0;
    Ctx X{R->d_words, R->len, R->num_sms, &R->ws, &R->last, &trial, d_cfg};
    std::vector<sa_result> out(n);
    for (int rep = 0; rep < 2; rep++)
        TRY(run_host(X, &q, sc, jobs, n, reads, reads_len, out.data(), nullptr, 0, nullptr, R->own));
    *ms = R->last.ms_fill + R->last.ms_rerun;
    return SA_OK;
}

}  // namespace

int sa_tune(sa_reference* R, const sa_params* P, const sa_job* jobs, uint32_t n_jobs, const char* reads,
            uint64_t reads_len, uint32_t* classes_tuned) {
    try {
        g_err[0] = 0;
        if (!R) return fail(SA_EINVAL, "reference is NULL");
        Score sc;
        TRY(check_params(P, &sc));
        if (n_jobs && (!jobs || !reads)) return fail(SA_EINVAL, "NULL jobs or reads");
        if (classes_tuned) *classes_tuned = 0;
        std::lock_guard<std::mutex> lk(R->mu);
        CU(cudaSetDevice(R->device));
        uint8_t* d_cfg = nullptr;
        CU(cudaMalloc(&d_cfg, sizeof(Plan::cfg)));
        struct Free { uint8_t* p; ~Free() { cudaFree(p); } } guard{d_cfg};
        const bool local16 = P->mode == SA_LOCAL && use16(P);
        uint32_t tuned = 0;
        for (int c0 = 0; c0 < kNumCfg; c0++) {
            // the length class that the default plan gives to configuration c0
            std::vector<uint32_t> idx;
            for (uint32_t k = 0; k < n_jobs && idx.size() < 65536; k++) {
                const uint32_t n = jobs[k].read_len;
                if (n >= 1 && n <= SA_MAX_READ && cfg_for_rows((int)n) == c0) idx.push_back(k);
            }
            if (idx.size() < 256) continue;
            // the timed batch repeats the class's jobs up to 2^18, so that every
            // candidate's persistent grid runs many items per lane group (a batch
            // of one item per group would time the tail, not the kernel)
            const size_t distinct = idx.size();
            while (idx.size() < (1u << 18)) idx.push_back(idx[idx.size() % distinct]);
            std::vector<sa_job> sj(idx.size());
            std::vector<char> sr;
            for (size_t t = 0; t < idx.size(); t++) {
                sj[t] = jobs[idx[t]];
                if (sj[t].read_off + sj[t].read_len > reads_len)
                    return fail(SA_EINVAL, "job %u: read outside the reads buffer", idx[t]);
                sj[t].read_off = sr.size();
                sr.insert(sr.end(), reads + jobs[idx[t]].read_off, reads + jobs[idx[t]].read_off + sj[t].read_len);
            }
            // candidates: c0, the next K with the same lane count, the first 32-lane
            // configuration that covers the class; 16- and 32-bit where 16-bit applies
            std::vector<int> cands{c0};
            if (c0 + 1 < kNumCfg && cfg_L(c0 + 1) == cfg_L(c0)) cands.push_back(c0 + 1);
            if (cfg_L(c0) == 8)
                for (int c = 0; c < kNumCfg; c++)
                    if (cfg_L(c) == 32 && cfg_L(c) * cfg_K(c) >= cfg_L(c0) * cfg_K(c0)) { cands.push_back(c); break; }
            std::vector<int> widths = local16 ? std::vector<int>{16, 32} : std::vector<int>{32};
            // the default (c0, automatic width) is timed first and kept unless a
            // candidate is more than 2 % faster
            float best_ms = 0.f;
            int best_c = c0, best_w = 0;
            {
                Plan trial = R->plan;
                for (int n = 1; n <= SA_MAX_READ; n++)
                    if (cfg_for_rows(n) == c0) trial.cfg[n] = (uint8_t)c0;
                trial.width[c0] = 0;
                TRY(time_trial(R, P, sc, trial, d_cfg, sj.data(), (uint32_t)sj.size(), sr.data(), sr.size(), &best_ms));
            }
            const float bar = 0.98f * best_ms;
            float cand_ms = bar;
            for (int c : cands) {
                for (int w : widths) {
                    Plan trial = R->plan;
                    for (int n = 1; n <= SA_MAX_READ; n++)
                        if (cfg_for_rows(n) == c0) trial.cfg[n] = (uint8_t)c;
                    trial.width[c] = (int8_t)w;
                    float ms = 0.f;
                    TRY(time_trial(R, P, sc, trial, d_cfg, sj.data(), (uint32_t)sj.size(), sr.data(), sr.size(), &ms));
                    if (ms < cand_ms) { cand_ms = ms; best_c = c; best_w = w; }
                }
            }
            for (int n = 1; n <= SA_MAX_READ; n++)
                if (cfg_for_rows(n) == c0) R->plan.cfg[n] = (uint8_t)best_c;
            R->plan.width[best_c] = (int8_t)(local16 ? best_w : 0);
            tuned++;
        }
        R->plan_default = false;           // the tuned plan serves every batch size
        TRY(upload_plan(R));
        if (classes_tuned) *classes_tuned = tuned;
        return SA_OK;
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

int sa_plan_get(const sa_reference* R, void* out, uint64_t size, uint64_t* needed) {
    if (!R) return fail(SA_EINVAL, "reference is NULL");
    if (needed) *needed = kPlanBytes;
    if (!out || size < kPlanBytes) return fail(SA_EOVERFLOW, "the plan needs %llu bytes", (unsigned long long)kPlanBytes);
    uint8_t* o = static_cast<uint8_t*>(out);
    std::memcpy(o, &kPlanMagic, 4);
    std::memcpy(o + 4, &kPlanVersion, 4);
    std::memcpy(o + 8, R->plan.cfg, sizeof(Plan::cfg));
    std::memcpy(o + 8 + sizeof(Plan::cfg), R->plan.width, sizeof(Plan::width));
    return SA_OK;
}

int sa_plan_set(sa_reference* R, const void* plan, uint64_t size) {
    try {
        g_err[0] = 0;
        if (!R) return fail(SA_EINVAL, "reference is NULL");
        if (!plan) {
            std::lock_guard<std::mutex> lk(R->mu);
            CU(cudaSetDevice(R->device));
            default_plan(&R->plan);
            R->plan_default = true;
            return upload_plan(R);
        }
        if (size != kPlanBytes) return fail(SA_EINVAL, "a plan has %llu bytes, got %llu",
                                            (unsigned long long)kPlanBytes, (unsigned long long)size);
        const uint8_t* b = static_cast<const uint8_t*>(plan);
        uint32_t magic = 0, version = 0;
        std::memcpy(&magic, b, 4);
        std::memcpy(&version, b + 4, 4);
        if (magic != kPlanMagic || version != kPlanVersion) return fail(SA_EINVAL, "not a plan of this version");
        Plan p;
        std::memcpy(p.cfg, b + 8, sizeof(Plan::cfg));
        std::memcpy(p.width, b + 8 + sizeof(Plan::cfg), sizeof(Plan::width));
        p.cfg[0] = (uint8_t)cfg_for_rows(1);
        if (!plan_valid(p)) return fail(SA_EINVAL, "invalid plan: a read length mapped to a configuration "
                                        "with fewer rows, or a width other than 0, 16, 32");
        std::lock_guard<std::mutex> lk(R->mu);
        CU(cudaSetDevice(R->device));
        R->plan = p;
        R->plan_default = false;
        return upload_plan(R);
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

int sa_server_create(sa_reference* R, const sa_params* P, uint64_t hbm_budget, uint32_t max_inflight,
                     sa_server** out) {
    try {
        g_err[0] = 0;
        if (!R || !out) return fail(SA_EINVAL, "NULL argument");
        *out = nullptr;
        Score sc;
        TRY(check_params(P, &sc));
        CU(cudaSetDevice(R->device));
        if (hbm_budget == 0) {
            size_t fr = 0, tot = 0;
            CU(cudaMemGetInfo(&fr, &tot));
            hbm_budget = (uint64_t)(0.8 * (double)fr);
        }
        if (max_inflight == 0) max_inflight = 4;
        if (max_inflight > 64) return fail(SA_EINVAL, "max_inflight must be <= 64");
        std::unique_ptr<sa_server> S(new (std::nothrow) sa_server());
        if (!S) return fail(SA_ENOMEM, "host allocation failed");
        S->ref = R;
        S->params = *P;
        S->params.profile = 0;
        S->sc = sc;
        S->budget = hbm_budget;
        for (uint32_t k = 0; k < max_inflight; k++) {
            auto slot = std::make_unique<sa_server::Slot>();
            CU(cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking));
            S->slots.push_back(std::move(slot));
        }
        for (auto& slot : S->slots) slot->th = std::thread(slot_main, S.get(), slot.get());
        *out = S.release();
        return SA_OK;
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

int sa_submit(sa_server* S, const sa_job* jobs, uint32_t n_jobs, const char* reads, uint64_t reads_len,
              uint64_t* ticket) {
    try {
        g_err[0] = 0;
        if (!S || !ticket) return fail(SA_EINVAL, "NULL argument");
        if (n_jobs && (!jobs || !reads)) return fail(SA_EINVAL, "NULL jobs or reads");
        auto rq = std::make_shared<Request>();
        rq->jobs.assign(jobs, jobs + n_jobs);
        rq->reads.assign(reads, reads + reads_len);
        rq->est_bytes = estimate_bytes(jobs, n_jobs, reads_len);
        if (rq->est_bytes > S->budget)
            return fail(SA_EBUSY, "request needs about %llu bytes of device memory, the budget is %llu",
                        (unsigned long long)rq->est_bytes, (unsigned long long)S->budget);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            rq->ticket = S->next_ticket++;
            S->tickets[rq->ticket] = rq;
            S->queue.push_back(rq);
            *ticket = rq->ticket;
            S->counters.submitted++;
            S->counters.max_queue = std::max<uint64_t>(S->counters.max_queue, S->queue.size());
        }
        S->cv_work.notify_all();
        return SA_OK;
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

int sa_poll(sa_server* S, uint64_t ticket, int timeout_ms, sa_result* out, uint32_t* cigar,
            uint64_t cigar_cap, uint64_t* cigar_used) {
    try {
        g_err[0] = 0;
        if (!S) return fail(SA_EINVAL, "server is NULL");
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return fail(SA_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
        std::shared_ptr<Request> rq = it->second;
        auto done = [&] { return rq->rc != SA_PENDING; };
        if (!done()) {
            if (timeout_ms == 0) return SA_PENDING;
            if (timeout_ms < 0) {
                S->cv_done.wait(lk, done);
            } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
                return fail(SA_ETIMEOUT, "ticket %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
            }
        }
        if (rq->rc != SA_OK) {
            const int rc = rq->rc;
            snprintf(g_err, sizeof(g_err), "%s", rq->err.c_str());
            S->tickets.erase(ticket);
            return rc;
        }
        if (cigar_used) *cigar_used = rq->cigar.size();
        if (rq->cigar.size() > cigar_cap || (!rq->cigar.empty() && !cigar))
            return fail(SA_EOVERFLOW, "CIGAR buffer holds %llu ops, %zu needed",
                        (unsigned long long)cigar_cap, rq->cigar.size());
        if (!rq->out.empty()) {
            if (!out) return fail(SA_EINVAL, "out is NULL");
            std::memcpy(out, rq->out.data(), rq->out.size() * sizeof(sa_result));
        }
        if (!rq->cigar.empty()) std::memcpy(cigar, rq->cigar.data(), rq->cigar.size() * 4);
        S->tickets.erase(ticket);
        return SA_OK;
    } catch (...) {
        return fail(SA_ENOMEM, "unexpected host exception");
    }
}

int sa_server_get_stats(sa_server* S, sa_server_stats* out) {
    if (!S || !out) return fail(SA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->counters;
    return SA_OK;
}

int sa_server_destroy(sa_server* S) {
    if (!S) return fail(SA_EINVAL, "server is NULL");
    try {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
            for (auto& rq : S->queue) {       // never started: fail them
                rq->rc = SA_ECUDA;
                rq->err = "server destroyed before the request ran";
            }
            S->queue.clear();
        }
        S->cv_work.notify_all();
        S->cv_done.notify_all();
        for (auto& slot : S->slots)
            if (slot->th.joinable()) slot->th.join();
        cudaSetDevice(S->ref->device);
        for (auto& slot : S->slots) {
            cudaStreamSynchronize(slot->stream);
            slot->ws.release();
            cudaStreamDestroy(slot->stream);
        }
        delete S;
        return SA_OK;
    } catch (...) {
        return fail(SA_ECUDA, "unexpected host exception");
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// read-only view of a reference handle for the other translation units

namespace sa {
RefView ref_view(const sa_reference* R) {
    return RefView{R->d_words, R->len, R->device, R->num_sms, R->own};
}

// Scores and mode of every alignment entry point.  The limits keep each kernel
// exact: a LOCAL best score must fit 21 bits (the 32-bit score pass forms keys
// H * 1024 + row tag in an int32); the 16-bit pass takes the schemes it holds
// exactly and leaves the rest to the 32-bit pass.
int check_scoring(const sa_params* p, Score* sc) {
    if (!p) return fail(SA_EINVAL, "params is NULL");
    const sa_scoring& s = p->sc;
    if (s.match < 0 || s.mismatch < 0 || s.gap_open < 0 || s.gap_extend < 0)
        return fail(SA_EINVAL, "scores are magnitudes and must be >= 0");
    if (s.match > 2047 || s.mismatch > 16383 || (int64_t)s.gap_open + s.gap_extend > 16383)
        return fail(SA_EINVAL, "match must be <= 2047, mismatch and gap_open + gap_extend <= 16383");
    if (p->mode != SA_LOCAL && p->mode != SA_GLOCAL) return fail(SA_EINVAL, "mode must be SA_LOCAL or SA_GLOCAL");
    sc->a = s.match;
    sc->b = -s.mismatch;
    sc->GO = -(s.gap_open + s.gap_extend);
    sc->GE = -s.gap_extend;
    sc->dm = sc->a - sc->GO;
    sc->dx = sc->b - sc->GO;
    sc->mode = p->mode;
    return SA_OK;
}

// the calling thread's sa_last_error() message, for the other translation units
int set_error(int code, const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
    return code;
}
}  // namespace sa
