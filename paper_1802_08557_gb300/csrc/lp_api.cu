// lp_api.cu -- host side of the C ABI declared in include/lpbatch.h.
//
// lp_batch_create uploads the LPs, checks them and plans the launches (the
// role of the batching routine, Algorithm 1 of Section 4.1: it sizes the
// work from each LP's tableau footprint, Eq. 5).  Instead of chunking by
// free memory and launching one block per LP of a single size, LPs are
// grouped by shared-memory footprint and each group is one launch of the
// SMEM-resident kernel.  lp_batch_solve enqueues the groups on the caller's
// stream; lp_batch_results copies the outputs.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda.h>

#include "lp_internal.h"
#include "lpbatch.h"

namespace lpb {

thread_local std::string g_last_error;

lpb_err api_fail(lpb_err e, const std::string& msg) {
    g_last_error = msg;
    return e;
}

lpb_err api_cuda_fail(cudaError_t err, const char* what) {
    return api_fail(LPB_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

void api_clear_error() { g_last_error.clear(); }

}  // namespace lpb

namespace {

using lpb::g_last_error;

lpb_err fail(lpb_err e, const std::string& msg) { return lpb::api_fail(e, msg); }

lpb_err cuda_fail(cudaError_t err, const char* what) { return lpb::api_cuda_fail(err, what); }

// Identity of the calling thread's current CUDA context (0 if there is none
// or the driver cannot say).  The per-device pool cache below holds a pool of
// one context and starts over when it changes: after cudaDeviceReset, or with
// another context current, the pool it held is gone or not ours.
unsigned long long context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return 0;
    if (!ctx) {
        // no context yet: the runtime's first call makes its primary context
        // current; do that now, so that what is cached belongs to it
        cudaFree(nullptr);
        if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    }
    unsigned long long id = 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// One stream-ordered memory pool per device and context that keeps freed
// memory cached, so that create/destroy cycles do not return memory to the
// driver.  A changed context (cudaDeviceReset, or another context current)
// gets a pool of its own; the old one is forgotten, not destroyed (it went
// with its context, or belongs to one that is not current).
struct DeviceCache {
    unsigned long long ctx = 0;
    cudaMemPool_t pool = nullptr;
};
std::mutex g_cache_mu;
std::map<int, DeviceCache> g_cache;

cudaError_t device_pool(int dev, cudaMemPool_t* out) {
    const unsigned long long ctx = context_id();
    std::lock_guard<std::mutex> lock(g_cache_mu);
    DeviceCache& c = g_cache[dev];
    if (c.pool && c.ctx == ctx) { *out = c.pool; return cudaSuccess; }
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    cudaError_t err = cudaMemPoolCreate(&pool, &props);
    if (err != cudaSuccess) return err;
    uint64_t keep = UINT64_MAX;
    err = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (err != cudaSuccess) return err;
    c.pool = pool;
    c.ctx = ctx;
    *out = pool;
    return cudaSuccess;
}

class DeviceGuard {
public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != prev_) cudaSetDevice(prev_);
    }
private:
    int prev_ = 0;
};

struct Group {
    int64_t offset;  // into the order array
    int32_t count;
    int32_t threads;
    size_t smem;             // shared memory of the block forms
    size_t smem_warp = 0;    // mixed groups: of the one-warp form (no block reduction scratch)
    int32_t gi = 0;          // index into the per-group device counters
    int32_t persistent = 0;  // 1: persistent CTAs over an atomic work queue
    int32_t ctas = 0;        // CTAs of the persistent form
    float tuned_ms = -1.0f;  // time of the chosen form (lp_batch_autotune), -1: not tuned
};

// Bound of Step 1's tie window in key units: ceil(tau * 2^54 * (1 + 2^-30)) + 4
// (covers tau*2^54*(1+2^-53) + 1.5, see step1_window in the kernel); -1 when
// tau is too large for the single-binade argument (tau > 2^-33).
long long step1_key_window(double tau) {
    if (!(tau <= std::ldexp(1.0, -33))) return -1;
    return (long long)std::ceil(tau * std::ldexp(1.0, 54) * (1.0 + std::ldexp(1.0, -30))) + 4;
}

// Internal streams per batch: launch groups of one solve overlap on them, so
// small groups do not wait for the large ones.
constexpr int kLanes = 4;

// Solves whose stage times lp_batch_stage_times can average.
constexpr int kTimingRing = 64;

// Cap of the streamed kernel's global workspace (slots x largest tableau).
constexpr int64_t kMaxWorkspaceBytes = int64_t(16) << 30;

// LPB_SCHED_SINGLE: the largest tableau kept in shared memory (two 512-thread
// CTAs per SM); larger ones go to the CTA's global workspace slot.
constexpr size_t kSingleSmemCap = 110 * 1024;

int pick_threads(int m, int n, int k, int requested) {
    if (requested > 0) return std::min(std::max(32, (requested + 31) / 32 * 32), lpb::kMaxThreads);
    const int64_t e = (int64_t)(m + 1 + (k > 0)) * (n + k + 1);
    // measured best on GB300 (mixed-sign dense m x m, m = 20..100)
    if (e <= 1024) return 32;
    if (e <= 3072) return 64;
    if (e <= 8192) return 128;
    if (e <= 32768) return 256;
    return 512;
}

// Threads per CTA of the mixed-precision kernel; 0 requested = from the
// tableau size.  32 selects the one-warp-per-LP variant (no block barriers):
// measured best up to 70x70 tableaux (50x50: 16.3 ms per 1e5 LPs against
// 19.7 ms at 64 threads), 128 best at 100x100.
// Rows with b_i < 0 (each gets an artificial variable in phase I).
int32_t count_negative(const double* b, int32_t m) {
    int32_t cnt = 0;
    for (int32_t i = 0; i < m; ++i) cnt += b[i] < 0.0 ? 1 : 0;
    return cnt;
}

int mixed_threads(int m, int n, int k, int requested) {
    if (requested > 0) return pick_threads(m, n, k, requested);
    const int64_t e = (int64_t)(m + 1 + (k > 0)) * (n + k + 1);
    if (e <= 8192) return 32;
    if (e <= 32768) return 128;
    return 256;
}

}  // namespace

struct lp_batch {
    int device = 0;
    int32_t num_lps = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<void*> allocs;
    lpb::DeviceBatch d{};
    int32_t* d_order = nullptr;
    std::vector<Group> groups;
    lpb::Tolerances tol{};
    int64_t total_x = 0, total_y = 0;
    cudaStream_t last_stream = nullptr;
    bool solved = false;
    int32_t num_phase1 = 0;
    size_t max_smem = 0;
    // streamed LPs: order[streamed_offset ...), persistent CTAs over slots
    int64_t streamed_offset = 0;
    int32_t num_streamed = 0;
    int32_t streamed_slots = 0;
    size_t slot_bytes = 0;
    unsigned char* workspace = nullptr;
    int32_t* counter = nullptr;
    // mixed precision: groups of the FP32 + certificate kernel, fallback queue
    std::vector<Group> mixed_groups;
    int32_t num_mixed = 0;
    lpb::MixedParams mp{};
    int32_t* fb_queue = nullptr;
    int32_t* fb_len = nullptr;
    int32_t* fb_counter = nullptr;
    int32_t* diag = nullptr;  // 8 int32: internal-consistency failures of the last solve
    // count of non-finite inputs when the check was left for the caller to
    // read (lp_solve_host); null when create read it
    unsigned long long* d_bad = nullptr;
    // internal streams: the launch groups of a solve run concurrently on them
    cudaStream_t lanes[kLanes] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kLanes] = {};
    int fb_threads = 0, fb_ctas = 0;
    size_t fb_smem = 0;
    int32_t num_fsmall = 0;  // mixed LPs whose FP64 re-solve fits one CTA (fb_queue's capacity)
    // mixed precision with the FP32 tableau in a global workspace slot
    int64_t mstream_offset = 0;
    int32_t num_mstream = 0;
    int32_t mstream_slots = 0;
    size_t mslot_bytes = 0;
    unsigned char* mworkspace = nullptr;
    int32_t* mcounter = nullptr;
    // FP64 streamed re-solve of uncertified mixed LPs whose FP64 tableau
    // exceeds one CTA
    int32_t num_fbig = 0;
    int32_t* fbig_queue = nullptr;
    int32_t* fbig_len = nullptr;
    int32_t* fbig_counter = nullptr;
    int32_t fbig_slots = 0;
    size_t fbig_slot_bytes = 0;
    unsigned char* fbig_workspace = nullptr;
    // ... on thread-block clusters of fbig_C CTAs when every such LP fits one
    // (0: on the streamed kernel)
    int fbig_C = 0, fbig_clusters = 0;
    size_t fbig_cluster_smem = 0;
    // optional stage timing: event triples (start, groups joined, re-solve
    // done) for the last kTimingRing solves
    std::vector<cudaEvent_t> tev;
    int64_t timed_solves = 0;
    // learned warm start (lp_batch_solve_warm): every LP's size when all are
    // equal (else -1), what the cold FP64 re-solve of any LP needs, and the
    // buffers, allocated by the first warm solve
    int32_t uniform_m = -1, uniform_n = -1;
    size_t cold_smem = 0;
    int cold_threads = 0;
    float* warm_x = nullptr;       // features [num_lps x (m+n)]
    float* warm_logits = nullptr;  // [num_lps x m]
    int32_t* warm_q = nullptr;     // LPs for the cold FP64 solve
    int32_t* warm_q2 = nullptr;    // LPs whose restricted LP outgrew the first pass's row cap
    int32_t* warm_stats = nullptr; // [0] queue length, [1] certified, [2] rounds, [3] queue counter,
                                   // [4] second-pass queue length
    bool last_warm = false;
    // per launch group: LP count and work counter of the persistent form
    int32_t* group_len = nullptr;
    int32_t* group_counter = nullptr;
    // LPs on thread-block clusters: one group per cluster size
    struct ClusterGroup {
        int64_t offset;
        int32_t count, C, clusters, gi;
        size_t smem;
    };
    std::vector<ClusterGroup> cluster_groups;
    int32_t* cluster_counter = nullptr;
    int32_t num_cluster = 0;
    // LPB_SCHED_SINGLE: every LP in one persistent launch over order[single_offset ...)
    int64_t single_offset = 0;
    int32_t num_single = 0, num_single_streamed = 0, single_ctas = 0;
    int32_t single_warp_from = 0;      // mixed: order[single_offset + single_warp_from ...) one LP per warp
    size_t single_smem = 0, single_slot_bytes = 0;
    uint8_t* d_resident = nullptr;     // per LP: 1 = tableau in shared memory
    unsigned char* single_workspace = nullptr;
    int32_t* single_counter = nullptr;
    // captured solve (lp_batch_solve_graph)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
};

namespace {

template <typename T>
cudaError_t alloc(lp_batch* h, T** p, size_t count, cudaStream_t s) {
    void* v = nullptr;
    cudaError_t err = cudaMallocFromPoolAsync(&v, std::max<size_t>(count, 1) * sizeof(T), h->pool, s);
    if (err != cudaSuccess) return err;
    h->allocs.push_back(v);
    *p = static_cast<T*>(v);
    return cudaSuccess;
}

void release(lp_batch* h, cudaStream_t s) {
    for (int i = 0; i < kLanes; ++i)
        if (h->lanes[i]) cudaStreamSynchronize(h->lanes[i]);
    for (void* p : h->allocs) cudaFreeAsync(p, s);
    h->allocs.clear();
    cudaStreamSynchronize(s);
    for (int i = 0; i < kLanes; ++i) {
        if (h->ev_join[i]) cudaEventDestroy(h->ev_join[i]);
        if (h->lanes[i]) cudaStreamDestroy(h->lanes[i]);
        h->ev_join[i] = nullptr;
        h->lanes[i] = nullptr;
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    h->ev_fork = nullptr;
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    h->tev.clear();
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
}

lpb::FallbackQueues fallback_queues(const lp_batch* h) {
    return lpb::FallbackQueues{h->fb_queue, h->fb_len, h->num_fsmall, h->fbig_queue, h->fbig_len, h->num_fbig};
}

// CTAs of a group's persistent form on `sms` SMs: CTAs per SM x SMs, at most
// one per LP.
void size_persistent(Group& g, int kind, int sms) {
    const int per_sm = kind == 0 ? lpb::mixed_queue_ctas_per_sm(g.threads, g.smem)
                                 : lpb::fp64_resident_queue_ctas_per_sm(g.threads, g.smem);
    g.ctas = (int32_t)std::min<int64_t>((int64_t)sms * per_sm, g.count);
}

// One launch group on stream ls: kind 0 mixed precision, 1 FP64 resident;
// one CTA per LP, or persistent CTAs over the group's work queue.
cudaError_t launch_group(lp_batch* h, int kind, const Group& g, cudaStream_t ls) {
    const int32_t* order = h->d_order + g.offset;
    if (kind == 0) {
        if (g.persistent)
            return lpb::launch_mixed_queue(h->d, h->tol, h->mp, order, h->group_len + g.gi, h->group_counter + g.gi,
                                           g.ctas, g.threads, g.smem, fallback_queues(h), h->diag, ls);
        return lpb::launch_mixed(h->d, h->tol, h->mp, order, g.count, g.threads, g.threads == 32 ? g.smem_warp : g.smem,
                                 fallback_queues(h), h->diag, ls);
    }
    if (g.persistent)
        return lpb::launch_fp64_resident_queue(h->d, h->tol, order, h->group_len + g.gi, g.count, h->num_lps,
                                               h->group_counter + g.gi, h->diag, g.ctas, g.threads, g.smem, ls);
    return lpb::launch_fp64_resident(h->d, h->tol, order, g.count, g.threads, g.smem, h->diag, ls);
}

// Everything a solve enqueues on stream s: counters reset, launch groups forked
// onto the internal streams (largest first, round robin) and joined back, the
// FP64 re-solve of uncertified LPs; with `timing`, the stage events.
lpb_err enqueue_solve(lp_batch* h, cudaStream_t s, bool timing) {
    cudaError_t err = cudaMemsetAsync(h->diag, 0, 8 * sizeof(int32_t), s);
    if (err != cudaSuccess) return cuda_fail(err, "diagnostic reset");
    if (h->num_mixed > 0 && ((err = cudaMemsetAsync(h->fb_len, 0, sizeof(int32_t), s)) ||
                             (err = cudaMemsetAsync(h->fbig_len, 0, sizeof(int32_t), s))))
        return cuda_fail(err, "fallback queue reset");
    // kind 0 mixed, 1 resident, 2 streamed, 3 cluster, 4 mixed streamed
    struct Job { int kind; const Group* g; int64_t count; };
    std::vector<Job> jobs;
    for (const Group& g : h->mixed_groups) jobs.push_back({0, &g, g.count});
    for (const Group& g : h->groups) jobs.push_back({1, &g, g.count});
    if (h->num_streamed > 0) jobs.push_back({2, nullptr, h->num_streamed});
    if (h->num_single > 0) jobs.push_back({5, nullptr, h->num_single});
    if (h->num_mstream > 0) jobs.push_back({4, nullptr, h->num_mstream});
    for (size_t ci = 0; ci < h->cluster_groups.size(); ++ci)
        jobs.push_back({3, reinterpret_cast<const Group*>(ci), h->cluster_groups[ci].count});
    std::stable_sort(jobs.begin(), jobs.end(), [](const Job& a, const Job& b) { return a.count > b.count; });
    cudaEvent_t* tev = (!timing || h->tev.empty()) ? nullptr : &h->tev[3 * (size_t)(h->timed_solves % kTimingRing)];
    if (tev && (err = cudaEventRecord(tev[0], s))) return cuda_fail(err, "timing");
    if ((err = cudaEventRecord(h->ev_fork, s))) return cuda_fail(err, "fork");
    bool used[kLanes] = {};
    for (size_t i = 0; i < jobs.size(); ++i) {
        const int lane = (int)(i % kLanes);
        cudaStream_t ls = h->lanes[lane];
        if (!used[lane]) {
            if ((err = cudaStreamWaitEvent(ls, h->ev_fork, 0))) return cuda_fail(err, "fork wait");
            used[lane] = true;
        }
        const Job& j = jobs[i];
        if (j.kind == 5 && h->num_mixed > 0) {
            err = lpb::launch_mixed_single(h->d, h->tol, h->mp, h->d_order + h->single_offset, h->d_resident,
                                           h->num_single, h->single_warp_from, h->single_ctas, h->single_smem,
                                           h->single_workspace, h->single_slot_bytes, h->single_counter,
                                           fallback_queues(h), h->diag, ls);
        } else if (j.kind == 5) {
            err = lpb::launch_fp64_single(h->d, h->tol, h->d_order + h->single_offset, h->d_resident, h->num_single,
                                          h->single_ctas, h->single_smem, h->single_workspace, h->single_slot_bytes,
                                          h->single_counter, h->diag, ls);
        } else if (j.kind == 2) {
            err = lpb::launch_fp64_streamed(h->d, h->tol, h->d_order + h->streamed_offset, h->num_streamed,
                                            h->streamed_slots, h->workspace, h->slot_bytes, h->counter, h->diag, ls);
        } else if (j.kind == 4) {
            err = lpb::launch_mixed_streamed(h->d, h->tol, h->mp, h->d_order + h->mstream_offset, h->num_mstream,
                                             h->mstream_slots, h->mworkspace, h->mslot_bytes, h->mcounter,
                                             fallback_queues(h), h->diag, ls);
        } else if (j.kind == 3) {
            const lp_batch::ClusterGroup& cg = h->cluster_groups[reinterpret_cast<size_t>(j.g)];
            err = lpb::launch_fp64_cluster(h->d, h->tol, h->d_order + cg.offset, cg.count, cg.C, cg.clusters, cg.smem,
                                           h->cluster_counter + cg.gi, h->diag, ls);
        } else {
            err = launch_group(h, j.kind, *j.g, ls);
        }
        if (err != cudaSuccess) return cuda_fail(err, "solver launch");
    }
    for (int lane = 0; lane < kLanes; ++lane) {
        if (!used[lane]) continue;
        if ((err = cudaEventRecord(h->ev_join[lane], h->lanes[lane])) ||
            (err = cudaStreamWaitEvent(s, h->ev_join[lane], 0)))
            return cuda_fail(err, "join");
    }
    if (tev && (err = cudaEventRecord(tev[1], s))) return cuda_fail(err, "timing");
    if (h->num_fsmall > 0) {
        err = lpb::launch_fp64_resident_queue(h->d, h->tol, h->fb_queue, h->fb_len, h->num_fsmall, h->num_lps,
                                              h->fb_counter, h->diag, h->fb_ctas, h->fb_threads, h->fb_smem, s);
        if (err != cudaSuccess) return cuda_fail(err, "fallback launch");
    }
    if (h->num_fbig > 0) {
        if (h->fbig_C > 0)
            err = lpb::launch_fp64_cluster(h->d, h->tol, h->fbig_queue, h->num_fbig, h->fbig_C, h->fbig_clusters,
                                           h->fbig_cluster_smem, h->fbig_counter, h->diag, s, h->fbig_len);
        else
            err = lpb::launch_fp64_streamed(h->d, h->tol, h->fbig_queue, h->num_fbig, h->fbig_slots,
                                            h->fbig_workspace, h->fbig_slot_bytes, h->fbig_counter, h->diag, s,
                                            h->fbig_len);
        if (err != cudaSuccess) return cuda_fail(err, "fallback launch");
    }
    if (tev) {
        if ((err = cudaEventRecord(tev[2], s))) return cuda_fail(err, "timing");
        ++h->timed_solves;
    }
    h->last_stream = s;
    h->solved = true;
    h->last_warm = false;
    return LPB_OK;
}

}  // namespace

extern "C" {

void lpb_default_opts(lp_batch_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = LP_PREC_FP64;
    o->max_iters = 0;
    o->eps_opt = 1e-9;
    o->eps_piv = 1e-9;
    o->eps_feas = 1e-9;
    o->tau = 1e-12;
    o->block_threads = 0;
}

const char* lpb_strerror(lpb_err e) {
    switch (e) {
        case LPB_OK: return "success";
        case LPB_EINVAL: return "invalid argument";
        case LPB_ENOMEM: return "out of memory";
        case LPB_ECUDA: return "CUDA runtime error";
        case LPB_ETOOBIG: return "LP too large";
        case LPB_ENOTSOLVED: return "no solve has been run on this batch";
    }
    return "unknown error";
}

const char* lpb_last_error(void) { return g_last_error.c_str(); }

// lp_batch_create, with three more parameters for lp_solve_host: `copied`
// (optional) is recorded on the stream right after the copies of A, b and c;
// with `defer_check` (host inputs only) the call returns without waiting for
// the stream, leaving the count of non-finite inputs in h->d_bad for the
// caller to read after its solve (the check zeroes every such entry, so the
// solve sees finite data).  Without it the call waits for the check and fails
// on a non-finite entry.  `phase1_rows` (host inputs only, optional): every
// LP's count of rows with b_i < 0, already counted by the caller.
static lpb_err create_batch(lp_batch** out, int32_t num_lps, const int32_t* m, const int32_t* n,
                            const int64_t* a_off, const double* A, int64_t a_len,
                            const int64_t* b_off, const double* b, int64_t b_len,
                            const int64_t* c_off, const double* c, int64_t c_len,
                            int32_t ptr_kind, const lp_batch_opts* opts, void* stream, cudaEvent_t copied,
                            bool defer_check, const int32_t* phase1_rows = nullptr) {
    g_last_error.clear();
    if (!out) return fail(LPB_EINVAL, "out is NULL");
    if (defer_check && ptr_kind != LPB_HOST) return fail(LPB_EINVAL, "a deferred input check needs host inputs");
    *out = nullptr;
    if (num_lps < 1) return fail(LPB_EINVAL, "num_lps < 1");
    if (!m || !n || !A || !b || !c) return fail(LPB_EINVAL, "m, n, A, b and c must be non-NULL");
    if (ptr_kind != LPB_HOST && ptr_kind != LPB_DEVICE) return fail(LPB_EINVAL, "ptr_kind must be LPB_HOST or LPB_DEVICE");
    lp_batch_opts o;
    lpb_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != LP_PREC_FP64 && o.precision != LP_PREC_FP32_REFINE)
        return fail(LPB_EINVAL, "unsupported precision");
    if (o.schedule != LPB_SCHED_AUTO && o.schedule != LPB_SCHED_STREAMED && o.schedule != LPB_SCHED_CLUSTER &&
        o.schedule != LPB_SCHED_SINGLE)
        return fail(LPB_EINVAL, "unknown schedule");
    if (!(o.eps_opt >= 0) || !(o.eps_piv >= 0) || !(o.eps_feas >= 0) || !(o.tau >= 0))
        return fail(LPB_EINVAL, "tolerances must be >= 0");

    // sizes and offsets (host)
    std::vector<int32_t> hm(m, m + num_lps), hn(n, n + num_lps);
    std::vector<int64_t> ha(num_lps), hb(num_lps), hc(num_lps), hx(num_lps), hy(num_lps);
    int64_t pa = 0, pb = 0, pc = 0, px = 0, py = 0;
    for (int32_t k = 0; k < num_lps; ++k) {
        const int64_t mk = hm[k], nk = hn[k];
        if (mk < 1 || nk < 1) return fail(LPB_EINVAL, "LP " + std::to_string(k) + ": m and n must be >= 1");
        if (mk > LPB_MAX_DIM || nk > LPB_MAX_DIM)
            return fail(LPB_ETOOBIG, "LP " + std::to_string(k) + ": m or n above LPB_MAX_DIM");
        ha[k] = a_off ? a_off[k] : pa;
        hb[k] = b_off ? b_off[k] : pb;
        hc[k] = c_off ? c_off[k] : pc;
        pa += mk * nk; pb += mk; pc += nk;
        if (ha[k] < 0 || ha[k] + mk * nk > a_len) return fail(LPB_EINVAL, "LP " + std::to_string(k) + ": A offset out of range");
        if (hb[k] < 0 || hb[k] + mk > b_len) return fail(LPB_EINVAL, "LP " + std::to_string(k) + ": b offset out of range");
        if (hc[k] < 0 || hc[k] + nk > c_len) return fail(LPB_EINVAL, "LP " + std::to_string(k) + ": c offset out of range");
        hx[k] = px; px += nk;
        hy[k] = py; py += mk;
    }

    lp_batch* h = new (std::nothrow) lp_batch();
    if (!h) return fail(LPB_ENOMEM, "host allocation failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaGetDevice(&h->device);
    if (err != cudaSuccess) { delete h; return cuda_fail(err, "cudaGetDevice"); }
    err = device_pool(h->device, &h->pool);
    if (err != cudaSuccess) { delete h; return cuda_fail(err, "memory pool"); }
    h->num_lps = num_lps;
    h->total_x = px;
    h->total_y = py;
    // FP32 ratio screen of Step 2: a window far wider than the float rounding
    // error of the screened ratios (< 8 * 2^-24 relative) and than the tie
    // window (tau relative, or tau absolute below 1).
    const float ratio_rel = (float)std::max(std::ldexp(1.0, -12), 8.0 * o.tau);
    const float ratio_abs = (float)std::max(std::ldexp(1.0, -20), 8.0 * o.tau);
    h->tol = {o.eps_opt, o.eps_piv, o.eps_feas, o.tau, o.max_iters, step1_key_window(o.tau), ratio_rel, ratio_abs};
    h->last_stream = s;

    auto bail = [&](lpb_err e, const std::string& msg) {
        release(h, s);
        delete h;
        return fail(e, msg);
    };
    auto bail_cuda = [&](cudaError_t e, const char* what) {
        std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
        release(h, s);
        delete h;
        return fail(e == cudaErrorMemoryAllocation ? LPB_ENOMEM : LPB_ECUDA, msg);
    };

    int32_t *dm, *dn, *dk, *dorder, *dstatus, *diters;
    int64_t *da, *db, *dc, *dx_off, *dy_off;
    double *dA, *dbv, *dcv, *dobj, *dx, *dy;
    unsigned long long* dbad;
    if ((err = alloc(h, &dm, num_lps, s)) || (err = alloc(h, &dn, num_lps, s)) ||
        (err = alloc(h, &dk, num_lps, s)) || (err = alloc(h, &dorder, num_lps, s)) ||
        (err = alloc(h, &dstatus, num_lps, s)) || (err = alloc(h, &diters, num_lps, s)) ||
        (err = alloc(h, &da, num_lps, s)) || (err = alloc(h, &db, num_lps, s)) ||
        (err = alloc(h, &dc, num_lps, s)) || (err = alloc(h, &dx_off, num_lps, s)) ||
        (err = alloc(h, &dy_off, num_lps, s)) || (err = alloc(h, &dA, (size_t)a_len, s)) ||
        (err = alloc(h, &dbv, (size_t)b_len, s)) || (err = alloc(h, &dcv, (size_t)c_len, s)) ||
        (err = alloc(h, &dobj, num_lps, s)) || (err = alloc(h, &dx, (size_t)px, s)) ||
        (err = alloc(h, &dy, (size_t)py, s)) || (err = alloc(h, &dbad, 1, s)))
        return bail_cuda(err, "device allocation");

    const cudaMemcpyKind kind = ptr_kind == LPB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t nl = (size_t)num_lps;
    if ((err = cudaMemcpyAsync(dm, hm.data(), nl * 4, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(dn, hn.data(), nl * 4, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(da, ha.data(), nl * 8, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(db, hb.data(), nl * 8, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(dc, hc.data(), nl * 8, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(dx_off, hx.data(), nl * 8, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(dy_off, hy.data(), nl * 8, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(dA, A, (size_t)a_len * 8, kind, s)) ||
        (err = cudaMemcpyAsync(dbv, b, (size_t)b_len * 8, kind, s)) ||
        (err = cudaMemcpyAsync(dcv, c, (size_t)c_len * 8, kind, s)))
        return bail_cuda(err, "copy of the LP data");
    if (copied && (err = cudaEventRecord(copied, s))) return bail_cuda(err, "event record");

    h->d = lpb::DeviceBatch{dm, dn, da, db, dc, dx_off, dy_off, dA, dbv, dcv, dstatus, diters, dobj, dx, dy};
    h->d_order = dorder;
    if (ptr_kind == LPB_DEVICE &&
        ((err = lpb::launch_input_check(dA, a_len, dbv, b_len, dcv, c_len, dbad, s)) ||
         (err = lpb::launch_count_negative_rhs(h->d, num_lps, dk, s))))
        return bail_cuda(err, "input check kernel");
    std::vector<int32_t> hk(num_lps);
    unsigned long long bad = 0;
    if (ptr_kind == LPB_HOST) {
        // phase-I rows counted here while the copies run (the plan below
        // overlaps them too); the input check is launched after the last
        // upload of the plan, so that no host call of this function waits for
        // a kernel (a kernel queued behind another stream's large grid can
        // wait for most of that grid)
        if (phase1_rows) {
            std::copy(phase1_rows, phase1_rows + num_lps, hk.begin());
        } else {
            for (int32_t k = 0; k < num_lps; ++k) hk[k] = count_negative(b + hb[k], hm[k]);
        }
    } else {
        if ((err = cudaMemcpyAsync(hk.data(), dk, nl * 4, cudaMemcpyDeviceToHost, s)) ||
            (err = cudaMemcpyAsync(&bad, dbad, sizeof bad, cudaMemcpyDeviceToHost, s)) ||
            (err = cudaStreamSynchronize(s)))
            return bail_cuda(err, "input check");
        if (bad) return bail(LPB_EINVAL, std::to_string(bad) + " non-finite entries in A, b or c");
    }

    // Plan: LPs whose tableau fits in one CTA's shared memory are grouped by
    // (threads per CTA, footprint rounded up to 4 KiB), one launch per group;
    // the others go to the streamed kernel (global workspace slots).
    std::map<std::pair<int, size_t>, std::vector<int32_t>> buckets, mixed_buckets;
    std::vector<int32_t> streamed;
    std::map<int, std::vector<int32_t>> cluster_buckets;  // cluster size -> LPs
    std::vector<int32_t> mstream;                         // mixed precision, tableau in global memory
    std::vector<int32_t> fbig_lps;                        // mixed LPs whose FP64 re-solve exceeds one CTA
    std::vector<int32_t> single;                          // LPB_SCHED_SINGLE: every LP
    std::vector<int32_t> single_warp;                     // ... (mixed) the ones solved one per warp
    std::vector<uint8_t> single_resident;                 // ... per LP: 1 = in shared memory
    const size_t queue_smem_cap = lpb::kMaxSmemPerBlock - 1024;
    h->uniform_m = hm[0];
    h->uniform_n = hn[0];
    for (int32_t k = 0; k < num_lps; ++k) {
        const size_t need = lpb::resident_smem_bytes(hm[k], hn[k], hk[k]);
        h->num_phase1 += hk[k] > 0;
        if (hm[k] != h->uniform_m || hn[k] != h->uniform_n) h->uniform_m = h->uniform_n = -1;
        h->cold_smem = std::max(h->cold_smem, need);
        h->cold_threads = std::max(h->cold_threads, pick_threads(hm[k], hn[k], hk[k], 0));
        if (o.precision == LP_PREC_FP32_REFINE) {
            // FP32 tableau + FP64 certificate: in shared memory when the FP32
            // tableau fits one CTA (AUTO), else in a global workspace slot.
            // The FP64 re-solve of an uncertified LP runs in one CTA when its
            // FP64 tableau fits, else streamed.
            if (need <= queue_smem_cap) {
                ++h->num_fsmall;
                h->fb_smem = std::max(h->fb_smem, need);
                // the re-solve runs after every mixed launch, over ~1% of the
                // LPs: its time is one LP's latency, so at least 256 threads per
                // LP (50x50: re-solve 0.77 -> 0.66 ms per 1e5; 512 was slower)
                h->fb_threads = std::max({h->fb_threads, pick_threads(hm[k], hn[k], hk[k], 0), 256});
            } else {
                ++h->num_fbig;
                h->fbig_slot_bytes = std::max(h->fbig_slot_bytes, lpb::streamed_slot_bytes(hm[k], hn[k], hk[k]));
                fbig_lps.push_back(k);
            }
            const size_t mneed = lpb::mixed_smem_bytes(hm[k], hn[k], hk[k]);
            if (o.schedule == LPB_SCHED_SINGLE) {
                // one launch for all: an LP the default plan gives one warp
                // and whose area fits a warp's share of the CTA in warp mode
                // (listed last); the others one per CTA, the LP's area in
                // shared memory up to kMixedSingleSmemCap (two CTAs per SM),
                // else in this CTA's global workspace slot
                if (single_resident.empty()) single_resident.assign((size_t)num_lps, 0);
                if (mixed_threads(hm[k], hn[k], hk[k], o.block_threads) == 32 &&
                    lpb::mixed_layout(hm[k], hn[k], hk[k]).total <= lpb::kMixedSingleWarpArea) {
                    single_resident[k] = 1;
                    single_warp.push_back(k);
                    h->single_smem = std::max(h->single_smem, lpb::kMixedSingleSmemCap);  // every warp's area
                    continue;
                }
                single.push_back(k);
                if (mneed <= lpb::kMixedSingleSmemCap) {
                    single_resident[k] = 1;
                    h->single_smem = std::max(h->single_smem, mneed);
                } else {
                    ++h->num_single_streamed;
                    h->single_slot_bytes = std::max(
                        h->single_slot_bytes, (lpb::mixed_layout(hm[k], hn[k], hk[k]).total + 255) & ~size_t(255));
                }
                continue;
            }
            if (o.schedule != LPB_SCHED_STREAMED && mneed <= queue_smem_cap) {
                const int threads = mixed_threads(hm[k], hn[k], hk[k], o.block_threads);
                // shared memory rounded to 1 KiB for the one-warp form (it sets
                // how many LPs share an SM), to 8 KiB otherwise: fewer, larger
                // launches (uneven workload: 1 KiB 280 groups 17.3 ms, 4 KiB
                // 123 groups 11.6 ms, 8 KiB 97 groups 11.2 ms, 16 KiB 84 groups
                // 11.4 ms)
                const size_t gran = threads == 32 ? 1024 : 8192;
                mixed_buckets[{threads, std::min(queue_smem_cap, (mneed + gran - 1) / gran * gran)}].push_back(k);
            } else {
                mstream.push_back(k);
                h->mslot_bytes = std::max(h->mslot_bytes, (lpb::mixed_layout(hm[k], hn[k], hk[k]).total + 255) &
                                                              ~size_t(255));
            }
            continue;
        }
        if (o.schedule == LPB_SCHED_SINGLE) {
            // one launch for all: shared memory up to kSingleSmemCap (two
            // 512-thread CTAs per SM), else this CTA's global workspace slot
            if (single_resident.empty()) single_resident.assign((size_t)num_lps, 0);
            single.push_back(k);
            if (need <= kSingleSmemCap) {
                single_resident[k] = 1;
                h->single_smem = std::max(h->single_smem, need);
            } else {
                ++h->num_single_streamed;
                h->single_slot_bytes = std::max(h->single_slot_bytes, lpb::streamed_slot_bytes(hm[k], hn[k], hk[k]));
            }
            continue;
        }
        // (measured on GB300: the streamed kernel, 304 LPs at once, beats the
        // clusters, ~50 LPs at once, on every large-LP workload tried --
        // 1.04-1.34x, more with more pivots -- so clusters are on request)
        if (need > lpb::kMaxSmemPerBlock && o.schedule == LPB_SCHED_CLUSTER) {
            // the smallest cluster whose CTAs hold the tableau's rows
            int C = 0;
            for (int c = 2; c <= lpb::kMaxClusterCtas && !C; ++c)
                if (lpb::cluster_smem_bytes(hm[k], hn[k], hk[k], c) <= lpb::kMaxSmemPerBlock - 1024) C = c;
            if (C) {
                cluster_buckets[C].push_back(k);
                continue;
            }
        }
        if (need > lpb::kMaxSmemPerBlock || o.schedule == LPB_SCHED_STREAMED) {
            streamed.push_back(k);
            h->slot_bytes = std::max(h->slot_bytes, lpb::streamed_slot_bytes(hm[k], hn[k], hk[k]));
            continue;
        }
        const size_t smem = std::min(lpb::kMaxSmemPerBlock, (need + 4095) / 4096 * 4096);
        const int threads = pick_threads(hm[k], hn[k], hk[k], o.block_threads);
        buckets[{threads, smem}].push_back(k);
        h->max_smem = std::max(h->max_smem, smem);
    }
    // Longest work first within every list (LPT): the tail of a launch is
    // made of small LPs.  Work estimate: (m+1)(n+k+1) per pivot, O(m+n) pivots.
    std::vector<double> work(num_lps);
    for (int32_t k = 0; k < num_lps; ++k)
        work[k] = (double)(hm[k] + 1) * (hn[k] + hk[k] + 1) * (hm[k] + hn[k]);
    auto lpt = [&](std::vector<int32_t>& v) {
        bool uniform = true;
        for (size_t i = 1; i < v.size() && uniform; ++i) uniform = work[v[i]] == work[v[0]];
        if (uniform) return;  // already in order
        std::stable_sort(v.begin(), v.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    };
    for (auto& kv : buckets) lpt(kv.second);
    for (auto& kv : mixed_buckets) lpt(kv.second);
    lpt(streamed);
    std::vector<int32_t> order;
    order.reserve(num_lps);
    for (auto& kv : buckets) {
        Group g;
        g.offset = (int64_t)order.size();
        g.count = (int32_t)kv.second.size();
        g.threads = kv.first.first;
        g.smem = kv.first.second;
        order.insert(order.end(), kv.second.begin(), kv.second.end());
        h->groups.push_back(g);
    }
    for (auto& kv : mixed_buckets) {
        Group g;
        g.offset = (int64_t)order.size();
        g.count = (int32_t)kv.second.size();
        g.threads = kv.first.first;
        g.smem = kv.first.second;
        // the one-warp form at its exact size (128-byte units): 13.5 KB, not
        // 14 KB, is what lets 16 CTAs of 50 x 50 LPs share an SM
        for (int32_t k : kv.second)
            g.smem_warp = std::max(g.smem_warp, (lpb::mixed_layout(hm[k], hn[k], hk[k]).total + 127) / 128 * 128);
        order.insert(order.end(), kv.second.begin(), kv.second.end());
        h->mixed_groups.push_back(g);
        h->num_mixed += g.count;
    }
    {
        // per-group device counters of the persistent form
        std::vector<int32_t> lens;
        for (Group& g : h->groups) { g.gi = (int32_t)lens.size(); lens.push_back(g.count); }
        for (Group& g : h->mixed_groups) { g.gi = (int32_t)lens.size(); lens.push_back(g.count); }
        if (!lens.empty()) {
            if ((err = alloc(h, &h->group_len, lens.size(), s)) || (err = alloc(h, &h->group_counter, lens.size(), s)) ||
                (err = cudaMemcpyAsync(h->group_len, lens.data(), lens.size() * 4, cudaMemcpyHostToDevice, s)))
                return bail_cuda(err, "group counters");
        }
    }
    // cluster groups (a cluster shape that cannot be placed goes to the streamed kernel)
    for (auto& kv : cluster_buckets) {
        const int C = kv.first;
        lpt(kv.second);
        size_t smem = 0;
        for (int32_t k : kv.second) smem = std::max(smem, lpb::cluster_smem_bytes(hm[k], hn[k], hk[k], C));
        smem = (smem + 1023) / 1024 * 1024;
        int active = 0;
        if ((err = lpb::cluster_kernel_prepare()) == cudaSuccess) active = lpb::cluster_max_active(C, smem);
        cudaGetLastError();
        if (active <= 0) {
            for (int32_t k : kv.second) {
                streamed.push_back(k);
                h->slot_bytes = std::max(h->slot_bytes, lpb::streamed_slot_bytes(hm[k], hn[k], hk[k]));
            }
            continue;
        }
        lp_batch::ClusterGroup g;
        g.offset = (int64_t)order.size();
        g.count = (int32_t)kv.second.size();
        g.C = C;
        g.clusters = std::min<int32_t>(g.count, active);
        g.gi = (int32_t)h->cluster_groups.size();
        g.smem = smem;
        order.insert(order.end(), kv.second.begin(), kv.second.end());
        h->cluster_groups.push_back(g);
        h->num_cluster += g.count;
    }
    if (!h->cluster_groups.empty() &&
        (err = alloc(h, &h->cluster_counter, h->cluster_groups.size(), s)))
        return bail_cuda(err, "cluster counters");
    lpt(mstream);
    h->mstream_offset = (int64_t)order.size();
    h->num_mstream = (int32_t)mstream.size();
    h->num_mixed += h->num_mstream;
    order.insert(order.end(), mstream.begin(), mstream.end());
    if (h->num_mstream > 0) {
        int sms = 0;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device)))
            return bail_cuda(err, "device query");
        int64_t slots = (int64_t)sms * lpb::mixed_streamed_ctas_per_sm();
        const int64_t cap = std::max<int64_t>(1, kMaxWorkspaceBytes / (int64_t)h->mslot_bytes);
        slots = std::min<int64_t>({slots, (int64_t)h->num_mstream, cap});
        h->mstream_slots = (int32_t)slots;
        if ((err = alloc(h, &h->mworkspace, (size_t)slots * h->mslot_bytes, s)) || (err = alloc(h, &h->mcounter, 1, s)))
            return bail_cuda(err, "mixed streamed workspace allocation");
    }
    lpt(single);
    lpt(single_warp);
    h->single_warp_from = (int32_t)single.size();
    single.insert(single.end(), single_warp.begin(), single_warp.end());
    h->single_offset = (int64_t)order.size();
    h->num_single = (int32_t)single.size();
    if (o.precision == LP_PREC_FP32_REFINE) h->num_mixed += h->num_single;
    order.insert(order.end(), single.begin(), single.end());
    lpt(streamed);
    h->streamed_offset = (int64_t)order.size();
    h->num_streamed = (int32_t)streamed.size();
    order.insert(order.end(), streamed.begin(), streamed.end());
    // the last upload from pageable host memory, ahead of every memset and
    // kernel of this function: such a copy may wait for the stream, and
    // returns once its data is staged (so the host vectors may go out of
    // scope before the copies run)
    if ((err = cudaMemcpyAsync(dorder, order.data(), nl * 4, cudaMemcpyHostToDevice, s)))
        return bail_cuda(err, "plan upload");
    if (h->num_single > 0) {
        if ((err = alloc(h, &h->d_resident, (size_t)num_lps, s)) ||
            (err = cudaMemcpyAsync(h->d_resident, single_resident.data(), (size_t)num_lps, cudaMemcpyHostToDevice, s)))
            return bail_cuda(err, "plan upload");
        int sms = 0;
        const bool mixed = o.precision == LP_PREC_FP32_REFINE;
        // (each LP's footprint above includes the reduction scratch its area follows)
        h->single_smem = std::max(h->single_smem, lpb::SmallLayout::total);
        // FP64 streamed LPs stage their update in the CTA's shared memory beyond the reduction scratch
        if (!mixed && h->num_single_streamed > 0)
            h->single_smem = std::max(h->single_smem, lpb::SmallLayout::total + lpb::kStreamStageBytes);
        h->single_smem = (h->single_smem + 1023) / 1024 * 1024;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device)) ||
            (err = mixed ? lpb::mixed_single_prepare(h->single_smem) : lpb::fp64_single_prepare(h->single_smem)))
            return bail_cuda(err, "single launch set-up");
        const int per_sm = std::max(1, mixed ? lpb::mixed_single_ctas_per_sm(h->single_smem)
                                             : lpb::fp64_single_ctas_per_sm(h->single_smem));
        int64_t ctas = std::min<int64_t>((int64_t)sms * per_sm, h->num_single);
        if (h->num_single_streamed > 0) {
            h->single_slot_bytes = (h->single_slot_bytes + 255) & ~size_t(255);
            ctas = std::min<int64_t>(ctas, std::max<int64_t>(1, kMaxWorkspaceBytes / (int64_t)h->single_slot_bytes));
            if ((err = alloc(h, &h->single_workspace, (size_t)ctas * h->single_slot_bytes, s)))
                return bail_cuda(err, "single-launch workspace allocation");
        }
        h->single_ctas = (int32_t)ctas;
        h->max_smem = std::max(h->max_smem, h->single_smem);
        if ((err = alloc(h, &h->single_counter, 1, s))) return bail_cuda(err, "single-launch counter");
    }
    if (h->num_streamed > 0) {
        int sms = 0;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device)))
            return bail_cuda(err, "device query");
        int64_t slots = (int64_t)sms * lpb::fp64_streamed_ctas_per_sm();
        const int64_t cap = std::max<int64_t>(1, kMaxWorkspaceBytes / (int64_t)h->slot_bytes);
        slots = std::min<int64_t>({slots, (int64_t)h->num_streamed, cap});
        h->streamed_slots = (int32_t)slots;
        if ((err = alloc(h, &h->workspace, (size_t)slots * h->slot_bytes, s)) || (err = alloc(h, &h->counter, 1, s)))
            return bail_cuda(err, "streamed workspace allocation");
    }
    if (h->num_mixed > 0) {
        h->mp.eps_opt32 = 1e-6f;
        h->mp.eps_piv32 = 1e-6f;
        h->mp.eps_feas32 = 1e-6f;
        h->mp.cert_tol = 1e-9;
        h->mp.conv_tol = std::ldexp(1.0, -43);  // componentwise backward error ~1.1e-13
        h->mp.fwd_tol = 1e-12;
        // a component at or near 0 (a degenerate basis, a ray) is accurate to
        // 1e-15 max|z| at best, not 1e-12 of itself
        h->mp.fwd_floor = 1e-3;
        // slow refinements (an ill-conditioned basis) that still converge are
        // certified rather than re-solved (50x50: 604 -> 372 re-solves per 1e5)
        h->mp.max_refine = 12;
        h->fb_smem = (h->fb_smem + 1023) / 1024 * 1024;
        if ((err = alloc(h, &h->fb_queue, (size_t)h->num_fsmall, s)) || (err = alloc(h, &h->fb_len, 1, s)) ||
            (err = alloc(h, &h->fb_counter, 1, s)) || (err = cudaMemsetAsync(h->fb_len, 0, 4, s)) ||
            (err = alloc(h, &h->fbig_queue, (size_t)h->num_fbig, s)) || (err = alloc(h, &h->fbig_len, 1, s)) ||
            (err = alloc(h, &h->fbig_counter, 1, s)) || (err = cudaMemsetAsync(h->fbig_len, 0, 4, s)))
            return bail_cuda(err, "fallback queue allocation");
        int sms = 0;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device)) ||
            (err = lpb::fp64_kernels_prepare()) || (err = lpb::mixed_kernel_prepare()))
            return bail_cuda(err, "device query");
        if (h->num_fsmall > 0)
            h->fb_ctas = sms * lpb::fp64_resident_queue_ctas_per_sm(h->fb_threads, h->fb_smem);
        if (h->num_fbig > 0) {
            // re-solve on clusters: the smallest cluster size that holds every
            // such LP (re-solves are few, so each gets many SMs' FP64 pipes)
            int C = 0;
            for (int32_t k : fbig_lps) {
                int ck = 0;
                for (int c = 2; c <= lpb::kMaxClusterCtas && !ck; ++c)
                    if (lpb::cluster_smem_bytes(hm[k], hn[k], hk[k], c) <= lpb::kMaxSmemPerBlock - 1024) ck = c;
                if (!ck) { C = 0; break; }
                C = std::max(C, ck);
            }
            if (C) {
                size_t smem = 0;
                for (int32_t k : fbig_lps) smem = std::max(smem, lpb::cluster_smem_bytes(hm[k], hn[k], hk[k], C));
                smem = (smem + 1023) / 1024 * 1024;
                int active = 0;
                if (lpb::cluster_kernel_prepare() == cudaSuccess) active = lpb::cluster_max_active(C, smem);
                cudaGetLastError();
                if (active > 0) {
                    h->fbig_C = C;
                    h->fbig_clusters = std::min<int32_t>(active, h->num_fbig);
                    h->fbig_cluster_smem = smem;
                }
            }
            if (!h->fbig_C) {
                // else streamed, one slot per SM
                const int64_t cap = std::max<int64_t>(1, kMaxWorkspaceBytes / (int64_t)h->fbig_slot_bytes);
                h->fbig_slots = (int32_t)std::min<int64_t>({(int64_t)sms, (int64_t)h->num_fbig, cap});
                if ((err = alloc(h, &h->fbig_workspace, (size_t)h->fbig_slots * h->fbig_slot_bytes, s)))
                    return bail_cuda(err, "fallback workspace allocation");
            }
        }
    }
    if ((err = alloc(h, &h->diag, 8, s)) || (err = cudaMemsetAsync(h->diag, 0, 32, s)))
        return bail_cuda(err, "diagnostic word allocation");
    if ((err = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)))
        return bail_cuda(err, "event creation");
    for (int i = 0; i < kLanes; ++i)
        if ((err = cudaStreamCreateWithFlags(&h->lanes[i], cudaStreamNonBlocking)) ||
            (err = cudaEventCreateWithFlags(&h->ev_join[i], cudaEventDisableTiming)))
            return bail_cuda(err, "stream creation");
    if ((err = lpb::fp64_kernels_prepare())) return bail_cuda(err, "plan upload");
    if (ptr_kind == LPB_HOST) {
        if ((err = lpb::launch_input_check(dA, a_len, dbv, b_len, dcv, c_len, dbad, s)))
            return bail_cuda(err, "input check kernel");
        if (defer_check) {
            h->d_bad = dbad;
            *out = h;
            return LPB_OK;
        }
        if ((err = cudaMemcpyAsync(&bad, dbad, sizeof bad, cudaMemcpyDeviceToHost, s)))
            return bail_cuda(err, "input check");
    }
    if ((err = cudaStreamSynchronize(s))) return bail_cuda(err, "plan upload");
    if (bad) return bail(LPB_EINVAL, std::to_string(bad) + " non-finite entries in A, b or c");
    *out = h;
    return LPB_OK;
}

lpb_err lp_batch_create(lp_batch** out, int32_t num_lps, const int32_t* m, const int32_t* n,
                        const int64_t* a_off, const double* A, int64_t a_len,
                        const int64_t* b_off, const double* b, int64_t b_len,
                        const int64_t* c_off, const double* c, int64_t c_len,
                        int32_t ptr_kind, const lp_batch_opts* opts, void* stream) {
    return create_batch(out, num_lps, m, n, a_off, A, a_len, b_off, b, b_len, c_off, c, c_len, ptr_kind, opts, stream,
                        nullptr, false);
}

lpb_err lp_batch_solve(lp_batch* h, void* stream) {
    g_last_error.clear();
    if (!h) return fail(LPB_EINVAL, "handle is NULL");
    DeviceGuard guard(h->device);
    return enqueue_solve(h, static_cast<cudaStream_t>(stream), true);
}

lpb_err lp_batch_solve_graph(lp_batch* h, void* stream) {
    g_last_error.clear();
    if (!h) return fail(LPB_EINVAL, "handle is NULL");
    DeviceGuard guard(h->device);
    cudaError_t err;
    if (!h->graph_exec) {
        if (!h->cap_stream && (err = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)))
            return cuda_fail(err, "capture stream");
        if ((err = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)))
            return cuda_fail(err, "begin capture");
        const lpb_err r = enqueue_solve(h, h->cap_stream, false);
        cudaGraph_t graph = nullptr;
        err = cudaStreamEndCapture(h->cap_stream, &graph);
        if (r != LPB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (err != cudaSuccess) return cuda_fail(err, "end capture");
        err = cudaGraphInstantiate(&h->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess) {
            h->graph_exec = nullptr;
            return cuda_fail(err, "graph instantiation");
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((err = cudaGraphLaunch(h->graph_exec, s))) return cuda_fail(err, "graph launch");
    h->last_stream = s;
    h->solved = true;
    h->last_warm = false;
    return LPB_OK;
}

lpb_err lp_batch_autotune(lp_batch* h, int32_t rounds, void* stream) {
    g_last_error.clear();
    if (!h) return fail(LPB_EINVAL, "handle is NULL");
    if (rounds < 1 || rounds > 100) return fail(LPB_EINVAL, "rounds must be in [1, 100]");
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    cudaError_t err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device))) return cuda_fail(err, "device query");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((err = cudaEventCreate(&e0)) || (err = cudaEventCreate(&e1))) return cuda_fail(err, "tuning events");
    auto time_group = [&](int kind, Group& g, float& best) -> cudaError_t {
        float t_min = 1e30f;
        for (int r = 0; r < rounds; ++r) {
            cudaError_t e;
            if ((e = cudaMemsetAsync(h->diag, 0, 32, s))) return e;
            if (kind == 0 && ((e = cudaMemsetAsync(h->fb_len, 0, 4, s)) || (e = cudaMemsetAsync(h->fbig_len, 0, 4, s))))
                return e;
            if ((e = cudaEventRecord(e0, s)) || (e = launch_group(h, kind, g, s)) || (e = cudaEventRecord(e1, s)) ||
                (e = cudaEventSynchronize(e1)))
                return e;
            float ms = 0.0f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1))) return e;
            t_min = std::min(t_min, ms);
        }
        best = t_min;
        return cudaSuccess;
    };
    auto tune = [&](int kind, std::vector<Group>& gs, std::initializer_list<int> cand) -> cudaError_t {
        for (Group& g : gs) {
            Group best_g = g;
            float best = 1e30f;
            // the queue kernels keep a word of static shared memory: the
            // largest groups run one CTA per LP only
            const int max_form = g.smem <= lpb::kMaxSmemPerBlock - 1024 ? 1 : 0;
            for (int persistent = 0; persistent <= max_form; ++persistent)
                for (int threads : cand) {
                    Group t = g;
                    t.threads = threads;
                    t.persistent = persistent;
                    if (persistent) size_persistent(t, kind, sms);
                    float ms = 0.0f;
                    cudaError_t e = time_group(kind, t, ms);
                    if (e != cudaSuccess) return e;
                    if (ms < best) { best = ms; best_g = t; }
                }
            best_g.tuned_ms = best;
            g = best_g;
        }
        return cudaSuccess;
    };
    err = tune(1, h->groups, {32, 64, 128, 256, 512});
    if (!err) err = tune(0, h->mixed_groups, {32, 64, 128, 256});
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err) return cuda_fail(err, "autotune");
    if (h->graph_exec) {  // the captured solve has the old launch forms
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    h->solved = false;  // the trial launches left partial outputs
    return LPB_OK;
}

lpb_err lp_batch_set_group_form(lp_batch* h, int32_t index, int32_t threads, int32_t persistent) {
    g_last_error.clear();
    if (!h) return fail(LPB_EINVAL, "handle is NULL");
    const int32_t nr = (int32_t)h->groups.size(), nm = (int32_t)h->mixed_groups.size();
    if (index < 0 || index >= nr + nm) return fail(LPB_EINVAL, "group index out of range (or a streamed group)");
    const int kind = index < nr ? 1 : 0;
    if (threads < 32 || threads > lpb::kMaxThreads || threads % 32)
        return fail(LPB_EINVAL, "threads must be a multiple of 32 within the kernel's range");
    if (persistent != 0 && persistent != 1) return fail(LPB_EINVAL, "persistent must be 0 or 1");
    DeviceGuard guard(h->device);
    Group& g = index < nr ? h->groups[index] : h->mixed_groups[index - nr];
    if (persistent && g.smem > lpb::kMaxSmemPerBlock - 1024)
        return fail(LPB_EINVAL, "this group's shared memory leaves no room for the persistent form");
    g.threads = threads;
    g.persistent = persistent;
    g.tuned_ms = -1.0f;
    if (persistent) {
        int sms = 0;
        cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (err) return cuda_fail(err, "device query");
        size_persistent(g, kind, sms);
    }
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    return LPB_OK;
}

lpb_err lp_batch_group_info(lp_batch* h, int32_t index, lp_batch_group* out) {
    if (!h || !out) return fail(LPB_EINVAL, "handle or out is NULL");
    const int32_t nr = (int32_t)h->groups.size(), nm = (int32_t)h->mixed_groups.size();
    const int32_t nc = (int32_t)h->cluster_groups.size();
    const int32_t ns = h->num_streamed > 0 ? 1 : 0;
    const int32_t nms = h->num_mstream > 0 ? 1 : 0;
    const int32_t total = nr + nm + nc + ns + nms + (h->num_single > 0 ? 1 : 0);
    if (index < 0 || index >= total) return fail(LPB_EINVAL, "group index out of range");
    std::memset(out, 0, sizeof *out);
    if (h->num_single > 0 && index == total - 1) {
        out->kind = 5;
        out->count = h->num_single;
        out->threads = h->num_mixed > 0 ? lpb::kMixedSingleThreads : lpb::kStreamedThreads;
        out->persistent = 1;
        out->smem_bytes = (int64_t)h->single_smem;
        out->tuned_ms = -1.0f;
        return LPB_OK;
    }
    if (index >= nr + nm && index < nr + nm + nc) {
        const lp_batch::ClusterGroup& g = h->cluster_groups[index - nr - nm];
        out->kind = 3;
        out->count = g.count;
        out->threads = 512;
        out->persistent = 1;
        out->smem_bytes = (int64_t)g.smem;
        out->tuned_ms = -1.0f;
        out->cluster_ctas = g.C;
        return LPB_OK;
    }
    if (index < nr + nm) {
        const Group& g = index < nr ? h->groups[index] : h->mixed_groups[index - nr];
        out->kind = index < nr ? 1 : 0;
        out->count = g.count;
        out->threads = g.threads;
        out->persistent = g.persistent;
        out->smem_bytes = (int64_t)(index >= nr && g.threads == 32 && !g.persistent ? g.smem_warp : g.smem);
        out->tuned_ms = g.tuned_ms;
    } else if (index < nr + nm + nc + ns) {
        out->kind = 2;
        out->count = h->num_streamed;
        out->threads = lpb::kStreamedThreads;
        out->persistent = 1;
        out->smem_bytes = 0;
        out->tuned_ms = -1.0f;
    } else {
        out->kind = 4;
        out->count = h->num_mstream;
        out->threads = lpb::kMixedStreamedThreads;
        out->persistent = 1;
        out->smem_bytes = 0;
        out->tuned_ms = -1.0f;
    }
    return LPB_OK;
}

lpb_err lp_batch_solve_warm(lp_batch* h, lp_mlp* net, float threshold, void* stream) {
    g_last_error.clear();
    if (!h || !net) return fail(LPB_EINVAL, "handle or network is NULL");
    if (!(threshold > 0.0f && threshold < 1.0f)) return fail(LPB_EINVAL, "threshold must be in (0, 1)");
    if (h->uniform_m < 0) return fail(LPB_EINVAL, "a warm solve needs LPs of one size");
    const int m = h->uniform_m, n = h->uniform_n;
    int n_in = 0, n_out = 0, net_dev = -1;
    lpb::mlp_shape(net, &n_in, &n_out, &net_dev);
    if (n_in != m + n || n_out != m) return fail(LPB_EINVAL, "network widths must be m + n inputs and m outputs");
    if (net_dev != h->device) return fail(LPB_EINVAL, "network and batch are on different devices");
    if (h->cold_smem > lpb::kMaxSmemPerBlock - 1024)
        return fail(LPB_ETOOBIG, "a warm solve needs every LP's FP64 tableau to fit in shared memory");
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t err;
    const int32_t N = h->num_lps;
    if (!h->warm_x) {
        if ((err = alloc(h, &h->warm_x, (size_t)N * (m + n), s)) || (err = alloc(h, &h->warm_logits, (size_t)N * m, s)) ||
            (err = alloc(h, &h->warm_q, (size_t)N, s)) || (err = alloc(h, &h->warm_q2, (size_t)N, s)) ||
            (err = alloc(h, &h->warm_stats, 8, s)) ||
            (err = lpb::fp64_kernels_prepare())) {
            h->warm_x = nullptr;
            return cuda_fail(err, "warm-start buffers");
        }
    }
    // restricted rows at most: a first pass with a cap of 16 (the shared
    // memory of a smaller tableau puts more LPs on an SM: 200 x 100 family,
    // ~6 active rows, 3.96 against 4.82 ms per 1e5 LPs with a cap of 32), then
    // a second pass with a cap of 32 over the LPs whose rows outgrew the
    // first; the cold solve gets what neither certifies
    const int kmax1 = std::min(m, 16), kmax2 = std::min(m, 32);
    const bool two_pass = kmax2 > kmax1;
    const float logit_thr = (float)std::log((double)threshold / (1.0 - (double)threshold));
    int sms = 0;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device))) return cuda_fail(err, "device query");
    const size_t cold_smem = (h->cold_smem + 1023) / 1024 * 1024;
    const int ctas = sms * lpb::fp64_resident_queue_ctas_per_sm(h->cold_threads, cold_smem);
    if ((err = cudaMemsetAsync(h->diag, 0, 8 * sizeof(int32_t), s)) ||
        (err = cudaMemsetAsync(h->warm_stats, 0, 8 * sizeof(int32_t), s)) ||
        (err = lpb::launch_warm_features(h->d, N, m, n, h->warm_x, s)))
        return cuda_fail(err, "warm-start features");
    lpb_err r = lp_mlp_forward(net, h->warm_x, N, h->warm_logits, stream);
    if (r != LPB_OK) return r;
    if ((err = lpb::launch_warm(h->d, h->warm_logits, N, m, n, kmax1, /*max_rounds=*/8, /*max_iters=*/50 * (kmax1 + n),
                                logit_thr, h->tol.eps_opt, h->tol.eps_piv, /*cert_tol=*/1e-9, h->warm_q,
                                h->warm_stats, N, nullptr, nullptr, two_pass ? h->warm_q2 : nullptr,
                                two_pass ? h->warm_stats + 4 : nullptr, h->warm_stats + 1, h->warm_stats + 2, h->diag,
                                s)) ||
        (two_pass &&
         (err = lpb::launch_warm(h->d, h->warm_logits, N, m, n, kmax2, /*max_rounds=*/8,
                                 /*max_iters=*/50 * (kmax2 + n), logit_thr, h->tol.eps_opt, h->tol.eps_piv,
                                 /*cert_tol=*/1e-9, h->warm_q, h->warm_stats, N, h->warm_q2, h->warm_stats + 4,
                                 nullptr, nullptr, h->warm_stats + 1, h->warm_stats + 2, h->diag, s))) ||
        (err = lpb::launch_fp64_resident_queue(h->d, h->tol, h->warm_q, h->warm_stats, N, N, h->warm_stats + 3,
                                               h->diag, ctas, h->cold_threads, cold_smem, s)))
        return cuda_fail(err, "warm solve");
    h->last_stream = s;
    h->solved = true;
    h->last_warm = true;
    return LPB_OK;
}

lpb_err lp_batch_features(lp_batch* h, float* x, void* stream) {
    g_last_error.clear();
    if (!h || !x) return fail(LPB_EINVAL, "handle or x is NULL");
    if (h->uniform_m < 0) return fail(LPB_EINVAL, "features need LPs of one size");
    DeviceGuard guard(h->device);
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, x) != cudaSuccess ||
        !(at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == h->device))) {
        cudaGetLastError();
        return fail(LPB_EINVAL, "x must be device memory of the batch's device");
    }
    cudaError_t err = lpb::launch_warm_features(h->d, h->num_lps, h->uniform_m, h->uniform_n, x,
                                                static_cast<cudaStream_t>(stream));
    return err ? cuda_fail(err, "features") : LPB_OK;
}

lpb_err lp_batch_active_labels(lp_batch* h, float* labels, void* stream) {
    g_last_error.clear();
    if (!h || !labels) return fail(LPB_EINVAL, "handle or labels is NULL");
    if (h->uniform_m < 0) return fail(LPB_EINVAL, "labels need LPs of one size");
    if (!h->solved) return fail(LPB_ENOTSOLVED, "lp_batch_solve has not been called");
    DeviceGuard guard(h->device);
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, labels) != cudaSuccess ||
        !(at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == h->device))) {
        cudaGetLastError();
        return fail(LPB_EINVAL, "labels must be device memory of the batch's device");
    }
    cudaError_t err = lpb::launch_warm_labels(h->d, h->num_lps, h->uniform_m, labels, static_cast<cudaStream_t>(stream));
    return err ? cuda_fail(err, "labels") : LPB_OK;
}

lpb_err lp_batch_results(lp_batch* h, int32_t* status, int32_t* iters, double* obj, double* x, double* y,
                         int32_t ptr_kind) {
    g_last_error.clear();
    if (!h) return fail(LPB_EINVAL, "handle is NULL");
    if (ptr_kind != LPB_HOST && ptr_kind != LPB_DEVICE) return fail(LPB_EINVAL, "ptr_kind must be LPB_HOST or LPB_DEVICE");
    if (!h->solved) return fail(LPB_ENOTSOLVED, "lp_batch_solve has not been called");
    DeviceGuard guard(h->device);
    cudaStream_t s = h->last_stream;
    const cudaMemcpyKind kind = ptr_kind == LPB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t nl = (size_t)h->num_lps;
    cudaError_t err = cudaSuccess;
    if (status && (err = cudaMemcpyAsync(status, h->d.status, nl * 4, kind, s))) return cuda_fail(err, "copy status");
    if (iters && (err = cudaMemcpyAsync(iters, h->d.iters, nl * 4, kind, s))) return cuda_fail(err, "copy iters");
    if (obj && (err = cudaMemcpyAsync(obj, h->d.obj, nl * 8, kind, s))) return cuda_fail(err, "copy obj");
    if (x && (err = cudaMemcpyAsync(x, h->d.x, (size_t)h->total_x * 8, kind, s))) return cuda_fail(err, "copy x");
    if (y && (err = cudaMemcpyAsync(y, h->d.y, (size_t)h->total_y * 8, kind, s))) return cuda_fail(err, "copy y");
    if ((err = cudaStreamSynchronize(s))) return cuda_fail(err, "solve");
    return LPB_OK;
}

lpb_err lp_batch_set_timing(lp_batch* h, int32_t enable) {
    g_last_error.clear();
    if (!h) return fail(LPB_EINVAL, "handle is NULL");
    DeviceGuard guard(h->device);
    if (!enable) {
        if (h->solved && !h->tev.empty()) cudaStreamSynchronize(h->last_stream);
        for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
        h->tev.clear();
        h->timed_solves = 0;
        return LPB_OK;
    }
    if (!h->tev.empty()) return LPB_OK;
    h->tev.assign(3 * (size_t)kTimingRing, nullptr);
    for (cudaEvent_t& e : h->tev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            for (cudaEvent_t& f : h->tev)
                if (f) cudaEventDestroy(f);
            h->tev.clear();
            return cuda_fail(err, "timing events");
        }
    }
    h->timed_solves = 0;
    return LPB_OK;
}

lpb_err lp_batch_stage_times(lp_batch* h, float* stage_ms, int32_t* num_solves) {
    g_last_error.clear();
    if (!h || !stage_ms || !num_solves) return fail(LPB_EINVAL, "handle, stage_ms or num_solves is NULL");
    *num_solves = 0;
    if (h->tev.empty()) return fail(LPB_EINVAL, "stage timing is not enabled (lp_batch_set_timing)");
    const int64_t n = std::min<int64_t>(h->timed_solves, kTimingRing);
    if (n == 0) return LPB_OK;
    DeviceGuard guard(h->device);
    const int64_t last = (h->timed_solves - 1) % kTimingRing;
    cudaError_t err = cudaEventSynchronize(h->tev[3 * last + 2]);
    if (err != cudaSuccess) return cuda_fail(err, "timing wait");
    double sum0 = 0.0, sum1 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        float a = 0.0f, b = 0.0f;
        if ((err = cudaEventElapsedTime(&a, h->tev[3 * i], h->tev[3 * i + 1])) ||
            (err = cudaEventElapsedTime(&b, h->tev[3 * i + 1], h->tev[3 * i + 2])))
            return cuda_fail(err, "timing read");
        sum0 += a;
        sum1 += b;
    }
    stage_ms[0] = (float)(sum0 / (double)n);
    stage_ms[1] = (float)(sum1 / (double)n);
    *num_solves = (int32_t)n;
    h->timed_solves = 0;
    return LPB_OK;
}

lpb_err lp_batch_plan_info(lp_batch* h, lp_batch_plan* plan) {
    if (!h || !plan) return fail(LPB_EINVAL, "handle or plan is NULL");
    plan->num_groups = (int32_t)(h->groups.size() + h->mixed_groups.size() + h->cluster_groups.size()) +
                       (h->num_streamed > 0 ? 1 : 0) + (h->num_mstream > 0 ? 1 : 0) + (h->num_fsmall > 0 ? 1 : 0) +
                       (h->num_fbig > 0 ? 1 : 0) + (h->num_single > 0 ? 1 : 0);
    plan->num_resident = h->num_lps - h->num_streamed - h->num_mstream - h->num_cluster - h->num_single_streamed;
    plan->num_cluster = h->num_cluster;
    plan->num_mixed = h->num_mixed;
    plan->num_fallback = 0;
    plan->num_warm_certified = 0;
    plan->num_warm_rounds = 0;
    plan->num_warm_retried = 0;
    plan->internal_errors = 0;
    plan->internal_error_code = 0;
    plan->internal_error_lp = -1;
    for (int i = 0; i < 5; ++i) plan->internal_error_detail[i] = 0;
    if (h->solved) {
        DeviceGuard guard(h->device);
        int32_t fb = 0, fbig = 0, dg[8] = {0, 0, -1, 0, 0, 0, 0, 0}, ws[5] = {0, 0, 0, 0, 0};
        cudaError_t err = cudaSuccess;
        if (h->last_warm)
            err = cudaMemcpyAsync(ws, h->warm_stats, sizeof ws, cudaMemcpyDeviceToHost, h->last_stream);
        else if (h->num_mixed > 0 &&
                 (err = cudaMemcpyAsync(&fb, h->fb_len, sizeof fb, cudaMemcpyDeviceToHost, h->last_stream)) == cudaSuccess)
            err = cudaMemcpyAsync(&fbig, h->fbig_len, sizeof fbig, cudaMemcpyDeviceToHost, h->last_stream);
        if (err == cudaSuccess) err = cudaMemcpyAsync(dg, h->diag, sizeof dg, cudaMemcpyDeviceToHost, h->last_stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(h->last_stream);
        if (err != cudaSuccess) return cuda_fail(err, "plan counters");
        plan->num_fallback = h->last_warm ? ws[0] : fb + fbig;
        plan->num_warm_certified = h->last_warm ? ws[1] : 0;
        plan->num_warm_rounds = h->last_warm ? ws[2] : 0;
        plan->num_warm_retried = h->last_warm ? ws[4] : 0;
        plan->internal_errors = dg[0];
        plan->internal_error_code = dg[0] ? dg[1] : 0;
        plan->internal_error_lp = dg[0] ? dg[2] : -1;
        for (int i = 0; i < 5; ++i) plan->internal_error_detail[i] = dg[0] ? dg[3 + i] : 0;
    }
    plan->num_streamed = h->num_streamed + h->num_mstream + h->num_single_streamed;
    plan->num_phase1 = h->num_phase1;
    plan->max_smem_bytes = (int64_t)h->max_smem;
    plan->workspace_bytes = (int64_t)h->streamed_slots * (int64_t)h->slot_bytes +
                            (int64_t)h->mstream_slots * (int64_t)h->mslot_bytes +
                            (int64_t)h->fbig_slots * (int64_t)h->fbig_slot_bytes +
                            (h->single_workspace ? (int64_t)h->single_ctas * (int64_t)h->single_slot_bytes : 0);
    return LPB_OK;
}

lpb_err lp_hyperbox_solve(int32_t num_lps, int32_t dim, const double* lo, const double* hi, int32_t box_per_lp,
                          const double* L, double* obj, double* x, int32_t ptr_kind, void* stream) {
    g_last_error.clear();
    if (num_lps < 0 || dim < 1) return fail(LPB_EINVAL, "num_lps must be >= 0 and dim >= 1");
    if (dim > LPB_MAX_HYPERBOX_DIM) return fail(LPB_ETOOBIG, "dim exceeds LPB_MAX_HYPERBOX_DIM");
    if (!lo || !hi || !L || !obj) return fail(LPB_EINVAL, "lo, hi, L and obj must not be NULL");
    if (ptr_kind != LPB_HOST && ptr_kind != LPB_DEVICE) return fail(LPB_EINVAL, "ptr_kind must be LPB_HOST or LPB_DEVICE");
    if (num_lps == 0) return LPB_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n_el = (size_t)num_lps * (size_t)dim;
    const size_t box_el = box_per_lp ? n_el : (size_t)dim;
    cudaError_t err;
    if (ptr_kind == LPB_DEVICE) {
        // every array must be memory the current device can address
        int dev = 0;
        if ((err = cudaGetDevice(&dev))) return cuda_fail(err, "cudaGetDevice");
        const void* ptrs[] = {lo, hi, L, obj, x};
        for (const void* p : ptrs) {
            if (!p) continue;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type == cudaMemoryTypeUnregistered ||
                at.type == cudaMemoryTypeHost || (at.type == cudaMemoryTypeDevice && at.device != dev)) {
                cudaGetLastError();
                return fail(LPB_EINVAL, "LPB_DEVICE pointer is not device memory of the current device");
            }
        }
        if ((err = lpb::launch_hyperbox(L, lo, hi, box_per_lp != 0, obj, x, num_lps, dim, s)))
            return cuda_fail(err, "hyperbox launch");
        return LPB_OK;
    }
    // host arrays: stage through stream-ordered device buffers
    double *dL = nullptr, *dlo = nullptr, *dhi = nullptr, *dobj = nullptr, *dx = nullptr;
    auto cleanup = [&]() {
        for (double* p : {dL, dlo, dhi, dobj, dx})
            if (p) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
    };
    if ((err = cudaMallocAsync((void**)&dL, n_el * 8, s)) || (err = cudaMallocAsync((void**)&dlo, box_el * 8, s)) ||
        (err = cudaMallocAsync((void**)&dhi, box_el * 8, s)) ||
        (err = cudaMallocAsync((void**)&dobj, (size_t)num_lps * 8, s)) ||
        (x && (err = cudaMallocAsync((void**)&dx, n_el * 8, s)))) {
        cleanup();
        return err == cudaErrorMemoryAllocation ? fail(LPB_ENOMEM, "device buffers") : cuda_fail(err, "device buffers");
    }
    if ((err = cudaMemcpyAsync(dL, L, n_el * 8, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(dlo, lo, box_el * 8, cudaMemcpyHostToDevice, s)) ||
        (err = cudaMemcpyAsync(dhi, hi, box_el * 8, cudaMemcpyHostToDevice, s)) ||
        (err = lpb::launch_hyperbox(dL, dlo, dhi, box_per_lp != 0, dobj, dx, num_lps, dim, s)) ||
        (err = cudaMemcpyAsync(obj, dobj, (size_t)num_lps * 8, cudaMemcpyDeviceToHost, s)) ||
        (x && (err = cudaMemcpyAsync(x, dx, n_el * 8, cudaMemcpyDeviceToHost, s)))) {
        cleanup();
        return cuda_fail(err, "hyperbox solve");
    }
    cleanup();
    if ((err = cudaGetLastError())) return cuda_fail(err, "hyperbox solve");
    return LPB_OK;
}

lpb_err lp_batch_destroy(lp_batch* h) {
    if (!h) return LPB_OK;
    DeviceGuard guard(h->device);
    cudaStreamSynchronize(h->last_stream);
    release(h, h->last_stream);
    delete h;
    return LPB_OK;
}

lpb_err lp_solve_host(int32_t num_lps, const int32_t* m, const int32_t* n,
                      const int64_t* a_off, const double* A, int64_t a_len,
                      const int64_t* b_off, const double* b, int64_t b_len,
                      const int64_t* c_off, const double* c, int64_t c_len,
                      const lp_batch_opts* opts, int32_t chunks,
                      int32_t* status, int32_t* iters, double* obj, double* x, double* y) {
    g_last_error.clear();
    if (num_lps < 1) return fail(LPB_EINVAL, "num_lps < 1");
    if (!m || !n || !A || !b || !c) return fail(LPB_EINVAL, "m, n, A, b and c must be non-NULL");
    if (!status || !iters || !obj || !x) return fail(LPB_EINVAL, "status, iters, obj and x must be non-NULL");
    if (chunks < 0 || chunks > LPB_MAX_HOST_CHUNKS) return fail(LPB_EINVAL, "chunks must be in [0, LPB_MAX_HOST_CHUNKS]");
    if (chunks == 0) {
        // one chunk per 256 MiB of input, at most 8: the first chunk's copy is
        // the one not overlapped with a solve (1e5 dense 50 x 50 LPs, 2.08 GB
        // from pinned memory at ~211 GB/s: 24.8 / 19.6 / 17.2 / 17.7 / 16.3 /
        // 18.6 / 23.9 ms for 1 / 2 / 4 / 6 / 8 / 12 / 16 chunks)
        const double per = 256.0 * 1024 * 1024;
        const double bytes = 8.0 * ((double)std::max<int64_t>(a_len, 0) + (double)std::max<int64_t>(b_len, 0) +
                                    (double)std::max<int64_t>(c_len, 0));
        chunks = (int32_t)std::min(8.0, std::max(1.0, std::ceil(bytes / per)));
    }
    chunks = std::min(chunks, num_lps);
    // every LP's offsets (packed when NULL); each chunk passes the smallest
    // ranges of A, b and c that hold its LPs, with offsets rebased to them
    std::vector<int64_t> ha(num_lps), hb(num_lps), hc(num_lps);
    int64_t pa = 0, pb = 0, pc = 0;
    for (int32_t k = 0; k < num_lps; ++k) {
        const int64_t mk = m[k], nk = n[k];
        if (mk < 1 || nk < 1) return fail(LPB_EINVAL, "LP " + std::to_string(k) + ": m and n must be >= 1");
        ha[k] = a_off ? a_off[k] : pa;
        hb[k] = b_off ? b_off[k] : pb;
        hc[k] = c_off ? c_off[k] : pc;
        pa += mk * nk; pb += mk; pc += nk;
        if (ha[k] < 0 || ha[k] + mk * nk > a_len || hb[k] < 0 || hb[k] + mk > b_len || hc[k] < 0 ||
            hc[k] + nk > c_len)
            return fail(LPB_EINVAL, "LP " + std::to_string(k) + ": offset out of range");
    }
    std::vector<cudaStream_t> streams(chunks, nullptr);
    std::vector<cudaEvent_t> copied(chunks, nullptr);
    std::vector<lp_batch*> hs(chunks, nullptr);
    std::vector<int32_t> k0s(chunks + 1);
    std::vector<int64_t> xs(chunks), ys(chunks);
    lpb_err e = LPB_OK;
    int64_t px = 0, py = 0;
    for (int32_t i = 0; i <= chunks; ++i) k0s[i] = (int32_t)((int64_t)num_lps * i / chunks);
    // The phase-I row counts of ranges 1.. are taken by a helper thread while
    // range 0 is created: each create would otherwise read its range's b on
    // the host path that issues the copies (~0.3 ms per 12,500 LPs of 50 rows
    // on the GPU machine's host).
    std::vector<int32_t> phase1(chunks > 1 ? (size_t)num_lps : 0);
    std::atomic<int32_t> counted{0};  // ranges 1 .. counted-1 are done
    std::thread counter;
    bool helper = false;
    if (chunks > 1) {
        counted.store(1, std::memory_order_relaxed);
        try {
            counter = std::thread([&] {
                for (int32_t i = 1; i < chunks; ++i) {
                    for (int32_t k = k0s[i]; k < k0s[i + 1]; ++k) phase1[k] = count_negative(b + hb[k], m[k]);
                    counted.store(i + 1, std::memory_order_release);
                }
            });
            helper = true;
        } catch (...) {
            helper = false;  // no thread: every create counts its own range
        }
    }
    // Every chunk is created and its solve enqueued without waiting for the
    // device: the copies run back to back (chunk i+1's copy waits for chunk
    // i's, so the first chunk has the bandwidth to itself), each solve starts
    // when its chunk's copy and input check end, and the input checks are
    // read after the solves.
    for (int32_t i = 0; i < chunks && e == LPB_OK; ++i) {
        const int32_t k0 = k0s[i], k1 = k0s[i + 1];
        xs[i] = px;
        ys[i] = py;
        int64_t alo = INT64_MAX, ahi = 0, blo = INT64_MAX, bhi = 0, clo = INT64_MAX, chi = 0;
        for (int32_t k = k0; k < k1; ++k) {
            px += n[k];
            py += m[k];
            alo = std::min(alo, ha[k]); ahi = std::max(ahi, ha[k] + (int64_t)m[k] * n[k]);
            blo = std::min(blo, hb[k]); bhi = std::max(bhi, hb[k] + (int64_t)m[k]);
            clo = std::min(clo, hc[k]); chi = std::max(chi, hc[k] + (int64_t)n[k]);
        }
        std::vector<int64_t> sa(k1 - k0), sb(k1 - k0), sc(k1 - k0);
        for (int32_t k = k0; k < k1; ++k) {
            sa[k - k0] = ha[k] - alo;
            sb[k - k0] = hb[k] - blo;
            sc[k - k0] = hc[k] - clo;
        }
        cudaError_t err = cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming);
        if (err == cudaSuccess && i > 0) err = cudaStreamWaitEvent(streams[i], copied[i - 1], 0);
        if (err != cudaSuccess) {
            e = cuda_fail(err, "stream creation");
            break;
        }
        if (helper && i > 0)
            while (counted.load(std::memory_order_acquire) <= i) std::this_thread::yield();
        e = create_batch(&hs[i], k1 - k0, m + k0, n + k0, sa.data(), A + alo, ahi - alo, sb.data(), b + blo,
                         bhi - blo, sc.data(), c + clo, chi - clo, LPB_HOST, opts, streams[i], copied[i], true,
                         helper && i > 0 ? phase1.data() + k0 : nullptr);
        if (e == LPB_OK) e = lp_batch_solve(hs[i], streams[i]);
    }
    if (helper) counter.join();
    // the input checks (each read waits for its chunk's solve); results only
    // when every chunk's inputs were finite
    for (int32_t i = 0; i < chunks && e == LPB_OK; ++i) {
        unsigned long long bad = 0;
        cudaError_t err = cudaMemcpyAsync(&bad, hs[i]->d_bad, sizeof bad, cudaMemcpyDeviceToHost, streams[i]);
        if (err == cudaSuccess) err = cudaStreamSynchronize(streams[i]);
        if (err != cudaSuccess)
            e = cuda_fail(err, "input check");
        else if (bad)
            e = fail(LPB_EINVAL, "LPs " + std::to_string(k0s[i]) + ".." + std::to_string(k0s[i + 1] - 1) + ": " +
                                     std::to_string(bad) + " non-finite entries in A, b or c");
    }
    for (int32_t i = 0; i < chunks && e == LPB_OK; ++i) {
        const int32_t k0 = k0s[i];
        e = lp_batch_results(hs[i], status + k0, iters + k0, obj + k0, x + xs[i], y ? y + ys[i] : nullptr, LPB_HOST);
    }
    const std::string msg = g_last_error;
    for (int32_t i = 0; i < chunks; ++i) {
        if (hs[i]) lp_batch_destroy(hs[i]);
        if (streams[i]) {
            cudaStreamSynchronize(streams[i]);
            cudaStreamDestroy(streams[i]);
        }
    }
    for (int32_t i = 0; i < chunks; ++i)
        if (copied[i]) cudaEventDestroy(copied[i]);
    if (e != LPB_OK) return fail(e, msg);
    return LPB_OK;
}

}  // extern "C"
