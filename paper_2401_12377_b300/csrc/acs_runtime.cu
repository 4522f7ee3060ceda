// Host side of libacs: the C ABI declared in include/acs.h.
//
// acs_submit* validates a task and writes its 320-byte descriptor straight
// into a pinned host ring that mirrors the stream's device ring position for
// position. acs_flush copies the new range with one cudaMemcpyAsync per stream
// (two where the ring wraps) and, in window mode, starts the persistent
// scheduler kernel with a cooperative launch (which fails instead of
// oversubscribing, so every scheduler and worker CTA is co-resident). That
// copy is the only host->device crossing per flush; nothing crosses per task.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "acs_internal.h"

namespace acs {
const void *persistent_kernel_fn();
const void *body_kernel_fn();
cudaError_t launch_init(unsigned long long *cells, uint32_t ncells, DevCtl *ctl, unsigned long long *done,
                        uint32_t nslots, cudaStream_t st);
}  // namespace acs

using namespace acs;

// The persistent kernel's dynamic shared-memory limit is per-function state
// of the process, shared by every context: it is only ever raised (under a
// lock), so that creating a context with a smaller window never makes a live
// context's launches fail.
cudaError_t acs::raise_kernel_smem_limit(uint32_t bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    const void *kfn = persistent_kernel_fn();
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kfn);
    if (e != cudaSuccess) return e;
    if ((uint32_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}


namespace {

struct StreamState {
    uint32_t submitted = 0;  // next seq
    uint32_t flushed = 0;    // seqs below were handed to the device
    uint32_t synced = 0;     // seqs below are known retired (last acs_sync)
    bool has_id = false;
    uint32_t last_id = 0;
    uint32_t emit_pending = 0;  // emit tasks submitted since the last flush
    bool emitting = false;      // flushed emit tasks not yet synced: the device owns the end
    uint32_t base = 0;          // position the stream was last restarted at (acs_stream_rebase)
};

// tasks a stream had before position `first` since its last restart, capped
// at 64 (the most predecessors a window tests)
uint8_t tasks_before(const StreamState &ss, uint32_t first) {
    const uint32_t n = first - ss.base;
    return (uint8_t)(n < 64u ? n : 64u);
}

int64_t wrap_diff(uint32_t a, uint32_t b) { return (int64_t)(int32_t)(a - b); }

struct TimedLaunch {
    cudaEvent_t a, b;
};

uint32_t log2_pow2(uint32_t v) {
    uint32_t l = 0;
    while ((1u << l) < v) ++l;
    return l;
}

}  // namespace

// ACS_MODE_SW: the paper's software scheduler on the host (Sec. IV-B, Alg. 2).
struct SwTask {
    uint32_t stream, q;             // stream and position
    uint32_t up = 0;                // upstream tasks not yet complete
    std::vector<uint32_t> down;     // tasks waiting on this one
};

struct SwState {
    std::mutex m;
    std::condition_variable work;   // threads: a ready task or shutdown
    std::condition_variable idle;   // flush: every task complete or an error
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;
    bool shutdown = false;
    std::vector<SwTask> tasks;                 // this flush's tasks, stream by stream
    std::deque<uint32_t> ready;                // oldest first
    std::vector<std::vector<uint32_t>> window; // per stream: tasks inserted and not complete
    std::vector<uint32_t> next, end;           // per stream: next task to insert, one past the last
    uint32_t remaining = 0;         // tasks of this flush not yet complete
    uint32_t inflight = 0;          // tasks a thread launched and has not completed
    int err = 0;
};

// A resident flush's descriptor copies (copy engine, beside the kernel) and
// the stream ends to publish once they completed.
struct PendingPub {
    cudaEvent_t ev;
    std::vector<std::pair<uint32_t, uint32_t>> ends;
};

struct acs_ctx {
    acs_config cfg{};
    uint32_t W = 0, S = 0, C = 0, cap_log2 = 0, LC = 0, log_log2 = 0;
    uint32_t Wact = 0;   // the window; W is the ring span (free-slot span, or window + ahead)
    uint32_t ahead = 0;  // dispatch lookahead (0: off)
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    TaskRec *h_ring = nullptr;  // pinned [S][C]
    TaskRec *d_ring = nullptr;
    DevCtl *d_ctl = nullptr;
    unsigned long long *d_done = nullptr;
    unsigned long long *d_cells = nullptr;
    TaskAux *d_taskaux = nullptr;
    uint32_t ncells = 0;
    unsigned long long *d_log_mask = nullptr, *d_log_start = nullptr, *d_log_retire = nullptr;
    SchedStats *d_sched_stats = nullptr;
    unsigned long long *d_trace = nullptr;
    StreamCtl *d_sctl = nullptr;
    HostStatus *h_status = nullptr, *d_status = nullptr;
    // resident launches (acs_start .. acs_stop)
    bool resident = false;
    Mailbox *h_mbox = nullptr, *d_mbox = nullptr;
    Mirror *d_mirror = nullptr;          // device copy of the mailbox's host-written words
    cudaStream_t side = nullptr;         // copies beside the resident kernel
    std::deque<PendingPub> pend;         // descriptor copies not yet published
    std::vector<cudaEvent_t> pub_events; // free events for them
    uint32_t *h_one = nullptr;           // pinned source of those copies
    std::vector<StreamState> st;
    int err = ACS_OK;
    uint32_t aborted = 0;                // acs_abort was called (atomic: any host thread)
    uint32_t grid = 0, cta_slots = 0, smem = 0;
    acs_stats stats{};
    std::vector<TimedLaunch> timed;     // launches whose events are not yet read
    std::vector<TimedLaunch> event_pool;
    // graph mode
    cudaGraphExec_t last_exec = nullptr;
    std::vector<cudaGraphExec_t> execs_pending;
    std::vector<cudaGraph_t> graphs_pending;
    // software scheduler (ACS_MODE_SW)
    SwState *sw = nullptr;
};

namespace {

int fail(acs_ctx *c, int code) {
    if (c && c->err == ACS_OK) c->err = code;
    return code;
}

int cuda_fail(acs_ctx *c, cudaError_t e) {
    if (e == cudaSuccess) return ACS_OK;
    if (e == cudaErrorMemoryAllocation) return fail(c, ACS_ERR_NOMEM);
    return fail(c, ACS_ERR_DEVICE);
}

TimedLaunch get_events(acs_ctx *c) {
    if (!c->event_pool.empty()) {
        TimedLaunch t = c->event_pool.back();
        c->event_pool.pop_back();
        return t;
    }
    TimedLaunch t{};
    cudaEventCreate(&t.a);
    cudaEventCreate(&t.b);
    return t;
}

// Segment validation and conversion to the inclusive form; returns false on
// overflow. Empty segments are skipped.
bool add_segs(const acs_segment *s, uint32_t n, bool write, Seg *out, uint32_t &cnt, uint16_t &wmask,
              uint64_t &bytes) {
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t a = s[i].start, z = s[i].size;
        if (z == 0) continue;
        Seg g;
        if (a == ACS_WHOLE_MEMORY_START && z == ACS_WHOLE_MEMORY_SIZE) {
            g.start = 0;
            g.last = UINT64_MAX;
        } else {
            if (a != 0 && z - 1 > UINT64_MAX - a) return false;  // end past 2^64
            g.start = a;
            g.last = a + (z - 1);
            bytes += z;
        }
        if (cnt >= (uint32_t)kMaxSegs) return false;
        if (write) wmask |= (uint16_t)(1u << cnt);
        out[cnt++] = g;
    }
    return true;
}

bool valid_op(uint16_t op) {
    switch (op) {
    case ACS_OP_NOP: case ACS_OP_AXPY: case ACS_OP_SCALE: case ACS_OP_ADD: case ACS_OP_GEMV:
    case ACS_OP_BIAS_RELU: case ACS_OP_RESID: case ACS_OP_RL_BROADPHASE: case ACS_OP_RL_SOLVE:
    case ACS_OP_RL_INTEGRATE: case ACS_OP_RL_EMIT: case ACS_OP_WAIT_FLAG: case ACS_OP_SLEEP:
        return true;
    default:
        return false;
    }
}

// conflict test of the host-side DAG builder (graph baseline): same rule as
// the device window test, over inclusive ranges.
bool recs_conflict(const TaskRec &i, const TaskRec &j) {
    for (int x = 0; x < j.nseg; ++x) {
        const bool xw = (j.wmask >> x) & 1u;
        for (int y = 0; y < i.nseg; ++y) {
            const bool yw = (i.wmask >> y) & 1u;
            if ((xw || yw) && j.seg[x].start <= i.seg[y].last && i.seg[y].start <= j.seg[x].last) return true;
        }
    }
    return false;
}

void collect_timing(acs_ctx *c) {
    for (auto &t : c->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) c->stats.kernel_ms += ms;
        c->event_pool.push_back(t);
    }
    c->timed.clear();
}

int copy_new_descriptors(acs_ctx *c) {
    for (uint32_t s = 0; s < c->S; ++s) {
        StreamState &ss = c->st[s];
        uint32_t a = ss.flushed, b = ss.submitted;
        while (a < b) {
            const uint32_t pa = a & (c->C - 1);
            const uint32_t n = std::min(b - a, c->C - pa);
            const size_t off = (size_t)s * c->C + pa;
            cudaError_t e = cudaMemcpyAsync(c->d_ring + off, c->h_ring + off, (size_t)n * sizeof(TaskRec),
                                            cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e);
            a += n;
        }
    }
    return ACS_OK;
}

void fill_params(acs_ctx *c, KParams &P) {
    std::memset(&P, 0, sizeof P);
    P.recs = c->d_ring;
    P.ctl = c->d_ctl;
    P.cells = c->d_cells;
    P.taskaux = c->d_taskaux;
    P.done = c->d_done;
    P.log_mask = c->d_log_mask;
    P.log_start = c->d_log_start;
    P.log_retire = c->d_log_retire;
    P.sched_stats = c->d_sched_stats;
    P.trace = c->d_trace;
    P.sctl = c->d_sctl;
    P.hstatus = c->d_status;
    P.timeout_ns = c->cfg.timeout_ns;
    P.cap_log2 = c->cap_log2;
    P.log_log2 = c->log_log2;
    P.cell_mask = c->ncells - 1;
    P.window = c->W;
    // ring: W = Wact; free-slot: at most Wact tasks active among W slots, candidates over W;
    // dispatch ahead: W slots, candidates and admission over Wact
    P.active_limit = c->ahead ? c->W : c->Wact;
    P.check_w = c->ahead ? c->Wact : c->W;
    P.admit = c->ahead ? 1u : 0u;
    P.n_streams = c->S;
    P.flags = c->cfg.flags;
    P.sched_smem = sched_smem_bytes(c->W);
    P.poll_ns = c->cfg.poll_ns ? c->cfg.poll_ns : 128u;
    P.mbox = c->d_mbox;
    P.mirror = c->d_mirror;
    P.idle_limit_ns = (unsigned long long)(c->cfg.idle_limit_ms ? c->cfg.idle_limit_ms : 10000u) * 1000000ull;
}

int launch_persistent(acs_ctx *c, KParams &P) {
    void *args[] = {&P};
    TimedLaunch t{};
    const bool timing = (c->cfg.flags & ACS_FLAG_TIMING) != 0;
    if (timing) {
        t = get_events(c);
        cudaEventRecord(t.a, c->stream);
    }
    cudaError_t e = cudaLaunchCooperativeKernel(persistent_kernel_fn(), dim3(c->grid), dim3(kBlock), args,
                                                c->smem, c->stream);
    if (e != cudaSuccess) {
        if (timing) c->event_pool.push_back(t);
        return cuda_fail(c, e);
    }
    if (timing) {
        cudaEventRecord(t.b, c->stream);
        c->timed.push_back(t);
    }
    c->stats.launches++;
    return ACS_OK;
}

int flush_window(acs_ctx *c) {
    int rc = copy_new_descriptors(c);
    if (rc) return rc;
    KParams P;
    fill_params(c, P);
    for (uint32_t s = 0; s < c->S; ++s) {
        P.first[s] = c->st[s].flushed;
        P.nprev[s] = tasks_before(c->st[s], P.first[s]);
        P.end[s] = c->st[s].submitted;
        P.open[s] = (uint8_t)std::min<uint32_t>(c->st[s].emit_pending, 255u);
    }
    return launch_persistent(c, P);
}

// ---- resident launches ---------------------------------------------------------------

void heartbeat(acs_ctx *c) {
    __atomic_fetch_add(&c->h_mbox->heartbeat, 1ull, __ATOMIC_RELAXED);
}

// Take in what the device reported for stream s: released tasks free ring
// space; an idle end at or past everything published means the stream's
// tasks (and any emitter chain they started) all retired.
void refresh_stream(acs_ctx *c, uint32_t s) {
    StreamState &ss = c->st[s];
    const uint32_t head = __atomic_load_n(&c->h_mbox->progress[s].head, __ATOMIC_ACQUIRE);
    const uint32_t idle = __atomic_load_n(&c->h_mbox->progress[s].idle_at, __ATOMIC_ACQUIRE);
    if (wrap_diff(head, ss.synced) > 0 && wrap_diff(head, ss.flushed) <= 0) ss.synced = head;
    if (wrap_diff(idle, ss.flushed) >= 0) {
        if (ss.emitting) {   // the chain's final end: the stream continues after it
            c->stats.tasks_emitted += idle - ss.flushed;
            ss.submitted = ss.flushed = idle;
            if (idle) { ss.has_id = true; ss.last_id = std::max(ss.last_id, idle - 1); }
            ss.emitting = false;
        }
        ss.synced = ss.flushed;
    }
}

int resident_status(acs_ctx *c) {
    const uint32_t e = __atomic_load_n(&c->h_mbox->err, __ATOMIC_ACQUIRE);
    if (e) return fail(c, (int)(int32_t)e);
    if (__atomic_load_n(&c->h_mbox->expired, __ATOMIC_ACQUIRE)) return fail(c, ACS_ERR_STOPPED);
    if (__atomic_load_n(&c->aborted, __ATOMIC_ACQUIRE)) return fail(c, ACS_ERR_STOPPED);
    return ACS_OK;
}

// Publish the ends of every resident flush whose descriptor copy completed,
// oldest first (wait: block on each copy).
int publish_ready(acs_ctx *c, bool wait) {
    while (!c->pend.empty()) {
        PendingPub &pp = c->pend.front();
        const cudaError_t q = wait ? cudaEventSynchronize(pp.ev) : cudaEventQuery(pp.ev);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return cuda_fail(c, q);
        // the descriptors are in the device ring; this store publishes them
        for (auto &se : pp.ends) __atomic_store_n(&c->h_mbox->host_end[se.first], se.second, __ATOMIC_RELEASE);
        c->pub_events.push_back(pp.ev);
        c->pend.pop_front();
    }
    return ACS_OK;
}

int flush_resident(acs_ctx *c) {
    int rc = resident_status(c);
    if (rc) return rc;
    PendingPub pp{};
    for (uint32_t s = 0; s < c->S; ++s) {
        StreamState &ss = c->st[s];
        if (ss.submitted == ss.flushed) continue;
        uint32_t a = ss.flushed;
        while (a != ss.submitted) {
            const uint32_t pa = a & (c->C - 1);
            const uint32_t n = std::min(ss.submitted - a, c->C - pa);
            const size_t off = (size_t)s * c->C + pa;
            cudaError_t e = cudaMemcpyAsync(c->d_ring + off, c->h_ring + off, (size_t)n * sizeof(TaskRec),
                                            cudaMemcpyHostToDevice, c->side);
            if (e != cudaSuccess) return cuda_fail(c, e);
            a += n;
        }
        pp.ends.emplace_back(s, ss.submitted);
    }
    if (!pp.ends.empty()) {
        if (c->pub_events.empty()) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(c, e);
            c->pub_events.push_back(ev);
        }
        pp.ev = c->pub_events.back();
        c->pub_events.pop_back();
        cudaError_t e = cudaEventRecord(pp.ev, c->side);
        if (e != cudaSuccess) return cuda_fail(c, e);
        c->pend.push_back(std::move(pp));
    }
    rc = publish_ready(c, false);
    heartbeat(c);
    return rc;
}

// ---- software scheduler (ACS_MODE_SW) ---------------------------------------------

const TaskRec &sw_rec(acs_ctx *c, const SwTask &t) {
    return c->h_ring[(size_t)t.stream * c->C + (t.q & (c->C - 1))];
}

// window module, insertion: the next tasks of stream s enter while the window
// has room; each is checked against every task still in the window (caller
// holds the lock)
void sw_insert(acs_ctx *c, uint32_t s) {
    SwState &w = *c->sw;
    auto &win = w.window[s];
    while (win.size() < c->Wact && w.next[s] < w.end[s]) {
        const uint32_t j = w.next[s]++;
        SwTask &tj = w.tasks[j];
        const TaskRec &rj = sw_rec(c, tj);
        for (uint32_t i : win)
            if (recs_conflict(sw_rec(c, w.tasks[i]), rj)) {
                w.tasks[i].down.push_back(j);
                tj.up++;
            }
        win.push_back(j);
        if (tj.up == 0) w.ready.push_back(j);
    }
}

// scheduler module: one thread, one CUDA stream, one task in flight
void sw_thread(acs_ctx *c, uint32_t k) {
    SwState &w = *c->sw;
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(w.m);
    while (true) {
        w.work.wait(lk, [&] { return w.shutdown || (!w.ready.empty() && !w.err); });
        if (w.shutdown) return;
        const uint32_t j = w.ready.front();
        w.ready.pop_front();
        w.inflight++;
        const TaskRec &r = sw_rec(c, w.tasks[j]);
        lk.unlock();
        TaskHdr h;
        std::memcpy(&h, &r, sizeof h);
        void *args[] = {&h};
        cudaError_t e = cudaLaunchKernel(body_kernel_fn(), dim3(r.ncta), dim3(kBlock), args, kBodySmem, w.streams[k]);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w.streams[k]);
        lk.lock();
        if (e != cudaSuccess && !w.err) w.err = e == cudaErrorMemoryAllocation ? ACS_ERR_NOMEM : ACS_ERR_DEVICE;
        // window module, completion: release dependents, free the slot
        SwTask &t = w.tasks[j];
        for (uint32_t d : t.down)
            if (--w.tasks[d].up == 0) w.ready.push_back(d);
        auto &win = w.window[t.stream];
        win.erase(std::find(win.begin(), win.end(), j));
        sw_insert(c, t.stream);
        c->stats.launches++;
        w.inflight--;
        if (--w.remaining == 0 || w.err || !w.inflight) w.idle.notify_all();
        w.work.notify_all();
    }
}

int sw_start(acs_ctx *c) {
    c->sw = new (std::nothrow) SwState();
    if (!c->sw) return ACS_ERR_NOMEM;
    const uint32_t K = c->cfg.sw_threads ? c->cfg.sw_threads : 8u;
    c->sw->streams.resize(K, nullptr);
    for (auto &st : c->sw->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return ACS_ERR_DEVICE;
    for (uint32_t k = 0; k < K; ++k) c->sw->threads.emplace_back(sw_thread, c, k);
    return ACS_OK;
}

void sw_stop(acs_ctx *c) {
    if (!c->sw) return;
    {
        std::lock_guard<std::mutex> g(c->sw->m);
        c->sw->shutdown = true;
    }
    c->sw->work.notify_all();
    for (auto &t : c->sw->threads) t.join();
    for (auto st : c->sw->streams)
        if (st) cudaStreamDestroy(st);
    delete c->sw;
    c->sw = nullptr;
}

int flush_sw(acs_ctx *c) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    // the caller's earlier work on its stream (buffer copies) comes first
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    SwState &w = *c->sw;
    std::unique_lock<std::mutex> lk(w.m);
    w.tasks.clear();
    w.ready.clear();
    w.window.assign(c->S, {});
    w.next.assign(c->S, 0);
    w.end.assign(c->S, 0);
    w.err = 0;
    for (uint32_t s = 0; s < c->S; ++s) {
        w.next[s] = (uint32_t)w.tasks.size();
        for (uint32_t q = c->st[s].flushed; q != c->st[s].submitted; ++q) w.tasks.push_back(SwTask{s, q});
        w.end[s] = (uint32_t)w.tasks.size();
    }
    w.remaining = (uint32_t)w.tasks.size();
    for (uint32_t s = 0; s < c->S; ++s) sw_insert(c, s);
    w.work.notify_all();
    const auto limit = std::chrono::nanoseconds(c->cfg.timeout_ns);
    uint32_t seen = w.remaining;
    auto last = clk::now();
    while (w.remaining && !w.err) {
        w.idle.wait_for(lk, std::chrono::milliseconds(10));
        if (w.remaining != seen) { seen = w.remaining; last = clk::now(); }
        else if (clk::now() - last > limit) { w.err = ACS_ERR_TIMEOUT; break; }
    }
    const int err = w.err;
    // threads launch nothing more after an error; wait for what they started
    // (each of their waits is a cudaStreamSynchronize, which returns)
    while (w.inflight) w.idle.wait_for(lk, std::chrono::milliseconds(1));
    w.ready.clear();
    lk.unlock();
    c->stats.kernel_ms += std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    return err ? fail(c, err) : ACS_OK;
}

int flush_inorder(acs_ctx *c) {
    const bool timing = (c->cfg.flags & ACS_FLAG_TIMING) != 0;
    TimedLaunch t{};
    if (timing) {
        t = get_events(c);
        cudaEventRecord(t.a, c->stream);
    }
    for (uint32_t s = 0; s < c->S; ++s) {
        StreamState &ss = c->st[s];
        for (uint32_t q = ss.flushed; q < ss.submitted; ++q) {
            const TaskRec &r = c->h_ring[(size_t)s * c->C + (q & (c->C - 1))];
            TaskHdr h;
            std::memcpy(&h, &r, sizeof h);
            void *args[] = {&h};
            cudaError_t e = cudaLaunchKernel(body_kernel_fn(), dim3(r.ncta), dim3(kBlock), args, kBodySmem, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e);
            c->stats.launches++;
        }
    }
    if (timing) {
        cudaEventRecord(t.b, c->stream);
        c->timed.push_back(t);
    }
    return ACS_OK;
}

int flush_graph(acs_ctx *c) {
    using clk = std::chrono::steady_clock;
    auto t0 = clk::now();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return cuda_fail(c, e);
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(body_kernel_fn());
    kp.blockDim = dim3(kBlock);
    kp.sharedMemBytes = kBodySmem;
    for (uint32_t s = 0; s < c->S; ++s) {
        StreamState &ss = c->st[s];
        const uint32_t n = ss.submitted - ss.flushed;
        if (!n) continue;
        std::vector<cudaGraphNode_t> nodes(n);
        const uint32_t words = (n + 63) / 64;
        std::vector<uint64_t> reach((size_t)n * words, 0);  // reach[j]: ancestors of j
        std::vector<cudaGraphNode_t> deps;
        for (uint32_t j = 0; j < n; ++j) {
            const TaskRec &rj = c->h_ring[(size_t)s * c->C + ((ss.flushed + j) & (c->C - 1))];
            uint64_t *rr = &reach[(size_t)j * words];
            deps.clear();
            // scan predecessors latest first; skip those already implied
            for (int64_t i = (int64_t)j - 1; i >= 0; --i) {
                if ((rr[i >> 6] >> (i & 63)) & 1u) continue;
                const TaskRec &ri = c->h_ring[(size_t)s * c->C + ((ss.flushed + i) & (c->C - 1))];
                if (!recs_conflict(ri, rj)) continue;
                deps.push_back(nodes[i]);
                const uint64_t *ra = &reach[(size_t)i * words];
                for (uint32_t w = 0; w < words; ++w) rr[w] |= ra[w];
                rr[i >> 6] |= 1ull << (i & 63);
            }
            TaskHdr h;
            std::memcpy(&h, &rj, sizeof h);
            void *args[] = {&h};
            kp.gridDim = dim3(rj.ncta);
            kp.kernelParams = args;
            e = cudaGraphAddKernelNode(&nodes[j], g, deps.empty() ? nullptr : deps.data(), deps.size(), &kp);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                return cuda_fail(c, e);
            }
            c->stats.graph_edges += deps.size();
        }
    }
    auto t1 = clk::now();
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    auto t2 = clk::now();
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, e);
    }
    c->stats.graph_build_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
    c->stats.graph_instantiate_ms += std::chrono::duration<double, std::milli>(t2 - t1).count();
    c->graphs_pending.push_back(g);
    c->execs_pending.push_back(x);
    c->last_exec = x;
    const bool timing = (c->cfg.flags & ACS_FLAG_TIMING) != 0;
    TimedLaunch t{};
    if (timing) {
        t = get_events(c);
        cudaEventRecord(t.a, c->stream);
    }
    e = cudaGraphLaunch(x, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (timing) {
        cudaEventRecord(t.b, c->stream);
        c->timed.push_back(t);
    }
    c->stats.launches++;
    return ACS_OK;
}

void release_graphs(acs_ctx *c, bool keep_last) {
    // everything launched has completed when this is called
    for (size_t i = 0; i < c->execs_pending.size(); ++i) {
        if (keep_last && c->execs_pending[i] == c->last_exec) continue;
        cudaGraphExecDestroy(c->execs_pending[i]);
        cudaGraphDestroy(c->graphs_pending[i]);
    }
    if (keep_last && c->last_exec) {
        for (size_t i = 0; i < c->execs_pending.size(); ++i) {
            if (c->execs_pending[i] == c->last_exec) {
                cudaGraphExec_t x = c->execs_pending[i];
                cudaGraph_t g = c->graphs_pending[i];
                c->execs_pending.assign(1, x);
                c->graphs_pending.assign(1, g);
                return;
            }
        }
    }
    c->execs_pending.clear();
    c->graphs_pending.clear();
    if (!keep_last) c->last_exec = nullptr;
}

}  // namespace

extern "C" {

void acs_config_default(acs_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->mode = ACS_MODE_WINDOW;
    cfg->n_streams = 1;
    cfg->capacity = 8192;
    cfg->timeout_ns = 5000000000ull;
    cfg->device = -1;
    cfg->lookahead = ACS_LOOKAHEAD_AUTO;
}

const char *acs_strerror(int code) {
    switch (code) {
    case ACS_OK: return "ok";
    case ACS_ERR_INVALID: return "invalid argument";
    case ACS_ERR_FULL: return "stream ring full (flush and sync, then retry)";
    case ACS_ERR_TIMEOUT: return "a bounded device wait made no progress before the timeout";
    case ACS_ERR_DEVICE: return "CUDA runtime error";
    case ACS_ERR_STOPPED: return "context stopped";
    case ACS_ERR_ORDER: return "task_id not strictly increasing within its stream";
    case ACS_ERR_NOMEM: return "out of memory";
    case ACS_ERR_RANGE: return "stream position reached 2^31 (acs_stream_rebase at an idle point)";
    default: return "unknown status";
    }
}

int acs_error(const acs_ctx *ctx) { return ctx ? ctx->err : ACS_ERR_INVALID; }

void acs_destroy(acs_ctx *c) {
    if (!c) return;
    if (c->resident) acs_stop(c);
    sw_stop(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    release_graphs(c, false);
    for (auto &t : c->timed) c->event_pool.push_back(t);
    for (auto &t : c->event_pool) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    cudaFree(c->d_ring);
    cudaFree(c->d_ctl);
    cudaFree(c->d_done);
    cudaFree(c->d_cells);
    cudaFree(c->d_taskaux);
    cudaFree(c->d_log_mask);
    cudaFree(c->d_log_start);
    cudaFree(c->d_log_retire);
    cudaFree(c->d_sched_stats);
    cudaFree(c->d_trace);
    cudaFree(c->d_sctl);
    cudaFree(c->d_mirror);
    if (c->h_ring) cudaFreeHost(c->h_ring);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_mbox) cudaFreeHost(c->h_mbox);
    if (c->h_one) cudaFreeHost(c->h_one);
    for (auto &pp : c->pend) c->pub_events.push_back(pp.ev);
    for (auto ev : c->pub_events) cudaEventDestroy(ev);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int acs_init(acs_ctx **out, uint32_t window, const acs_config *cfg_in) {
    if (!out) return ACS_ERR_INVALID;
    acs_config cfg;
    acs_config_default(&cfg);
    if (cfg_in) {
        cfg = *cfg_in;
        for (uint32_t r : cfg.reserved)
            if (r) return ACS_ERR_INVALID;
        if (!cfg.n_streams) cfg.n_streams = 1;
        if (!cfg.capacity) cfg.capacity = 8192;
        if (!cfg.timeout_ns) cfg.timeout_ns = 5000000000ull;
    }
    if (window < 1 || window > (uint32_t)kMaxWindow) return ACS_ERR_INVALID;
    if (cfg.span && (cfg.span < window || cfg.span > (uint32_t)kMaxWindow)) return ACS_ERR_INVALID;
    // dispatch ahead of the window (window mode only; not with a free-slot span)
    uint32_t ahead = cfg.lookahead;
    // (auto: single-stream contexts only; with several streams the lookahead's
    // claimed-but-waiting CTAs hold workers the other streams could use)
    if (ahead == ACS_LOOKAHEAD_AUTO)
        ahead = (cfg.span || cfg.mode != ACS_MODE_WINDOW || cfg.n_streams > 1) ? 0u
                                                                               : std::min(2u * window, (uint32_t)kMaxWindow - window);
    if (ahead && (cfg.span || cfg.mode != ACS_MODE_WINDOW || ahead > (uint32_t)kMaxWindow - window)) return ACS_ERR_INVALID;
    if (cfg.n_streams > ACS_MAX_STREAMS) return ACS_ERR_INVALID;
    if (cfg.mode > ACS_MODE_SW) return ACS_ERR_INVALID;
    if (cfg.capacity > (1u << 24)) return ACS_ERR_INVALID;

    acs_ctx *c = new (std::nothrow) acs_ctx();
    if (!c) return ACS_ERR_NOMEM;
    c->cfg = cfg;
    c->W = cfg.span ? cfg.span : window + ahead;
    c->Wact = window;
    c->ahead = ahead;
    c->S = cfg.n_streams;
    uint32_t cap = std::max<uint32_t>(cfg.capacity, kMinCapacity);
    cap = std::max<uint32_t>(cap, 2u * c->W + kPrefetch);
    c->cap_log2 = log2_pow2(cap);
    c->C = 1u << c->cap_log2;
    if ((uint64_t)c->S * c->C > (1ull << 24)) {  // work-ring payload holds a 24-bit descriptor index
        delete c;
        return ACS_ERR_INVALID;
    }
    uint32_t lc = cfg.log_capacity ? cfg.log_capacity : c->C;
    c->log_log2 = log2_pow2(std::max<uint32_t>(lc, 64));
    c->LC = 1u << c->log_log2;
    c->st.resize(c->S);

    cudaError_t e;
    if (cfg.device >= 0) {
        e = cudaSetDevice(cfg.device);
        if (e != cudaSuccess) { delete c; return ACS_ERR_DEVICE; }
    }
    cudaGetDevice(&c->device);
    int rc = ACS_OK;
    auto chk = [&](cudaError_t e2) {
        if (e2 != cudaSuccess && rc == ACS_OK) rc = (e2 == cudaErrorMemoryAllocation) ? ACS_ERR_NOMEM : ACS_ERR_DEVICE;
    };
    if (cfg.cuda_stream) {
        c->stream = (cudaStream_t)cfg.cuda_stream;
    } else {
        chk(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    const size_t nrec = (size_t)c->S * c->C;
    chk(cudaHostAlloc(&c->h_ring, nrec * sizeof(TaskRec), cudaHostAllocDefault));
    chk(cudaMalloc(&c->d_ring, nrec * sizeof(TaskRec)));
    chk(cudaMalloc(&c->d_ctl, sizeof(DevCtl)));
    const uint32_t nslots = c->S * c->C;   // one done word per descriptor ring position
    chk(cudaMalloc(&c->d_done, (size_t)nslots * sizeof(unsigned long long)));
    // work ring: at most (2W - 1) * ACS_MAX_NCTA units of one stream are in flight
    uint32_t cells = 1;
    while (cells < std::min<uint32_t>(2u * c->W * ACS_MAX_NCTA * std::max<uint32_t>(1u, std::min<uint32_t>(c->S, 8u)), 1u << 20)) cells <<= 1;
    c->ncells = std::max<uint32_t>(cells, 4096);
    chk(cudaMalloc(&c->d_cells, (size_t)c->ncells * sizeof(unsigned long long)));
    chk(cudaMalloc(&c->d_taskaux, nrec * sizeof(TaskAux)));
    const bool keep_log = (cfg.flags & (ACS_FLAG_LOG | ACS_FLAG_TRACE)) != 0;
    if (!keep_log) c->log_log2 = 0, c->LC = 1;
    const size_t nlog = keep_log ? (size_t)c->S * c->LC : 1;
    chk(cudaMalloc(&c->d_trace, nlog * kTraceFields * sizeof(unsigned long long)));
    chk(cudaMalloc(&c->d_log_mask, nlog * sizeof(unsigned long long)));
    chk(cudaMalloc(&c->d_log_start, nlog * sizeof(unsigned long long)));
    chk(cudaMalloc(&c->d_log_retire, nlog * sizeof(unsigned long long)));
    chk(cudaMalloc(&c->d_sched_stats, c->S * sizeof(SchedStats)));
    chk(cudaMalloc(&c->d_sctl, c->S * sizeof(StreamCtl)));
    chk(cudaMalloc(&c->d_mirror, sizeof(Mirror)));
    chk(cudaHostAlloc(&c->h_status, sizeof(HostStatus), cudaHostAllocMapped));
    chk(cudaHostAlloc(&c->h_mbox, sizeof(Mailbox), cudaHostAllocMapped));
    chk(cudaHostAlloc(&c->h_one, sizeof(uint32_t), cudaHostAllocDefault));
    if (rc) { acs_destroy(c); return rc; }
    std::memset((void *)c->h_status, 0, sizeof(HostStatus));
    std::memset((void *)c->h_mbox, 0, sizeof(Mailbox));
    *c->h_one = 1u;
    chk(cudaHostGetDevicePointer((void **)&c->d_status, (void *)c->h_status, 0));
    chk(cudaHostGetDevicePointer((void **)&c->d_mbox, (void *)c->h_mbox, 0));
    chk(cudaMemsetAsync(c->d_sched_stats, 0, c->S * sizeof(SchedStats), c->stream));
    chk(cudaMemsetAsync(c->d_sctl, 0, c->S * sizeof(StreamCtl), c->stream));
    chk(cudaMemsetAsync(c->d_log_mask, 0, nlog * sizeof(unsigned long long), c->stream));
    chk(launch_init(c->d_cells, c->ncells, c->d_ctl, c->d_done, nslots, c->stream));

    // grid: one scheduler CTA per stream + worker CTAs, all co-resident
    c->smem = dyn_smem_bytes(c->W);
    if (cfg.ctas_per_sm) {
        // reserve enough shared memory that at most ctas_per_sm CTAs fit an SM
        int per_sm_smem = 0, per_block_optin = 0;
        chk(cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device));
        chk(cudaDeviceGetAttribute(&per_block_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        const uint32_t want = (uint32_t)per_sm_smem / (cfg.ctas_per_sm + 1) + 1024u;
        c->smem = std::max<uint32_t>(c->smem, std::min<uint32_t>(want, (uint32_t)per_block_optin));
    }
    const void *kfn = persistent_kernel_fn();
    chk(raise_kernel_smem_limit(c->smem));
    int per_sm = 0, sms = 0;
    chk(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBlock, c->smem));
    chk(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    chk(cudaStreamSynchronize(c->stream));
    if (rc) { acs_destroy(c); return rc; }
    const uint32_t max_grid = (uint32_t)per_sm * (uint32_t)sms;
    if (cfg.mode == ACS_MODE_WINDOW && max_grid <= c->S) { acs_destroy(c); return ACS_ERR_INVALID; }
    uint32_t slots = cfg.cta_slots ? cfg.cta_slots : (max_grid > c->S ? max_grid - c->S : 0);
    if (cfg.mode == ACS_MODE_WINDOW && (slots == 0 || slots + c->S > max_grid)) { acs_destroy(c); return ACS_ERR_INVALID; }
    if (cfg.mode == ACS_MODE_SW) {
        rc = sw_start(c);
        if (rc) { acs_destroy(c); return rc; }
    }
    c->cta_slots = slots;
    c->grid = slots + c->S;
    c->stats.cta_slots = c->cta_slots;
    c->stats.grid = c->grid;
    *out = c;
    return ACS_OK;
}

int acs_get_addresses(const acs_args *a, acs_segment *r, uint32_t *nr, acs_segment *w, uint32_t *nw) {
    if (!a || !r || !nr || !w || !nw) return ACS_ERR_INVALID;
    uint32_t R = 0, Wn = 0;
    auto rd = [&](uint64_t p, uint64_t n) { r[R++] = acs_segment{p, n}; };
    auto wr = [&](uint64_t p, uint64_t n) { w[Wn++] = acs_segment{p, n}; };
    const uint64_t F = 4, S = ACS_RL_SPHERES;
    switch (a->op) {
    case ACS_OP_NOP: break;
    case ACS_OP_AXPY: {
        acs_axpy_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.x, x.n * F); rd(x.y, x.n * F); wr(x.y, x.n * F);
        break;
    }
    case ACS_OP_SCALE: {
        acs_axpy_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.x, x.n * F); wr(x.y, x.n * F);
        break;
    }
    case ACS_OP_ADD: {
        acs_add_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.x, x.n * F); rd(x.y, x.n * F); wr(x.z, x.n * F);
        break;
    }
    case ACS_OP_GEMV: {  // reads W (m*k) and x (k), writes y (m): Fig. get_addresses with k = 1 column
        acs_gemv_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.W, (uint64_t)x.m * x.k * F); rd(x.x, x.k * F); wr(x.y, x.m * F);
        break;
    }
    case ACS_OP_BIAS_RELU: {
        acs_bias_relu_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.t, x.n * F); rd(x.b, x.n * F); wr(x.t, x.n * F);
        break;
    }
    case ACS_OP_RESID: {
        acs_resid_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.h, x.n * F); rd(x.u, x.n * F); rd(x.b, x.n * F); wr(x.h, x.n * F);
        break;
    }
    case ACS_OP_RL_BROADPHASE: {
        acs_rl_broadphase_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.pos, x.nenv * S * 3 * F); rd(x.prop, x.nenv * S * 2 * F);
        wr(x.cont, (uint64_t)x.nenv * ACS_RL_REC_BYTES); wr(x.nisl, x.nenv * F);
        break;
    }
    case ACS_OP_RL_SOLVE: {
        acs_rl_solve_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.pos, S * 3 * F); rd(x.prop, S * 2 * F); rd(x.cont, ACS_RL_REC_BYTES); rd(x.vel, S * 3 * F);
        wr(x.vel, S * 3 * F);
        break;
    }
    case ACS_OP_RL_INTEGRATE: {
        acs_rl_integrate_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.pos, x.nenv * S * 3 * F); rd(x.vel, x.nenv * S * 3 * F); rd(x.prop, x.nenv * S * 2 * F);
        wr(x.pos, x.nenv * S * 3 * F); wr(x.vel, x.nenv * S * 3 * F);
        break;
    }
    case ACS_OP_RL_EMIT: {  // reads nisl, the cfg block and the CTA table; writes the token
        acs_rl_emit_args x; std::memcpy(&x, a->bytes, sizeof x);
        if (!x.chunk || x.n_env % x.chunk) return ACS_ERR_INVALID;
        rd(x.nisl, (uint64_t)x.n_env * F); rd(x.cfg, sizeof(acs_rl_emit_cfg));
        rd(x.ncta_table, (uint64_t)(x.steps + 1) * 2 * (x.n_env / x.chunk)); wr(x.token, F);
        break;
    }
    case ACS_OP_WAIT_FLAG: {
        acs_wait_args x; std::memcpy(&x, a->bytes, sizeof x);
        rd(x.flag, 4);
        break;
    }
    case ACS_OP_SLEEP: {
        acs_sleep_args x; std::memcpy(&x, a->bytes, sizeof x);
        wr(x.y, 4);
        break;
    }
    default:
        return ACS_ERR_INVALID;
    }
    *nr = R;
    *nw = Wn;
    return ACS_OK;
}

int acs_submit_stream(acs_ctx *c, uint32_t stream, uint32_t task_id, const acs_args *args,
                      const acs_segment *reads, uint32_t n_reads, const acs_segment *writes, uint32_t n_writes) {
    if (!c) return ACS_ERR_INVALID;
    if (c->err) return c->err;
    if (!args || stream >= c->S || (n_reads && !reads) || (n_writes && !writes)) return ACS_ERR_INVALID;
    if (!valid_op(args->op) || args->ncta < 1 || args->ncta > ACS_MAX_NCTA || args->reserved) return ACS_ERR_INVALID;
    StreamState &ss = c->st[stream];
    const bool full = (uint64_t)ss.submitted + c->W - 1 - ss.synced + 1 > c->C - kPrefetch;
    if (c->resident && (ss.emitting || full)) refresh_stream(c, stream);
    if (ss.emitting) return ACS_ERR_INVALID;   // sync first: the device appends to this stream
    if (args->op == ACS_OP_RL_EMIT && c->cfg.mode != ACS_MODE_WINDOW) return ACS_ERR_INVALID;
    if (ss.submitted >= ACS_MAX_POSITION) return ACS_ERR_RANGE;   // acs_stream_rebase at an idle point
    if (ss.has_id && task_id <= ss.last_id) return ACS_ERR_ORDER;
    if ((uint64_t)ss.submitted + c->W - 1 - ss.synced + 1 > c->C - kPrefetch) return ACS_ERR_FULL;
    TaskRec &r = c->h_ring[(size_t)stream * c->C + (ss.submitted & (c->C - 1))];
    uint32_t cnt = 0;
    uint16_t wmask = 0;
    uint64_t bytes = 0;
    if (!add_segs(reads, n_reads, false, r.seg, cnt, wmask, bytes) ||
        !add_segs(writes, n_writes, true, r.seg, cnt, wmask, bytes))
        return ACS_ERR_INVALID;
    r.task_id = task_id;
    r.op = args->op;
    r.ncta = args->ncta;
    r.wmask = wmask;
    r.nseg = (uint8_t)cnt;
    r.flags = 0;
    fold_reads(r);
    r.seq = ss.submitted;
    std::memcpy(r.args, args->bytes, sizeof r.args);
    ss.has_id = true;
    ss.last_id = task_id;
    ss.submitted++;
    if (args->op == ACS_OP_RL_EMIT) ss.emit_pending++;
    c->stats.tasks_submitted++;
    c->stats.seg_bytes += bytes;
    return ACS_OK;
}

int acs_submit(acs_ctx *c, uint32_t task_id, const acs_args *args, const acs_segment *reads, uint32_t n_reads,
               const acs_segment *writes, uint32_t n_writes) {
    return acs_submit_stream(c, 0, task_id, args, reads, n_reads, writes, n_writes);
}

int acs_submit_ops(acs_ctx *c, uint32_t stream, uint32_t n, const uint32_t *task_ids, const acs_args *args) {
    if (!c) return ACS_ERR_INVALID;
    if (c->err) return c->err;
    if (n && (!task_ids || !args)) return ACS_ERR_INVALID;
    acs_segment r[ACS_MAX_SEGS], w[ACS_MAX_SEGS];
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t nr = 0, nw = 0;
        int rc = acs_get_addresses(&args[i], r, &nr, w, &nw);
        if (rc) return rc;
        rc = acs_submit_stream(c, stream, task_ids[i], &args[i], r, nr, w, nw);
        if (rc) return rc;
    }
    return ACS_OK;
}

int acs_flush(acs_ctx *c) {
    if (!c) return ACS_ERR_INVALID;
    if (__atomic_load_n(&c->aborted, __ATOMIC_ACQUIRE)) fail(c, ACS_ERR_STOPPED);
    if (c->err) return c->err;
    uint32_t n = 0;
    for (auto &s : c->st) n += s.submitted - s.flushed;
    if (!n) return ACS_OK;
    int rc;
    if (c->resident) rc = flush_resident(c);
    else if (c->cfg.mode == ACS_MODE_WINDOW) rc = flush_window(c);
    else if (c->cfg.mode == ACS_MODE_INORDER) rc = flush_inorder(c);
    else if (c->cfg.mode == ACS_MODE_SW) rc = flush_sw(c);
    else rc = flush_graph(c);
    if (rc) return rc;
    for (auto &s : c->st) {
        c->stats.tasks_flushed += s.submitted - s.flushed;
        s.flushed = s.submitted;
        if (s.emit_pending) s.emitting = true;
        s.emit_pending = 0;
    }
    return ACS_OK;
}

// Resident: wait on the host, without ending the kernel, until every
// published task (and the emitter chains they started) retired.
int sync_resident(acs_ctx *c) {
    using clk = std::chrono::steady_clock;
    auto last = clk::now();
    std::vector<uint32_t> seen(c->S, 0);
    // spin first (short requests finish in microseconds), then poll every 20 us
    for (uint32_t iter = 0;; ++iter) {
        int rc = resident_status(c);
        if (rc) return rc;
        rc = publish_ready(c, false);
        if (rc) return rc;
        bool all = true, moved = false;
        for (uint32_t s = 0; s < c->S; ++s) {
            refresh_stream(c, s);
            const StreamState &ss = c->st[s];
            const uint32_t h = __atomic_load_n(&c->h_mbox->progress[s].head, __ATOMIC_RELAXED);
            if (h != seen[s]) { seen[s] = h; moved = true; }
            if (ss.emitting || ss.synced != ss.flushed) all = false;
        }
        if (all) return ACS_OK;
        const bool spinning = iter < 4096;
        if (spinning && (iter & 63) != 0) continue;
        heartbeat(c);
        const cudaError_t q = cudaStreamQuery(c->stream);
        if (q != cudaErrorNotReady) {     // the kernel is gone before the work retired
            return q == cudaSuccess ? fail(c, ACS_ERR_STOPPED) : cuda_fail(c, q);
        }
        const auto now = clk::now();
        if (moved) last = now;
        else if ((uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - last).count() >
                 c->cfg.timeout_ns)
            return fail(c, ACS_ERR_TIMEOUT);
        if (!spinning) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int acs_sync(acs_ctx *c) {
    if (!c) return ACS_ERR_INVALID;
    if (c->resident) return sync_resident(c);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    collect_timing(c);
    if (c->cfg.mode == ACS_MODE_WINDOW) {
        const uint32_t derr = c->h_status->err;
        if (derr) fail(c, (int)(int32_t)derr);
        if (__atomic_load_n(&c->aborted, __ATOMIC_ACQUIRE)) fail(c, ACS_ERR_STOPPED);
    }
    if (c->cfg.mode == ACS_MODE_GRAPH) release_graphs(c, true);
    if (c->err) return c->err;
    bool any = false;
    for (auto &s : c->st) any |= s.emitting;
    if (any) {   // the device appended tasks: continue the streams after them
        std::vector<StreamCtl> sc(c->S);
        e = cudaMemcpy(sc.data(), c->d_sctl, c->S * sizeof(StreamCtl), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e);
        for (uint32_t i = 0; i < c->S; ++i) {
            StreamState &s = c->st[i];
            if (!s.emitting) continue;
            const uint32_t added = sc[i].end - s.flushed;
            c->stats.tasks_emitted += added;
            s.submitted = s.flushed = sc[i].end;
            if (sc[i].end) { s.has_id = true; s.last_id = std::max(s.last_id, sc[i].end - 1); }
            s.emitting = false;
        }
    }
    for (auto &s : c->st) s.synced = s.flushed;
    return ACS_OK;
}

int acs_graph_replay(acs_ctx *c) {
    if (!c) return ACS_ERR_INVALID;
    if (c->err) return c->err;
    if (c->cfg.mode != ACS_MODE_GRAPH || !c->last_exec) return ACS_ERR_INVALID;
    const bool timing = (c->cfg.flags & ACS_FLAG_TIMING) != 0;
    TimedLaunch t{};
    if (timing) {
        t = get_events(c);
        cudaEventRecord(t.a, c->stream);
    }
    cudaError_t e = cudaGraphLaunch(c->last_exec, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (timing) {
        cudaEventRecord(t.b, c->stream);
        c->timed.push_back(t);
    }
    c->stats.launches++;
    return ACS_OK;
}

int acs_get_log(acs_ctx *c, uint32_t stream, uint64_t first, uint32_t n, uint64_t *masks, uint64_t *start,
                uint64_t *retire) {
    if (!c || stream >= c->S || !(c->cfg.flags & ACS_FLAG_LOG)) return ACS_ERR_INVALID;
    const StreamState &ss = c->st[stream];
    if (first + n > ss.synced || n > c->LC || first + c->LC < ss.synced) return ACS_ERR_INVALID;
    uint64_t *dst[3] = {masks, start, retire};
    unsigned long long *src[3] = {c->d_log_mask, c->d_log_start, c->d_log_retire};
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        uint64_t a = first, done = 0;
        while (done < n) {
            const uint64_t pa = a & (c->LC - 1);
            const uint64_t m = std::min<uint64_t>(n - done, c->LC - pa);
            cudaError_t e = cudaMemcpy(dst[k] + done, src[k] + (size_t)stream * c->LC + pa, m * sizeof(uint64_t),
                                       cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return ACS_ERR_DEVICE;
            a += m;
            done += m;
        }
    }
    return ACS_OK;
}

int acs_get_trace(acs_ctx *c, uint32_t stream, uint64_t first, uint32_t n, uint64_t *t) {
    if (!c || !t || stream >= c->S || !(c->cfg.flags & ACS_FLAG_TRACE)) return ACS_ERR_INVALID;
    const StreamState &ss = c->st[stream];
    if (first + n > ss.synced || n > c->LC || first + c->LC < ss.synced) return ACS_ERR_INVALID;
    uint64_t a = first, done = 0;
    while (done < n) {
        const uint64_t pa = a & (c->LC - 1);
        const uint64_t m = std::min<uint64_t>(n - done, c->LC - pa);
        cudaError_t e = cudaMemcpy(t + done * kTraceFields, c->d_trace + ((size_t)stream * c->LC + pa) * kTraceFields,
                                   m * kTraceFields * sizeof(uint64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return ACS_ERR_DEVICE;
        a += m;
        done += m;
    }
    return ACS_OK;
}

int acs_start(acs_ctx *c) {
    if (!c) return ACS_ERR_INVALID;
    if (c->err) return c->err;
    if (c->cfg.mode != ACS_MODE_WINDOW || c->resident) return ACS_ERR_INVALID;
    for (auto &s : c->st)
        if (s.flushed != s.synced || s.emitting) return ACS_ERR_INVALID;   // acs_sync first
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    collect_timing(c);
    Mailbox *m = c->h_mbox;
    std::memset((void *)m, 0, sizeof(Mailbox));
    for (uint32_t s = 0; s < c->S; ++s) {
        m->host_end[s] = c->st[s].flushed;
        m->progress[s].head = m->progress[s].idle_at = c->st[s].flushed;
    }
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    Mirror mir;
    std::memset(&mir, 0, sizeof mir);
    for (uint32_t s = 0; s < c->S; ++s) mir.end[s] = c->st[s].flushed;
    e = cudaMemcpy(c->d_mirror, &mir, sizeof mir, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e);
    KParams P;
    fill_params(c, P);
    P.resident = 1;
    for (uint32_t s = 0; s < c->S; ++s) {
        P.first[s] = c->st[s].flushed;
        P.nprev[s] = tasks_before(c->st[s], P.first[s]);
        P.end[s] = c->st[s].flushed;
        P.open[s] = 0;
    }
    if (!c->side) {
        e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    int rc = launch_persistent(c, P);
    if (rc) return rc;
    c->resident = true;
    // tasks submitted before the start are published now
    return acs_flush(c);
}

int acs_progress(acs_ctx *c, uint32_t *head, uint32_t *idle_at) {
    if (!c) return ACS_ERR_INVALID;
    if (!c->resident) {   // what the last acs_sync established
        for (uint32_t s = 0; s < c->S; ++s) {
            if (head) head[s] = c->st[s].synced;
            if (idle_at) idle_at[s] = c->st[s].synced;
        }
        return c->err;
    }
    heartbeat(c);
    int prc = publish_ready(c, false);
    if (prc) return prc;
    for (uint32_t s = 0; s < c->S; ++s) {
        refresh_stream(c, s);
        if (head) head[s] = __atomic_load_n(&c->h_mbox->progress[s].head, __ATOMIC_ACQUIRE);
        if (idle_at) idle_at[s] = __atomic_load_n(&c->h_mbox->progress[s].idle_at, __ATOMIC_ACQUIRE);
    }
    return resident_status(c);
}

int acs_stop(acs_ctx *c) {
    if (!c) return ACS_ERR_INVALID;
    if (!c->resident) return c->err;
    using clk = std::chrono::steady_clock;
    // publish what is staged, then ask every scheduler to leave once idle
    if (!c->err) acs_flush(c);
    publish_ready(c, true);
    __atomic_store_n(&c->h_mbox->drain, 1u, __ATOMIC_RELEASE);
    heartbeat(c);
    auto last = clk::now();
    std::vector<uint32_t> seen(c->S, 0);
    bool aborted = false;
    while (true) {
        const cudaError_t q = cudaStreamQuery(c->stream);
        if (q != cudaErrorNotReady) break;
        bool moved = false;
        for (uint32_t s = 0; s < c->S; ++s) {
            const uint32_t h = __atomic_load_n(&c->h_mbox->progress[s].head, __ATOMIC_RELAXED);
            if (h != seen[s]) { seen[s] = h; moved = true; }
        }
        const auto now = clk::now();
        if (moved) last = now;
        const uint64_t still = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - last).count();
        if (!aborted && (c->err || still > c->cfg.timeout_ns)) {
            // no progress: raise the device stop flag through a copy that runs
            // beside the kernel; every device wait then ends
            if (!c->side) cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
            if (c->side) {
                cudaMemcpyAsync(&c->d_ctl->stop, c->h_one, sizeof(uint32_t), cudaMemcpyHostToDevice, c->side);
                cudaStreamSynchronize(c->side);
            }
            if (!c->err) fail(c, ACS_ERR_TIMEOUT);
            aborted = true;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    c->resident = false;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    collect_timing(c);
    const uint32_t derr = c->h_status->err;
    if (derr) fail(c, (int)(int32_t)derr);
    // final ends of every stream, emitter chains included
    std::vector<StreamCtl> sc(c->S);
    e = cudaMemcpy(sc.data(), c->d_sctl, c->S * sizeof(StreamCtl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e);
    for (uint32_t i = 0; i < c->S; ++i) {
        StreamState &s = c->st[i];
        if (s.emitting && !c->err) {
            c->stats.tasks_emitted += sc[i].end - s.flushed;
            s.submitted = s.flushed = sc[i].end;
            if (sc[i].end) { s.has_id = true; s.last_id = std::max(s.last_id, sc[i].end - 1); }
        }
        s.emitting = false;
        s.emit_pending = 0;
        if (!c->err) s.synced = s.flushed;
    }
    if (!c->err && __atomic_load_n(&c->h_mbox->expired, __ATOMIC_ACQUIRE)) return ACS_ERR_STOPPED;
    return c->err;
}

int acs_abort(acs_ctx *c) {
    if (!c) return ACS_ERR_INVALID;
    if (c->cfg.mode != ACS_MODE_WINDOW) return ACS_ERR_INVALID;
    __atomic_store_n(&c->aborted, 1u, __ATOMIC_RELEASE);
    // the device stop word, written by the copy engine on a stream of this
    // call's own (non-blocking, so it never waits behind the running kernel)
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return ACS_ERR_DEVICE;
    if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return ACS_ERR_DEVICE;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        e = cudaMemcpyAsync(&c->d_ctl->stop, c->h_one, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
        const cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(s);
    }
    if (prev != c->device) cudaSetDevice(prev);
    return e == cudaSuccess ? ACS_OK : ACS_ERR_DEVICE;
}

int acs_stream_tail(acs_ctx *c, uint32_t stream, uint32_t *tail) {
    if (!c || !tail || stream >= c->S) return ACS_ERR_INVALID;
    *tail = c->st[stream].submitted;
    return ACS_OK;
}

// Nothing on the device that outlives a launch is keyed to the old positions
// in a way a later launch consults: a launch writes the done words of its own
// tasks before any of them is published, counts the tasks before its first one
// as complete (workers' admission) and loads and tests as candidates only the
// tasks the stream had since its restart (KParams::nprev).
int acs_stream_rebase(acs_ctx *c, uint32_t stream, uint32_t pos) {
    if (!c || stream >= c->S || pos >= ACS_MAX_POSITION) return ACS_ERR_INVALID;
    if (c->err) return c->err;
    if (c->resident) return ACS_ERR_INVALID;   // acs_stop first
    StreamState &ss = c->st[stream];
    if (ss.submitted != ss.flushed || ss.flushed != ss.synced || ss.emitting || ss.emit_pending)
        return ACS_ERR_INVALID;                // acs_flush + acs_sync first
    ss.submitted = ss.flushed = ss.synced = ss.base = pos;
    ss.has_id = false;
    ss.last_id = 0;
    return ACS_OK;
}

int acs_get_stats(acs_ctx *c, acs_stats *out) {
    if (!c || !out) return ACS_ERR_INVALID;
    if (c->cfg.mode == ACS_MODE_WINDOW) {
        std::vector<SchedStats> ss(c->S);
        if (cudaMemcpy(ss.data(), c->d_sched_stats, c->S * sizeof(SchedStats), cudaMemcpyDeviceToHost) == cudaSuccess) {
            c->stats.sched_cycles = c->stats.sched_busy_cycles = c->stats.sched_inserts = 0;
            c->stats.sched_iterations = 0;
            // the submitted tasks' bytes (counted by acs_submit*) and the
            // appended ones' (counted by the emitters)
            c->stats.device_seg_bytes = c->stats.seg_bytes;
            for (int k = 0; k < kPhases; ++k) c->stats.sched_phase_cycles[k] = 0;
            c->stats.check_cycles = c->stats.starved_iters = 0;
            for (auto &x : ss) {
                c->stats.device_seg_bytes += x.seg_bytes;
                c->stats.check_cycles += x.check_cycles;
                c->stats.starved_iters += x.starved_iters;
                for (int k = 0; k < kPhases; ++k) c->stats.sched_phase_cycles[k] += x.phase[k];
                c->stats.sched_cycles += x.cycles;
                c->stats.sched_busy_cycles += x.busy_cycles;
                c->stats.sched_inserts += x.inserts;
                c->stats.sched_iterations += x.iterations;
            }
        }
    }
    *out = c->stats;
    return ACS_OK;
}

}  // extern "C"
