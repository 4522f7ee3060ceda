// Internal layouts shared by the host runtime (acs_runtime.cu) and the device
// code (acs_kernels.cu). Not part of the C ABI.
#pragma once

#include <cstdint>

#include "acs.h"

namespace acs {

constexpr int kBlock = ACS_BLOCK_THREADS;
constexpr int kMaxSegs = ACS_MAX_SEGS;
constexpr int kMaxWindow = ACS_MAX_WINDOW;
constexpr int kPrefetch = 16;          // descriptors per loader batch (one round trip)
constexpr int kBodySmem = 24576;       // shared memory reserved for task bodies
constexpr uint32_t kMinCapacity = 64;

// An inclusive byte range [start, last]; empty segments are never stored.
struct Seg {
    uint64_t start;
    uint64_t last;
};

// One task descriptor, 320 bytes, at ring position (seq mod capacity) of its
// stream. The first 64 bytes are what a worker CTA needs; the segments are
// what the scheduler needs.
struct alignas(16) TaskRec {
    uint32_t task_id;
    uint16_t op;
    uint16_t ncta;
    uint16_t wmask;      // bit k set: seg[k] is a write segment
    uint8_t nseg;
    uint8_t flags;       // bit k (k < 8): seg[k] is written and also read (see fold_reads)
    uint32_t seq;        // position of the task in its stream
    uint8_t args[48];
    Seg seg[kMaxSegs];
};
static_assert(sizeof(TaskRec) == 320, "TaskRec layout");

// Drops every read segment that lies inside a write segment of the same task.
// The dependency relation is unchanged: a write segment conflicts with every
// segment of another task that a read segment inside it could conflict with
// (read-after-write, write-after-read and write-after-write alike), so the
// checks see fewer segment pairs and give the same masks. A read equal to a
// write sets that write's bit in `flags`, so byte counts still see two
// accesses (a read-modify-write range).
__host__ __device__ inline void fold_reads(TaskRec &r) {
    const uint32_t n = r.nseg < kMaxSegs ? r.nseg : kMaxSegs;
    uint32_t drop = 0, rw = 0;
    for (uint32_t x = 0; x < n; ++x) {
        if ((r.wmask >> x) & 1u) continue;
        for (uint32_t y = 0; y < n; ++y) {
            if (!((r.wmask >> y) & 1u)) continue;
            if (r.seg[x].start >= r.seg[y].start && r.seg[x].last <= r.seg[y].last) {
                drop |= 1u << x;
                if (r.seg[x].start == r.seg[y].start && r.seg[x].last == r.seg[y].last) rw |= 1u << y;
                break;
            }
        }
    }
    if (!drop) return;
    uint32_t out = 0, wm = 0, fl = 0;
    for (uint32_t k = 0; k < n; ++k) {
        if ((drop >> k) & 1u) continue;
        r.seg[out] = r.seg[k];
        if ((r.wmask >> k) & 1u) wm |= 1u << out;
        if (((rw >> k) & 1u) && out < 8) fl |= 1u << out;
        ++out;
    }
    r.nseg = (uint8_t)out;
    r.wmask = (uint16_t)wm;
    r.flags = (uint8_t)fl;
}

// A descriptor in a scheduler's shared-memory history, padded to 336 bytes so
// that 16-byte segment loads of consecutive records by the lanes of a warp hit
// distinct banks.
// For a narrow record the loader also writes the low 32 bits of its segments'
// starts into r.seg[4] and of their lasts into r.seg[5] (four words each,
// unused entries 0): entries a narrow record never uses, so that a checker
// reads a candidate in three 16-byte loads (these two and hi .. nsw).
struct alignas(16) HistRec {
    TaskRec r;
    uint32_t hi;        // the upper 32 address bits of every segment, when `narrow`
    uint32_t narrow;    // 1: at most 4 segments, each inside the 4 GiB window [hi << 32, (hi + 1) << 32)
    uint32_t nsw;       // nseg | wmask << 8
    uint32_t pad;
};
static_assert(sizeof(HistRec) == 336, "HistRec layout");

struct alignas(16) TaskHdr {   // the first 64 bytes of a TaskRec
    uint32_t task_id;
    uint16_t op;
    uint16_t ncta;
    uint16_t wmask;
    uint8_t nseg;
    uint8_t flags;
    uint32_t seq;
    uint8_t args[48];
};
static_assert(sizeof(TaskHdr) == 64, "TaskHdr layout");

// Device-resident counters of one context; hot words on separate 128 B lines.
struct alignas(128) DevCtl {
    uint32_t ring_head;     // work-ring positions claimed by worker CTAs
    uint32_t pad0[31];
    uint32_t ring_tail;     // work-ring positions reserved by scheduler warps
    uint32_t pad1[31];
    uint32_t stop;          // 1: every CTA leaves its loop
    uint32_t sched_done;    // scheduler warps that finished their streams
    uint32_t exit_count;    // CTAs that left the kernel
    uint32_t err;           // first error (ACS_ERR_*), 0 = none
    uint32_t err_info;      // where: enum ErrSite
    uint32_t pad2[27];
    unsigned long long ticket;  // legality-log ticket counter
    uint32_t pad3[30];
};

// Written by the last CTA of each persistent launch into mapped host memory.
struct HostStatus {
    volatile uint32_t err;
    volatile uint32_t err_info;
    volatile uint32_t launches_done;
    volatile uint32_t pad;
};

// Per-stream scheduler statistics (device), accumulated over launches.
// scheduler-loop phases timed with clock64: 0 descriptor loads, 1 inserts,
// 2 retire (incl. waiting for the done polls), 3 dispatch selection,
// 4 ring-cell checks, 5 aux words, 6 publication fence, 7 cell stores
constexpr int kPhases = 8;

struct SchedStats {
    unsigned long long cycles;
    unsigned long long busy_cycles;
    unsigned long long inserts;
    unsigned long long iterations;
    unsigned long long phase[kPhases];
    unsigned long long seg_bytes;   // read + write segment bytes of the tasks emitters appended
    unsigned long long emitted;     // descriptors appended by device-side emitters
    unsigned long long check_cycles;    // tracing: cycles checker warps spent testing
    unsigned long long starved_iters;   // tracing: iterations with a free slot but no checked task
};

// per-task trace fields (globaltimer ns): insert, dispatch, first CTA start,
// last CTA end, retirement seen by the scheduler
constexpr int kTraceFields = 5;

// Per-stream words shared by the scheduler and device-side emitters. A stream
// holding emit tasks is open: its end grows as emitters append descriptors.
struct StreamCtl {
    uint32_t end;        // one past the last published descriptor
    uint32_t open;       // emit tasks whose chain has not finished
    uint32_t head_pub;   // oldest unreleased task (emitters wait for ring space)
};

// Host-mapped words of a resident launch (pinned host memory the device reads
// and writes over the bus). The host copies a stream's new descriptors into
// the device ring (copy engine) and, once that copy completed, publishes the
// new end with a release store; the device reports progress back.
struct StreamProgress {
    uint32_t head;      // device -> host: tasks below were released (published every few tasks)
    uint32_t idle_at;   // device -> host: the stream was idle (all tasks below retired,
                        // no emitter alive) with this end
};

struct Mailbox {
    uint32_t host_end[ACS_MAX_STREAMS];   // host -> device: published end of each stream
    uint32_t drain;                       // host -> device: finish published work, then exit
    uint32_t err;                         // device -> host: first error (as DevCtl::err)
    uint32_t expired;                     // device -> host: exited after the idle limit
    uint32_t pad0;
    unsigned long long heartbeat;         // host -> device: changes with every host call
    unsigned long long pad1[6];
    StreamProgress progress[ACS_MAX_STREAMS];
};

// A device-memory copy of the host-written mailbox words, refreshed about
// every microsecond by one warp (the loader warp of stream 0) so that every
// other poll of a resident launch stays in device memory: polls of mapped
// host memory from many SMs slow the whole GPU down.
struct alignas(128) Mirror {
    uint32_t end[ACS_MAX_STREAMS];
    uint32_t drain;
    uint32_t pad;
    unsigned long long heartbeat;
};

// What a worker needs beside its cell's payload, written once per task by the
// checker warp and indexed like the descriptor ring: the conflicting
// candidates it must wait for (bit k: the task k + 1 positions earlier) and
// the task's seq. Task q + capacity reuses the entry only after task q retired,
// and every CTA of q reads it before q can retire.
struct alignas(16) TaskAux {
    unsigned long long up;
    uint32_t seq;
    uint32_t pad;
};

struct KParams {
    TaskRec *recs;            // [n_streams][capacity]
    DevCtl *ctl;
    unsigned long long *cells;// work ring: low 32 bits sequence, high 32 payload
                              // (descriptor index << 8 | CTA index)
    TaskAux *taskaux;         // [n_streams][capacity], like recs
    // [n_streams][capacity] done words, indexed like recs: (seq + 1) << 32 |
    // CTAs not yet finished, of the position's latest task (set when the loader
    // takes the task; each CTA subtracts one with release semantics)
    unsigned long long *done;
    unsigned long long *log_mask, *log_start, *log_retire;   // [n_streams][log_capacity]
    SchedStats *sched_stats;  // [n_streams]
    unsigned long long *trace;  // [n_streams][log_capacity][kTraceFields] (ACS_FLAG_TRACE)
    StreamCtl *sctl;          // [n_streams]
    HostStatus *hstatus;      // mapped host memory
    unsigned long long timeout_ns;
    uint32_t cap_log2;        // capacity = 1 << cap_log2
    uint32_t log_log2;        // log_capacity = 1 << log_log2
    uint32_t cell_mask;       // work-ring cells - 1 (power of two)
    uint32_t window;          // ring span M: slots (tasks inserted and not released)
    uint32_t active_limit;    // tasks inserted and not retired, at most (<= window)
    uint32_t check_w;         // candidates: the check_w - 1 previous tasks (log masks by slot
                              // mod check_w); = window except with dispatch ahead
    uint32_t admit;           // 1: dispatch ahead: a task's workers wait until every task
                              // check_w or more positions back completed (their done words)
    uint32_t n_streams;       // = scheduler CTAs (CTA s < n_streams schedules stream s)
    uint32_t flags;
    uint32_t sched_smem;      // bytes of dynamic shared memory a scheduler uses
    uint32_t poll_ns;         // longest sleep of an idle worker between ring polls
    uint32_t resident;        // 1: serve host-published work until drained (Mailbox)
    Mailbox *mbox;            // mapped host memory (resident launches)
    Mirror *mirror;           // device copy of the mailbox's host-written words
    unsigned long long idle_limit_ns;  // resident: exit after this long without host activity
    uint32_t first[ACS_MAX_STREAMS];  // first seq of this launch, per stream
    uint32_t end[ACS_MAX_STREAMS];    // one past the last seq submitted by the host
    uint8_t open[ACS_MAX_STREAMS];    // emit tasks among the stream's new tasks
    uint8_t nprev[ACS_MAX_STREAMS];   // tasks the stream had before `first` since it was last
                                      // restarted (acs_stream_rebase), at most 64: the
                                      // candidates and ring slots below `first` that exist
};
static_assert(sizeof(KParams) <= 4096, "KParams fits the classic kernel-parameter limit");

// descriptors kept in a scheduler's shared-memory history ring: the W - 1
// predecessors of every task being checked plus look-ahead
__host__ __device__ inline uint32_t hist_size(uint32_t window) { return window <= 32 ? 64u : 128u; }

// Insertion batches handed from the scheduler warp to the publisher warp
// (shared memory): per task its seq, work-ring offset, CTA count and upstream
// mask still to wait for.
constexpr uint32_t kPubSlots = 4;
struct PubBatch {
    uint32_t q[32], off[32], n[32];
    uint32_t nins, p0, total, pad;
};
struct PubQueue {
    uint32_t produced, consumed, pad[2];
    PubBatch b[kPubSlots];
};

inline uint32_t sched_smem_bytes(uint32_t window) {
    const uint32_t H = hist_size(window);
    const uint32_t base = H * 336u + H * 8 + H * 4 + 32 + kMaxWindow * 4 * 2;   // hist, pmask, ptag, sh, expect, slotpos
    return (base + 15u) / 16u * 16u + (uint32_t)sizeof(PubQueue);
}

// Raises the persistent kernel's dynamic shared-memory limit (process-wide,
// per-function state) to at least `bytes`; never lowers it (acs_runtime.cu).
cudaError_t raise_kernel_smem_limit(uint32_t bytes);

inline uint32_t dyn_smem_bytes(uint32_t window) {
    uint32_t s = sched_smem_bytes(window);
    return s > (uint32_t)kBodySmem ? s : (uint32_t)kBodySmem;
}

// Task states of a window slot (scheduler registers).
enum SlotState : uint32_t { kEmpty = 0, kPending = 1, kReady = 2, kExec = 3, kRetired = 4 };

// error-site codes stored in DevCtl::err_info
enum ErrSite : uint32_t {
    kSiteSched = 1, kSiteWorker = 2, kSiteRing = 3, kSitePrefetch = 4, kSiteEmit = 8,
    // self-checks (ACS_ERR_INVALID): a descriptor or work unit that is not what it must be
    kSiteCheckRecord = 5, kSiteWorkerPayload = 6, kSiteWorkerRecord = 7
};

}  // namespace acs
