// Device side of the scheduler: one cooperative persistent kernel.
//
// CTAs [0, n_streams) are schedulers, one per stream, 8 warps each:
//   warp 0 owns the stream's scheduling window (W slots, Sec. III-C): the
//          per-slot state machine (pending / ready / executing / retired,
//          Sec. III-C) and upstream masks live in its registers (lane l holds
//          slots l and l + 32). Each iteration it retires the slots the poller
//          saw complete, releases them in program order, and inserts checked
//          tasks (upstream = candidates still active), oldest first;
//   warps 1..4 run the segment-overlap test of Alg. 1 (extended to
//          read-after-write) of each task against its W - 1 predecessors,
//          one predecessor per lane; a ballot turns the per-lane results into
//          the task's upstream-candidate mask, which goes to the task's aux
//          word (what its worker CTAs wait for);
//   warp 5 publishes the pending insertion batches to the work ring (one
//          fence per pass, then the cells' sequence words);
//   warp 6 polls the done words of executing tasks (acquire loads);
//   warp 7 streams descriptors into a shared-memory history ring ahead of
//          use, setting each new task's done word (and, in a resident launch,
//          follows the host-published ends).
//
// CTAs [n_streams, grid) are workers: each claims work-ring positions one at a
// time, runs the body for one (task, CTA index) unit, then takes itself off
// its task's done word (seq + 1, CTAs still running; one per descriptor ring
// position) with a release reduction.
//
// Every wait is bounded by timeout_ns of no progress (a resident launch's
// waits for the host by its idle limit); on expiry the waiter records
// ACS_ERR_TIMEOUT, raises the stop flag and leaves, so the kernel always
// terminates.
#include <cstdint>

#include "acs_bodies.cuh"
#include "acs_internal.h"

namespace acs {

// ---- PTX helpers ------------------------------------------------------------

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// CTA scope on shared memory: flags between the warps of a scheduler CTA
__device__ __forceinline__ uint32_t ld_acquire_cta_shared(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta_shared(uint32_t *p, uint32_t v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// Bulk prefetch of [p, p + bytes) into L2 (a hint: no data moves to the SM);
// p and bytes multiples of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// A done word shows task `want - 1` (want = seq + 1) complete when it names
// that task with no CTA left, or names a later task of the same ring position
// (which the position takes only after the earlier task retired).
__device__ __forceinline__ bool slot_done(unsigned long long w, uint32_t want) {
    const uint32_t hi = (uint32_t)(w >> 32);
    return (int32_t)(hi - want) > 0 || (hi == want && (uint32_t)w == 0u);
}
// system scope: words in mapped host memory (resident launches)
__device__ __forceinline__ uint32_t ld_acquire_sys_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_sys_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_sys_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }
__device__ __forceinline__ void st_relaxed_sys_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void raise_error(const KParams &P, uint32_t code, uint32_t site) {
    if (atomicCAS(&P.ctl->err, 0u, code) == 0u) {
        P.ctl->err_info = site;
        if (P.resident) st_relaxed_sys_u32(&P.mbox->err, code);   // a waiting host sees it at once
    }
    __threadfence();
    atomicExch(&P.ctl->stop, 1u);
}

__device__ __forceinline__ bool stopped(const KParams &P) { return ld_volatile_u32(&P.ctl->stop) != 0; }

// ---- scheduler CTA ----------------------------------------------------------------
//
// Shared memory of a scheduler CTA (stream s):
//   hist[H]     the descriptors of tasks seq mod H, copied in by the loader
//               warp in batches of up to kPrefetch; it holds the
//               W - 1 predecessors of every task still to be checked
//   pmask[H]    upstream-candidate mask of task seq mod H (bit i mod W for
//               each conflicting predecessor i in [seq - W + 1, seq - 1])
//   ptag[H]     seq + 1 once pmask of seq is written (0: not yet)
//   sh          counters shared by the warps
//   expect[64]  the done value each executing slot waits for (0: none)
//   pub         the insertion batches handed from warp 0 to the publisher
//
// Warps 1..4 ("checkers") compute the upstream-candidate mask of tasks
// j = first + w + 4k: the segment-overlap test of Alg. 1 (extended to RAW) of
// task j against its W - 1 predecessors, one predecessor per lane, ballot ->
// mask (bit i mod W for each conflicting i in [j - W + 1, j - 1]). The
// candidate set of a task is fixed by the stream, so the test runs ahead of
// execution, in parallel with it. Warp 5 publishes insertion batches to the
// work ring. Warp 6 polls the done words of executing slots. Warp 7 loads
// descriptors. Warp 0 owns the window: it inserts checked tasks into the
// W-slot ring, dispatching each at once (its workers wait for the
// predecessors its mask names: the pending -> ready transition happens at the
// worker), retires tasks the poller saw complete and releases slots in
// program order.

struct SchedShared {
    uint32_t complete_upto;  // hist holds every seq below (loaded), from `lo`
    uint32_t next;           // tasks below are inserted
    uint32_t quit;           // 1: checkers and loader leave
    uint32_t end;            // stream end known to the CTA (grows while the stream is open)
    uint32_t head_pos;       // sole producer: work-ring position of the oldest unreleased task's
                             // first unit (every unit below it belongs to a retired task)
    uint32_t released;       // every task below it retired (the window's release point)
    uint32_t pad[2];
};
static_assert(sizeof(SchedShared) == 32, "SchedShared size (sched_smem_bytes)");

struct SchedSmem {
    uint32_t *expect;        // [kMaxWindow] done value of each executing slot (0: none)
    uint32_t *slotpos;       // [kMaxWindow] sole producer: first work-ring position of the slot's task
    HistRec *hist;
    unsigned long long *pmask;
    uint32_t *ptag;
    SchedShared *sh;
    PubQueue *pub;
    uint32_t H;
};

__device__ __forceinline__ SchedSmem carve(uint8_t *smem, uint32_t W) {
    SchedSmem s;
    s.H = hist_size(W);
    uint8_t *p = smem;
    s.hist = reinterpret_cast<HistRec *>(p);
    p += s.H * sizeof(HistRec);
    s.pmask = reinterpret_cast<unsigned long long *>(p);
    p += s.H * sizeof(unsigned long long);
    s.ptag = reinterpret_cast<uint32_t *>(p);
    p += s.H * sizeof(uint32_t);
    s.sh = reinterpret_cast<SchedShared *>(p);
    p += sizeof(SchedShared);
    s.expect = reinterpret_cast<uint32_t *>(p);
    p += kMaxWindow * sizeof(uint32_t);
    s.slotpos = reinterpret_cast<uint32_t *>(p);
    p += kMaxWindow * sizeof(uint32_t);
    p = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 15u) & ~(uintptr_t)15u);
    s.pub = reinterpret_cast<PubQueue *>(p);
    return s;
}

__device__ __forceinline__ uint32_t lds_volatile(const uint32_t *p) { return *(const volatile uint32_t *)p; }
__device__ __forceinline__ void sts_volatile(uint32_t *p, uint32_t v) { *(volatile uint32_t *)p = v; }

// Alg. 1's overlap test between task i (earlier) and task j on inclusive
// ranges; a segment pair counts unless both are reads (RAW, WAR, WAW).
// The task being checked, its first kRegSegs segments held in registers
// (the same for every lane; tasks with more segments read the rest from
// shared memory).
constexpr int kRegSegs = 4;
struct NewTask {
    Seg a[kRegSegs];
    uint32_t n, w;
    uint32_t hi, narrow;   // as HistRec
    uint32_t s[kRegSegs], l[kRegSegs];   // narrow: low 32 bits of the starts and lasts
};

__device__ __forceinline__ NewTask load_new_task(const HistRec &hj) {
    const TaskRec &rj = hj.r;
    NewTask t;
    t.n = min((uint32_t)rj.nseg, (uint32_t)kMaxSegs);
    t.w = rj.wmask;
    t.hi = hj.hi;
    t.narrow = hj.narrow;
#pragma unroll
    for (int x = 0; x < kRegSegs; ++x) t.a[x] = x < (int)t.n ? rj.seg[x] : Seg{0, 0};   // unused beyond n
    if (t.narrow) {
        const uint4 cs = *reinterpret_cast<const uint4 *>(&rj.seg[4]), cl = *reinterpret_cast<const uint4 *>(&rj.seg[5]);
        t.s[0] = cs.x; t.s[1] = cs.y; t.s[2] = cs.z; t.s[3] = cs.w;
        t.l[0] = cl.x; t.l[1] = cl.y; t.l[2] = cl.z; t.l[3] = cl.w;
    } else {
#pragma unroll
        for (int x = 0; x < kRegSegs; ++x) { t.s[x] = 0; t.l[x] = 0; }
    }
    return t;
}

// Whether every segment of a record lies in one 4 GiB-aligned window (and
// there are at most kRegSegs of them): then overlap tests against another such
// record in the same window compare the low 32 bits only, which decide them
// exactly. Computed once per record by the loader, with the compact 32-bit
// copies of a narrow record's segments (see HistRec).
__device__ __forceinline__ void set_narrow(HistRec &h) {
    const uint32_t n = min((uint32_t)h.r.nseg, (uint32_t)kMaxSegs);
    const uint32_t hi = n ? (uint32_t)(h.r.seg[0].start >> 32) : 0u;
    bool ok = n <= (uint32_t)kRegSegs;
    for (uint32_t k = 0; k < n && ok; ++k)
        ok = (uint32_t)(h.r.seg[k].start >> 32) == hi && (uint32_t)(h.r.seg[k].last >> 32) == hi;
    h.hi = hi;
    h.narrow = ok ? 1u : 0u;
    h.nsw = n | ((uint32_t)h.r.wmask << 8);
    if (ok) {
        uint32_t s4[kRegSegs], l4[kRegSegs];
#pragma unroll
        for (int k = 0; k < kRegSegs; ++k) {
            s4[k] = (uint32_t)k < n ? (uint32_t)h.r.seg[k].start : 0u;
            l4[k] = (uint32_t)k < n ? (uint32_t)h.r.seg[k].last : 0u;
        }
        *reinterpret_cast<uint4 *>(&h.r.seg[4]) = make_uint4(s4[0], s4[1], s4[2], s4[3]);
        *reinterpret_cast<uint4 *>(&h.r.seg[5]) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
    }
}

// Every segment pair of a candidate (ri) and the new task (t, all segments
// also in rj), from shared memory: tasks with more than kRegSegs segments.
__device__ __noinline__ bool rec_conflict_all(const TaskRec &ri, const TaskRec &rj) {
    const int ni = min((int)ri.nseg, kMaxSegs), nj = min((int)rj.nseg, kMaxSegs);
    const uint32_t wi = ri.wmask, wj = rj.wmask;
    for (int y = 0; y < ni; ++y) {
        const Seg b = ri.seg[y];
        const bool yw = (wi >> y) & 1u;
        for (int x = 0; x < nj; ++x) {
            const Seg a = rj.seg[x];
            if ((yw || ((wj >> x) & 1u)) && a.start <= b.last && b.start <= a.last) return true;
        }
    }
    return false;
}

// Every segment pair of the candidate and the new task is tested (predicated,
// no early exit): when both records lie in the same 4 GiB window, on the low
// 32 address bits from their compact copies (three 16-byte loads of the
// candidate); else on the full 64 bits of the candidate's first kRegSegs
// segments, loaded together, and on the rest from shared memory.
__device__ __forceinline__ bool rec_conflict(const HistRec &hi_, const NewTask &t, const TaskRec &rj) {
    const TaskRec &ri = hi_.r;
    const uint4 meta = *reinterpret_cast<const uint4 *>(&hi_.hi);   // hi, narrow, nsw, pad
    if (t.narrow && meta.y && meta.x == t.hi) {
        const uint4 cs = *reinterpret_cast<const uint4 *>(&ri.seg[4]), cl = *reinterpret_cast<const uint4 *>(&ri.seg[5]);
        const uint32_t bs[kRegSegs] = {cs.x, cs.y, cs.z, cs.w}, bl[kRegSegs] = {cl.x, cl.y, cl.z, cl.w};
        const uint32_t ni = meta.z & 0xffu, wi = meta.z >> 8;
        // which segment pairs count (x and y valid, one of them written) as a
        // 16-bit mask (bit 4x + y), which overlap as another: one AND decides
        // (fewer instructions than testing the conditions pair by pair)
        const uint32_t yv = (1u << ni) - 1u, yw = wi & yv;
        uint32_t elig = 0, ov = 0;
#pragma unroll
        for (int x = 0; x < kRegSegs; ++x) {
            const uint32_t ym = (uint32_t)x < t.n ? (((t.w >> x) & 1u) ? yv : yw) : 0u;
            elig |= ym << (4 * x);
#pragma unroll
            for (int y = 0; y < kRegSegs; ++y)
                ov |= (t.s[x] <= bl[y] && bs[y] <= t.l[x]) ? (1u << (4 * x + y)) : 0u;
        }
        return (elig & ov) != 0u;
    }
    const uint32_t ni = min((uint32_t)ri.nseg, (uint32_t)kMaxSegs);
    const uint32_t wi = ri.wmask;
    Seg b[kRegSegs];
#pragma unroll
    for (int y = 0; y < kRegSegs; ++y) b[y] = ri.seg[y];    // unused entries are masked below
    bool hit = false;
    {
#pragma unroll
        for (int y = 0; y < kRegSegs; ++y) {
            const bool yv = (uint32_t)y < ni, yw = (wi >> y) & 1u;
#pragma unroll
            for (int x = 0; x < kRegSegs; ++x)
                hit |= yv && (uint32_t)x < t.n && (yw || ((t.w >> x) & 1u)) && t.a[x].start <= b[y].last &&
                       b[y].start <= t.a[x].last;
        }
    }
    if (!hit && (ni > (uint32_t)kRegSegs || t.n > (uint32_t)kRegSegs)) hit = rec_conflict_all(ri, rj);
    return hit;
}

// Warp 7: copies descriptors from the stream's device ring into hist with
// ordinary loads, a batch of kPrefetch at a time (every load of a batch in
// flight at once: one round trip), and publishes them through
// complete_upto after a CTA-scope fence. hist[s mod H] may take seq s once the
// record it replaces (s - H) is neither a candidate of an unchecked task nor
// uninserted: s < next + H - W + 1.
// Refresh the device mirror of the mailbox (one warp, resident launches). The
// drain word is read before the stream ends and written after them, so a
// reader that sees drain in the mirror sees every end published before it;
// the sys-scope fences carry the host's release of an end (its descriptors
// were copied before it) to the readers of the mirror.
__device__ void mirror_poll(const KParams &P, uint32_t lane) {
    uint32_t d = 0;
    unsigned long long hb = 0;
    if (lane == 0) {
        d = ld_relaxed_sys_u32(&P.mbox->drain);
        hb = ld_relaxed_sys_u64(&P.mbox->heartbeat);
    }
    fence_acq_rel_sys();
    constexpr uint32_t kPer = ACS_MAX_STREAMS / 32;
    uint32_t he[kPer];
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k)
        if (lane + 32 * k < P.n_streams) he[k] = ld_relaxed_sys_u32(&P.mbox->host_end[lane + 32 * k]);
    fence_acq_rel_sys();
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k)
        if (lane + 32 * k < P.n_streams) st_relaxed_u32(&P.mirror->end[lane + 32 * k], he[k]);
    __syncwarp();
    if (lane == 0) {
        fence_acq_rel_gpu();
        st_relaxed_u64(&P.mirror->heartbeat, hb);
        st_relaxed_u32(&P.mirror->drain, d);
    }
    __syncwarp();
}

__device__ void loader_warp(const KParams &P, uint32_t stream, uint8_t *smem_raw) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t W = P.window;
    const uint32_t C = 1u << P.cap_log2;
    const uint32_t first = P.first[stream];
    uint32_t end = P.end[stream];
    const bool open = P.open[stream] != 0;
    const TaskRec *recs = P.recs + (size_t)stream * C;
    SchedSmem S = carve(smem_raw, W);
    const uint32_t H = S.H, HM = H - 1;
    uint32_t load_upto = first - min(W - 1u, (uint32_t)P.nprev[stream]);   // the predecessors that exist
    unsigned long long tw = 0;
    uint32_t spins = 0, backoff = 32;
    uint32_t host_seen = end;                      // resident: host end last read
    const bool mirror_keeper = P.resident && stream == 0;
    unsigned long long mirror_t = 0;
    while (true) {
        if (mirror_keeper) {
            const unsigned long long now = globaltimer_ns();
            if (now - mirror_t >= 1000ull) {
                mirror_poll(P, lane);
                mirror_t = now;
            }
        }
        bool wait = false, host_wait = false;
        if (load_upto >= end) {
            if (!open && !P.resident) return;      // a closed stream is fully loaded
            if (P.resident) {
                // host-published descriptors first: at most 64 per round are
                // copied from the pinned host ring into the device ring (the
                // host appends only while no emitter of the stream is alive)
                if ((int32_t)(host_seen - end) <= 0) {   // nothing known beyond end (emitters may have moved it)
                    // the mirrored end (device memory); acquire when it moved
                    uint32_t he = 0;
                    if (lane == 0) {
                        he = ld_relaxed_u32(&P.mirror->end[stream]);
                        if (he != host_seen) fence_acq_rel_gpu();
                    }
                    host_seen = __shfl_sync(0xffffffffu, he, 0);
                }
                if ((int32_t)(host_seen - end) > 0) {
                    // the host published descriptors already copied into the
                    // device ring (by the copy engine, before the release
                    // store); take up to 256 per round, counting the emit
                    // tasks among them: each starts one emitter chain
                    const uint32_t n = min(host_seen - end, 256u);
                    const TaskRec *ring = P.recs + (size_t)stream * C;
                    uint32_t emits = 0;
#pragma unroll
                    for (uint32_t k = 0; k < 8; ++k) {
                        const uint32_t r = k * 32 + lane;
                        if (r < n) {
                            const uint4 h = __ldcg(reinterpret_cast<const uint4 *>(ring + ((end + r) & (C - 1))));
                            if ((h.y & 0xffffu) == ACS_OP_RL_EMIT) ++emits;
                        }
                    }
                    emits = __reduce_add_sync(0xffffffffu, emits);
                    if (lane == 0 && emits) atomicAdd(&P.sctl[stream].open, emits);
                    __syncwarp();
                    __threadfence();                   // chains counted before the new end
                    end += n;
                    if (lane == 0) {
                        st_relaxed_u32(&P.sctl[stream].end, end);
                        sts_volatile(&S.sh->end, end);
                    }
                    __syncwarp();
                    tw = 0;
                    backoff = 32;
                    continue;
                }
            }
            // an open stream grows when an emitter publishes a larger end (an
            // acquire load: the emitter's descriptors are visible once it reads it)
            const uint32_t e = ld_acquire_u32(&P.sctl[stream].end);
            if ((int32_t)(e - end) > 0) {
                __syncwarp();
                end = e;
                if (lane == 0) sts_volatile(&S.sh->end, end);
                continue;
            }
            wait = true;
            host_wait = P.resident;                // idle until the host publishes work
        } else {
            // a batch of up to kPrefetch stops at the stream's end and at the
            // device ring's end (the first 16 descriptors an emitter publishes
            // arrive in one batch, whatever their position)
            const uint32_t nb = min(min((uint32_t)kPrefetch, end - load_upto), C - (load_upto & (C - 1u)));
            const uint32_t bhi = load_upto + nb;
            const uint32_t nx = lds_volatile(&S.sh->next);
            if (bhi + W > nx + H + 1) {
                wait = true;
            } else {
                tw = 0;
                backoff = 32;
                // every load of the batch issued before the first store to
                // shared memory (one round trip, not one per vector)
                constexpr uint32_t kRec16 = sizeof(TaskRec) / 16;    // 20 vectors per record
                constexpr uint32_t kPerLane = (kPrefetch * kRec16 + 31) / 32;
                const uint32_t n16 = (bhi - load_upto) * kRec16;
                const uint4 *src = reinterpret_cast<const uint4 *>(recs + (load_upto & (C - 1)));
                uint4 v[kPerLane];
#pragma unroll
                for (uint32_t r = 0; r < kPerLane; ++r) {
                    const uint32_t i = lane + 32u * r;
                    if (i < n16) v[r] = __ldcg(src + i);
                }
#pragma unroll
                for (uint32_t r = 0; r < kPerLane; ++r) {
                    const uint32_t i = lane + 32u * r;
                    if (i < n16) {
                        const uint32_t rec = i / kRec16, part = i - rec * kRec16;
                        reinterpret_cast<uint4 *>(&S.hist[(load_upto + rec) & HM])[part] = v[r];
                    }
                }
                __syncwarp();
                if (lane < bhi - load_upto) {
                    HistRec &h = S.hist[(load_upto + lane) & HM];
                    set_narrow(h);
                    // the task's done word: (seq + 1, all its CTAs to go). The
                    // ring position's previous task (seq - capacity) retired
                    // before this descriptor was written, so waiters of it read
                    // the new word as complete, as they must. Tasks below `first`
                    // belong to earlier launches and have retired: untouched.
                    const uint32_t q = load_upto + lane;
                    if ((int32_t)(q - first) >= 0)
                        st_relaxed_u64(&P.done[((size_t)stream << P.cap_log2) | (q & (C - 1))],
                                       ((unsigned long long)(q + 1u) << 32) | h.r.ncta);
                }
                __syncwarp();
                __threadfence_block();
                load_upto = bhi;
                if (lane == 0) sts_volatile(&S.sh->complete_upto, load_upto);
            }
        }
        if (wait) {
            if (lds_volatile(&S.sh->quit)) return;
            if (host_wait) {
                // waiting for the host is not a stall: the scheduler warp bounds
                // it (idle limit) and raises quit; the mirror is device memory
                tw = 0;
                __nanosleep(backoff);
                if (backoff < 512) backoff <<= 1;
                continue;
            }
            if ((++spins & 63) == 0) {
                const unsigned long long now = globaltimer_ns();
                if (tw == 0) tw = now;
                else if (now - tw > 4ull * P.timeout_ns) {
                    if (lane == 0) raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSitePrefetch);
                    return;
                }
            }
            __nanosleep(backoff);
            if (backoff < 64) backoff <<= 1;
        }
    }
}

// Warp 6: polls the done word of every executing slot's task (acquire loads)
// and clears the slot's expect word once its task completed; those acquires, with
// the publisher's fence before it publishes work, order the retired tasks'
// writes before every dependent's start. Warp 0 never waits on global memory
// to retire tasks.
__device__ void poller_warp(const KParams &P, uint32_t stream, uint8_t *smem_raw) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t W = P.window;
    SchedSmem S = carve(smem_raw, W);
    const uint32_t CM = (1u << P.cap_log2) - 1u;
    const unsigned long long *done = P.done + ((size_t)stream << P.cap_log2);
    uint32_t backoff = 32;
    while (!lds_volatile(&S.sh->quit)) {
        const uint32_t e0 = lane < W ? lds_volatile(&S.expect[lane]) : 0u;
        const uint32_t e1 = lane + 32 < W ? lds_volatile(&S.expect[lane + 32]) : 0u;
        bool h0 = false, h1 = false;
        // acquire loads: a done word read at its task's value orders the
        // task's writes before what this lane does next
        if (e0) h0 = slot_done(ld_acquire_u64(&done[(e0 - 1u) & CM]), e0);
        if (e1) h1 = slot_done(ld_acquire_u64(&done[(e1 - 1u) & CM]), e1);
        const uint32_t b0 = __ballot_sync(0xffffffffu, h0), b1 = __ballot_sync(0xffffffffu, h1);
        if (b0 | b1) {
            // release at CTA scope: warp 0 retires a slot once it reads 0 here
            __threadfence_block();
            if (h0) sts_volatile(&S.expect[lane], 0u);
            if (h1) sts_volatile(&S.expect[lane + 32], 0u);
            backoff = 32;
        } else {
            const bool any = __any_sync(0xffffffffu, e0 | e1);
            if (!any) {
                __nanosleep(backoff);
                if (backoff < 256) backoff <<= 1;
            }
        }
    }
}

__device__ void checker_warp(const KParams &P, uint32_t stream, uint8_t *smem_raw, uint32_t w) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t W = P.check_w;   // candidates: the W - 1 previous tasks
    const uint32_t first = P.first[stream], end = P.end[stream];
    // open or resident: tasks beyond `end` may still come
    const bool open = P.open[stream] != 0 || P.resident != 0;
    SchedSmem S = carve(smem_raw, P.window);
    const uint32_t H = S.H, HM = H - 1;   // H is a power of two
    constexpr uint32_t kCheckers = kBlock / 32 - 4;   // warps 1 .. 4
    unsigned long long tw = 0;
    unsigned long long check_cycles = 0;
    const bool tracing = (P.flags & ACS_FLAG_TRACE) != 0;
    const bool logging = (P.flags & ACS_FLAG_LOG) != 0;
    // the loader's and the scheduler warp's progress as last read: both only
    // grow, so while they cover a task no new read is needed (the acquire that
    // returned cu_seen ordered every record below it); until the first read,
    // values that cover nothing
    uint32_t cu_seen = first, nx_seen = first - H;
    for (uint32_t j = first + w; open || j < end; j += kCheckers) {
        // wait: record j loaded and pmask slot j mod H consumed (j < next + H)
        uint32_t spins = 0, backoff = 32;
        while (!((int32_t)(cu_seen - j) > 0 && (int32_t)(j - (nx_seen + H)) < 0)) {
            // an acquire load: the loader released the records below it
            const uint32_t cu = ld_acquire_cta_shared(&S.sh->complete_upto);
            const uint32_t nx = lds_volatile(&S.sh->next);
            cu_seen = cu;
            nx_seen = nx;
            if (cu > j && j < nx + H) break;
            if (lds_volatile(&S.sh->quit)) {
                if (lane == 0 && check_cycles) atomicAdd(&P.sched_stats[stream].check_cycles, check_cycles);
                return;
            }
            // a resident stream waits for the host without bound here; the
            // scheduler warp's idle limit ends the wait through quit
            if (!P.resident && (++spins & 63) == 0) {
                const unsigned long long now = globaltimer_ns();
                if (tw == 0) tw = now;
                else if (now - tw > 4ull * P.timeout_ns) {
                    if (lane == 0) raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSiteSched);
                    return;
                }
            }
            __nanosleep(backoff);
            if (backoff < 64) backoff <<= 1;
        }
        tw = 0;
        const unsigned long long tc0 = tracing ? clock64() : 0ull;
        const TaskRec &rj = S.hist[j & HM].r;
        if (rj.seq != j || rj.nseg > kMaxSegs) {   // self-check: the record must be task j
            if (lane == 0) raise_error(P, (uint32_t)ACS_ERR_INVALID, kSiteCheckRecord);
            return;
        }
        bool c0 = false, c1 = false;
        const uint32_t d0 = lane + 1, d1 = lane + 33;      // distances to the candidates
        const uint32_t have = j - first + P.nprev[stream];   // tasks of the stream before j (capped)
        const NewTask nt = load_new_task(S.hist[j & HM]);
        // Without a log, a candidate that already retired is not tested: its
        // done word reads as complete to the task's workers anyway, and the
        // publisher's fence orders its writes before this task's units, as for
        // every conflict farther back than the window. (A stale release point
        // only means more tests.) With a log, every candidate is tested: the
        // log holds the window DAG.
        const uint32_t rel = logging ? 0u : lds_volatile(&S.sh->released);
        if (d0 <= W - 1 && d0 <= have && (int32_t)(j - d0 - rel) >= 0)
            c0 = rec_conflict(S.hist[(j - d0) & HM], nt, rj);
        if (d1 <= W - 1 && d1 <= have && (int32_t)(j - d1 - rel) >= 0)
            c1 = rec_conflict(S.hist[(j - d1) & HM], nt, rj);
        // The workers' mask is by distance: bit k for the candidate at distance
        // k + 1, bit 32 + k for distance k + 33 (two ballots). The log's mask is
        // by window slot, the candidate at distance d sitting in slot
        // (j - d) mod W; only a logging launch builds it.
        const uint32_t dlo = __ballot_sync(0xffffffffu, c0), dhi = __ballot_sync(0xffffffffu, c1);
        uint32_t mlo = 0, mhi = 0;
        if (logging) {
            const uint32_t js = j % W;
            if (c0) {
                const uint32_t sl = js >= d0 ? js - d0 : js + W - d0;
                if (sl < 32) mlo |= 1u << sl; else mhi |= 1u << (sl - 32);
            }
            if (c1) {
                const uint32_t sl = js >= d1 ? js - d1 : js + W - d1;
                if (sl < 32) mlo |= 1u << sl; else mhi |= 1u << (sl - 32);
            }
            mlo = __reduce_or_sync(0xffffffffu, mlo);
            mhi = __reduce_or_sync(0xffffffffu, mhi);
        }
        if (lane == 0) {
            if (logging) S.pmask[j & HM] = (unsigned long long)mlo | ((unsigned long long)mhi << 32);
            // what the task's worker CTAs wait for: every conflicting candidate
            // (one that has retired by then reads as complete); published to them
            // by the publisher's fence after the task's insertion
            *reinterpret_cast<uint4 *>(&P.taskaux[((size_t)stream << P.cap_log2) | (j & ((1u << P.cap_log2) - 1u))]) =
                make_uint4(dlo, dhi, j, 0u);
            st_release_cta_shared(&S.ptag[j & HM], j + 1u);   // after the aux word
            if (tracing) check_cycles += clock64() - tc0;
        }
        // no warp barrier here: the other lanes go on to the next task's
        // loads and tests while lane 0 publishes (the next ballots reconverge)
    }
    if (lane == 0 && check_cycles) atomicAdd(&P.sched_stats[stream].check_cycles, check_cycles);
}

// Shared-memory set-up of a scheduler CTA, before its warps take their roles
// (followed by __syncthreads in the caller).
__device__ void sched_init(const KParams &P, uint32_t stream, uint8_t *smem_raw) {
    const uint32_t W = P.window;
    const uint32_t first = P.first[stream];
    SchedSmem S = carve(smem_raw, W);
    for (uint32_t i = threadIdx.x; i < S.H; i += blockDim.x) S.ptag[i] = 0;
    for (uint32_t i = threadIdx.x; i < (uint32_t)kMaxWindow; i += blockDim.x) S.expect[i] = 0;
    if (threadIdx.x == 0) {
        S.pub->produced = 0;
        S.pub->consumed = 0;
        S.sh->complete_upto = first - min(W - 1u, (uint32_t)P.nprev[stream]);
        S.sh->next = first;
        S.sh->quit = 0;
        S.sh->end = P.end[stream];
        S.sh->head_pos = 0;
        S.sh->released = first;
        if (P.open[stream] || P.resident) {   // published before any emitter of this launch can run
            StreamCtl *sc = &P.sctl[stream];
            sc->end = P.end[stream];
            sc->open = P.open[stream];
            sc->head_pub = first;
            __threadfence();
        }
    }
}

// Warp 5: publishes the scheduler's insertion batches, oldest first, every
// batch pending at the time in one pass: a check that every work-ring cell it
// fills is free (its sequence word reads its position), one fence.acq_rel.gpu
// for the pass, then the cells' sequence words. The fence orders what the
// other warps wrote or saw before the batches were handed over (the loader's
// done words, the checkers' aux words, log entries, retirements the poller
// acquired) before the new units. A pass costs about one fence whatever the
// number of batches, so batches that queue while one is published go out
// together in the next.
__device__ void publisher_warp(const KParams &P, uint32_t stream, uint8_t *smem_raw) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t C = 1u << P.cap_log2;
    SchedSmem S = carve(smem_raw, P.window);
    const bool sole_producer = P.n_streams == 1;
    const bool tracing = (P.flags & ACS_FLAG_TRACE) != 0;
    uint32_t done_b = 0, backoff = 32;
    const uint32_t ncells = P.cell_mask + 1u;
    while (true) {
        const uint32_t prod = lds_volatile(&S.pub->produced);
        if (prod == done_b) {
            if (lds_volatile(&S.sh->quit)) return;
            __nanosleep(backoff);
            if (backoff < 64) backoff <<= 1;
            continue;
        }
        backoff = 32;
        __threadfence_block();
        // sole producer: a cell whose previous unit lies below head_pos was
        // read by its worker before that unit's task retired (the fence below
        // orders this read of head_pos before the cells are written)
        const uint32_t head_pos = sole_producer ? lds_volatile(&S.sh->head_pos) : 0u;
        // 1. every pending batch: its cells checked free
        bool ok = true;
        for (uint32_t b = done_b; b != prod && ok; ++b) {
            const PubBatch &B = S.pub->b[b % kPubSlots];
            const uint32_t p0 = B.p0, total = B.total;
            for (uint32_t u = lane; u < total && ok; u += 32) {
                const uint32_t x = p0 + u;
                if (sole_producer && (int32_t)(x - ncells - head_pos) < 0) continue;
                unsigned long long *cell = &P.cells[x & P.cell_mask];
                unsigned long long tw = 0;
                uint32_t spins = 0;
                while ((uint32_t)ld_relaxed_u64(cell) != x) {
                    if ((++spins & 63) == 0) {
                        const unsigned long long now = globaltimer_ns();
                        if (tw == 0) tw = now;
                        else if (now - tw > P.timeout_ns) {
                            raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSiteRing);
                            ok = false;
                            break;
                        }
                        if (stopped(P)) { ok = false; break; }
                    }
                }
            }
        }
        if (!__all_sync(0xffffffffu, ok)) return;
        fence_acq_rel_gpu();
        __syncwarp();
        // 2. the cells of every pending batch
        for (uint32_t b = done_b; b != prod; ++b) {
            const PubBatch &B = S.pub->b[b % kPubSlots];
            const uint32_t nins = B.nins, p0 = B.p0;
            if (lane < nins) {
                const uint32_t q = B.q[lane], off = B.off[lane], n = B.n[lane];
                const uint32_t gidx = (stream << P.cap_log2) | (q & (C - 1));
                if (tracing)   // publication: the units become visible from here on
                    P.trace[(((size_t)stream << P.log_log2) + (q & ((1u << P.log_log2) - 1u))) * kTraceFields + 1] =
                        globaltimer_ns();
                for (uint32_t c = 0; c < n; ++c) {
                    const uint32_t pos = p0 + off + c;
                    const uint32_t payload = (gidx << 8) | c;
                    st_relaxed_u64(&P.cells[pos & P.cell_mask],
                                   ((unsigned long long)payload << 32) | (unsigned long long)(pos + 1u));
                }
            }
        }
        done_b = prod;
        __syncwarp();
        if (lane == 0) sts_volatile(&S.pub->consumed, done_b);
    }
}

__device__ void scheduler_warp(const KParams &P, uint32_t stream, uint8_t *smem_raw) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t W = P.window;
    const uint32_t first = P.first[stream];
    const bool resident = P.resident != 0;
    const bool open = P.open[stream] != 0 || resident;
    uint32_t end = P.end[stream];              // grows while the stream is open
    const bool logging = (P.flags & ACS_FLAG_LOG) != 0;
    const bool tracing = (P.flags & ACS_FLAG_TRACE) != 0;
    const uint32_t LM = (1u << P.log_log2) - 1u;
    const size_t lbase = (size_t)stream << P.log_log2;
    SchedSmem S = carve(smem_raw, W);
    const uint32_t H = S.H, HM = H - 1;
    const unsigned long long t_begin = clock64();
    unsigned long long busy = 0, inserts = 0, starved = 0;

    // per-lane slot registers: slot lane (index 0) and lane + 32 (index 1)
    uint32_t st0 = kEmpty, st1 = kEmpty, sq0 = 0, sq1 = 0;

    uint32_t head = first, next = first;
    uint32_t hslot = first % W, nslot = first % W;   // head % W, next % W
    const bool sole_producer = P.n_streams == 1;
    uint32_t tail = sole_producer ? ld_volatile_u32(&P.ctl->ring_tail) : 0u;
    if (sole_producer && lane == 0) sts_volatile(&S.sh->head_pos, tail);   // earlier launches' units are consumed
    uint32_t pub_prod = 0;                          // batches handed to the publisher
    unsigned long long idle_since = 0;
    uint32_t iter = 0;
    bool failed = false;
    unsigned long long ph[kPhases] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long tp = 0;
// per-phase cycle counters, only when tracing (each clock read sits on the warp's path)
#define ACS_PHASE(k) do { if (tracing) { const unsigned long long _t = clock64(); ph[k] += _t - tp; tp = _t; } } while (0)

    uint32_t head_pub = first;
    // resident launches: progress reported to the host, idle bookkeeping
    uint32_t head_host = first, idle_pub = first - 1u, idle_polls = 0, idle_sleep = 256;
    unsigned long long last_hb = 0, hb_time = 0;
    while (first < end || open) {
        bool progress = false;
        const unsigned long long t0 = tracing ? clock64() : 0ull;
        tp = t0;
        if (open) end = lds_volatile(&S.sh->end);

        ACS_PHASE(0);
        const unsigned long long full = W == 64 ? ~0ull : ((1ull << W) - 1ull);
        // 1. retire the slots the poller warp saw complete, first, so that a
        //    slot released now takes a task in this same iteration: an
        //    executing slot whose expect word the poller cleared (each lane
        //    reads the words of its own two slots)
        const bool ret0 = st0 == kExec && lds_volatile(&S.expect[lane]) == 0u;
        const bool ret1 = W > 32 && st1 == kExec && lds_volatile(&S.expect[lane + 32]) == 0u;
        if (__any_sync(0xffffffffu, ret0 || ret1)) {
            __threadfence_block();   // acquire: what the poller acquired before clearing ...
            __syncwarp();            // ... for every lane of the warp
            progress = true;
            if (ret0) st0 = kRetired;
            if (ret1) st1 = kRetired;
            if (tracing) {
                const unsigned long long now = globaltimer_ns();
                if (ret0) P.trace[(lbase + (sq0 & LM)) * kTraceFields + 4] = now;
                if (ret1) P.trace[(lbase + (sq1 & LM)) * kTraceFields + 4] = now;
            }
            // release in program order: the run of retired slots from the head
            unsigned long long RT = __ballot_sync(0xffffffffu, st0 == kRetired);
            if (W > 32) RT |= (unsigned long long)__ballot_sync(0xffffffffu, st1 == kRetired) << 32;
            const unsigned long long rrt = hslot ? (((RT >> hslot) | (RT << (W - hslot))) & full) : RT;
            uint32_t run = rrt == ~0ull ? 64u : (uint32_t)(__ffsll((long long)~rrt) - 1);
            run = min(run, next - head);
            head += run;
            hslot += run;
            if (hslot >= W) hslot -= W;
            // for the checkers: candidates below it need no test
            if (lane == 0 && run) st_release_cta_shared(&S.sh->released, head);
            if (sole_producer && run) {
                // every unit below the first one of the oldest unreleased task
                // belongs to a retired task, so its worker has read it
                const uint32_t hp = head == next ? tail : S.slotpos[hslot];
                __threadfence_block();   // after the retirements taken above
                if (lane == 0) sts_volatile(&S.sh->head_pos, hp);
            }
        }
        ACS_PHASE(2);
        // 2. how many tasks are checked and have a free slot (at most 32 per
        //    iteration); one CTA-scope fence orders the tag reads before the
        //    mask reads (before the global polls below, so it never waits on them)
        uint32_t nins = 0;
        {
            // room: ring positions (span W) and, with a smaller active limit,
            // tasks not yet retired (retired ones free their place at once,
            // out of order, while ring positions are released in order)
            uint32_t room = min(W - (next - head), 32u);
            if (P.active_limit < W) {
                uint32_t act_n = __popc(__ballot_sync(0xffffffffu, st0 == kExec));
                if (W > 32) act_n += __popc(__ballot_sync(0xffffffffu, st1 == kExec));
                room = min(room, P.active_limit > act_n ? P.active_limit - act_n : 0u);
            }
            const uint32_t cap = min(end - next, room);
            const bool ok = lane < cap && lds_volatile(&S.ptag[(next + lane) & HM]) == next + lane + 1u;
            const uint32_t okm = __ballot_sync(0xffffffffu, ok);
            nins = __ffs(~okm) - 1;          // leading run of checked tasks
            if (okm == 0xffffffffu) nins = 32;
            if (tracing && nins == 0 && cap > 0) ++starved;
        }
        if (nins) __threadfence_block();

        // values of this iteration's insertion batch, handed to the publisher below
        bool mine = false;
        uint32_t q = 0, my_n = 0, my_off = 0, js = 0, p0 = 0, total = 0;
        // 3. insert and dispatch, lane k taking task next + k. Every task is
        //    dispatched when it enters the window: its worker CTAs wait for the
        //    checker's mask and then for the done words of the predecessors it
        //    names. Units enter the FIFO work ring in program order, after
        //    those of every upstream task, so the oldest unfinished unit never
        //    waits on a later one: no deadlock.
        if (nins) {
            mine = lane < nins;
            q = next + lane;
            my_n = mine ? (uint32_t)S.hist[q & HM].r.ncta : 0u;
            // the checker's candidate mask, for the log (the task's workers
            // read it from its aux word, which the checker wrote)
            const unsigned long long pre = (mine && logging) ? S.pmask[q & HM] : 0ull;
            // exclusive prefix sum of the CTA counts, one ballot per bit plane
            // (independent of each other, unlike a shuffle scan)
            const uint32_t planes = 32u - (uint32_t)__clz(__reduce_or_sync(0xffffffffu, my_n));
            const uint32_t below = (1u << lane) - 1u;
            uint32_t excl = 0;
            total = 0;
            for (uint32_t b = 0; b < planes; ++b) {
                const uint32_t m = __ballot_sync(0xffffffffu, (my_n >> b) & 1u);
                excl += (uint32_t)__popc(m & below) << b;
                total += (uint32_t)__popc(m) << b;
            }
            if (sole_producer) {
                p0 = tail;
            } else {
                p0 = 0;
                if (lane == 0) p0 = atomicAdd(&P.ctl->ring_tail, total);
                p0 = __shfl_sync(0xffffffffu, p0, 0);
            }
            tail = p0 + total;
            ACS_PHASE(3);
            ACS_PHASE(4);
            js = nslot + lane >= W ? nslot + lane - W : nslot + lane;
            my_off = excl;
            if (mine) {
                S.slotpos[js] = p0 + my_off;
                if (logging || tracing) {
                    const size_t li = lbase + (q & LM);
                    if (logging) {
                        P.log_mask[li] = pre;
                        P.log_start[li] = ~0ull;
                        P.log_retire[li] = 0ull;
                    }
                    if (tracing) {
                        const unsigned long long now = globaltimer_ns();
                        P.trace[li * kTraceFields + 0] = now;   // field 1: the publisher warp
                        P.trace[li * kTraceFields + 2] = ~0ull;   // first-CTA start: atomicMin target
                        P.trace[li * kTraceFields + 3] = 0ull;    // last-CTA end: atomicMax target
                    }
                }
            }
            ACS_PHASE(5);
            // slot states for in-order release: the owner of slot s takes task
            // next + ((s - nslot) mod W)
            const uint32_t k0 = lane >= nslot ? lane - nslot : lane + W - nslot;
            if (lane < W && k0 < nins) { st0 = kExec; sq0 = next + k0; }
            if (W > 32) {
                const uint32_t s1 = lane + 32u;
                const uint32_t k1 = s1 >= nslot ? s1 - nslot : s1 + W - nslot;
                if (s1 < W && k1 < nins) { st1 = kExec; sq1 = next + k1; }
            }
            next += nins;
            nslot += nins;
            if (nslot >= W) nslot -= W;
            inserts += nins;
            progress = true;
            if (lane == 0) sts_volatile(&S.sh->next, next);
            __syncwarp();
        }
        ACS_PHASE(1);
        // 4. hand this iteration's insertion batch to the publisher warp (its
        //    fence then orders the log entries above and the retirements seen
        //    through the poller before the new units: conflicts farther back
        //    than W - 1 rely on that alone); a slot's expect word is set here,
        //    after its task is marked executing, and read again only in a
        //    later iteration
        if (nins) {
            uint32_t spins = 0;
            unsigned long long tw = 0;
            bool ok = true;
            while (pub_prod - lds_volatile(&S.pub->consumed) >= kPubSlots) {   // queue full: wait (bounded)
                if ((++spins & 63) == 0) {
                    const unsigned long long now = globaltimer_ns();
                    if (tw == 0) tw = now;
                    else if (now - tw > P.timeout_ns) {
                        if (lane == 0) raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSiteRing);
                        ok = false;
                        break;
                    }
                    if (stopped(P)) { ok = false; break; }
                }
            }
            if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
            PubBatch &B = S.pub->b[pub_prod % kPubSlots];
            if (mine) {
                B.q[lane] = q;
                B.off[lane] = my_off;
                B.n[lane] = my_n;
                S.expect[js] = q + 1u;             // the poller watches the slot from now on
            }
            if (lane == 0) {
                B.nins = nins;
                B.p0 = p0;
                B.total = total;
            }
            __syncwarp();
            __threadfence_block();
            ++pub_prod;
            if (lane == 0) sts_volatile(&S.pub->produced, pub_prod);
            ACS_PHASE(6);
        }
        if (open && head != head_pub && lane == 0) {   // emitters wait on it for ring space
            st_relaxed_u32(&P.sctl[stream].head_pub, head);
        }
        head_pub = head;
        if (resident && head - head_host >= 16u && lane == 0) {   // the host's ring-space check
            st_relaxed_sys_u32(&P.mbox->progress[stream].head, head);
            head_host = head;
        }
        bool idle = false;
        if (head == end) {
            if (!open) { if (tracing) busy += clock64() - t0; break; }
            // open stream: finished once no emitter is left and nothing was appended
            // (an acquire load, not a fence: idle streams poll this often)
            uint32_t fin = 0;
            if (lane == 0 && ld_acquire_u32(&P.sctl[stream].open) == 0)
                fin = ld_relaxed_u32(&P.sctl[stream].end) == end;
            fin = __shfl_sync(0xffffffffu, fin, 0);
            if (fin && !resident) { if (tracing) busy += clock64() - t0; break; }
            if (fin) {
                // resident and idle: every task below end retired. Tell the host
                // (its results are visible system-wide first), then look for
                // the host's drain request or its absence, every 8th idle pass.
                idle = true;
                uint32_t leave = 0;
                if (lane == 0) {
                    if (end != idle_pub) {
                        __threadfence_system();
                        st_relaxed_sys_u32(&P.mbox->progress[stream].head, head);
                        st_relaxed_sys_u32(&P.mbox->progress[stream].idle_at, end);
                        idle_pub = end;
                        head_host = head;
                    }
                    if ((++idle_polls & 7) == 0) {
                        const unsigned long long now = globaltimer_ns();
                        const unsigned long long hb = ld_relaxed_u64(&P.mirror->heartbeat);
                        if (hb != last_hb || hb_time == 0) { last_hb = hb; hb_time = now; }
                        // (emitters may have taken the end past the host's)
                        if (ld_acquire_u32(&P.mirror->drain) &&
                            (int32_t)(ld_relaxed_u32(&P.mirror->end[stream]) - end) <= 0) {
                            leave = 1;
                        } else if (now - hb_time > P.idle_limit_ns) {
                            st_relaxed_sys_u32(&P.mbox->expired, 1u);
                            leave = 1;
                        }
                    }
                }
                if (__shfl_sync(0xffffffffu, leave, 0)) { if (tracing) busy += clock64() - t0; break; }
            }
        }

        ACS_PHASE(7);

        if (progress) {
            if (tracing) busy += clock64() - t0;
            idle_since = 0;
            idle_sleep = 256;
        } else if (idle) {
            // resident and waiting for the host: bounded by the idle limit
            // above (the polls stay in device memory and take no fence)
            idle_since = 0;
            __nanosleep(idle_sleep);
            if (idle_sleep < 1024) idle_sleep <<= 1;
        } else {
            const unsigned long long now = globaltimer_ns();
            if (idle_since == 0) idle_since = now;
            else if (now - idle_since > P.timeout_ns) {
                if (lane == 0) raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSiteSched);
                failed = true;
                break;
            }
        }
        if ((++iter & 31) == 0 && stopped(P)) { failed = true; break; }
    }
    (void)failed;
    if (sole_producer && lane == 0) st_relaxed_u32(&P.ctl->ring_tail, tail);
    if (lane == 0) sts_volatile(&S.sh->quit, 1u);
    if (lane == 0) {
        SchedStats *ss = &P.sched_stats[stream];
        ss->cycles += clock64() - t_begin;
        ss->busy_cycles += busy;
        ss->inserts += inserts;
        ss->iterations += iter;
        for (int k = 0; k < kPhases; ++k) ss->phase[k] += ph[k];
        ss->starved_iters += starved;
        __threadfence();
        if (atomicAdd(&P.ctl->sched_done, 1u) == P.n_streams - 1u) {
            __threadfence();
            atomicExch(&P.ctl->stop, 1u);
        }
    }
}

// ---- device-side emission (rigid-sphere stream) -----------------------------------

struct EmitSmem {
    acs_rl_emit_cfg cfg;
    uint32_t base, ok, pad[2];
    int wcnt[kBlock / 32];
    uint16_t env[1024];        // environments with islands, ascending
    uint8_t nisl[1024];        // their island counts
    uint8_t tab_int[1024];     // CTA counts of this step's integrate tasks, by chunk
    uint8_t tab_bp[1024];      // CTA counts of the next step's broadphase tasks, by chunk
};

static_assert(sizeof(EmitSmem) <= kBodySmem, "emit smem");

// One descriptor written straight into the stream's device ring: header, args
// and the segments acs_get_addresses derives for the same args. Returns the
// bytes its segments name (a read-modify-write segment twice), as the host
// counts a submitted task's.
__device__ __forceinline__ unsigned long long put_rec(TaskRec *r, uint32_t seq, uint16_t op, uint16_t ncta,
                                                      const void *args, uint32_t args_bytes, const Seg *segs,
                                                      uint32_t nseg, uint16_t wmask, uint8_t rw) {
    TaskHdr h;
    uint32_t *hw = reinterpret_cast<uint32_t *>(&h);
#pragma unroll
    for (int i = 0; i < 16; ++i) hw[i] = 0;
    h.task_id = seq;
    h.op = op;
    h.ncta = ncta;
    h.wmask = wmask;
    h.nseg = (uint8_t)nseg;
    h.flags = rw;
    h.seq = seq;
    const uint32_t *aw = reinterpret_cast<const uint32_t *>(args);
    for (uint32_t i = 0; i < args_bytes / 4; ++i) hw[4 + i] = aw[i];
    uint4 *dst = reinterpret_cast<uint4 *>(r);
    const uint4 *src = reinterpret_cast<const uint4 *>(&h);
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[i] = src[i];
    unsigned long long bytes = 0;
    for (uint32_t k = 0; k < nseg; ++k) {
        r->seg[k] = segs[k];
        bytes += (segs[k].last - segs[k].start + 1) * (1u + ((rw >> k) & 1u));
    }
    return bytes;
}

__device__ __forceinline__ Seg seg_of(uint64_t a, uint64_t n) { return Seg{a, a + n - 1}; }

// The emit task of step t (one CTA): appends solves, integrates, the next
// broadphase and the next emit task after the current end of its stream, and
// publishes the new end with release semantics in two steps (the first 32
// descriptors, then all). Every global read it needs
// (the cfg block, the island counts, the chunk CTA counts, the stream's end
// and oldest unreleased task) is issued at once, so the task costs one memory
// round trip before it writes.
__device__ void body_rl_emit(const KParams &P, uint32_t stream, const TaskHdr &hdr, uint8_t *smem) {
    EmitSmem &E = *reinterpret_cast<EmitSmem *>(smem);
    const acs_rl_emit_args a = load_args<acs_rl_emit_args>(hdr.args);
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t C = 1u << P.cap_log2, W = P.window;
    StreamCtl *sc = &P.sctl[stream];
    TaskRec *ring = P.recs + (size_t)stream * C;
    const uint32_t n_env = a.n_env, chunk = a.chunk;
    if (!(n_env <= 1024 && chunk > 0 && n_env % chunk == 0)) {   // self-check of the args (uniform)
        if (tid == 0) raise_error(P, (uint32_t)ACS_ERR_INVALID, kSiteEmit);
        return;
    }
    const uint32_t n_chunks = n_env / chunk;
    const bool more = a.step + 1 < a.steps;
    constexpr int kPer = 1024 / kBlock;            // environments (and chunks) per thread, at most
    const uint32_t *nisl_g = reinterpret_cast<const uint32_t *>(a.nisl);
    const uint8_t *table = reinterpret_cast<const uint8_t *>(a.ncta_table);
    uint32_t cfgw = 0, base = 0, head = 0, isl[kPer];
    uint8_t ti[kPer], tb[kPer];
    if (tid < sizeof(acs_rl_emit_cfg) / 4) cfgw = reinterpret_cast<const uint32_t *>(a.cfg)[tid];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const uint32_t e = tid + r * kBlock;
        isl[r] = e < n_env ? nisl_g[e] : 0u;
        ti[r] = e < n_chunks ? table[(a.step * 2 + 1) * n_chunks + e] : (uint8_t)1;
        tb[r] = more && e < n_chunks ? table[((a.step + 1) * 2 + 0) * n_chunks + e] : (uint8_t)1;
    }
    if (tid == 0) {
        base = ld_relaxed_u32(&sc->end);
        head = ld_relaxed_u32(&sc->head_pub);
    }
    if (tid < sizeof(acs_rl_emit_cfg) / 4) reinterpret_cast<uint32_t *>(&E.cfg)[tid] = cfgw;
    // the chunk CTA counts this task copies from the table must be 1 .. 255 (a
    // 0 would leave its task unrun): checked before anything is appended
    bool bad = false;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const uint32_t c = tid + r * kBlock;
        if (c < n_chunks) {
            E.tab_int[c] = ti[r];
            E.tab_bp[c] = tb[r];
            bad |= ti[r] == 0 || tb[r] == 0;
        }
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) raise_error(P, (uint32_t)ACS_ERR_INVALID, kSiteEmit);
        return;
    }
    // environments with islands, in ascending order (ballot scan per 256)
    uint32_t count = 0;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        if ((uint32_t)r * kBlock >= n_env) break;     // uniform
        const uint32_t e = r * kBlock + tid;
        const uint32_t k = isl[r];
        const bool has = k > 0;
        const uint32_t bal = __ballot_sync(0xffffffffu, has);
        if (lane == 0) E.wcnt[warp] = __popc(bal);
        __syncthreads();
        uint32_t off = count;
        for (uint32_t w = 0; w < warp; ++w) off += E.wcnt[w];
        if (has) {
            const uint32_t pos = off + __popc(bal & ((1u << lane) - 1u));
            E.env[pos] = (uint16_t)e;
            E.nisl[pos] = (uint8_t)min(k, 255u);
        }
        for (uint32_t w = 0; w < kBlock / 32; ++w) count += E.wcnt[w];
        __syncthreads();
    }
    const uint32_t n_solve = count;
    const uint32_t n_new = n_solve + n_chunks + (more ? n_chunks + 1 : 0);
    // the ring positions the new tasks overwrite must hold only released
    // tasks no window still looks at: wait (bounded) while they do not
    if (tid == 0) {
        unsigned long long tw = 0;
        uint32_t ok = 1;
        while ((int32_t)(base + n_new + W - (head + C)) > 0) {
            if (stopped(P)) { ok = 0; break; }
            const unsigned long long now = globaltimer_ns();
            if (tw == 0) tw = now;
            else if (now - tw > P.timeout_ns) {
                raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSiteEmit);
                ok = 0;
                break;
            }
            __nanosleep(256);
            head = ld_relaxed_u32(&sc->head_pub);
        }
        E.base = base;
        E.ok = ok;
    }
    __syncthreads();
    if (!E.ok) return;
    base = E.base;
    const acs_rl_emit_cfg &cfg = E.cfg;
    constexpr uint64_t kPos = 32 * 3 * 4, kProp = 32 * 2 * 4, kRec = ACS_RL_REC_BYTES;
    unsigned long long bytes = 0;    // segment bytes of the descriptors this thread writes
    auto put = [&](uint32_t k) {
        const uint32_t seq = base + k;
        TaskRec *r = ring + (seq & (C - 1));
        Seg sg[5];
        if (k < n_solve) {
            const uint64_t e = E.env[k];
            acs_rl_solve_args x{cfg.pos + e * kPos, cfg.prop + e * kProp, cfg.cont + e * kRec, cfg.vel + e * kPos,
                                cfg.beta_dt, cfg.slop};
            // reads pos, prop, cont; reads and writes vel (one write segment: see fold_reads)
            sg[0] = seg_of(x.pos, kPos); sg[1] = seg_of(x.prop, kProp); sg[2] = seg_of(x.cont, kRec);
            sg[3] = seg_of(x.vel, kPos);
            const uint16_t nc = (uint16_t)min(max((uint32_t)E.nisl[k], 1u), 16u);
            bytes += put_rec(r, seq, ACS_OP_RL_SOLVE, nc, &x, sizeof x, sg, 4, 1u << 3, 1u << 3);
        } else if (k < n_solve + n_chunks) {
            const uint64_t c = k - n_solve, e0 = c * chunk;
            acs_rl_integrate_args x{cfg.pos + e0 * kPos, cfg.vel + e0 * kPos, cfg.prop + e0 * kProp, chunk,
                                    cfg.dt, cfg.gdt, cfg.box};
            // reads prop, reads and writes pos and vel (the host's folded order)
            sg[0] = seg_of(x.prop, chunk * kProp);
            sg[1] = seg_of(x.pos, chunk * kPos); sg[2] = seg_of(x.vel, chunk * kPos);
            bytes += put_rec(r, seq, ACS_OP_RL_INTEGRATE, E.tab_int[c], &x, sizeof x, sg, 3, 6u, 6u);
        } else if (k < n_solve + 2 * n_chunks) {
            const uint64_t c = k - n_solve - n_chunks, e0 = c * chunk;
            acs_rl_broadphase_args x{cfg.pos + e0 * kPos, cfg.prop + e0 * kProp, cfg.cont + e0 * kRec,
                                     a.nisl + e0 * 4, chunk, 0};
            sg[0] = seg_of(x.pos, chunk * kPos); sg[1] = seg_of(x.prop, chunk * kProp);
            sg[2] = seg_of(x.cont, chunk * kRec); sg[3] = seg_of(x.nisl, chunk * 4);
            bytes += put_rec(r, seq, ACS_OP_RL_BROADPHASE, E.tab_bp[c], &x, sizeof x, sg, 4, (1u << 2) | (1u << 3), 0u);
        } else {
            acs_rl_emit_args x = a;
            x.step = a.step + 1;
            sg[0] = seg_of(x.nisl, (uint64_t)n_env * 4);
            sg[1] = seg_of(x.cfg, sizeof(acs_rl_emit_cfg));
            sg[2] = seg_of(x.ncta_table, (uint64_t)(x.steps + 1) * 2 * n_chunks);
            sg[3] = seg_of(x.token, 4);
            bytes += put_rec(r, seq, ACS_OP_RL_EMIT, 1, &x, sizeof x, sg, 4, 1u << 3, 0u);
        }
    };
    // Warp 0 writes the first 32 descriptors and publishes them at once, so
    // that the scheduler loads and checks them while the other warps write the
    // rest; the full end follows below.
    const uint32_t k1 = min(n_new, 32u);
    if (warp == 0) {
        if (lane < k1) put(lane);
        __syncwarp();
        if (lane == 0) st_release_u32(&sc->end, base + k1);   // the warp's descriptors before it
    } else {
        for (uint32_t k = k1 + tid - 32u; k < n_new; k += kBlock - 32u) put(k);
    }
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    if (lane == 0 && bytes) atomicAdd(&P.sched_stats[stream].seg_bytes, bytes);
    __syncthreads();
    if (tid == 0) {
        st_release_u32(&sc->end, base + n_new);   // every descriptor before the new end
        atomicAdd(&P.sched_stats[stream].emitted, (unsigned long long)n_new);
        if (!more) {
            __threadfence();                   // the final end before the stream closes
            atomicSub(&sc->open, 1u);
        }
    }
}

// ---- worker CTAs ----------------------------------------------------------------

__device__ void worker_loop(const KParams &P, uint8_t *smem) {
    __shared__ unsigned long long s_cell;
    __shared__ uint32_t s_quit;
    __shared__ uint4 s_aux;
    __shared__ TaskHdr s_hdr;
    const bool logging = (P.flags & ACS_FLAG_LOG) != 0;
    const bool tracing = (P.flags & ACS_FLAG_TRACE) != 0;
    const uint32_t ncells = P.cell_mask + 1u;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t nrec = P.n_streams << P.cap_log2;
    const uint32_t CM = (1u << P.cap_log2) - 1u;
    // warps 1 and 2 watch the done words of the tasks at distance d = 1 .. 64
    // back (lane k of warp 1: d = k + 1; of warp 2: d = k + 33), up to the ring's span
    const uint32_t d = warp * 32u + lane - 31u;
    const bool watcher = (warp == 1 || warp == 2) && d <= P.window;
    while (true) {
        if (threadIdx.x == 0) {
            // claim the next work-ring position and wait for its unit
            const uint32_t pos = atomicAdd(&P.ctl->ring_head, 1u);
            unsigned long long *cell = &P.cells[pos & P.cell_mask];
            uint32_t quit = 0, spins = 0, backoff = 32;
            unsigned long long tw = 0, v;
            while (true) {
                // an acquire load: reading the publisher's cell (written after
                // its fence) orders everything it published before this unit
                v = ld_acquire_u64(cell);
                if ((uint32_t)v == pos + 1u) break;
                if ((++spins & 7) == 0) {
                    if (stopped(P)) { quit = 1; break; }
                    const unsigned long long now = globaltimer_ns();
                    if (tw == 0) tw = now;
                    else if (now - tw > 4ull * P.timeout_ns + (P.resident ? P.idle_limit_ns : 0ull)) {
                        // idle workers outwait the schedulers' bounds
                        raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSiteWorker);
                        quit = 1;
                        break;
                    }
                }
                __nanosleep(backoff);
                if (backoff < P.poll_ns) backoff <<= 1;
            }
            if (!quit) st_relaxed_u64(cell, (unsigned long long)(pos + ncells));  // free for the next lap
            s_cell = v;
            s_quit = quit;
        }
        // the barrier passes thread 0's acquire of the cell to every thread
        __syncthreads();
        if (s_quit) break;
        const uint32_t payload = (uint32_t)(s_cell >> 32);
        const uint32_t gidx = payload >> 8, cta = payload & 255u;
        if (gidx >= nrec) {   // self-check: payload names a ring entry
            if (threadIdx.x == 0) raise_error(P, (uint32_t)ACS_ERR_INVALID, kSiteWorkerPayload);
            __syncthreads();
            continue;
        }
        const uint32_t stream = gidx >> P.cap_log2;
        const unsigned long long *done = P.done + (gidx & ~CM);   // the stream's done words
        // one round trip for the task's header and aux word (warp 0) and the
        // first look at the done words (warps 1, 2: acquire loads, one per
        // thread, issued before the unit knows which of them it needs; the
        // words lie inside the stream's ring, so every load is in bounds)
        unsigned long long dw = 0;
        if (warp == 0 && lane < 5) {
            const uint4 *src = lane < 4 ? reinterpret_cast<const uint4 *>(P.recs + gidx) + lane
                                        : reinterpret_cast<const uint4 *>(&P.taskaux[gidx]);
            const uint4 w = __ldcg(src);
            if (lane < 4) reinterpret_cast<uint4 *>(&s_hdr)[lane] = w;
            else s_aux = w;
        }
        if (watcher) dw = ld_acquire_u64(&done[(gidx - d) & CM]);
        __syncthreads();
        const uint32_t seq = s_aux.z;
        const unsigned long long up = (unsigned long long)s_aux.x | ((unsigned long long)s_aux.y << 32);
        // a GEMV unit's weight rows depend on no task: start moving them into L2
        // now, while the unit may still wait for its upstream tasks
        if (threadIdx.x == 0 && s_hdr.op == ACS_OP_GEMV && cta < s_hdr.ncta) {
            const acs_gemv_args g = load_args<acs_gemv_args>(s_hdr.args);
            const uint32_t rpc = (g.m + s_hdr.ncta - 1) / s_hdr.ncta;
            const uint32_t r0 = min(g.m, rpc * cta), r1 = min(g.m, r0 + rpc);
            const uint64_t a = g.W + (uint64_t)r0 * g.k * 4u, bytes = (uint64_t)(r1 - r0) * g.k * 4u;
            if (((a | bytes) & 15u) == 0)
                for (uint64_t o = 0; o < bytes; o += 32768u)
                    prefetch_l2_bulk(reinterpret_cast<const void *>(a + o),
                                     (uint32_t)(bytes - o < 32768u ? bytes - o : 32768u));
        }
        // The unit starts once every task it must follow completed:
        // - the conflicting candidates: bit d - 1 of the checker's mask names
        //   task seq - d (d <= check_w);
        // - with dispatch ahead, every task check_w or more positions back
        //   (what a ring of check_w slots ensures before it inserts a task).
        //   The scheduler inserted this task only once every task a whole ring
        //   span (window) or more back had retired, so the tasks at distance
        //   check_w .. window - 1 remain; those below the launch's first task
        //   finished in earlier launches.
        // A done word shows its task complete (or a later task at the same ring
        // position, which it takes only after the earlier one retired).
        bool ok = true;
        if (watcher) {
            const uint32_t t = seq - d;
            bool needed = d <= P.check_w && ((up >> (d - 1u)) & 1ull);
            if (P.admit && d >= P.check_w && d < P.window)
                needed = needed || (int32_t)(t - P.first[stream]) >= 0;
            ok = !needed || slot_done(dw, t + 1u);
        }
        if (!__syncthreads_and(ok)) {
            uint32_t spins = 0, backoff = 16;
            unsigned long long tw = 0;
            while (true) {
                __nanosleep(backoff);
                if (backoff < 64) backoff <<= 1;
                if (!ok) {
                    ok = slot_done(ld_acquire_u64(&done[(gidx - d) & CM]), seq - d + 1u);
                    if (!ok && (++spins & 7) == 0) {
                        const unsigned long long now = globaltimer_ns();
                        if (tw == 0) tw = now;
                        const bool expired = now - tw > 4ull * P.timeout_ns;
                        if (expired) raise_error(P, (uint32_t)ACS_ERR_TIMEOUT, kSiteWorker);
                        if (expired || stopped(P)) ok = true;   // leave; the run has failed
                    }
                }
                if (__syncthreads_and(ok)) break;
            }
        }
        if (s_hdr.seq != seq || cta >= s_hdr.ncta) {     // self-check: the unit matches its record
            if (threadIdx.x == 0) raise_error(P, (uint32_t)ACS_ERR_INVALID, kSiteWorkerRecord);
            __syncthreads();
            continue;
        }
        if (tracing && threadIdx.x == 0)
            atomicMin(&P.trace[(((size_t)stream << P.log_log2) + (seq & ((1u << P.log_log2) - 1u))) * kTraceFields + 2],
                      globaltimer_ns());
        if (logging && threadIdx.x == 0) {
            const unsigned long long t = atomicAdd(&P.ctl->ticket, 1ull);
            atomicMin(&P.log_start[((size_t)stream << P.log_log2) + (seq & ((1u << P.log_log2) - 1u))], t);
        }
        if (s_hdr.op == ACS_OP_RL_EMIT) body_rl_emit(P, stream, s_hdr, smem);
        else run_body(s_hdr, (int)cta, smem, &P.ctl->stop);
        __syncthreads();
        if (threadIdx.x == 0) {
            // every CTA stamps its end (the task's is the latest) and then
            // takes itself off the done word's CTA count with release
            // semantics: the CTA that reaches zero completes the task, with
            // no round trip and no reset for the slot's next task
            const size_t li = ((size_t)stream << P.log_log2) + (seq & ((1u << P.log_log2) - 1u));
            if (tracing) atomicMax(&P.trace[li * kTraceFields + 3], globaltimer_ns());
            if (logging) atomicMax(&P.log_retire[li], atomicAdd(&P.ctl->ticket, 1ull));
            red_release_add_u64(&P.done[((size_t)stream << P.cap_log2) | (seq & ((1u << P.cap_log2) - 1u))],
                                ~0ull);   // - 1 in the low half
        }
    }
}

// ---- kernels ----------------------------------------------------------------------

__global__ void __launch_bounds__(kBlock, 2) acs_persistent_kernel(const __grid_constant__ KParams P) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (blockIdx.x < P.n_streams) {
        sched_init(P, blockIdx.x, smem);
        __syncthreads();
        const uint32_t warp = threadIdx.x / 32;
        if (warp == 0) scheduler_warp(P, blockIdx.x, smem);
        else if (warp == kBlock / 32 - 1) loader_warp(P, blockIdx.x, smem);
        else if (warp == kBlock / 32 - 2) poller_warp(P, blockIdx.x, smem);
        else if (warp == kBlock / 32 - 3) publisher_warp(P, blockIdx.x, smem);
        else checker_warp(P, blockIdx.x, smem, warp - 1);
    } else {
        worker_loop(P, smem);
    }
    // exit protocol: the last CTA out resets the work ring for the next launch
    // and reports the error word to the host.
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&P.ctl->exit_count, 1u) == gridDim.x - 1u) {
            __threadfence();
            const uint32_t err = atomicAdd(&P.ctl->err, 0u);
            P.ctl->ring_head = atomicAdd(&P.ctl->ring_tail, 0u);
            P.ctl->stop = 0u;
            P.ctl->sched_done = 0u;
            P.ctl->exit_count = 0u;
            __threadfence();
            P.hstatus->err = err;
            P.hstatus->err_info = P.ctl->err_info;
            P.hstatus->launches_done = P.hstatus->launches_done + 1u;
            __threadfence_system();
        }
    }
}

__global__ void acs_init_kernel(unsigned long long *cells, uint32_t ncells, DevCtl *ctl, unsigned long long *done,
                                uint32_t nslots) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t q = i; q < ncells; q += gridDim.x * blockDim.x) cells[q] = q;
    for (uint32_t q = i; q < nslots; q += gridDim.x * blockDim.x) done[q] = 0;
    if (i == 0) {
        ctl->ring_head = 0; ctl->ring_tail = 0; ctl->stop = 0; ctl->sched_done = 0;
        ctl->exit_count = 0; ctl->err = 0; ctl->err_info = 0; ctl->ticket = 0;
    }
}

// One task as a standalone kernel (in-order and graph baselines): the same
// body code the persistent kernel runs.
__global__ void __launch_bounds__(kBlock) acs_body_kernel(const __grid_constant__ TaskHdr h) {
    extern __shared__ __align__(128) uint8_t smem[];
    run_body(h, (int)blockIdx.x, smem, nullptr);
}

}  // namespace acs

// Host-visible launch helpers (defined here so the kernels stay in one TU).
namespace acs {
const void *persistent_kernel_fn() { return (const void *)acs_persistent_kernel; }
const void *body_kernel_fn() { return (const void *)acs_body_kernel; }
cudaError_t launch_init(unsigned long long *cells, uint32_t ncells, DevCtl *ctl, unsigned long long *done,
                        uint32_t nslots, cudaStream_t st) {
    acs_init_kernel<<<148, 256, 0, st>>>(cells, ncells, ctl, done, nslots);
    return cudaGetLastError();
}
}  // namespace acs
