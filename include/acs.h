/*
 * acs.h -- C ABI of the B300 out-of-order task scheduler (libacs.so).
 *
 * Implements the runtime problem of ACS (arXiv 2401.12377): small GPU tasks are
 * submitted in program order together with the byte ranges each reads and
 * writes; dependencies between them are found at run time by testing those
 * ranges for overlap within a sliding scheduling window (Sec. III-C, Alg. 1),
 * and every task is issued as soon as its upstream tasks have retired
 * (ready / pending / executing states, Sec. III-C and Sec. IV-C).
 *
 * Here the window, the dependency test, the state machine and the dispatch all
 * live in one persistent, cooperatively launched CUDA kernel (sm_103a): one
 * scheduler warp per stream keeps the stream's window in shared memory and
 * hands ready tasks' CTAs to resident worker CTAs through a device work ring,
 * so no task costs a host round trip.
 *
 * Conventions for every entry point:
 *   - Return value: ACS_OK (0) or a negative ACS_ERR_* code.
 *   - Errors are sticky: after the first error a context returns it from every
 *     later call except acs_get_stats / acs_get_log / acs_destroy.
 *   - A context belongs to one host thread; calls on one context must not race.
 *   - Pointers inside acs_args are DEVICE addresses of caller-owned memory,
 *     which must stay allocated until acs_sync has returned for the tasks using
 *     it. All other pointer arguments are HOST memory, read or written only
 *     during the call.
 */
#ifndef ACS_H
#define ACS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define ACS_OK              0
#define ACS_ERR_INVALID    (-1)  /* bad argument: window, stream, op, ncta, segment */
#define ACS_ERR_FULL       (-2)  /* stream ring full: acs_flush + acs_sync, then retry */
#define ACS_ERR_TIMEOUT    (-3)  /* a bounded device wait expired (no progress) */
#define ACS_ERR_DEVICE     (-4)  /* a CUDA runtime call failed */
#define ACS_ERR_STOPPED    (-5)  /* the context was stopped */
#define ACS_ERR_ORDER      (-6)  /* task_id not strictly increasing within a stream */
#define ACS_ERR_NOMEM      (-7)  /* host or device allocation failed */
#define ACS_ERR_RANGE      (-8)  /* the stream's position reached 2^31: acs_stream_rebase first */

/* ---- limits ------------------------------------------------------------- */
#define ACS_MAX_WINDOW     64    /* W: slots of the scheduling window per stream */
#define ACS_MAX_SEGS       16    /* read + write segments per task (non-empty ones) */
#define ACS_MAX_NCTA       256   /* CTAs per task */
#define ACS_MAX_STREAMS    256   /* independent streams per context */
#define ACS_BLOCK_THREADS  256   /* threads of every task CTA */

/*
 * A byte range [start, start + size) of device memory that a task reads or
 * writes (the paper's read_segments / write_segments entries, Sec. III-C and
 * Sec. IV-A). size == 0 is dropped (it never conflicts). {0, UINT64_MAX} is
 * "all of memory", the paper's rule for kernels with indirect accesses whose
 * ranges are unknown (Sec. IV-A). Any other range whose end overflows 2^64 is
 * rejected with ACS_ERR_INVALID.
 */
typedef struct acs_segment {
    uint64_t start;
    uint64_t size;
} acs_segment;

#define ACS_WHOLE_MEMORY_START 0ull
#define ACS_WHOLE_MEMORY_SIZE  UINT64_MAX

/* ---- task bodies ---------------------------------------------------------
 * Every task runs one of these bodies on ncta CTAs of ACS_BLOCK_THREADS
 * threads. Arithmetic is fp32 with round-to-nearest and no contraction of
 * multiply-add except where stated, so a task's output does not depend on ncta
 * or on the schedule. */
enum acs_op {
    ACS_OP_NOP = 0,           /* no body; segments as given                     */
    ACS_OP_AXPY = 1,          /* y[i] = a*x[i] + y[i]              acs_axpy_args */
    ACS_OP_SCALE = 2,         /* y[i] = a*x[i]                     acs_axpy_args */
    ACS_OP_ADD = 3,           /* z[i] = x[i] + y[i]                acs_add_args  */
    ACS_OP_GEMV = 4,          /* y = W x, W row-major m x k, fp32 fused-multiply-add
                                 accumulation in a fixed order    acs_gemv_args */
    ACS_OP_BIAS_RELU = 5,     /* t[i] = max(t[i] + b[i], +0)       acs_bias_relu_args */
    ACS_OP_RESID = 6,         /* h[i] = h[i] + (u[i] + b[i])       acs_resid_args */
    ACS_OP_RL_BROADPHASE = 10,/* sphere contacts + islands per env acs_rl_broadphase_args */
    ACS_OP_RL_SOLVE = 11,     /* Gauss-Seidel contact impulses, 1 env acs_rl_solve_args */
    ACS_OP_RL_INTEGRATE = 12, /* semi-implicit Euler + box walls   acs_rl_integrate_args */
    ACS_OP_RL_EMIT = 13,      /* device-side task emission: append the next
                                 simulation step's tasks to this task's own
                                 stream from the island counts   acs_rl_emit_args */
    ACS_OP_WAIT_FLAG = 30,    /* test body: wait until *flag != 0, the stop flag, or
                                 limit_ns elapsed                  acs_wait_args */
    ACS_OP_SLEEP = 31         /* spin ns, then y[0] = y[0]*0.5 + tag (CTA 0)
                                                                   acs_sleep_args */
};

/* Packed launch arguments of one task: op, CTA count and up to 48 bytes of
 * op-specific arguments (one of the acs_*_args structs below, memcpy'd into
 * bytes). Copied by acs_submit*. */
typedef struct acs_args {
    uint16_t op;        /* enum acs_op */
    uint16_t ncta;      /* 1 .. ACS_MAX_NCTA */
    uint32_t reserved;  /* must be 0 */
    uint8_t bytes[48];
} acs_args;

typedef struct { uint64_t x, y; uint32_t n; float a; } acs_axpy_args;
typedef struct { uint64_t x, y, z; uint32_t n; uint32_t pad; } acs_add_args;
typedef struct { uint64_t W, x, y; uint32_t m, k; } acs_gemv_args;
typedef struct { uint64_t t, b; uint32_t n; uint32_t pad; } acs_bias_relu_args;
typedef struct { uint64_t h, u, b; uint32_t n; uint32_t pad; } acs_resid_args;

/* Rigid-sphere workload: 32 spheres per environment.
 *   pos  fp32 [env][32][3]    vel fp32 [env][32][3]    prop fp32 [env][32][2] (radius, 1/mass)
 *   cont contact record per env, ACS_RL_REC_BYTES bytes:
 *        u32 ncontact, u32 nisland, u8 label[32] (smallest sphere index of its
 *        component), u8 root[32] (labels of islands with >= 1 contact, ascending),
 *        u16 pair[496] (i | j << 8, i < j, lexicographic), zero padding.
 *   nisl u32 [env] island count (copy of the record's nisland). */
#define ACS_RL_SPHERES   32
#define ACS_RL_REC_BYTES 1088
typedef struct { uint64_t pos, prop, cont, nisl; uint32_t nenv; uint32_t pad; } acs_rl_broadphase_args;
typedef struct { uint64_t pos, prop, cont, vel; float beta_dt, slop; } acs_rl_solve_args;
typedef struct { uint64_t pos, vel, prop; uint32_t nenv; float dt, gdt, box; } acs_rl_integrate_args;
/* Device-side emission for the rigid-sphere stream. The emit task of step t
 * reads the island counts of step t and appends, in this order: one
 * ACS_OP_RL_SOLVE per environment with islands (ascending, ncta =
 * clamp(islands, 1, 16)), one ACS_OP_RL_INTEGRATE per chunk of step t, and if
 * t + 1 < steps one ACS_OP_RL_BROADPHASE per chunk of step t + 1 followed by
 * the emit task of step t + 1. Appended tasks get task_id = their position in
 * the stream. Chunk CTA counts come from ncta_table[(t * 2 + k) * n_chunks + c]
 * (k = 0 broadphase of step t, k = 1 integrate of step t; bytes, each 1 .. 255:
 * an emit task that finds a 0 among the entries it copies appends nothing and
 * fails the launch with ACS_ERR_INVALID, returned by acs_sync). Segments: reads
 * nisl, the cfg block and the table; writes the 4-byte token (so emit tasks of
 * one stream are ordered). A stream holding an emit task stays open until the
 * last emit task ran: acs_sync returns once every appended task retired. */
typedef struct {
    uint64_t pos, vel, prop, cont;   /* device buffers of all environments */
    float beta_dt, slop, dt, gdt, box;
    uint32_t pad[3];
} acs_rl_emit_cfg;                   /* device memory, read by emit tasks */
typedef struct { uint64_t cfg, nisl, token, ncta_table; uint32_t n_env, step, steps, chunk; } acs_rl_emit_args;
typedef struct { uint64_t flag; uint64_t limit_ns; } acs_wait_args;
typedef struct { uint64_t y; uint64_t ns; float tag; uint32_t pad; } acs_sleep_args;

/* ---- context configuration ----------------------------------------------- */
enum acs_mode {
    ACS_MODE_WINDOW = 0,   /* the method: persistent device scheduler (default) */
    ACS_MODE_INORDER = 1,  /* baseline: one kernel launch per task, one CUDA stream */
    ACS_MODE_GRAPH = 2,    /* baseline: per flush, a CUDA graph of the full DAG */
    ACS_MODE_SW = 3        /* baseline: the paper's software scheduler (Sec. IV-B, Alg. 2):
                              a host-side window of W tasks per stream checked with the
                              same overlap test, completed tasks leave the window out of
                              order; sw_threads host threads each launch one ready task
                              at a time into their own CUDA stream and wait for it with
                              cudaStreamSynchronize. acs_flush returns when every
                              flushed task completed; kernel_ms then holds the flushes'
                              host wall time */
};

enum acs_flags {
    ACS_FLAG_LOG = 1,      /* record per-task upstream-candidate masks and
                              start / retire tickets (window mode) */
    ACS_FLAG_TIMING = 2,   /* time each device launch with CUDA events */
    ACS_FLAG_TRACE = 4     /* record per-task timestamps (window mode, see acs_get_trace) */
};

typedef struct acs_config {
    uint32_t mode;          /* enum acs_mode */
    uint32_t n_streams;     /* independent task streams, 1 .. ACS_MAX_STREAMS (0 -> 1) */
    uint32_t cta_slots;     /* worker CTAs of the persistent kernel (0 -> every
                               co-resident CTA not used by a scheduler) */
    uint32_t capacity;      /* ring entries per stream, rounded up to a power of
                               two >= 64 (0 -> 8192); bounds tasks in flight */
    uint32_t log_capacity;  /* log entries per stream (0 -> capacity) */
    uint32_t flags;         /* enum acs_flags */
    uint64_t timeout_ns;    /* bound on every device wait without progress (0 -> 5 s) */
    void *cuda_stream;      /* cudaStream_t for all device work (NULL -> a
                               non-blocking stream owned by the context) */
    int32_t device;         /* CUDA device ordinal (-1 -> current) */
    uint32_t poll_ns;       /* longest sleep of an idle worker between polls of
                               the work ring (0 -> 128 ns; a tuning knob) */
    uint32_t ctas_per_sm;   /* cap on co-resident persistent CTAs per SM, enforced
                               through their shared-memory reservation (0 -> as
                               many as registers allow; a tuning knob) */
    uint32_t idle_limit_ms; /* resident launches (acs_start): the kernel leaves by
                               itself after this long idle without any host call
                               (0 -> 10 000 ms), so it always terminates */
    uint32_t sw_threads;    /* ACS_MODE_SW: host threads, one CUDA stream each (0 -> 8) */
    uint32_t span;          /* window mode: ring span M, window <= M <= 64 (0 -> M = window).
                               M = window is the in-order ring: task j enters once every
                               task <= j - W retired, and its candidates are tasks
                               j - W + 1 .. j - 1. M > window is the free-slot variant
                               (Sec. IV-B/IV-C): at most `window` tasks are inserted and
                               not retired, a retired task frees its place at once (out
                               of order), and candidates are the unretired tasks among
                               j - M + 1 .. j - 1 (the M bound of the upstream load
                               module); logs then give the masks over M - 1 predecessors */
    uint32_t lookahead;     /* window mode, with span = 0: dispatch tasks ahead of the window.
                               With L > 0 the scheduler inserts task j (checks it against its
                               window - 1 predecessors, as in the ring, and publishes its
                               CTAs to the work ring) once every task <= j - window - L has
                               retired; j's worker CTAs then wait, besides its conflicting
                               predecessors, until every task <= j - window has completed
                               before they run it (read from the done words of the L tasks
                               in between: every task <= j - window - L had retired when j
                               was inserted). What runs, the masks (logs give the same
                               window DAG as L = 0) and legality are those of the ring;
                               only the dispatch (claiming a task's CTAs, reading its
                               descriptor) overlaps the window's wait. window + L <= 64.
                               0 -> off; ACS_LOOKAHEAD_AUTO (acs_config_default) ->
                               L = min(2 window, 64 - window) for one stream, 0 with several
                               streams or a span (CTAs that wait for their stream's window
                               would hold workers the other streams could use). */
    uint32_t reserved[1];   /* must be 0 */
} acs_config;

#define ACS_LOOKAHEAD_AUTO 0xFFFFFFFFu

typedef struct acs_stats {
    uint64_t tasks_submitted;
    uint64_t tasks_flushed;
    uint64_t launches;          /* persistent launches (window) / kernels (in-order) / graphs */
    uint64_t seg_bytes;         /* sum of read + write segment sizes of flushed tasks,
                                   whole-memory segments excluded */
    double kernel_ms;           /* ACS_FLAG_TIMING: device time of the launches, summed */
    double graph_build_ms;      /* graph mode: host time to build graphs (incl. DAG) */
    double graph_instantiate_ms;/* graph mode: host time in cudaGraphInstantiate */
    uint64_t graph_edges;       /* graph mode: edges after transitive reduction */
    uint64_t sched_cycles;      /* window mode: SM clock cycles the scheduler warps ran */
    uint64_t sched_busy_cycles; /* ... of which spent inserting, retiring, dispatching */
    uint64_t sched_inserts;     /* tasks inserted into windows */
    uint64_t sched_iterations;  /* scheduler loop iterations */
    uint64_t sched_phase_cycles[8]; /* ACS_FLAG_TRACE: scheduler-warp cycles by loop phase:
                                   [0] loop top, [1] slot-state updates (with nothing to
                                   insert: the room check), [2] retirement and in-order
                                   release, [3] insertion (room, checked tasks, upstream
                                   masks, work-ring offsets), [4] unused, [5] log and trace
                                   entries, [6] hand-off to the publisher warp, [7] progress
                                   and idle bookkeeping */
    uint64_t tasks_emitted;     /* tasks appended on the device by emit tasks */
    uint64_t device_seg_bytes;  /* window mode: segment bytes of every task, submitted by the
                                   host (seg_bytes) or appended on the device by emit tasks */
    uint64_t check_cycles;      /* ACS_FLAG_TRACE: SM cycles the checker warps spent testing */
    uint64_t starved_iters;     /* ACS_FLAG_TRACE: scheduler iterations with a free slot but no
                                   checked task */
    uint32_t cta_slots;         /* worker CTAs of the persistent kernel */
    uint32_t grid;              /* total CTAs of the persistent kernel */
} acs_stats;

typedef struct acs_ctx acs_ctx;

/* Fill *cfg with the defaults (all zero fields mean "default"). */
void acs_config_default(acs_config *cfg);

/*
 * Create a context with a scheduling window of `window` slots per stream
 * (Sec. III-C: a fixed-size window of N kernels filled in FIFO order; the paper
 * evaluates N = 16 and 32, Sec. VI-D). 1 <= window <= ACS_MAX_WINDOW. cfg may
 * be NULL. Allocates the context's device rings and pinned host rings; frees
 * them in acs_destroy. *out is set only on success.
 * Errors: ACS_ERR_INVALID (window, n_streams, mode, reserved fields),
 * ACS_ERR_DEVICE, ACS_ERR_NOMEM.
 */
int acs_init(acs_ctx **out, uint32_t window, const acs_config *cfg);

/*
 * Resolve the read and write segments of a task from its packed arguments:
 * the get_addresses wrapper of Sec. IV-A (Fig. get_addresses: a matrix product
 * reads its two inputs, m*n and n*k elements, and writes its m*k output). The
 * result is what acs_submit_ops submits. reads / writes must hold
 * ACS_MAX_SEGS entries; *n_reads / *n_writes receive the counts.
 * Errors: ACS_ERR_INVALID (unknown op, sizes overflowing 64 bits).
 */
int acs_get_addresses(const acs_args *args, acs_segment *reads, uint32_t *n_reads,
                      acs_segment *writes, uint32_t *n_writes);

/*
 * Append one task to stream 0 in program order (Sec. III-D: invoked kernels
 * and their segments enter the input FIFO). Copies args and both segment
 * arrays. task_id must be strictly greater than the previous task_id of the
 * stream (it names the task in logs). At most ACS_MAX_SEGS non-empty segments.
 * Nothing runs until acs_flush.
 * Errors: ACS_ERR_INVALID (also: an emit task outside window mode, or a stream
 * whose flushed emit tasks were not yet synced), ACS_ERR_ORDER, ACS_ERR_FULL
 * (more than capacity - window + 1 tasks since the last acs_sync).
 */
int acs_submit(acs_ctx *ctx, uint32_t task_id, const acs_args *args,
               const acs_segment *reads, uint32_t n_reads,
               const acs_segment *writes, uint32_t n_writes);

/* acs_submit on stream `stream` (0 <= stream < n_streams). Streams are
 * independent programs: no dependency is ever detected across streams. */
int acs_submit_stream(acs_ctx *ctx, uint32_t stream, uint32_t task_id, const acs_args *args,
                      const acs_segment *reads, uint32_t n_reads,
                      const acs_segment *writes, uint32_t n_writes);

/* Submit n tasks to `stream`, each with the segments acs_get_addresses
 * derives from its args. task_ids and args are arrays of n entries. Stops at
 * the first failing task and returns its error (earlier tasks stay submitted). */
int acs_submit_ops(acs_ctx *ctx, uint32_t stream, uint32_t n, const uint32_t *task_ids,
                   const acs_args *args);

/*
 * Make every task submitted since the last flush runnable and start running it,
 * without blocking the host. Window mode: copies the new descriptors into the
 * device rings and launches the persistent scheduler kernel (cooperative
 * launch) over them; windows continue across flushes, so dependency detection
 * is identical however a stream is split into flushes. In-order mode: launches
 * one kernel per task. Graph mode: builds, instantiates and launches a CUDA
 * graph of the flushed tasks' full DAG.
 * Errors: ACS_ERR_DEVICE (launch failed, e.g. the grid cannot be co-resident).
 */
int acs_flush(acs_ctx *ctx);

/*
 * Block until every flushed task retired (all CTAs finished, their global
 * writes visible). Returns the context's first error, e.g. ACS_ERR_TIMEOUT if
 * a device wait made no progress for timeout_ns.
 */
int acs_sync(acs_ctx *ctx);

/*
 * Copy the window-mode log of tasks [first, first + n) of `stream` (positions in
 * submission order) into host arrays of n entries each (any may be NULL):
 *   masks[i]  upstream candidates of the task at insertion: bit b set iff the
 *             task in window slot b (the unique earlier task t with
 *             t mod window == b among the window - 1 previous tasks)
 *             conflicts with it, whether or not that task had already retired;
 *   start[i]  smallest ticket drawn by the task's CTAs when they began;
 *   retire[i] ticket drawn when its last CTA finished.
 * Tickets come from one device counter. Needs ACS_FLAG_LOG and a completed
 * acs_sync; the range must lie within the last log_capacity tasks.
 * Errors: ACS_ERR_INVALID.
 */
int acs_get_log(acs_ctx *ctx, uint32_t stream, uint64_t first, uint32_t n,
                uint64_t *masks, uint64_t *start, uint64_t *retire);

/*
 * Copy the window-mode timestamps (device %globaltimer, ns) of tasks [first,
 * first + n) of `stream` into t[5*n]: for task i, t[5i+0] insertion into the
 * window, t[5i+1] publication of its work units to the worker CTAs, t[5i+2]
 * start of its first CTA, t[5i+3] end of its last CTA, t[5i+4] retirement
 * seen by the scheduler. Needs ACS_FLAG_TRACE and a completed acs_sync; same
 * range rules as acs_get_log. Errors: ACS_ERR_INVALID.
 */
int acs_get_trace(acs_ctx *ctx, uint32_t stream, uint64_t first, uint32_t n, uint64_t *t);

/* Position of `stream`: the number of tasks it has had so far (host submitted
 * plus device appended, the latter known after acs_sync); the next task's seq.
 * Errors: ACS_ERR_INVALID. */
int acs_stream_tail(acs_ctx *ctx, uint32_t stream, uint32_t *tail);

/* Restarts an idle stream's positions: its next task gets seq `pos` (normally
 * 0). Positions are 32-bit and a stream takes host-submitted tasks only below
 * ACS_MAX_POSITION (2^31; ACS_ERR_RANGE there), which keeps every comparison
 * of positions on the device, and the seq + 1 words that mark a task done or
 * checked, clear of the 2^32 wrap; a long-lived stream calls this at an idle
 * point. Idle: everything submitted was flushed and synced (acs_sync), no
 * emitter chain is alive, no resident launch runs (acs_stop first). After it
 * the tasks before `pos` count as complete and are no candidates; the logs and
 * traces of the earlier tasks are no longer readable and task ids may start
 * over. pos < ACS_MAX_POSITION.
 * Errors: ACS_ERR_INVALID (bad stream or pos, not idle, resident launch). */
#define ACS_MAX_POSITION 0x80000000u
int acs_stream_rebase(acs_ctx *ctx, uint32_t stream, uint32_t pos);

/*
 * Resident (serving) launches. acs_start launches the persistent scheduler
 * kernel and leaves it on the device: every stream's window stays in its
 * scheduler CTA between flushes, and new work reaches a running kernel with
 * no launch. While resident:
 *   - acs_submit / acs_submit_stream / acs_submit_ops stage descriptors in the
 *     context's pinned host ring as before (ACS_ERR_FULL when the ring lacks
 *     room for the task plus the window behind it: call acs_progress or
 *     acs_sync, then retry);
 *   - acs_flush copies each stream's new descriptors into its device ring
 *     with the copy engine (a stream of the context's own, beside the
 *     kernel) and publishes the stream's new end, with one release store into
 *     mapped host memory, once that copy has completed: at once if it has,
 *     else from the next acs_flush, acs_progress or acs_sync. The kernel's
 *     loader warp polls the published ends and schedules the new tasks;
 *   - acs_progress reports, without blocking, per stream: head (tasks below
 *     it were released, refreshed every 16 tasks and when idle) and idle_at
 *     (the stream was last seen idle with this end: all tasks below it
 *     retired and no emitter chain alive). Work published up to end E of a
 *     stream is complete once idle_at >= E (mod 2^32); for a stream whose
 *     flushed tasks hold emit tasks the tail (acs_stream_tail) then becomes
 *     idle_at. The task outputs are visible to the host and to other CUDA
 *     streams once idle_at covers them. A stream with emitter chains in
 *     flight accepts no new tasks (ACS_ERR_INVALID) until that point;
 *   - acs_sync waits on the host until every published task retired (bounded
 *     by timeout_ns without progress) and leaves the kernel running.
 * acs_start needs window mode, no launch in flight (acs_sync first), and
 * publishes tasks already staged. acs_stop publishes what is staged, waits
 * until all of it retired, and lets the kernel end (when nothing moves for
 * timeout_ns it raises the device stop flag instead and returns
 * ACS_ERR_TIMEOUT); acs_destroy stops a resident context first. The kernel
 * also ends by itself after idle_limit_ms without any host call (then calls
 * return ACS_ERR_STOPPED). Errors: ACS_ERR_INVALID, ACS_ERR_DEVICE, the
 * device's first error.
 */
int acs_start(acs_ctx *ctx);
int acs_progress(acs_ctx *ctx, uint32_t *head, uint32_t *idle_at);   /* arrays of n_streams, either NULL */
int acs_stop(acs_ctx *ctx);

/*
 * acs_abort -- stop the context's work from the host (window mode).
 *
 * Raises the device stop word of the context: every wait of a running
 * persistent launch (scheduler, workers, task bodies that poll it) ends, and
 * the launch exits without running the tasks it had not started. The context's
 * error becomes ACS_ERR_STOPPED (sticky): acs_sync returns it once the launch
 * has ended, and acs_submit / acs_flush return it from then on; destroy the
 * context and create a new one to run more work. Other CUDA work and other
 * contexts are unaffected. The stop word is written by a copy on a
 * non-blocking stream of the call's own, so the call never waits behind the
 * running kernel; it returns once the word is written. Unlike every other
 * entry point it may be called from a host thread other than the context's
 * owner (e.g. a watchdog while the owner blocks in acs_sync), and with no
 * launch in flight. Errors: ACS_ERR_INVALID (NULL, or a mode other than
 * ACS_MODE_WINDOW), ACS_ERR_DEVICE (the copy failed).
 */
int acs_abort(acs_ctx *ctx);

/* Copy the context's counters into *out (after acs_sync for device figures). */
int acs_get_stats(acs_ctx *ctx, acs_stats *out);

/* Graph mode: launch the most recently instantiated graph again (timing of a
 * prebuilt graph; re-runs its tasks). Errors: ACS_ERR_INVALID if none. */
int acs_graph_replay(acs_ctx *ctx);

/*
 * acs_run_noalloc -- run one stream of tasks without allocating anything.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they run their tasks, e.g. code embedded
 * in a framework that owns the device memory budget and forbids side
 * allocations, or paths that cannot absorb an allocator's latency or failure.
 * It runs the same persistent scheduler kernel as acs_flush (window of
 * `window` slots, one stream, tasks in program order with the segments
 * acs_get_addresses derives), but every byte of scratch comes from one
 * fixed-size array in the library's device memory that every GPU loading the
 * library holds until exit (under 2 MiB).
 *
 *   window      1 .. ACS_MAX_WINDOW
 *   n           number of tasks, 0 .. ACS_NOALLOC_MAX_TASKS (more: ACS_ERR_INVALID)
 *   task_ids    n strictly increasing ids (host memory)
 *   args        n packed tasks (host memory); their pointers name the caller's
 *               device buffers, which are the inputs and outputs. Every op but
 *               ACS_OP_RL_EMIT (which needs a context's emitter state).
 *   cuda_stream cudaStream_t to run on (NULL: the legacy default stream)
 *
 * Every task is checked on the host before anything reaches the device:
 * ACS_ERR_INVALID for an unknown op, an emit task, ncta outside
 * 1 .. ACS_MAX_NCTA, a nonzero reserved word or a bad segment; ACS_ERR_ORDER
 * for ids that do not increase; ACS_ERR_INVALID, before the stream is used,
 * if `cuda_stream` is in capture mode. The call then blocks until the tasks
 * retired (it synchronizes `cuda_stream` and copies the error word back) and
 * returns ACS_OK or the first device error (ACS_ERR_TIMEOUT, ACS_ERR_INVALID from a device self-check,
 * ACS_ERR_DEVICE). The first call on a device resolves the array's device
 * address and sets the kernel's attributes with that device current. Calls
 * share the array (each re-initialises what must start at zero); calls whose
 * device work overlaps race on it and must not be made. Not thread-safe. Calls
 * no cudaMalloc, cudaFree or other allocating routine.
 */
#define ACS_NOALLOC_MAX_TASKS 4096
int acs_run_noalloc(uint32_t window, uint32_t n, const uint32_t *task_ids, const acs_args *args,
                    void *cuda_stream);

/* The context's sticky error (ACS_OK if none). */
int acs_error(const acs_ctx *ctx);

/* Static description of a status code. */
const char *acs_strerror(int code);

/* Synchronize, then free everything the context allocated. NULL is a no-op. */
void acs_destroy(acs_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* ACS_H */
