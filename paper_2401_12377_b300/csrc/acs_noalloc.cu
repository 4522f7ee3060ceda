// acs_run_noalloc: the window scheduler for callers that must not allocate.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they want to run a batch of tasks: code inside another framework that
// owns the device memory budget and forbids side allocations, or
// latency-critical paths that cannot absorb an allocator's cost or failure.
// For them this entry point runs one stream of tasks through the same
// persistent scheduler kernel as acs_flush, but takes every byte of scratch
// (descriptor ring, work ring, counters, status) from one file-scope device
// array that exists for as long as the library is loaded. The caller provides
// only the tasks; their data buffers stay the caller's.
//
// The call blocks: it synchronizes the caller's stream and reads the error
// word back. A stream in capture mode is refused (ACS_ERR_INVALID) before the
// call uses it.
//
// The array is a host-side symbol: its device address is obtained once per
// device with cudaGetSymbolAddress (with that device current) on the first
// call on that device. Every call shares the array and finds the previous
// call's contents; each call re-initialises what must start from zero. Calls
// whose device work overlaps (e.g. on two streams) race on the array and must
// not be issued.
#include <cuda_runtime.h>

#include <cstring>

#include "acs_internal.h"

namespace acs {
const void *persistent_kernel_fn();
cudaError_t launch_init(unsigned long long *cells, uint32_t ncells, DevCtl *ctl, unsigned long long *done,
                        uint32_t nslots, cudaStream_t st);
}  // namespace acs

using namespace acs;

namespace {

constexpr uint32_t kNoAllocCapLog2 = 12;                 // descriptor ring: ACS_NOALLOC_MAX_TASKS
// work-ring cells: up to (2W - 1) tasks of ACS_MAX_NCTA units each can be in
// flight (W inserted, W - 1 more checked and waiting), rounded up to a power of two
constexpr uint32_t pow2_at_least(uint32_t x) { return x <= 1u ? 1u : 2u * pow2_at_least((x + 1u) / 2u); }
constexpr uint32_t kNoAllocCells = pow2_at_least((2u * ACS_MAX_WINDOW - 1u) * ACS_MAX_NCTA);
static_assert((kNoAllocCells & (kNoAllocCells - 1u)) == 0 && kNoAllocCells >= (2u * ACS_MAX_WINDOW - 1u) * ACS_MAX_NCTA,
              "work ring holds every unit that can be in flight");
constexpr size_t kAlign = 256;

constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// byte offsets of the parts of the scratch array
constexpr size_t kOffRing = 0;
constexpr size_t kOffCells = kOffRing + up(sizeof(TaskRec) * ACS_NOALLOC_MAX_TASKS);
constexpr size_t kOffAux = kOffCells + up(sizeof(unsigned long long) * kNoAllocCells);
constexpr size_t kOffCtl = kOffAux + up(sizeof(TaskAux) * ACS_NOALLOC_MAX_TASKS);
constexpr size_t kOffDone = kOffCtl + up(sizeof(DevCtl));
constexpr size_t kOffLog = kOffDone + up(sizeof(unsigned long long) * ACS_NOALLOC_MAX_TASKS);   // 3 x 1 entry
constexpr size_t kOffTrace = kOffLog + up(3 * sizeof(unsigned long long));
constexpr size_t kOffStats = kOffTrace + up(kTraceFields * sizeof(unsigned long long));
constexpr size_t kOffStatus = kOffStats + up(sizeof(SchedStats));
constexpr size_t kScratchBytes = kOffStatus + up(sizeof(HostStatus));
static_assert(kScratchBytes < (2u << 20), "scratch stays below 2 MiB");

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of acs_noalloc_scratch
    uint32_t grid = 0;
};

DeviceSetup g_setup[kMaxDevices];
TaskRec g_stage[ACS_NOALLOC_MAX_TASKS];   // host staging of descriptors (static, not heap)

}  // namespace

// The scratch itself: one array per loaded library and device.
static __device__ __align__(256) unsigned char acs_noalloc_scratch[kScratchBytes];

namespace {

int setup_device(int dev, DeviceSetup &d) {
    if (d.ready) return ACS_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, acs_noalloc_scratch) != cudaSuccess || !p) return ACS_ERR_DEVICE;
    const void *kfn = persistent_kernel_fn();
    // the largest dynamic shared memory any window needs (only ever raised)
    const uint32_t smem_max = dyn_smem_bytes(kMaxWindow);
    if (raise_kernel_smem_limit(smem_max) != cudaSuccess) return ACS_ERR_DEVICE;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBlock, smem_max) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
        return ACS_ERR_DEVICE;
    d.scratch = static_cast<unsigned char *>(p);
    d.grid = (uint32_t)(per_sm * sms);
    d.ready = true;
    return ACS_OK;
}

bool segs_to_rec(const acs_segment *s, uint32_t n, bool write, TaskRec &r, uint32_t &cnt, uint16_t &wmask) {
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t a = s[i].start, z = s[i].size;
        if (z == 0) continue;
        Seg g;
        if (a == ACS_WHOLE_MEMORY_START && z == ACS_WHOLE_MEMORY_SIZE) {
            g.start = 0;
            g.last = UINT64_MAX;
        } else {
            if (a != 0 && z - 1 > UINT64_MAX - a) return false;
            g.start = a;
            g.last = a + (z - 1);
        }
        if (cnt >= (uint32_t)kMaxSegs) return false;
        if (write) wmask |= (uint16_t)(1u << cnt);
        r.seg[cnt++] = g;
    }
    return true;
}

}  // namespace

extern "C" int acs_run_noalloc(uint32_t window, uint32_t n, const uint32_t *task_ids, const acs_args *args,
                               void *cuda_stream) {
    if (window < 1 || window > (uint32_t)kMaxWindow) return ACS_ERR_INVALID;
    if (n > ACS_NOALLOC_MAX_TASKS) return ACS_ERR_INVALID;   // beyond the scratch array's capacity
    if (n && (!task_ids || !args)) return ACS_ERR_INVALID;
    if (n == 0) return ACS_OK;

    // descriptors (the same layout acs_submit writes), checked as acs_submit
    // does, on the host before anything reaches the device. Emit tasks need a
    // context's per-stream emitter words, which this entry point does not
    // have: they are refused.
    for (uint32_t i = 0; i < n; ++i) {
        const acs_args &a = args[i];
        if (a.ncta < 1 || a.ncta > ACS_MAX_NCTA || a.reserved || a.op == ACS_OP_RL_EMIT) return ACS_ERR_INVALID;
        if (i && task_ids[i] <= task_ids[i - 1]) return ACS_ERR_ORDER;
        acs_segment rd[ACS_MAX_SEGS], wr[ACS_MAX_SEGS];
        uint32_t nr = 0, nw = 0;
        if (acs_get_addresses(&a, rd, &nr, wr, &nw) != ACS_OK) return ACS_ERR_INVALID;   // unknown op too
        TaskRec &r = g_stage[i];
        std::memset(&r, 0, sizeof r);
        uint32_t cnt = 0;
        uint16_t wmask = 0;
        if (!segs_to_rec(rd, nr, false, r, cnt, wmask) || !segs_to_rec(wr, nw, true, r, cnt, wmask))
            return ACS_ERR_INVALID;
        r.task_id = task_ids[i];
        r.op = a.op;
        r.ncta = a.ncta;
        r.wmask = wmask;
        r.nseg = (uint8_t)cnt;
        fold_reads(r);
        r.seq = i;
        std::memcpy(r.args, a.bytes, sizeof r.args);
    }

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the call synchronizes and copies back: a stream in capture mode is refused
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return ACS_ERR_DEVICE;
    if (cap != cudaStreamCaptureStatusNone) return ACS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ACS_ERR_DEVICE;
    DeviceSetup &d = g_setup[dev];
    int rc = setup_device(dev, d);
    if (rc) return rc;

    unsigned char *base = d.scratch;
    TaskRec *ring = reinterpret_cast<TaskRec *>(base + kOffRing);
    unsigned long long *cells = reinterpret_cast<unsigned long long *>(base + kOffCells);
    TaskAux *aux = reinterpret_cast<TaskAux *>(base + kOffAux);
    DevCtl *ctl = reinterpret_cast<DevCtl *>(base + kOffCtl);
    unsigned long long *done = reinterpret_cast<unsigned long long *>(base + kOffDone);
    unsigned long long *logs = reinterpret_cast<unsigned long long *>(base + kOffLog);
    unsigned long long *trace = reinterpret_cast<unsigned long long *>(base + kOffTrace);
    SchedStats *stats = reinterpret_cast<SchedStats *>(base + kOffStats);
    HostStatus *status = reinterpret_cast<HostStatus *>(base + kOffStatus);

    // what must start from zero: ring cells, counters, done words, status
    if (launch_init(cells, kNoAllocCells, ctl, done, ACS_NOALLOC_MAX_TASKS, st) != cudaSuccess) return ACS_ERR_DEVICE;
    if (cudaMemsetAsync(stats, 0, sizeof(SchedStats), st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(HostStatus), st) != cudaSuccess ||
        cudaMemcpyAsync(ring, g_stage, (size_t)n * sizeof(TaskRec), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ACS_ERR_DEVICE;

    KParams P;
    std::memset(&P, 0, sizeof P);
    P.recs = ring;
    P.ctl = ctl;
    P.cells = cells;
    P.taskaux = aux;
    P.done = done;
    P.log_mask = logs;
    P.log_start = logs + 1;
    P.log_retire = logs + 2;
    P.sched_stats = stats;
    P.trace = trace;
    P.hstatus = status;
    P.timeout_ns = 5000000000ull;
    P.cap_log2 = kNoAllocCapLog2;
    P.log_log2 = 0;
    P.cell_mask = kNoAllocCells - 1;
    P.window = window;
    P.active_limit = window;
    P.check_w = window;   // the ring: candidates over window - 1, no dispatch ahead (admit 0)
    P.n_streams = 1;
    P.flags = 0;
    P.sched_smem = sched_smem_bytes(window);
    P.poll_ns = 128;
    P.first[0] = 0;
    P.end[0] = n;
    // The kernel's shared-memory limit is per-function state every context
    // shares and only raises; make sure it covers this launch.
    const void *kfn = persistent_kernel_fn();
    const uint32_t smem = dyn_smem_bytes(kMaxWindow);
    if (raise_kernel_smem_limit(smem) != cudaSuccess) return ACS_ERR_DEVICE;
    void *kargs[] = {&P};
    if (cudaLaunchCooperativeKernel(kfn, dim3(d.grid), dim3(kBlock), kargs, smem, st) != cudaSuccess)
        return ACS_ERR_DEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACS_ERR_DEVICE;
    uint32_t err = 0;
    if (cudaMemcpy(&err, &ctl->err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess) return ACS_ERR_DEVICE;
    return (int)(int32_t)err;
}
