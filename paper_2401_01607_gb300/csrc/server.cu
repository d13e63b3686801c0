// server.cu -- continuous batching of many independent streams (tc_server_*).
//
// Real-time use of the taches-algorithm (Sec. 5.1 and Sec. 6: low-latency
// output, multichannel use, IRs that change while running) with many
// audio streams at once. Each stream has its own IR length, block size and IR
// versions. A step collects the queued blocks of every stream (up to kMerge
// consecutive blocks of a stream become one work item) and runs them all as
// one batch:
//   one host->device copy of the packed input and work list, one ingest
//   kernel into the streams' history rows (with any row compactions), one K1
//   work-list launch (one item per stream), one push of each shared-IR group
//   on the group's own CUDA stream (K2 in the BF16 modes, beside the gather;
//   ordered by events), one device->host copy of the packed output.
// The worker thread (tc_server_start) keeps two steps in flight: while the
// GPU runs step k, the host collects and launches step k+1 (its own pinned
// buffers; device buffers are shared because one CUDA stream orders them).
// Blocks submitted, or released by a live source, while a step is on the GPU
// join the next step. Streams are admitted while their device state fits the
// memory budget (TC_ENOMEM otherwise) and release it when removed.
//
// Threads: submit/poll take only the queue mutex and never wait for the GPU;
// add/set_ir upload on their own CUDA stream and take the state mutex only
// briefly; steps take the state mutex while packing and delivering.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/taches.h"
#include "tc_internal.h"

namespace {

constexpr int kMaxVer = 16;
constexpr int kMerge = 8;  // consecutive blocks of one stream merged into one work item
constexpr size_t kLogSteps = 1 << 16;
constexpr int kTuneTries = 2;
constexpr int kTuneWorkBins = 48, kTuneLBins = 24;
// Chunk-tasks per tile stay within K1's pairwise stack with the smallest chunk.
constexpr size_t kMaxL = (size_t)tc::K1_MAX_CHUNK_TASKS * 32 * tc::K1_SEG - 8;

struct DevTable {
    long long vstart[kMaxVer];
    int vslot[kMaxVer];
    int nver;
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

long long rup(long long a, long long m) { return (a + m - 1) / m * m; }
long long fl8(long long a) { return a >= 0 ? (a & ~7LL) : -(((-a) + 7) & ~7LL); }

struct Block {
    std::vector<float> own;  // copied input (submit, flush tail)
    const float *src;        // or input read in place from a live source
    long long n;
    double t_submit;  // ready time of the block (latency is measured from it)
    bool tail;        // zero input of the flush: output goes to the tail buffer
    const float *data() const { return src ? src : own.data(); }
};

struct OutBlock {
    std::vector<float> y;
    double t_submit;
    double t_done;
};

struct SStream {
    uint64_t id = 0;
    long long L = 0, block = 0, Lpad = 0, keep = 0, cap = 0, base = 0;
    long long pos = 0;       // input samples launched (history written up to here)
    long long pos_done = 0;  // input samples whose outputs are on the host
    long long stagger = 0;   // early-compaction offset in [0, keep / 2)
    int inflight = 0;        // work items launched, not yet delivered (queue mutex)
    int nslots = 3;
    bool ended = false;   // a short block was submitted: input is over
    bool flushed = false;
    long long x_end = -1;  // once flushed: input samples before the tail (later samples are zero)
    bool discard = false;  // keep no output blocks (latency is still recorded)
    // Group (tc_server_add_group): `channels` rows sharing one IR. Blocks hold
    // [channels][n] samples; the group stream of the C ABI (K2 on the tensor
    // cores in the BF16 modes, K1 in FP32) runs them after the step's K1 work
    // list. hist, ir and d_vt stay unused.
    long long channels = 1;
    int kind = 0;  // latency-log tag: 0 a plain stream (FP32 gather), 1 + precision for a group
    tc_stream *grp = nullptr;
    cudaEvent_t gdone = nullptr;  // the group's push of the current step is done
    std::mutex gmu;           // the group stream: worker pushes vs IR uploads
    long long tail_fill = 0;  // flush tail samples delivered so far (per row)
    size_t arena_off = 0, arena_len = 0;  // the stream's range of the server's arena (len 0: pool memory)
    float *hist = nullptr;       // [cap]
    float *ir = nullptr;         // [nslots][4][Lpad]
    DevTable *d_vt = nullptr;
    struct Ver {
        long long start;
        int slot;
    };
    std::vector<Ver> vt;
    std::vector<char> slot_used;
    bool vt_dirty = true;
    size_t bytes = 0;            // device footprint
    std::deque<Block> pending;   // guarded by the queue mutex
    bool in_ready = false;       // in the server's ready queue (queue mutex): pending is not empty
    std::deque<OutBlock> done;   // guarded by the queue mutex
    std::vector<float> tail_out; // output of the flush's zero blocks

    // Live input source (tc_server_attach_source): x[0, src_n) arriving at
    // src_fs samples/s from clock time src_t0; block b is released at its
    // ready time src_t0 + min((b + 1) * block, src_n) / src_fs.
    const float *src = nullptr;
    long long src_n = 0, src_next = 0;
    double src_t0 = 0.0, src_fs = 0.0;
    double src_ready(long long b) const
    {
        return src_t0 + (double)std::min((b + 1) * block, src_n) / src_fs;
    }
};

}  // namespace

// Device memory reserved by tc_server_reserve: one allocation that stream
// states are carved from by first fit, so that admitting a stream never maps
// device memory while steps run. A removed stream's range is reused only once
// an event recorded after the steps that read it has completed.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length, coalesced
    struct Freed {
        cudaEvent_t ev;
        size_t off, len;
    };
    std::deque<Freed> freed;          // waiting for the steps in flight
    std::vector<cudaEvent_t> spare;   // events to reuse
};

struct tc_server {
    size_t budget = 0, used = 0;
    Arena arena;
    std::mutex mu_arena;  // the arena's lists (add on the admin path, remove on the caller's)
    size_t max_step_samples = 0;
    int device = 0;
    cudaStream_t cs = nullptr;     // steps; frees of removed streams
    cudaStream_t admin = nullptr;  // allocations and IR uploads of add / set_ir_at
    cudaMemPool_t pool = nullptr;  // stream-ordered device memory of the streams
    std::mutex mu_admin;  // admin stream and IR staging (add / set_ir_at serialise on it)
    std::mutex mu_state;  // host state the steps read (positions, versions, budget)
    std::mutex mu_queue;  // pending input / finished output queues
    std::condition_variable cv;
    std::unordered_map<uint64_t, std::unique_ptr<SStream>> streams;  // O(1) lookups per released block
    uint64_t next_id = 1;
    size_t npending = 0;  // blocks queued over all streams (queue mutex)
    // Streams with queued blocks, in the order they became ready (queue
    // mutex). A step visits only these, not every admitted stream, and a
    // stream whose blocks did not all fit goes back to the end (round robin).
    std::deque<SStream *> ready;
    // Live sources by next ready time (queue mutex).
    std::priority_queue<std::pair<double, uint64_t>, std::vector<std::pair<double, uint64_t>>,
                        std::greater<std::pair<double, uint64_t>>>
        src_heap;

    // Step staging, one set per step in flight. Input side: a pinned buffer
    // laid out per step as [K1 items][CTA offsets][ingest table][history
    // pointers][packed input] (16-byte aligned regions), copied with one
    // host-to-device copy into d_stage. Output side: [error word, padded to
    // 16 bytes][packed output], copied back with one device-to-host copy.
    struct Item {
        SStream *s;
        uint32_t first, count;  // the item's blocks: StepBuf::blocks[first, first + count)
        long long off, n;       // packed input / output offset (floats); samples per row
    };
    struct StepBuf {
        char *pin_stage = nullptr;
        size_t items_cap = 0;
        float *pin_out = nullptr;  // [4 + max_step_samples]
        DevTable *pin_tables = nullptr;
        cudaEvent_t done = nullptr;
        cudaEvent_t in_ready = nullptr;  // the step's packed input is on the device (groups wait on it)
        std::vector<Item> items;
        std::vector<Block> blocks;  // every item's blocks, in item order (kept allocated across steps)
        size_t total = 0;
        double t_begin = 0.0, t_launch = 0.0;
        long long ctas = 0;
        int variant = 0;
        cudaEvent_t k1_start = nullptr, k1_stop = nullptr;  // timing of the gather (autotuner)
        int tune_key = -1;
        double tune_work = 0.0;
        double k1_work = 0.0;  // tap-MACs of the step's K1 work list (0: no K1 launch)
    } buf[2];

    // Autotuner of the gather's chunk variant: per step class (magnitude of
    // the step's tap-MACs, magnitude of its longest IR), the best measured
    // time per tap-MAC of each variant; each variant is tried kTuneTries
    // times per class, then the fastest is used.
    struct Tune {
        float best[tc::K1_NVARIANTS];
        uint8_t tries[tc::K1_NVARIANTS];
    };
    std::vector<Tune> tune;
    bool autotune = true;

    // CUDA-graph replay of a step: per chunk variant, a graph of
    // [H2D copy] -> [ingest] -> [event] -> [gather] -> [event] -> [D2H copy]
    // whose nodes get each step's sizes, grids, arguments and events. The
    // source graph stays alive: node updates name its nodes.
    struct StepGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t h2d, ingest, ev0, k1, ev1, d2h;
    };
    StepGraph graphs[tc::K1_NVARIANTS];
    bool use_graph = false;
    // Shared device buffers (steps run in order on the step stream).
    char *d_stage = nullptr;
    size_t d_stage_items = 0;
    float *d_out = nullptr;  // [4 + max_step_samples]
    float *scratch = nullptr;
    size_t scratch_floats = 0;
    unsigned *counters = nullptr;
    size_t counters_n = 0;
    double last_done = 0.0;
    float *ir_stage = nullptr;
    size_t ir_stage_floats = 0;
    float *ir_stage_host = nullptr;  // page-locked copy of the IR being uploaded (kMaxL floats)

    // Worker.
    std::thread worker;
    std::atomic<bool> run{false};
    std::atomic<bool> stop{false};
    std::string worker_error;

    long long k1_slots = 1;  // resident K1 CTAs on the GPU (SMs x CTAs per SM)

    // Stats. Latencies (t_done - ready time) of finished blocks, drained by
    // tc_server_latencies; guarded by the queue mutex.
    // Chunked storage: growing never copies or faults in a large array on the
    // worker thread.
    std::deque<double> lat;
    std::deque<uint32_t> lat_block;  // nominal block size of each recorded latency
    // Parts of each recorded latency: ready -> collected into a step, collected
    // -> copies and kernels enqueued, enqueued -> results on the host.
    std::deque<std::array<float, 3>> lat_parts;
    std::deque<uint8_t> lat_kind;  // the block's stream: 0 plain, 1 + precision for a group
    // Step log (tracing): the last kLogSteps steps, oldest first once full.
    std::vector<tc_server_step_rec> steplog;
    size_t steplog_next = 0;
    // A reader swaps the log with this spare under the queue mutex and copies
    // it out without holding that mutex (a copy under it held the worker's
    // next step back by milliseconds). mu_log_reader serialises readers.
    std::vector<tc_server_step_rec> steplog_spare;
    std::mutex mu_log_reader;
    uint64_t steps = 0, blocks = 0, rejected = 0;
    double busy_s = 0.0;
    double tap_macs = 0.0;
    uint64_t tensor_launches = 0, fp32_fallbacks = 0;  // group pushes (state mutex)
    uint64_t pool_admissions = 0;  // admissions whose state did not fit the reservation (state mutex)
    double host_collect_s = 0.0, host_pack_s = 0.0, host_deliver_s = 0.0;  // worker host time per phase
    uint64_t grows = 0;            // step-buffer growths (allocations inside steps)
    double k1_ms = 0.0, k1_macs = 0.0;                  // K1 work-list launches: event time, tap-MACs
};

namespace {

tc_status sfail(tc_status st, const std::string &m)
{
    tc::set_last_error(m.c_str());
    return st;
}

#define S_CU(call)                                                                                    \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return sfail(e_ == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA,                      \
                         std::string(#call ": ") + cudaGetErrorString(e_));                           \
    } while (0)

#define S_TRY(expr)             \
    do {                        \
        tc_status st_ = (expr); \
        if (st_ != TC_OK)       \
            return st_;         \
    } while (0)

// Ingest kernel, CTA i for work item i (table row sc[5i..5i+4] = input
// offset, n, history column, compaction shift, compaction length):
//   1. compaction, if length > 0: history columns [shift, shift + length)
//      move to [0, length) (the two ranges do not overlap: shift >= length;
//      shift and the row start are multiples of 8 floats);
//   2. the item's n new samples go from the packed input to the history at
//      its column.
__global__ void ingest_kernel(const float *__restrict__ in, const long long *__restrict__ sc, float *const *dst,
                             int nitems)
{
    const int it = blockIdx.x;
    if (it >= nitems)
        return;
    const long long *r = sc + 5 * (long long)it;
    const long long src = r[0], n = r[1], col = r[2], shift = r[3], len = r[4];
    float *row = dst[it];
    if (len > 0) {
        const float4 *from = reinterpret_cast<const float4 *>(row + shift);
        float4 *to = reinterpret_cast<float4 *>(row);
        const long long n4 = len >> 2;
        for (long long j = threadIdx.x; j < n4; j += blockDim.x)
            to[j] = from[j];
        for (long long j = (n4 << 2) + threadIdx.x; j < len; j += blockDim.x)
            row[j] = row[shift + j];
        __syncthreads();
    }
    float *d = row + col;
    for (long long j = threadIdx.x; j < n; j += blockDim.x)
        d[j] = in[src + j];
}

// Carries a group stream's device error word (a bounded wait that gave up)
// into the step's error word.
__global__ void err_merge_kernel(int *dst, const int *src)
{
    if (threadIdx.x == 0 && *src != 0)
        *dst = *src;
}

// History row of a stream: `keep` samples behind the launch position (L taps
// plus one tap chunk and the alignment shift), room for kMerge blocks and a
// tile's overrun, and a stagger window of keep / 2 samples: each stream
// compacts its row at its own point of that window, so streams that started
// together do not all compact in the same step.
size_t stream_bytes(long long L, long long block, int nslots, long long *keep, long long *cap, long long *Lpad)
{
    *keep = rup(L + tc::K1_KC_MAX + 16, 8);
    *cap = rup(2 * *keep + kMerge * block + 512 + 160 + *keep / 2, 64);
    *Lpad = rup(L + 4 + tc::K1_KC_MAX, 4);
    return (size_t)*cap * 4 + (size_t)nslots * 4 * (size_t)*Lpad * 4 + sizeof(DevTable);
}

constexpr size_t kArenaAlign = 256;

// Returns the ranges whose steps have completed to the free list (coalesced).
// Caller holds mu_arena.
void arena_reclaim(Arena &a)
{
    while (!a.freed.empty() && (!a.freed.front().ev || cudaEventQuery(a.freed.front().ev) == cudaSuccess)) {
        Arena::Freed f = a.freed.front();
        a.freed.pop_front();
        if (f.ev)
            a.spare.push_back(f.ev);
        auto it = a.free_.emplace(f.off, f.len).first;
        auto nx = std::next(it);
        if (nx != a.free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            a.free_.erase(nx);
        }
        if (it != a.free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                a.free_.erase(it);
            }
        }
    }
}

// First fit of len bytes (a multiple of kArenaAlign); SIZE_MAX if none.
size_t arena_alloc(tc_server *srv, size_t len)
{
    std::lock_guard<std::mutex> lk(srv->mu_arena);
    Arena &a = srv->arena;
    if (!a.base)
        return SIZE_MAX;
    arena_reclaim(a);
    for (auto it = a.free_.begin(); it != a.free_.end(); ++it) {
        if (it->second < len)
            continue;
        const size_t off = it->first, rest = it->second - len;
        a.free_.erase(it);
        if (rest)
            a.free_.emplace(off + len, rest);
        return off;
    }
    return SIZE_MAX;
}

// Frees a range after the work already enqueued on the step stream.
void arena_free(tc_server *srv, size_t off, size_t len)
{
    std::lock_guard<std::mutex> lk(srv->mu_arena);
    Arena &a = srv->arena;
    cudaEvent_t ev = nullptr;
    if (!a.spare.empty()) {
        ev = a.spare.back();
        a.spare.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(srv->cs);  // no event: wait instead, then the range is free at once
        a.freed.push_back({nullptr, off, len});
        return;
    }
    cudaEventRecord(ev, srv->cs);
    a.freed.push_back({ev, off, len});
}

// Returns a removed stream's device memory to the arena or the pool, ordered
// after every step that used it (no host synchronisation).
void free_stream(tc_server *srv, SStream *s)
{
    if (s->grp) {
        tc_close(s->grp);  // waits for the steps that used it
        s->grp = nullptr;
    }
    if (s->gdone) {
        cudaEventDestroy(s->gdone);
        s->gdone = nullptr;
    }
    if (s->arena_len) {
        arena_free(srv, s->arena_off, s->arena_len);
        s->arena_len = 0;
    } else {
        if (s->hist)
            cudaFreeAsync(s->hist, srv->cs);
        if (s->ir)
            cudaFreeAsync(s->ir, srv->cs);
        if (s->d_vt)
            cudaFreeAsync(s->d_vt, srv->cs);
    }
    s->hist = nullptr;
    s->ir = nullptr;
    s->d_vt = nullptr;
}

// Drops versions no future output needs: the next version started at or
// before the oldest input sample that an output not yet delivered reads.
// (pos_done, not pos: a step in flight may still read an older version.)
void retire(SStream *s)
{
    const long long oldest = s->pos_done - s->L + 1;
    size_t drop = 0;
    while (drop + 1 < s->vt.size() && s->vt[drop + 1].start <= oldest)
        ++drop;
    for (size_t i = 0; i < drop; ++i)
        s->slot_used[(size_t)s->vt[i].slot] = 0;
    if (drop) {
        s->vt.erase(s->vt.begin(), s->vt.begin() + (long)drop);
        s->vt_dirty = true;
    }
}

// Queued input samples of s not yet run (queue mutex held by the caller).
long long queued_samples(const SStream *s)
{
    long long q = 0;
    for (auto &b : s->pending)
        q += b.n;
    return q;
}

// Uploads IR h[0..n) (zero-padded to L) as the four shifted copies into IR
// slot `slot` of s on the admin stream and waits for it. Caller holds
// mu_admin (not mu_state: steps keep running meanwhile; the slot is one no
// live version uses).
tc_status upload_ir(tc_server *srv, SStream *s, int slot, const float *h, size_t n)
{
    if (n > srv->ir_stage_floats) {
        S_CU(cudaStreamSynchronize(srv->admin));
        cudaFree(srv->ir_stage);
        srv->ir_stage = nullptr;
        srv->ir_stage_floats = 0;
        S_CU(cudaMalloc(&srv->ir_stage, n * sizeof(float)));
        srv->ir_stage_floats = n;
    }
    // Through page-locked memory: one direct DMA instead of a driver-staged
    // copy of pageable memory that shares the copy engines with the steps.
    const float *src = h;
    if (srv->ir_stage_host && n <= kMaxL) {
        std::memcpy(srv->ir_stage_host, h, n * sizeof(float));
        src = srv->ir_stage_host;
    }
    S_CU(cudaMemcpyAsync(srv->ir_stage, src, n * sizeof(float), cudaMemcpyHostToDevice, srv->admin));
    float *dst = s->ir + (size_t)slot * 4 * (size_t)s->Lpad;
    S_CU(tc::ir_prep_launch(srv->ir_stage, (long long)n, (long long)n, 1, dst, 4 * s->Lpad, s->Lpad, s->Lpad,
                            srv->admin));
    S_CU(cudaStreamSynchronize(srv->admin));  // h and the staging buffer are free on return
    return TC_OK;
}

// New IR version of s from input sample `sample` on. Three phases so that
// steps are not held up by the upload: pick a free slot (state lock), upload
// (admin lock only), publish the version (state lock). Caller holds mu_admin.
tc_status set_ir(tc_server *srv, uint64_t id, const float *h, size_t n, long long sample)
{
    SStream *s = nullptr;
    int slot = -1;
    bool replace = false, group = false;
    {
        std::lock_guard<std::mutex> lk(srv->mu_state);
        auto it = srv->streams.find(id);
        if (it == srv->streams.end())
            return sfail(TC_EINVAL, "tc_server_set_ir_at: unknown stream");
        s = it->second.get();
        if (!h || n == 0 || (long long)n > s->L)
            return sfail(TC_EINVAL, "tc_server: IR length must be in [1, L]");
        long long queued;
        {
            std::lock_guard<std::mutex> lq(srv->mu_queue);
            queued = queued_samples(s);
        }
        if (sample < s->pos + queued)
            return sfail(TC_EINVAL, "tc_server_set_ir_at: the switch sample was already submitted");
        if (s->grp)
            group = true;  // the group stream keeps its own version table
        else if (!s->vt.empty() && sample < s->vt.back().start)
            return sfail(TC_EINVAL, "tc_server_set_ir_at: switch before the latest version");
    }
    if (group) {
        // Uploads on the step stream, ordered after the pushes already made;
        // a push of the switch sample waits for this (group mutex).
        std::lock_guard<std::mutex> g(s->gmu);
        return tc_set_ir_at(s->grp, h, n, (uint64_t)sample);
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu_state);
        retire(s);
        // Replacing the newest version in place is only safe while no block
        // that uses it has been submitted.
        replace = !s->vt.empty() && s->vt.back().start == sample;
        for (int i = 0; i < s->nslots && slot < 0; ++i)
            if (!s->slot_used[(size_t)i])
                slot = i;
        if (slot < 0)
            return sfail(TC_ENOMEM, "tc_server: every IR slot of the stream holds a live version");
        s->slot_used[(size_t)slot] = 1;  // reserved: retire() never frees a slot outside the table
    }
    tc_status st = upload_ir(srv, s, slot, h, n);
    std::lock_guard<std::mutex> lk(srv->mu_state);
    if (st != TC_OK) {
        s->slot_used[(size_t)slot] = 0;
        return st;
    }
    long long queued;
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        queued = queued_samples(s);
    }
    if (sample < s->pos + queued) {
        // A live source released the switch sample during the upload.
        s->slot_used[(size_t)slot] = 0;
        return sfail(TC_ESTATE, "tc_server_set_ir_at: the switch sample became due during the upload");
    }
    if (replace) {
        s->slot_used[(size_t)s->vt.back().slot] = 0;
        s->vt.back().slot = slot;
    } else {
        s->vt.push_back({sample, slot});
    }
    s->vt_dirty = true;
    return TC_OK;
}

size_t a16(size_t b) { return (b + 15) & ~(size_t)15; }

struct StageLayout {
    size_t items, cta, sc, dst, in, end;
};

StageLayout stage_layout(size_t ni, size_t samples)
{
    StageLayout l;
    l.items = 0;
    l.cta = a16(ni * sizeof(tc::K1Params));
    l.sc = a16(l.cta + (ni + 1) * sizeof(long long));
    l.dst = a16(l.sc + 5 * ni * sizeof(long long));
    l.in = a16(l.dst + ni * sizeof(float *));
    l.end = l.in + samples * sizeof(float);
    return l;
}

// Grows step buffer b and the shared device buffers. Device buffers grow in
// stream order (the old one is freed after the steps in flight, the new one
// comes from the library's pool): no host wait. Only a larger pinned staging
// buffer waits for the step in flight (rare: a step larger than any before).
tc_status grow(tc_server *srv, tc_server::StepBuf &b, size_t items, size_t scratch_floats, size_t counters)
{
    if (items > b.items_cap || items > srv->d_stage_items || scratch_floats > srv->scratch_floats ||
        counters > srv->counters_n)
        srv->grows++;
    if (items > b.items_cap) {
        S_CU(cudaStreamSynchronize(srv->cs));
        const size_t m = std::max(items, b.items_cap * 2 + 64);
        cudaFreeHost(b.pin_stage);
        cudaFreeHost(b.pin_tables);
        b.pin_stage = nullptr;
        b.pin_tables = nullptr;
        b.items_cap = 0;
        S_CU(cudaHostAlloc(&b.pin_stage, stage_layout(m, srv->max_step_samples).end, cudaHostAllocDefault));
        S_CU(cudaHostAlloc(&b.pin_tables, m * sizeof(DevTable), cudaHostAllocDefault));
        b.items_cap = m;
    }
    if (items > srv->d_stage_items) {
        const size_t m = std::max(items, srv->d_stage_items * 2 + 64);
        if (srv->d_stage)
            cudaFreeAsync(srv->d_stage, srv->cs);
        srv->d_stage = nullptr;
        srv->d_stage_items = 0;
        S_CU(tc::pool_alloc(reinterpret_cast<void **>(&srv->d_stage), stage_layout(m, srv->max_step_samples).end,
                            srv->cs));
        srv->d_stage_items = m;
    }
    if (scratch_floats > srv->scratch_floats) {
        const size_t m = std::max(scratch_floats, srv->scratch_floats * 2);
        if (srv->scratch)
            cudaFreeAsync(srv->scratch, srv->cs);
        srv->scratch = nullptr;
        srv->scratch_floats = 0;
        S_CU(tc::pool_alloc(reinterpret_cast<void **>(&srv->scratch), m * sizeof(float), srv->cs));
        srv->scratch_floats = m;
    }
    if (counters > srv->counters_n) {
        const size_t m = std::max(counters, srv->counters_n * 2);
        if (srv->counters)
            cudaFreeAsync(srv->counters, srv->cs);
        srv->counters = nullptr;
        srv->counters_n = 0;
        S_CU(tc::pool_alloc(reinterpret_cast<void **>(&srv->counters), m * sizeof(unsigned), srv->cs));
        S_CU(cudaMemsetAsync(srv->counters, 0, m * sizeof(unsigned), srv->cs));
        srv->counters_n = m;
    }
    return TC_OK;
}

// Appends block b to the queue of s, and s to the ready queue if it was not
// there. Caller holds the queue mutex.
void enqueue(tc_server *srv, SStream *s, Block &&b)
{
    s->pending.push_back(std::move(b));
    srv->npending++;
    if (!s->in_ready) {
        s->in_ready = true;
        srv->ready.push_back(s);
    }
}

// Moves every live-source block whose ready time has passed into its
// stream's queue. Caller holds the queue mutex. Returns the next ready time
// (+inf if no source is live).
double release_sources(tc_server *srv, double now)
{
    while (!srv->src_heap.empty() && srv->src_heap.top().first <= now) {
        const uint64_t id = srv->src_heap.top().second;
        srv->src_heap.pop();
        auto it = srv->streams.find(id);
        if (it == srv->streams.end())
            continue;  // removed
        SStream *s = it->second.get();
        if (!s->src || s->src_next * s->block >= s->src_n)
            continue;
        Block b;
        b.n = std::min(s->block, s->src_n - s->src_next * s->block);
        if (s->channels == 1) {
            b.src = s->src + s->src_next * s->block;
        } else {
            // A group's source is [channels][src_n]: gather the block's rows.
            b.src = nullptr;
            b.own.resize((size_t)(s->channels * b.n));
            for (long long c = 0; c < s->channels; ++c)
                std::memcpy(b.own.data() + c * b.n, s->src + c * s->src_n + s->src_next * s->block,
                            (size_t)b.n * sizeof(float));
        }
        b.t_submit = s->src_ready(s->src_next);
        b.tail = false;
        enqueue(srv, s, std::move(b));
        s->src_next++;
        if (s->src_next * s->block < s->src_n)
            srv->src_heap.push({s->src_ready(s->src_next), id});
        else
            s->ended = true;  // the source is exhausted: input is over
    }
    return srv->src_heap.empty() ? 1e300 : srv->src_heap.top().first;
}

// The blocks of item w of step buffer b.
struct BlockSpan {
    Block *b, *e;
    Block *begin() const { return b; }
    Block *end() const { return e; }
};
BlockSpan blocks_of(tc_server::StepBuf &b, const tc_server::Item &w)
{
    Block *p = b.blocks.data() + w.first;
    return {p, p + w.count};
}

// Takes the queued blocks of every ready stream (up to kMerge consecutive
// blocks of a stream as one item) into step buffer b. Round robin: when a
// step is full, the next one starts with the streams that did not fit.
// Caller holds mu_state. Returns the number of blocks taken.
size_t collect(tc_server *srv, tc_server::StepBuf &b)
{
    tc::Range nvtx_range("server step: collect");
    b.items.clear();
    b.blocks.clear();
    b.total = 0;
    size_t nblocks = 0;
    std::lock_guard<std::mutex> lk(srv->mu_queue);
    b.t_begin = now_s();
    release_sources(srv, b.t_begin);
    if (srv->npending == 0)
        return 0;
    // A step also stays within the gather's buffers as they are: work items,
    // tile tickets and chunk-sum scratch, the latter bounded with the most
    // chunks any variant may use (640-tap chunks), so that serving never
    // grows them (growing allocates, and allocating under running steps
    // stalled them). Only a step's first item may exceed them.
    const size_t items_cap = std::min(b.items_cap, srv->d_stage_items);
    size_t tiles = 0, scratch = 0;
    // take(s): up to kMerge queued blocks of s as one item; false if a block
    // of s did not fit the step (it stays queued).
    auto take = [&](SStream *s) {
        bool fits = true;
        tc_server::Item it{s, (uint32_t)b.blocks.size(), 0, (long long)b.total, 0};
        const long long nch_max = (s->L + 3 + tc::k1_chunk_taps(tc::K1_P1) - 1) / tc::k1_chunk_taps(tc::K1_P1);
        while (!s->pending.empty() && (int)it.count < kMerge) {
            Block &blk = s->pending.front();
            const size_t fl = (size_t)(blk.n * s->channels);  // packed floats
            if (b.total + fl > srv->max_step_samples) {
                fits = false;
                break;  // stays for the next step
            }
            if (!s->grp) {
                const size_t dt = (size_t)((it.n + blk.n + tc::K1_MO - 1) / tc::K1_MO - (it.n + tc::K1_MO - 1) / tc::K1_MO);
                const size_t ds = dt * (size_t)nch_max * tc::K1_MO;
                const bool first = b.items.empty() && it.count == 0;
                if (!first && (tiles + dt > srv->counters_n || scratch + ds > srv->scratch_floats ||
                               (it.count == 0 && b.items.size() + 1 > items_cap))) {
                    fits = false;
                    break;
                }
                tiles += dt;
                scratch += ds;
            }
            b.total += fl;
            it.n += blk.n;
            b.blocks.push_back(std::move(blk));
            it.count++;
            s->pending.pop_front();
            srv->npending--;
        }
        if (it.count) {
            nblocks += it.count;
            s->inflight++;
            b.items.push_back(it);
        }
        return fits;
    };
    // Visit the streams that were ready when the step began, in order. A
    // stream with more than kMerge blocks queued goes to the back; streams
    // whose blocks did not fit lead the next step, in their order.
    std::vector<SStream *> unfit;
    const size_t nready = srv->ready.size();
    for (size_t k = 0; k < nready; ++k) {
        SStream *s = srv->ready.front();
        srv->ready.pop_front();
        const bool fits = take(s);
        if (s->pending.empty())
            s->in_ready = false;
        else if (!fits)
            unfit.push_back(s);
        else
            srv->ready.push_back(s);
    }
    for (auto it = unfit.rbegin(); it != unfit.rend(); ++it)
        srv->ready.push_front(*it);
    return nblocks;
}

// Builds (once per chunk variant) and replays the step graph with this
// step's copies, grids, arguments and timing events. Parameter updates do
// not touch launches already enqueued.
tc_status graph_launch(tc_server *srv, tc_server::StepBuf &b, int variant, size_t in_bytes, const float *a_in,
                       const long long *a_sc, float *const *a_dst, int ni, const tc::K1Params *a_items,
                       const long long *a_cta, long long ctas, size_t out_bytes)
{
    tc_server::StepGraph &g = srv->graphs[variant];
    size_t k1_smem = 0;
    const void *k1_fn = tc::k1_list_kernel(variant, &k1_smem);
    if (!k1_fn)
        return sfail(TC_ECUDA, "tc_server: no gather kernel for the variant");
    tc::K1Params none{};
    int nlist = ni;
    void *k1_args[4] = {&none, &a_items, &a_cta, &nlist};
    void *in_args[4] = {&a_in, &a_sc, &a_dst, &nlist};
    cudaKernelNodeParams kin{};
    kin.func = reinterpret_cast<void *>(&ingest_kernel);
    kin.gridDim = dim3((unsigned)ni);
    kin.blockDim = dim3(256);
    kin.kernelParams = in_args;
    cudaKernelNodeParams kk{};
    kk.func = const_cast<void *>(k1_fn);
    kk.gridDim = dim3((unsigned)ctas);
    kk.blockDim = dim3(tc::K1_THREADS);
    kk.sharedMemBytes = (unsigned)k1_smem;
    kk.kernelParams = k1_args;
    if (!g.exec) {
        S_CU(cudaGraphCreate(&g.graph, 0));
        S_CU(cudaGraphAddMemcpyNode1D(&g.h2d, g.graph, nullptr, 0, srv->d_stage, b.pin_stage, in_bytes,
                                      cudaMemcpyHostToDevice));
        S_CU(cudaGraphAddKernelNode(&g.ingest, g.graph, &g.h2d, 1, &kin));
        S_CU(cudaGraphAddEventRecordNode(&g.ev0, g.graph, &g.ingest, 1, b.k1_start));
        S_CU(cudaGraphAddKernelNode(&g.k1, g.graph, &g.ev0, 1, &kk));
        S_CU(cudaGraphAddEventRecordNode(&g.ev1, g.graph, &g.k1, 1, b.k1_stop));
        S_CU(cudaGraphAddMemcpyNode1D(&g.d2h, g.graph, &g.ev1, 1, b.pin_out, srv->d_out, out_bytes,
                                      cudaMemcpyDeviceToHost));
        S_CU(cudaGraphInstantiate(&g.exec, g.graph, 0));
    } else {
        S_CU(cudaGraphExecMemcpyNodeSetParams1D(g.exec, g.h2d, srv->d_stage, b.pin_stage, in_bytes,
                                                cudaMemcpyHostToDevice));
        S_CU(cudaGraphExecKernelNodeSetParams(g.exec, g.ingest, &kin));
        S_CU(cudaGraphExecEventRecordNodeSetEvent(g.exec, g.ev0, b.k1_start));
        S_CU(cudaGraphExecKernelNodeSetParams(g.exec, g.k1, &kk));
        S_CU(cudaGraphExecEventRecordNodeSetEvent(g.exec, g.ev1, b.k1_stop));
        S_CU(cudaGraphExecMemcpyNodeSetParams1D(g.exec, g.d2h, b.pin_out, srv->d_out, out_bytes,
                                                cudaMemcpyDeviceToHost));
    }
    S_CU(cudaGraphLaunch(g.exec, srv->cs));
    tc::count_launch(2);
    return TC_OK;
}

// Packs step buffer b and enqueues its copies and kernels on the step stream
// (no wait). Caller holds mu_state. Advances each stream's launch position.
tc_status pack_launch(tc_server *srv, tc_server::StepBuf &b)
{
    tc::Range nvtx_range("server step: pack and launch");
    if (tc::inject_take(TC_INJECT_SERVER_STEP))
        return sfail(TC_ECUDA, "tc_server: injected failure of a step's launch (tc_test_inject)");
    // Plain streams go into the K1 work list; groups run after it.
    std::vector<size_t> plain, group;
    for (size_t i = 0; i < b.items.size(); ++i)
        (b.items[i].s->grp ? group : plain).push_back(i);
    // One chunk variant for the whole list: the largest chunk that still
    // gives the GPU about four waves of CTAs with < 10 % padded taps, else the
    // smallest (short IRs, small batches: latency first).
    int variant = tc::K1_P1;
    for (int v : {tc::K1_P11, tc::K1_P4}) {
        const long long kcv = tc::k1_chunk_taps(v);
        long long ctas = 0, taps = 0, padded = 0;
        for (size_t i : plain) {
            const tc_server::Item &w = b.items[i];
            const long long ntile = (w.n + tc::K1_MO - 1) / tc::K1_MO;
            const long long nch = (w.s->L + 3 + kcv - 1) / kcv;
            ctas += ntile * nch;
            taps += ntile * w.s->L;
            padded += ntile * nch * kcv;
        }
        if (ctas >= 4LL * srv->k1_slots && padded * 10 <= taps * 11) {
            variant = v;
            break;
        }
    }
    b.tune_key = -1;
    if (srv->autotune && !plain.empty()) {
        // Step class: magnitudes of the step's tap-MACs and of its longest IR.
        double work = 0.0;
        long long maxL = 1;
        for (size_t i : plain) {
            const tc_server::Item &w = b.items[i];
            work += (double)w.n * (double)w.s->L;
            maxL = std::max(maxL, w.s->L);
        }
        const int wb = std::min(kTuneWorkBins - 1, (int)std::log2(std::max(work, 1.0)));
        const int lb = std::min(kTuneLBins - 1, (int)std::log2((double)maxL));
        const int key = wb * kTuneLBins + lb;
        const tc_server::Tune &t = srv->tune[(size_t)key];
        int pick = -1;
        for (int v = 0; v < tc::K1_NVARIANTS && pick < 0; ++v)
            if (t.tries[v] < kTuneTries)
                pick = v;  // still exploring this class
        if (pick < 0) {
            pick = variant;
            for (int v = 0; v < tc::K1_NVARIANTS; ++v)
                if (t.best[v] < t.best[pick])
                    pick = v;
        }
        variant = pick;
        b.tune_key = key;
        b.tune_work = work;
    }
    const long long kc = tc::k1_chunk_taps(variant);
    b.k1_work = 0.0;
    for (size_t i : plain)
        b.k1_work += (double)b.items[i].n * (double)b.items[i].s->L;
    size_t scratch = 0, ctrs = 0;
    for (size_t i : plain) {
        const tc_server::Item &w = b.items[i];
        const long long ntile = (w.n + tc::K1_MO - 1) / tc::K1_MO;
        scratch += (size_t)(ntile * ((w.s->L + 3 + kc - 1) / kc) * tc::K1_MO);
        ctrs += (size_t)ntile;
    }
    S_TRY(grow(srv, b, plain.size(), scratch, ctrs));

    const StageLayout lay = stage_layout(plain.size(), b.total);
    auto *st_items = reinterpret_cast<tc::K1Params *>(b.pin_stage + lay.items);
    auto *st_cta = reinterpret_cast<long long *>(b.pin_stage + lay.cta);
    auto *st_sc = reinterpret_cast<long long *>(b.pin_stage + lay.sc);
    auto *st_dst = reinterpret_cast<float **>(b.pin_stage + lay.dst);
    auto *st_in = reinterpret_cast<float *>(b.pin_stage + lay.in);
    float *const d_y = srv->d_out + 4;
    int *const d_err = reinterpret_cast<int *>(srv->d_out);
    // Packed input of every item: [rows][n] (rows = 1 for plain streams).
    for (auto &w : b.items) {
        const long long C = w.s->channels;
        long long o = 0;
        for (auto &blk : blocks_of(b, w)) {
            for (long long c = 0; c < C; ++c)
                std::memcpy(st_in + w.off + c * w.n + o, blk.data() + c * blk.n, (size_t)blk.n * sizeof(float));
            o += blk.n;
        }
    }
    size_t si = 0, ci = 0;
    long long cta = 0;
    for (size_t j = 0; j < plain.size(); ++j) {
        tc_server::Item &w = b.items[plain[j]];
        SStream *s = w.s;
        const long long n = w.n;
        retire(s);
        long long c_shift = 0, c_len = 0;
        if (s->pos + n + tc::K1_MO + 8 + s->stagger > s->base + s->cap) {
            // Compaction (done by the ingest kernel, ordered after the steps
            // in flight, which read the old layout): keep `keep` samples
            // behind the launch position.
            const long long nb = fl8(s->pos - s->keep);
            c_len = s->pos - nb;
            c_shift = nb - s->base;
            if (c_shift < c_len || c_len + n + tc::K1_MO + 8 > s->cap)
                return sfail(TC_EINVAL, "tc_server: internal: history compaction would overlap");
            s->base = nb;
        }
        if (s->vt_dirty) {
            DevTable &t = b.pin_tables[j];
            std::memset(&t, 0, sizeof t);
            t.nver = (int)s->vt.size();
            for (size_t v = 0; v < s->vt.size(); ++v) {
                t.vstart[v] = s->vt[v].start;
                t.vslot[v] = s->vt[v].slot;
            }
            S_CU(cudaMemcpyAsync(s->d_vt, &t, sizeof t, cudaMemcpyHostToDevice, srv->cs));
            s->vt_dirty = false;
        }
        st_sc[5 * j] = w.off;
        st_sc[5 * j + 1] = n;
        st_sc[5 * j + 2] = s->pos - s->base;
        st_sc[5 * j + 3] = c_shift;
        st_sc[5 * j + 4] = c_len;
        st_dst[j] = s->hist;

        tc::K1Params p{};
        p.hist = s->hist;
        p.pitch = s->cap;
        p.base = s->base;
        p.x_item_rows = 1;
        p.x_in_rows = 0;
        p.ir = s->ir;
        p.ir_slot = 4 * s->Lpad;
        p.ir_item = 0;
        p.ir_in = 0;
        p.ir_phase = s->Lpad;
        p.L = (int)s->L;
        p.vstart = s->d_vt->vstart;
        p.vslot = s->d_vt->vslot;
        p.nver = &s->d_vt->nver;
        p.vt_item = 0;
        p.nitems = 1;
        p.nin = 1;
        p.t0 = s->pos;
        p.nout = (int)n;
        p.ntile = (int)((n + tc::K1_MO - 1) / tc::K1_MO);
        p.e = tc::k1_shift_e(s->pos, s->base);
        p.nchunk = (int)((s->L + p.e + kc - 1) / kc);
        p.y = d_y + w.off;
        p.y_pitch = n;
        p.partial = srv->scratch + si;
        p.counter = srv->counters + ci;
        p.err = d_err;
        if (s->x_end >= 0) {  // the flush's zero blocks: taps that read only them are skipped
            p.has_end = 1;
            p.x_end = s->x_end;
        }
        si += (size_t)p.ntile * p.nchunk * tc::K1_MO;
        ci += (size_t)p.ntile;
        st_items[j] = p;
        st_cta[j] = cta;
        cta += (long long)p.ntile * p.nchunk;
        s->pos += n;
    }
    st_cta[plain.size()] = cta;
    const int ni = (int)plain.size();
    char *const ds = srv->d_stage;
    b.t_launch = now_s();
    b.ctas = cta;
    b.variant = variant;
    if (cta > 0x7fffffffLL)
        return sfail(TC_EINVAL, "tc_server: internal: gather grid too large");
    const float *a_in = reinterpret_cast<const float *>(ds + lay.in);
    const long long *a_sc = reinterpret_cast<const long long *>(ds + lay.sc);
    float *const *a_dst = reinterpret_cast<float *const *>(ds + lay.dst);
    const tc::K1Params *a_items = reinterpret_cast<const tc::K1Params *>(ds + lay.items);
    const long long *a_cta = reinterpret_cast<const long long *>(ds + lay.cta);
    const size_t out_bytes = (4 + b.total) * sizeof(float);
    if (srv->use_graph && group.empty()) {
        S_TRY(graph_launch(srv, b, variant, lay.end, a_in, a_sc, a_dst, ni, a_items, a_cta, cta, out_bytes));
    } else {
        S_CU(cudaMemcpyAsync(ds, b.pin_stage, lay.end, cudaMemcpyHostToDevice, srv->cs));
        if (!group.empty())
            S_CU(cudaEventRecord(b.in_ready, srv->cs));
        if (ni > 0) {
            ingest_kernel<<<(unsigned)ni, 256, 0, srv->cs>>>(a_in, a_sc, a_dst, ni);
            tc::count_launch();
            S_CU(cudaGetLastError());
            S_CU(cudaEventRecord(b.k1_start, srv->cs));
            S_CU(tc::k1_launch_list(a_items, a_cta, ni, cta, variant, srv->cs));
            S_CU(cudaEventRecord(b.k1_stop, srv->cs));
        }
        // Groups: one push of each group's stream (history copy, bf16 split,
        // K2 or K1, K-part reduce) on the group's own CUDA stream, after the
        // packed input has landed and beside the gather: groups run
        // concurrently. Each reads the packed input on the device and writes
        // its part of the packed output; its error word joins the step's; the
        // step's output copy waits for all of them.
        for (size_t i : group) {
            tc_server::Item &w = b.items[i];
            SStream *s = w.s;
            std::lock_guard<std::mutex> g(s->gmu);
            cudaStream_t gcs = static_cast<cudaStream_t>(tc::group_stream(s->grp));
            S_CU(cudaStreamWaitEvent(gcs, b.in_ready, 0));
            tc_info before{}, after{};
            tc_get_info(s->grp, &before);
            tc_status st = tc::group_push(s->grp, a_in + w.off, (size_t)w.n, d_y + w.off);
            if (st != TC_OK)
                return st;
            tc_get_info(s->grp, &after);
            srv->tensor_launches += after.tensor_launches - before.tensor_launches;
            srv->fp32_fallbacks += after.fp32_fallbacks - before.fp32_fallbacks;
            err_merge_kernel<<<1, 1, 0, gcs>>>(d_err, tc::group_err(s->grp));
            tc::count_launch();
            S_CU(cudaGetLastError());
            S_CU(cudaEventRecord(s->gdone, gcs));
            S_CU(cudaStreamWaitEvent(srv->cs, s->gdone, 0));
            s->pos += w.n;
        }
        S_CU(cudaMemcpyAsync(b.pin_out, srv->d_out, out_bytes, cudaMemcpyDeviceToHost, srv->cs));
    }
    S_CU(cudaEventRecord(b.done, srv->cs));
    return TC_OK;
}

// Drops the work items of a step that will not complete (after a failure):
// their blocks are lost and their streams stop counting them as in flight,
// so that they can be removed.
void drop_items(tc_server *srv, tc_server::StepBuf &b)
{
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    for (auto &w : b.items)
        w.s->inflight--;
    b.items.clear();
}

// Waits for step buffer b (no lock held while waiting), then delivers its
// outputs: finished blocks, latencies, flush tails, positions, stats.
tc_status complete(tc_server *srv, tc_server::StepBuf &b)
{
    tc::Range nvtx_range("server step: wait and deliver");
    S_CU(cudaEventSynchronize(b.done));
    const double t_done = now_s();
    struct DeliverTimer {  // host time spent delivering this step's outputs
        tc_server *srv;
        double t0;
        ~DeliverTimer() { srv->host_deliver_s += now_s() - t0; }
    } deliver_timer{srv, t_done};
    std::lock_guard<std::mutex> lk(srv->mu_state);
    if (*reinterpret_cast<int *>(b.pin_out)) {
        cudaMemsetAsync(srv->d_out, 0, sizeof(int), srv->cs);
        cudaMemsetAsync(srv->counters, 0, srv->counters_n * sizeof(unsigned), srv->cs);
        cudaStreamSynchronize(srv->cs);
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        for (auto &w : b.items)
            w.s->inflight--;
        b.items.clear();
        return sfail(TC_ETIMEOUT, "tc_server: a kernel's bounded wait gave up");
    }
    if (b.k1_work > 0.0) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b.k1_start, b.k1_stop) == cudaSuccess && ms > 0.f) {
            srv->k1_ms += ms;
            srv->k1_macs += b.k1_work;
        }
    }
    if (b.tune_key >= 0 && b.tune_work > 0.0) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b.k1_start, b.k1_stop) == cudaSuccess && ms > 0.f) {
            tc_server::Tune &t = srv->tune[(size_t)b.tune_key];
            const float per = (float)(ms / b.tune_work);
            t.best[b.variant] = std::min(t.best[b.variant], per);
            if (t.tries[b.variant] < 255)
                t.tries[b.variant]++;
        }
    }
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    size_t nblocks = 0;
    for (auto &w : b.items) {
        SStream *s = w.s;
        const long long C = s->channels;
        const float *yo = b.pin_out + 4 + w.off;  // [C][w.n]
        long long boff = 0;
        for (auto &blk : blocks_of(b, w)) {
            if (blk.tail) {
                const long long tail = s->L - 1;  // tail_out is [C][tail]
                if (s->tail_fill + blk.n <= tail && (long long)s->tail_out.size() == C * tail)
                    for (long long c = 0; c < C; ++c)
                        std::memcpy(s->tail_out.data() + c * tail + s->tail_fill, yo + c * w.n + boff,
                                    (size_t)blk.n * sizeof(float));
                s->tail_fill += blk.n;
            } else {
                srv->lat.push_back(t_done - blk.t_submit);
                srv->lat_block.push_back((uint32_t)s->block);
                srv->lat_parts.push_back({(float)(b.t_begin - blk.t_submit), (float)(b.t_launch - b.t_begin),
                                          (float)(t_done - b.t_launch)});
                srv->lat_kind.push_back((uint8_t)s->kind);
                srv->tap_macs += (double)blk.n * (double)s->L * (double)C;
                if (!s->discard) {
                    OutBlock o;
                    o.y.resize((size_t)(C * blk.n));
                    for (long long c = 0; c < C; ++c)
                        std::memcpy(o.y.data() + c * blk.n, yo + c * w.n + boff, (size_t)blk.n * sizeof(float));
                    o.t_submit = blk.t_submit;
                    o.t_done = t_done;
                    s->done.push_back(std::move(o));
                }
            }
            boff += blk.n;
            ++nblocks;
        }
        s->pos_done += w.n;
        s->inflight--;
    }
    tc_server_step_rec rec{b.t_begin, b.t_launch, t_done, (uint32_t)nblocks, (uint32_t)b.total, (uint32_t)b.ctas,
                           (uint32_t)b.variant};
    if (srv->steplog.size() < kLogSteps)
        srv->steplog.push_back(rec);
    else
        srv->steplog[srv->steplog_next] = rec;
    srv->steplog_next = (srv->steplog_next + 1) % kLogSteps;
    srv->steps++;
    srv->blocks += nblocks;
    srv->busy_s += t_done - std::max(b.t_begin, srv->last_done);
    srv->last_done = t_done;
    b.items.clear();
    return TC_OK;
}

// One step on the calling thread: collect, launch, wait, deliver.
tc_status step_sync(tc_server *srv, size_t *nblocks)
{
    tc_server::StepBuf &b = srv->buf[0];
    {
        std::lock_guard<std::mutex> lk(srv->mu_state);
        *nblocks = collect(srv, b);
        if (*nblocks == 0)
            return TC_OK;
        tc_status st = pack_launch(srv, b);
        if (st != TC_OK) {
            cudaDeviceSynchronize();  // whatever the failed launch had enqueued
            drop_items(srv, b);
            return st;
        }
    }
    const tc_status st = complete(srv, b);
    if (st != TC_OK)
        drop_items(srv, b);
    return st;
}

void worker_main(tc_server *srv)
{
    cudaSetDevice(srv->device);
    int inflight = -1;  // step buffer launched and not yet delivered
    bool failed = false;
    auto fail = [&](const char *where) {
        const std::string msg = tc_last_error();
        srv->worker_error = msg.empty() ? std::string(where) + " failed" : msg;
        failed = true;
    };
    while (true) {
        const bool stopping = srv->stop.load();
        const int nb = inflight < 0 ? 0 : 1 - inflight;
        bool launched = false;
        if (!stopping) {
            std::lock_guard<std::mutex> lk(srv->mu_state);
            const double h0 = now_s();
            if (collect(srv, srv->buf[nb]) > 0) {
                const double h1 = now_s();
                if (pack_launch(srv, srv->buf[nb]) != TC_OK) {
                    fail("launch");
                    break;
                }
                srv->host_collect_s += h1 - h0;
                srv->host_pack_s += now_s() - h1;
                launched = true;
            }
        }
        if (inflight >= 0 && complete(srv, srv->buf[inflight]) != TC_OK) {
            fail("complete");
            inflight = launched ? nb : -1;
            break;
        }
        inflight = launched ? nb : -1;
        if (inflight >= 0)
            continue;  // keep the GPU fed: collect the next step at once
        if (stopping)
            break;
        // Idle: sleep until the next source block is due (waking ~60 us
        // early, then yielding) or a submit arrives.
        std::unique_lock<std::mutex> lq(srv->mu_queue);
        const double now = now_s();
        const double next = release_sources(srv, now);
        if (srv->npending > 0)
            continue;
        const double wake = std::min(next, now + 1e-3);
        if (wake - now > 80e-6) {
            const auto until = std::chrono::steady_clock::time_point(
                std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                    std::chrono::duration<double>(wake - 60e-6)));
            srv->cv.wait_until(lq, until, [&] { return srv->stop.load() || srv->npending > 0; });
        } else {
            lq.unlock();
            std::this_thread::yield();
        }
    }
    if (failed) {
        // Error path: wait for what is still on the GPU (either step, the
        // groups' streams), then drop the blocks of both step buffers. They
        // will not be delivered; tc_server_stop reports the failure.
        cudaDeviceSynchronize();
        for (auto &b : srv->buf)
            drop_items(srv, b);
    }
}

SStream *find(tc_server *srv, uint64_t id)
{
    auto it = srv->streams.find(id);
    return it == srv->streams.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

tc_status tc_server_open(size_t mem_budget_bytes, size_t max_step_samples, tc_server **out)
{
    if (!out || mem_budget_bytes == 0)
        return sfail(TC_EINVAL, "tc_server_open: out is NULL or budget is 0");
    *out = nullptr;
    if (max_step_samples == 0)
        max_step_samples = (size_t)1 << 22;
    auto srv = std::make_unique<tc_server>();
    srv->budget = mem_budget_bytes;
    srv->max_step_samples = max_step_samples;
    S_CU(cudaGetDevice(&srv->device));
    int sms = 0;
    S_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, srv->device));
    srv->k1_slots = 3LL * sms;
    S_CU(cudaStreamCreateWithFlags(&srv->cs, cudaStreamNonBlocking));
    S_CU(cudaStreamCreateWithFlags(&srv->admin, cudaStreamNonBlocking));
    // Streams' memory comes from a pool of this server that keeps freed
    // memory for reuse (no driver mapping work while serving).
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = srv->device;
    S_CU(cudaMemPoolCreate(&srv->pool, &props));
    uint64_t keep_all = ~0ull;
    S_CU(cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep_all));
    for (auto &b : srv->buf) {
        S_CU(cudaHostAlloc(&b.pin_out, (4 + max_step_samples) * sizeof(float), cudaHostAllocDefault));
        S_CU(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
        S_CU(cudaEventCreateWithFlags(&b.in_ready, cudaEventDisableTiming));
        S_CU(cudaEventCreate(&b.k1_start));
        S_CU(cudaEventCreate(&b.k1_stop));
    }
    tc_server::Tune t0{};
    for (auto &v : t0.best)
        v = 3.4e38f;
    srv->tune.assign((size_t)kTuneWorkBins * kTuneLBins, t0);
    S_CU(cudaMalloc(&srv->d_out, (4 + max_step_samples) * sizeof(float)));
    S_CU(cudaMemset(srv->d_out, 0, 4 * sizeof(float)));
    // IR upload staging for the longest IR a stream may have: growing it while
    // serving would need a cudaFree, which waits for the whole device.
    S_CU(cudaMalloc(&srv->ir_stage, kMaxL * sizeof(float)));
    srv->ir_stage_floats = kMaxL;
    S_CU(cudaHostAlloc(reinterpret_cast<void **>(&srv->ir_stage_host), kMaxL * sizeof(float), cudaHostAllocDefault));
    // Size the step buffers for a few thousand streams and load the kernels
    // now, so that the first steps do not pay for allocations or module loads.
    for (auto &b : srv->buf)
        S_TRY(grow(srv.get(), b, 4096, (size_t)1 << 26, 16384));
    srv->grows = 0;  // counts growths while serving only
    cudaFuncAttributes fa;
    S_CU(cudaFuncGetAttributes(&fa, ingest_kernel));
    tc::K1Plan plan{};
    S_CU(tc::k1_plan(1000, 0, 1, 1, 1, -1, &plan));
    srv->steplog.reserve(kLogSteps);
    srv->steplog_spare.reserve(kLogSteps);
    *out = srv.release();
    return TC_OK;
}

tc_status tc_server_close(tc_server *srv)
{
    if (!srv)
        return TC_OK;
    tc_server_stop(srv);
    cudaSetDevice(srv->device);
    if (srv->cs) {
        for (auto &kv : srv->streams)
            free_stream(srv, kv.second.get());
        cudaStreamSynchronize(srv->cs);
    }
    if (srv->admin)
        cudaStreamSynchronize(srv->admin);
    for (auto &b : srv->buf) {
        cudaFreeHost(b.pin_stage);
        cudaFreeHost(b.pin_out);
        cudaFreeHost(b.pin_tables);
        if (b.done)
            cudaEventDestroy(b.done);
        if (b.in_ready)
            cudaEventDestroy(b.in_ready);
        if (b.k1_start)
            cudaEventDestroy(b.k1_start);
        if (b.k1_stop)
            cudaEventDestroy(b.k1_stop);
    }
    for (auto &g : srv->graphs) {
        if (g.exec)
            cudaGraphExecDestroy(g.exec);
        if (g.graph)
            cudaGraphDestroy(g.graph);
    }
    cudaFree(srv->d_stage);
    cudaFree(srv->d_out);
    cudaFree(srv->scratch);
    cudaFree(srv->counters);
    cudaFree(srv->ir_stage);
    cudaFreeHost(srv->ir_stage_host);
    for (auto &f : srv->arena.freed)
        if (f.ev)
            cudaEventDestroy(f.ev);
    for (cudaEvent_t ev : srv->arena.spare)
        cudaEventDestroy(ev);
    if (srv->arena.base)
        cudaFree(srv->arena.base);  // the streams were freed and both streams synchronised above
    if (srv->pool)
        cudaMemPoolDestroy(srv->pool);
    if (srv->admin)
        cudaStreamDestroy(srv->admin);
    if (srv->cs)
        cudaStreamDestroy(srv->cs);
    delete srv;
    tc::pool_trim();
    return TC_OK;
}

tc_status tc_server_reserve(tc_server *srv, size_t bytes)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_reserve: server is NULL");
    bytes = std::min(bytes, srv->budget) / kArenaAlign * kArenaAlign;
    std::lock_guard<std::mutex> la(srv->mu_admin);
    std::lock_guard<std::mutex> lk(srv->mu_arena);
    if (srv->arena.base)
        return sfail(TC_ESTATE, "tc_server_reserve: the server already has a reservation");
    if (bytes == 0)
        return TC_OK;
    S_CU(cudaSetDevice(srv->device));
    void *ptr = nullptr;
    const cudaError_t e = cudaMalloc(&ptr, bytes);  // before serving: one mapping, now
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA,
                     std::string("tc_server_reserve: ") + cudaGetErrorString(e));
    }
    srv->arena.base = static_cast<char *>(ptr);
    srv->arena.size = bytes;
    srv->arena.free_.emplace(0, bytes);
    return TC_OK;
}

tc_status tc_server_add(tc_server *srv, size_t L, size_t block, const float *h, size_t n, int flags, uint64_t *id)
{
    if (!srv || !id || !h || L == 0 || block == 0 || n == 0 || n > L)
        return sfail(TC_EINVAL, "tc_server_add: bad arguments");
    if (block > srv->max_step_samples)
        return sfail(TC_EINVAL, "tc_server_add: block larger than one step");
    if (L > kMaxL)
        return sfail(TC_EINVAL, "tc_server_add: L too long for one K1 tile's chunk stack");
    if (flags & ~TC_SERVER_DISCARD_OUTPUT)
        return sfail(TC_EINVAL, "tc_server_add: unknown flag");
    auto s = std::make_unique<SStream>();
    s->L = (long long)L;
    s->block = (long long)block;
    s->discard = (flags & TC_SERVER_DISCARD_OUTPUT) != 0;
    s->bytes = stream_bytes(s->L, s->block, s->nslots, &s->keep, &s->cap, &s->Lpad);
    {
        std::lock_guard<std::mutex> lk(srv->mu_state);
        if (srv->used + s->bytes > srv->budget) {
            srv->rejected++;
            return sfail(TC_ENOMEM, "tc_server_add: the stream does not fit the device memory budget now");
        }
        srv->used += s->bytes;  // reserved
    }
    // Device state is built on the admin stream while steps keep running.
    std::lock_guard<std::mutex> la(srv->mu_admin);
    S_CU(cudaSetDevice(srv->device));
    auto unreserve = [&](tc_status st, const std::string &m) {
        cudaStreamSynchronize(srv->admin);  // allocations complete before the ordered frees
        free_stream(srv, s.get());
        std::lock_guard<std::mutex> lk(srv->mu_state);
        srv->used -= s->bytes;
        if (st == TC_ENOMEM)
            srv->rejected++;
        return sfail(st, m);
    };
    // From the reservation if it has room (one range: history, IR slots,
    // version table), else from the pool (which may map memory now).
    const size_t b_hist = rup((long long)s->cap * 4, kArenaAlign);
    const size_t b_ir = rup((long long)s->nslots * 4 * s->Lpad * 4, kArenaAlign);
    const size_t b_vt = rup((long long)sizeof(DevTable), kArenaAlign);
    cudaError_t e = cudaSuccess;
    const size_t off = arena_alloc(srv, b_hist + b_ir + b_vt);
    if (off != SIZE_MAX) {
        s->arena_off = off;
        s->arena_len = b_hist + b_ir + b_vt;
        char *base = srv->arena.base + off;
        s->hist = reinterpret_cast<float *>(base);
        s->ir = reinterpret_cast<float *>(base + b_hist);
        s->d_vt = reinterpret_cast<DevTable *>(base + b_hist + b_ir);
    } else {
        {
            std::lock_guard<std::mutex> lk(srv->mu_state);
            srv->pool_admissions++;
        }
        e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&s->hist), (size_t)s->cap * sizeof(float), srv->pool,
                                    srv->admin);
        if (e == cudaSuccess)
            e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&s->ir),
                                        (size_t)s->nslots * 4 * (size_t)s->Lpad * sizeof(float), srv->pool,
                                        srv->admin);
        if (e == cudaSuccess)
            e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&s->d_vt), sizeof(DevTable), srv->pool, srv->admin);
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->hist, 0, (size_t)s->cap * sizeof(float), srv->admin);
    if (e != cudaSuccess)
        return unreserve(e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA,
                         std::string("tc_server_add: ") + cudaGetErrorString(e));
    s->base = -s->keep;
    s->slot_used.assign((size_t)s->nslots, 0);
    s->slot_used[0] = 1;
    tc_status st = upload_ir(srv, s.get(), 0, h, n);
    if (st != TC_OK)
        return unreserve(st, tc_last_error());
    s->vt.push_back({0, 0});
    s->vt_dirty = true;
    std::lock_guard<std::mutex> lk(srv->mu_state);
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    s->id = srv->next_id++;
    s->stagger = (long long)((s->id * 0x9E3779B97F4A7C15ull) >> 33) % std::max<long long>(1, s->keep / 2);
    *id = s->id;
    srv->streams[s->id] = std::move(s);
    return TC_OK;
}

tc_status tc_server_add_group(tc_server *srv, size_t channels, size_t L, size_t block, const float *h, size_t n,
                              int precision, int flags, uint64_t *id)
{
    if (!srv || !id || !h || channels == 0 || L == 0 || block == 0 || n == 0 || n > L)
        return sfail(TC_EINVAL, "tc_server_add_group: bad arguments");
    if (channels > 4096 || channels * block > srv->max_step_samples)
        return sfail(TC_EINVAL, "tc_server_add_group: channels x block must fit one step (channels <= 4096)");
    if (precision != TC_FP32 && precision != TC_BF16 && precision != TC_BF16_SPLIT)
        return sfail(TC_EINVAL, "tc_server_add_group: unknown precision");
    if (flags & ~TC_SERVER_DISCARD_OUTPUT)
        return sfail(TC_EINVAL, "tc_server_add_group: unknown flag");
    auto s = std::make_unique<SStream>();
    s->L = (long long)L;
    s->block = (long long)block;
    s->channels = (long long)channels;
    s->kind = 1 + precision;
    s->discard = (flags & TC_SERVER_DISCARD_OUTPUT) != 0;
    std::lock_guard<std::mutex> la(srv->mu_admin);
    S_CU(cudaSetDevice(srv->device));
    size_t bytes = 0;
    S_TRY(tc::group_open(channels, L, (size_t)kMerge * block, precision, &s->grp, &bytes));
    if (cudaEventCreateWithFlags(&s->gdone, cudaEventDisableTiming) != cudaSuccess) {
        tc_close(s->grp);
        s->grp = nullptr;
        return sfail(TC_ECUDA, "tc_server_add_group: event creation failed");
    }
    s->bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(srv->mu_state);
        if (srv->used + s->bytes > srv->budget) {
            srv->rejected++;
            free_stream(srv, s.get());
            return sfail(TC_ENOMEM, "tc_server_add_group: the group does not fit the device memory budget now");
        }
        srv->used += s->bytes;
    }
    tc_status st = tc_set_ir_at(s->grp, h, n, 0);
    if (st != TC_OK) {
        const std::string m = tc_last_error();
        free_stream(srv, s.get());
        std::lock_guard<std::mutex> lk(srv->mu_state);
        srv->used -= s->bytes;
        return sfail(st, m);
    }
    std::lock_guard<std::mutex> lk(srv->mu_state);
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    s->id = srv->next_id++;
    *id = s->id;
    srv->streams[s->id] = std::move(s);
    return TC_OK;
}

tc_status tc_server_set_ir_at(tc_server *srv, uint64_t id, const float *h, size_t n, uint64_t sample)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_set_ir_at: server is NULL");
    std::lock_guard<std::mutex> la(srv->mu_admin);
    S_CU(cudaSetDevice(srv->device));
    return set_ir(srv, id, h, n, (long long)sample);
}

tc_status tc_server_submit(tc_server *srv, uint64_t id, const float *x, size_t n)
{
    const double t = now_s();
    return tc_server_submit_many(srv, 1, &id, &x, &n, &t);
}

tc_status tc_server_submit_many(tc_server *srv, size_t count, const uint64_t *ids, const float *const *xs,
                                const size_t *ns, const double *t_ready)
{
    if (!srv || (count && (!ids || !xs || !ns)))
        return sfail(TC_EINVAL, "tc_server_submit: bad arguments");
    const double now = now_s();
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    // Validate everything first: all or nothing.
    std::vector<SStream *> ss(count);
    std::unordered_set<uint64_t> ended_here;
    for (size_t i = 0; i < count; ++i) {
        auto it = srv->streams.find(ids[i]);
        if (it == srv->streams.end())
            return sfail(TC_EINVAL, "tc_server_submit: unknown stream");
        SStream *s = it->second.get();
        if (!xs[i] || ns[i] == 0 || (long long)ns[i] > s->block)
            return sfail(TC_EINVAL, "tc_server_submit: x is NULL or n not in [1, block]");
        if (s->ended || s->flushed || ended_here.count(ids[i]))
            return sfail(TC_ESTATE, "tc_server_submit: the stream's input has ended");
        if (s->src)
            return sfail(TC_ESTATE, "tc_server_submit: the stream reads a live source");
        if ((long long)ns[i] < s->block)
            ended_here.insert(ids[i]);
        ss[i] = s;
    }
    for (size_t i = 0; i < count; ++i) {
        SStream *s = ss[i];
        if ((long long)ns[i] < s->block)
            s->ended = true;  // a short block is the last one
        Block b;
        b.own.assign(xs[i], xs[i] + ns[i] * (size_t)s->channels);  // [channels][n]
        b.src = nullptr;
        b.n = (long long)ns[i];
        b.t_submit = t_ready ? t_ready[i] : now;
        b.tail = false;
        enqueue(srv, s, std::move(b));
    }
    srv->cv.notify_one();
    return TC_OK;
}

tc_status tc_server_latencies_ex(tc_server *srv, double *out, uint32_t *block, float *parts, uint8_t *kind,
                                 size_t cap, size_t *n_out)
{
    if (!srv || !n_out || (cap && !out))
        return sfail(TC_EINVAL, "tc_server_latencies: bad arguments");
    // Take the records out under the queue mutex in O(1) when they all fit
    // (the usual case), then copy them without it: the worker needs that
    // mutex for every step.
    std::deque<double> lat;
    std::deque<uint32_t> lat_block;
    std::deque<std::array<float, 3>> lat_parts;
    std::deque<uint8_t> lat_kind;
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        if (srv->lat.size() <= cap) {
            lat.swap(srv->lat);
            lat_block.swap(srv->lat_block);
            lat_parts.swap(srv->lat_parts);
            lat_kind.swap(srv->lat_kind);
        } else {
            const long c = (long)cap;
            lat.assign(srv->lat.begin(), srv->lat.begin() + c);
            lat_block.assign(srv->lat_block.begin(), srv->lat_block.begin() + c);
            lat_parts.assign(srv->lat_parts.begin(), srv->lat_parts.begin() + c);
            lat_kind.assign(srv->lat_kind.begin(), srv->lat_kind.begin() + c);
            srv->lat.erase(srv->lat.begin(), srv->lat.begin() + c);
            srv->lat_block.erase(srv->lat_block.begin(), srv->lat_block.begin() + c);
            srv->lat_parts.erase(srv->lat_parts.begin(), srv->lat_parts.begin() + c);
            srv->lat_kind.erase(srv->lat_kind.begin(), srv->lat_kind.begin() + c);
        }
    }
    const size_t n = lat.size();
    std::copy(lat.begin(), lat.end(), out);
    if (block)
        std::copy(lat_block.begin(), lat_block.end(), block);
    if (parts)
        for (size_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k)
                parts[3 * i + (size_t)k] = lat_parts[i][(size_t)k];
    if (kind)
        std::copy(lat_kind.begin(), lat_kind.end(), kind);
    *n_out = n;
    return TC_OK;
}

tc_status tc_server_latencies(tc_server *srv, double *out, uint32_t *block, size_t cap, size_t *n_out)
{
    return tc_server_latencies_ex(srv, out, block, nullptr, nullptr, cap, n_out);
}

tc_status tc_server_attach_source(tc_server *srv, uint64_t id, const float *x, size_t n, double t0, double fs)
{
    if (!srv || !x || n == 0 || !(fs > 0.0))
        return sfail(TC_EINVAL, "tc_server_attach_source: bad arguments");
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    auto it = srv->streams.find(id);
    if (it == srv->streams.end())
        return sfail(TC_EINVAL, "tc_server_attach_source: unknown stream");
    SStream *s = it->second.get();
    if (s->src || s->ended || s->flushed || !s->pending.empty())
        return sfail(TC_ESTATE, "tc_server_attach_source: the stream has a source, queued blocks or ended input");
    s->src = x;
    s->src_n = (long long)n;
    s->src_next = 0;
    s->src_t0 = t0;
    s->src_fs = fs;
    srv->src_heap.push({s->src_ready(0), id});
    srv->cv.notify_one();
    return TC_OK;
}

tc_status tc_server_stream_state(tc_server *srv, uint64_t id, int *state)
{
    if (!srv || !state)
        return sfail(TC_EINVAL, "tc_server_stream_state: bad arguments");
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    auto it = srv->streams.find(id);
    if (it == srv->streams.end())
        return sfail(TC_EINVAL, "tc_server_stream_state: unknown stream");
    const SStream *s = it->second.get();
    *state = !s->ended ? 0 : (s->pending.empty() && s->inflight == 0 ? 2 : 1);
    return TC_OK;
}

tc_status tc_server_step(tc_server *srv, size_t *blocks_done)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_step: server is NULL");
    if (srv->run.load())
        return sfail(TC_ESTATE, "tc_server_step: the worker thread is running");
    S_CU(cudaSetDevice(srv->device));
    size_t n = 0;
    tc_status st = step_sync(srv, &n);
    if (blocks_done)
        *blocks_done = n;
    return st;
}

tc_status tc_server_start(tc_server *srv)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_start: server is NULL");
    if (srv->run.load())
        return TC_OK;
    srv->stop = false;
    srv->worker_error.clear();
    srv->run = true;
    srv->worker = std::thread(worker_main, srv);
    return TC_OK;
}

tc_status tc_server_stop(tc_server *srv)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_stop: server is NULL");
    if (!srv->run.load())
        return TC_OK;
    srv->stop = true;
    srv->cv.notify_all();
    if (srv->worker.joinable())
        srv->worker.join();
    srv->run = false;
    if (!srv->worker_error.empty())
        return sfail(TC_ECUDA, "tc_server worker: " + srv->worker_error);
    return TC_OK;
}

tc_status tc_server_poll(tc_server *srv, uint64_t id, float *y, size_t cap, size_t *n_out, double *t_submit,
                         double *t_done)
{
    if (!srv || !n_out)
        return sfail(TC_EINVAL, "tc_server_poll: bad arguments");
    *n_out = 0;
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    auto it = srv->streams.find(id);
    if (it == srv->streams.end())
        return sfail(TC_EINVAL, "tc_server_poll: unknown stream");
    SStream *s = it->second.get();
    if (s->done.empty())
        return TC_OK;
    OutBlock &o = s->done.front();
    if (o.y.size() > cap || (!y && cap))
        return sfail(TC_EINVAL, "tc_server_poll: y too small for the next block");
    if (y)
        std::memcpy(y, o.y.data(), o.y.size() * sizeof(float));
    *n_out = o.y.size();
    if (t_submit)
        *t_submit = o.t_submit;
    if (t_done)
        *t_done = o.t_done;
    s->done.pop_front();
    return TC_OK;
}

tc_status tc_server_flush(tc_server *srv, uint64_t id, float *y, size_t cap, size_t *n_out)
{
    if (!srv || !y)
        return sfail(TC_EINVAL, "tc_server_flush: bad arguments");
    if (srv->run.load())
        return sfail(TC_ESTATE, "tc_server_flush: stop the worker first");
    std::unique_lock<std::mutex> lk(srv->mu_state);
    SStream *s = find(srv, id);
    if (!s)
        return sfail(TC_EINVAL, "tc_server_flush: unknown stream");
    const long long tail = s->L - 1;
    const long long C = s->channels;
    if ((long long)cap < C * tail)
        return sfail(TC_EINVAL, "tc_server_flush: cap < channels x (L - 1)");
    if (s->flushed)
        return sfail(TC_ESTATE, "tc_server_flush: already flushed");
    if (s->src && s->src_next * s->block < s->src_n)
        return sfail(TC_ESTATE, "tc_server_flush: the stream's live source has not ended");
    S_CU(cudaSetDevice(srv->device));
    // The tail is the output of L - 1 zero samples (the accumulator drained,
    // Sec. 4.2): zero blocks of `block` samples run through ordinary steps
    // (other streams' pending blocks ride along).
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        s->x_end = s->pos + queued_samples(s);  // real input: launched + still queued
        s->tail_out.assign((size_t)(C * tail), 0.f);
        s->tail_fill = 0;
        for (long long off = 0; off < tail; off += s->block) {
            Block b;
            b.n = std::min<long long>(s->block, tail - off);
            b.own.assign((size_t)(C * b.n), 0.f);
            b.src = nullptr;
            b.t_submit = now_s();
            b.tail = true;
            enqueue(srv, s, std::move(b));
        }
        s->ended = true;
        s->flushed = true;
    }
    lk.unlock();  // steps take the state lock themselves (the worker is stopped)
    for (;;) {
        {
            std::lock_guard<std::mutex> lq(srv->mu_queue);
            if (s->pending.empty())
                break;
        }
        size_t nb = 0;
        S_TRY(step_sync(srv, &nb));
        if (nb == 0)
            return sfail(TC_ESTATE, "tc_server_flush: internal: a step made no progress");
    }
    lk.lock();
    if (s->tail_fill != tail)
        return sfail(TC_ESTATE, "tc_server_flush: internal: tail length");
    if (tail > 0)
        std::memcpy(y, s->tail_out.data(), (size_t)(C * tail) * sizeof(float));
    s->tail_out.clear();
    s->tail_out.shrink_to_fit();
    if (n_out)
        *n_out = (size_t)(C * tail);
    return TC_OK;
}

tc_status tc_server_remove(tc_server *srv, uint64_t id)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_remove: server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu_state);
    std::unique_ptr<SStream> s;
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        auto it = srv->streams.find(id);
        if (it == srv->streams.end())
            return sfail(TC_EINVAL, "tc_server_remove: unknown stream");
        if (!it->second->pending.empty() || it->second->inflight > 0)
            return sfail(TC_ESTATE, "tc_server_remove: the stream still has blocks queued or running");
        if (it->second->in_ready)  // not reached (a ready stream has queued blocks); kept for safety
            srv->ready.erase(std::find(srv->ready.begin(), srv->ready.end(), it->second.get()));
        s = std::move(it->second);
        srv->streams.erase(it);
    }
    cudaSetDevice(srv->device);
    srv->used -= s->bytes;
    if (!s->grp) {
        free_stream(srv, s.get());  // stream-ordered frees after the steps that used it
        return TC_OK;
    }
    lk.unlock();  // closing a group stream waits for the steps in flight
    free_stream(srv, s.get());
    return TC_OK;
}

tc_status tc_server_get_stats(tc_server *srv, tc_server_stats *st)
{
    if (!srv || !st)
        return sfail(TC_EINVAL, "tc_server_get_stats: bad arguments");
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    st->streams = srv->streams.size();
    st->mem_used = srv->used;
    st->mem_budget = srv->budget;
    st->steps = srv->steps;
    st->blocks = srv->blocks;
    st->rejected = srv->rejected;
    st->busy_s = srv->busy_s;
    st->tap_macs = srv->tap_macs;
    st->tensor_launches = srv->tensor_launches;
    st->k1_ms = srv->k1_ms;
    st->k1_macs = srv->k1_macs;
    st->pool_admissions = srv->pool_admissions;
    st->grows = srv->grows;
    st->host_collect_s = srv->host_collect_s;
    st->host_pack_s = srv->host_pack_s;
    st->host_deliver_s = srv->host_deliver_s;
    st->fp32_fallbacks = srv->fp32_fallbacks;
    return TC_OK;
}

double tc_server_clock(void) { return now_s(); }

tc_status tc_server_set_option(tc_server *srv, int option, int value)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_set_option: server is NULL");
    if (value != 0 && value != 1)
        return sfail(TC_EINVAL, "tc_server_set_option: value must be 0 or 1");
    std::lock_guard<std::mutex> lk(srv->mu_state);
    switch (option) {
    case TC_SERVER_AUTOTUNE: srv->autotune = value != 0; return TC_OK;
    case TC_SERVER_GRAPH: srv->use_graph = value != 0; return TC_OK;
    default: return sfail(TC_EINVAL, "tc_server_set_option: unknown option");
    }
}

tc_status tc_server_step_log(tc_server *srv, tc_server_step_rec *out, size_t cap, size_t *n_out)
{
    if (!srv || !n_out || (cap && !out))
        return sfail(TC_EINVAL, "tc_server_step_log: bad arguments");
    std::lock_guard<std::mutex> lr(srv->mu_log_reader);
    size_t next = 0;
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        srv->steplog.swap(srv->steplog_spare);  // O(1): the worker continues on the empty spare
        next = srv->steplog_next;
        srv->steplog_next = 0;
    }
    const std::vector<tc_server_step_rec> &log = srv->steplog_spare;
    const size_t n = log.size();
    const size_t first = n < kLogSteps ? 0 : next;
    const size_t k = std::min(cap, n);
    for (size_t i = 0; i < k; ++i)  // the newest k, oldest first
        out[i] = log[(first + (n - k) + i) % n];
    srv->steplog_spare.clear();  // keeps its capacity
    *n_out = k;
    return TC_OK;
}

}  // extern "C"
