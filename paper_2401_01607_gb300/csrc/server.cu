// server.cu -- continuous batching of many independent streams (tc_server_*).
//
// Real-time use of the taches-algorithm (Sec. 5.1 and Sec. 6: low-latency
// output, multichannel use, IRs that change while running) with many
// audio streams at once. Each stream has its own IR length, block size and IR
// versions. A step collects every block that is pending on any stream and
// runs them all as one batch:
//   one host->device copy of the packed input, one scatter kernel into the
//   streams' history rows, one K1 work-list launch (one item per stream), one
//   device->host copy of the packed output.
// Blocks submitted while a step is on the GPU join the next step. A worker
// thread (tc_server_start) runs steps back to back whenever blocks are
// pending. Streams are admitted while their device state fits the memory
// budget (TC_ENOMEM otherwise) and release it when removed.
//
// Threads: submit/poll take only the queue mutex and never wait for the GPU;
// add/remove/set_ir and step take the state mutex.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/taches.h"
#include "tc_internal.h"

namespace {

constexpr int kMaxVer = 16;
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
    std::vector<float> x;
    double t_submit;  // ready time of the block (latency is measured from it)
    bool tail;        // zero input of the flush: output goes to the tail buffer
};

struct OutBlock {
    std::vector<float> y;
    double t_submit;
    double t_done;
};

struct SStream {
    uint64_t id = 0;
    long long L = 0, block = 0, Lpad = 0, keep = 0, cap = 0, base = 0, pos = 0;
    int nslots = 3;
    bool ended = false;   // a short block was submitted: input is over
    bool flushed = false;
    bool discard = false;  // keep no output blocks (latency is still recorded)
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
    std::deque<OutBlock> done;   // guarded by the queue mutex
    std::vector<float> tail_out; // output of the flush's zero blocks
};

}  // namespace

struct tc_server {
    size_t budget = 0, used = 0;
    size_t max_step_samples = 0;
    int device = 0;
    cudaStream_t cs = nullptr;
    std::mutex mu_state;  // device state of streams, steps
    std::mutex mu_queue;  // pending input / finished output queues
    std::condition_variable cv;
    std::map<uint64_t, std::unique_ptr<SStream>> streams;
    uint64_t next_id = 1;
    uint64_t rr = 0;  // first stream id visited by the next step

    // Step staging.
    // Step staging. Input side: ONE pinned buffer and its device mirror, laid
    // out per step as [K1 items][CTA offsets][scatter table][history
    // pointers][packed input] (16-byte aligned regions) and copied with one
    // host-to-device copy. Output side: [error word, padded to 16 bytes]
    // [packed output], copied back with one device-to-host copy.
    char *pin_stage = nullptr, *d_stage = nullptr;
    size_t stage_bytes = 0;
    size_t max_items = 0;
    float *pin_out = nullptr, *d_out = nullptr;  // [4 + max_step_samples]
    DevTable *pin_tables = nullptr;
    float *scratch = nullptr;
    size_t scratch_floats = 0;
    unsigned *counters = nullptr;
    size_t counters_n = 0;
    float *ir_stage = nullptr;
    size_t ir_stage_floats = 0;

    // Worker.
    std::thread worker;
    std::atomic<bool> run{false};
    std::atomic<bool> stop{false};
    std::string worker_error;

    long long k1_slots = 1;  // resident K1 CTAs on the GPU (SMs x CTAs per SM)

    // Stats. Latencies (t_done - ready time) of finished blocks, drained by
    // tc_server_latencies; guarded by the queue mutex.
    std::vector<double> lat;
    uint64_t steps = 0, blocks = 0, rejected = 0;
    double busy_s = 0.0;
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

// Scatter kernel: CTA i copies the n_i samples of item i from the packed input
// at src_i into its stream's history row at column col_i.
__global__ void scatter_kernel(const float *__restrict__ in, const long long *__restrict__ sc, float *const *dst,
                               int nitems)
{
    const int it = blockIdx.x;
    if (it >= nitems)
        return;
    const long long src = sc[3 * it], n = sc[3 * it + 1], col = sc[3 * it + 2];
    float *d = dst[it] + col;
    for (long long j = threadIdx.x; j < n; j += blockDim.x)
        d[j] = in[src + j];
}

size_t stream_bytes(long long L, long long block, int nslots, long long *keep, long long *cap, long long *Lpad)
{
    *keep = rup(L + tc::K1_KC_MAX + 16, 8);
    *cap = rup(2 * *keep + block + 512 + 160, 64);
    *Lpad = rup(L + 4 + tc::K1_KC_MAX, 4);
    return (size_t)*cap * 4 + (size_t)nslots * 4 * (size_t)*Lpad * 4 + sizeof(DevTable);
}

void free_stream(SStream *s)
{
    cudaFree(s->hist);
    cudaFree(s->ir);
    cudaFree(s->d_vt);
}

// Drops versions no future output needs (next version started >= L-1 ago).
void retire(SStream *s)
{
    const long long oldest = s->pos - s->L + 1;
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

tc_status set_ir(tc_server *srv, SStream *s, const float *h, size_t n, long long sample)
{
    if (!h || n == 0 || (long long)n > s->L)
        return sfail(TC_EINVAL, "tc_server: IR length must be in [1, L]");
    if (sample < s->pos || (!s->vt.empty() && sample < s->vt.back().start))
        return sfail(TC_EINVAL, "tc_server: IR switch before the next sample or the latest version");
    retire(s);
    int slot = -1;
    const bool replace = !s->vt.empty() && s->vt.back().start == sample;
    if (replace) {
        slot = s->vt.back().slot;
    } else {
        for (int i = 0; i < s->nslots; ++i)
            if (!s->slot_used[(size_t)i]) {
                slot = i;
                break;
            }
        if (slot < 0)
            return sfail(TC_ENOMEM, "tc_server: every IR slot of the stream holds a live version");
    }
    if (n > srv->ir_stage_floats) {
        S_CU(cudaStreamSynchronize(srv->cs));
        cudaFree(srv->ir_stage);
        srv->ir_stage = nullptr;
        S_CU(cudaMalloc(&srv->ir_stage, n * sizeof(float)));
        srv->ir_stage_floats = n;
    }
    S_CU(cudaMemcpyAsync(srv->ir_stage, h, n * sizeof(float), cudaMemcpyHostToDevice, srv->cs));
    float *dst = s->ir + (size_t)slot * 4 * (size_t)s->Lpad;
    S_CU(tc::ir_prep_launch(srv->ir_stage, (long long)n, (long long)n, 1, dst, 4 * s->Lpad, s->Lpad, s->Lpad, srv->cs));
    S_CU(cudaStreamSynchronize(srv->cs));  // h and the staging buffer are free on return
    if (!replace) {
        s->vt.push_back({sample, slot});
        s->slot_used[(size_t)slot] = 1;
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
    l.dst = a16(l.sc + 3 * ni * sizeof(long long));
    l.in = a16(l.dst + ni * sizeof(float *));
    l.end = l.in + samples * sizeof(float);
    return l;
}

tc_status grow(tc_server *srv, size_t items, size_t scratch_floats, size_t counters)
{
    if (items > srv->max_items) {
        const size_t m = std::max(items, srv->max_items * 2 + 64);
        cudaFreeHost(srv->pin_stage);
        cudaFree(srv->d_stage);
        cudaFreeHost(srv->pin_tables);
        srv->pin_stage = srv->d_stage = nullptr;
        srv->pin_tables = nullptr;
        srv->max_items = 0;
        const size_t bytes = stage_layout(m, srv->max_step_samples).end;
        S_CU(cudaHostAlloc(&srv->pin_stage, bytes, cudaHostAllocDefault));
        S_CU(cudaMalloc(&srv->d_stage, bytes));
        S_CU(cudaHostAlloc(&srv->pin_tables, m * sizeof(DevTable), cudaHostAllocDefault));
        srv->stage_bytes = bytes;
        srv->max_items = m;
    }
    if (scratch_floats > srv->scratch_floats) {
        cudaFree(srv->scratch);
        srv->scratch = nullptr;
        const size_t m = std::max(scratch_floats, srv->scratch_floats * 2);
        S_CU(cudaMalloc(&srv->scratch, m * sizeof(float)));
        srv->scratch_floats = m;
    }
    if (counters > srv->counters_n) {
        cudaFree(srv->counters);
        srv->counters = nullptr;
        const size_t m = std::max(counters, srv->counters_n * 2);
        S_CU(cudaMalloc(&srv->counters, m * sizeof(unsigned)));
        S_CU(cudaMemsetAsync(srv->counters, 0, m * sizeof(unsigned), srv->cs));
        srv->counters_n = m;
    }
    return TC_OK;
}

// One batched step over every pending block. Caller holds mu_state.
tc_status step_locked(tc_server *srv, size_t *nblocks)
{
    *nblocks = 0;
    struct Work {
        SStream *s;
        Block b;
        long long in_off, out_off;
    };
    std::vector<Work> work;
    size_t total = 0;
    {
        // Round robin: when a step fills up, the next one starts at the first
        // stream that did not fit, so no stream waits more than a few steps.
        std::lock_guard<std::mutex> lk(srv->mu_queue);
        bool capped = false;
        auto take = [&](SStream *s) {
            if (s->pending.empty())
                return;
            Block &b = s->pending.front();
            if (total + b.x.size() > srv->max_step_samples) {
                if (!capped)
                    srv->rr = s->id;
                capped = true;
                return;  // stays for the next step
            }
            work.push_back({s, std::move(b), (long long)total, (long long)total});
            s->pending.pop_front();
            total += work.back().b.x.size();
        };
        const auto start = srv->streams.lower_bound(srv->rr);
        for (auto it = start; it != srv->streams.end(); ++it)
            take(it->second.get());
        for (auto it = srv->streams.begin(); it != start; ++it)
            take(it->second.get());
        if (!capped)
            srv->rr = 0;
    }
    if (work.empty())
        return TC_OK;
    const double t_start = now_s();

    // Plan: one chunk variant for the whole list -- the largest chunk that
    // still gives the GPU about four waves of CTAs with < 10 % padded taps,
    // else the smallest (short IRs, small batches: latency first).
    int variant = tc::K1_P1;
    for (int v : {tc::K1_P13, tc::K1_P4}) {
        const long long kcv = tc::k1_chunk_taps(v);
        long long ctas = 0, taps = 0, padded = 0;
        for (auto &w : work) {
            const long long ntile = ((long long)w.b.x.size() + tc::K1_MO - 1) / tc::K1_MO;
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
    const long long kc = tc::k1_chunk_taps(variant);
    size_t scratch = 0, ctrs = 0;
    for (auto &w : work) {
        const long long n = (long long)w.b.x.size();
        const long long ntile = (n + tc::K1_MO - 1) / tc::K1_MO;
        const long long nchunk = (w.s->L + 3 + kc - 1) / kc;
        scratch += (size_t)(ntile * nchunk * tc::K1_MO);
        ctrs += (size_t)ntile;
    }
    S_TRY(grow(srv, work.size(), scratch, ctrs));

    // Input packing, history room, version tables.
    const StageLayout lay = stage_layout(work.size(), total);
    auto *st_items = reinterpret_cast<tc::K1Params *>(srv->pin_stage + lay.items);
    auto *st_cta = reinterpret_cast<long long *>(srv->pin_stage + lay.cta);
    auto *st_sc = reinterpret_cast<long long *>(srv->pin_stage + lay.sc);
    auto *st_dst = reinterpret_cast<float **>(srv->pin_stage + lay.dst);
    auto *st_in = reinterpret_cast<float *>(srv->pin_stage + lay.in);
    float *const d_y = srv->d_out + 4;
    int *const d_err = reinterpret_cast<int *>(srv->d_out);
    size_t si = 0, ci = 0;
    long long cta = 0;
    for (size_t i = 0; i < work.size(); ++i) {
        Work &w = work[i];
        SStream *s = w.s;
        const long long n = (long long)w.b.x.size();
        std::memcpy(st_in + w.in_off, w.b.x.data(), (size_t)n * sizeof(float));
        retire(s);
        if (s->pos + n + tc::K1_MO + 8 > s->base + s->cap) {
            const long long nb = fl8(s->pos - s->keep);
            const long long len = s->pos - nb, shift = nb - s->base;
            if (shift < len || len + n + tc::K1_MO + 8 > s->cap)
                return sfail(TC_EINVAL, "tc_server: internal: history compaction would overlap");
            S_CU(cudaMemcpyAsync(s->hist, s->hist + shift, (size_t)len * sizeof(float), cudaMemcpyDeviceToDevice,
                                 srv->cs));
            s->base = nb;
        }
        if (s->vt_dirty) {
            DevTable &t = srv->pin_tables[i];
            std::memset(&t, 0, sizeof t);
            t.nver = (int)s->vt.size();
            for (size_t v = 0; v < s->vt.size(); ++v) {
                t.vstart[v] = s->vt[v].start;
                t.vslot[v] = s->vt[v].slot;
            }
            S_CU(cudaMemcpyAsync(s->d_vt, &t, sizeof t, cudaMemcpyHostToDevice, srv->cs));
            s->vt_dirty = false;
        }
        st_sc[3 * i] = w.in_off;
        st_sc[3 * i + 1] = n;
        st_sc[3 * i + 2] = s->pos - s->base;
        st_dst[i] = s->hist;

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
        p.y = d_y + w.out_off;
        p.y_pitch = n;
        p.partial = srv->scratch + si;
        p.counter = srv->counters + ci;
        p.err = d_err;
        si += (size_t)p.ntile * p.nchunk * tc::K1_MO;
        ci += (size_t)p.ntile;
        st_items[i] = p;
        st_cta[i] = cta;
        cta += (long long)p.ntile * p.nchunk;
    }
    st_cta[work.size()] = cta;
    const int ni = (int)work.size();
    char *const ds = srv->d_stage;
    S_CU(cudaMemcpyAsync(ds, srv->pin_stage, lay.end, cudaMemcpyHostToDevice, srv->cs));
    scatter_kernel<<<(unsigned)ni, 128, 0, srv->cs>>>(reinterpret_cast<const float *>(ds + lay.in),
                                                       reinterpret_cast<const long long *>(ds + lay.sc),
                                                       reinterpret_cast<float *const *>(ds + lay.dst), ni);
    tc::count_launch();
    S_CU(cudaGetLastError());
    S_CU(tc::k1_launch_list(reinterpret_cast<const tc::K1Params *>(ds + lay.items),
                            reinterpret_cast<const long long *>(ds + lay.cta), ni, cta, variant, srv->cs));
    S_CU(cudaMemcpyAsync(srv->pin_out, srv->d_out, (4 + total) * sizeof(float), cudaMemcpyDeviceToHost, srv->cs));
    S_CU(cudaStreamSynchronize(srv->cs));
    if (*reinterpret_cast<int *>(srv->pin_out)) {
        cudaMemsetAsync(srv->d_out, 0, sizeof(int), srv->cs);
        cudaMemsetAsync(srv->counters, 0, srv->counters_n * sizeof(unsigned), srv->cs);
        cudaStreamSynchronize(srv->cs);
        return sfail(TC_ETIMEOUT, "tc_server: a kernel's bounded wait gave up");
    }
    const double t_done = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu_queue);
        for (auto &w : work) {
            const long long n = (long long)w.b.x.size();
            const float *yo = srv->pin_out + 4 + w.out_off;
            if (w.b.tail) {
                w.s->tail_out.insert(w.s->tail_out.end(), yo, yo + n);
            } else if (w.s->discard) {
                srv->lat.push_back(t_done - w.b.t_submit);
            } else {
                srv->lat.push_back(t_done - w.b.t_submit);
                OutBlock o;
                o.y.assign(yo, yo + n);
                o.t_submit = w.b.t_submit;
                o.t_done = t_done;
                w.s->done.push_back(std::move(o));
            }
            w.s->pos += n;
        }
    }
    srv->steps++;
    srv->blocks += work.size();
    srv->busy_s += t_done - t_start;
    *nblocks = work.size();
    return TC_OK;
}

bool any_pending(tc_server *srv)
{
    for (auto &kv : srv->streams)
        if (!kv.second->pending.empty())
            return true;
    return false;
}

void worker_main(tc_server *srv)
{
    cudaSetDevice(srv->device);
    while (!srv->stop.load()) {
        {
            std::unique_lock<std::mutex> lk(srv->mu_queue);
            srv->cv.wait_for(lk, std::chrono::microseconds(200), [&] { return srv->stop.load() || any_pending(srv); });
        }
        if (srv->stop.load())
            break;
        std::lock_guard<std::mutex> lk(srv->mu_state);
        size_t n = 0;
        if (step_locked(srv, &n) != TC_OK) {
            srv->worker_error = tc_last_error();
            break;
        }
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
    S_CU(cudaHostAlloc(&srv->pin_out, (4 + max_step_samples) * sizeof(float), cudaHostAllocDefault));
    S_CU(cudaMalloc(&srv->d_out, (4 + max_step_samples) * sizeof(float)));
    S_CU(cudaMemset(srv->d_out, 0, 4 * sizeof(float)));
    *out = srv.release();
    return TC_OK;
}

tc_status tc_server_close(tc_server *srv)
{
    if (!srv)
        return TC_OK;
    tc_server_stop(srv);
    cudaSetDevice(srv->device);
    if (srv->cs)
        cudaStreamSynchronize(srv->cs);
    for (auto &kv : srv->streams)
        free_stream(kv.second.get());
    cudaFreeHost(srv->pin_stage);
    cudaFree(srv->d_stage);
    cudaFreeHost(srv->pin_out);
    cudaFree(srv->d_out);
    cudaFreeHost(srv->pin_tables);
    cudaFree(srv->scratch);
    cudaFree(srv->counters);
    cudaFree(srv->ir_stage);
    if (srv->cs)
        cudaStreamDestroy(srv->cs);
    delete srv;
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
    std::lock_guard<std::mutex> lk(srv->mu_state);
    S_CU(cudaSetDevice(srv->device));
    auto s = std::make_unique<SStream>();
    if (flags & ~TC_SERVER_DISCARD_OUTPUT)
        return sfail(TC_EINVAL, "tc_server_add: unknown flag");
    s->L = (long long)L;
    s->block = (long long)block;
    s->discard = (flags & TC_SERVER_DISCARD_OUTPUT) != 0;
    s->bytes = stream_bytes(s->L, s->block, s->nslots, &s->keep, &s->cap, &s->Lpad);
    if (srv->used + s->bytes > srv->budget) {
        srv->rejected++;
        return sfail(TC_ENOMEM, "tc_server_add: the stream does not fit the device memory budget now");
    }
    cudaError_t e = cudaMalloc(&s->hist, (size_t)s->cap * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&s->ir, (size_t)s->nslots * 4 * (size_t)s->Lpad * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&s->d_vt, sizeof(DevTable));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->hist, 0, (size_t)s->cap * sizeof(float), srv->cs);
    if (e != cudaSuccess) {
        free_stream(s.get());
        srv->rejected++;
        return sfail(e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA,
                     std::string("tc_server_add: ") + cudaGetErrorString(e));
    }
    s->base = -s->keep;
    s->slot_used.assign((size_t)s->nslots, 0);
    tc_status st = set_ir(srv, s.get(), h, n, 0);
    if (st != TC_OK) {
        free_stream(s.get());
        return st;
    }
    s->id = srv->next_id++;
    srv->used += s->bytes;
    *id = s->id;
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    srv->streams[s->id] = std::move(s);
    return TC_OK;
}

tc_status tc_server_set_ir_at(tc_server *srv, uint64_t id, const float *h, size_t n, uint64_t sample)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_set_ir_at: server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu_state);
    SStream *s = find(srv, id);
    if (!s)
        return sfail(TC_EINVAL, "tc_server_set_ir_at: unknown stream");
    // Blocks already submitted but not yet run come before the switch point.
    long long queued = 0;
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        for (auto &b : s->pending)
            queued += (long long)b.x.size();
    }
    if ((long long)sample < s->pos + queued)
        return sfail(TC_EINVAL, "tc_server_set_ir_at: the switch sample was already submitted");
    S_CU(cudaSetDevice(srv->device));
    return set_ir(srv, s, h, n, (long long)sample);
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
    for (size_t i = 0; i < count; ++i) {
        auto it = srv->streams.find(ids[i]);
        if (it == srv->streams.end())
            return sfail(TC_EINVAL, "tc_server_submit: unknown stream");
        const SStream *s = it->second.get();
        if (!xs[i] || ns[i] == 0 || (long long)ns[i] > s->block)
            return sfail(TC_EINVAL, "tc_server_submit: x is NULL or n not in [1, block]");
        if (s->ended || s->flushed)
            return sfail(TC_ESTATE, "tc_server_submit: the stream's input has ended");
        for (size_t j = 0; j < i; ++j)
            if (ids[j] == ids[i] && (long long)ns[j] < s->block)
                return sfail(TC_ESTATE, "tc_server_submit: block after the stream's last (short) block");
    }
    for (size_t i = 0; i < count; ++i) {
        SStream *s = srv->streams[ids[i]].get();
        if ((long long)ns[i] < s->block)
            s->ended = true;  // a short block is the last one
        Block b;
        b.x.assign(xs[i], xs[i] + ns[i]);
        b.t_submit = t_ready ? t_ready[i] : now;
        b.tail = false;
        s->pending.push_back(std::move(b));
    }
    srv->cv.notify_one();
    return TC_OK;
}

tc_status tc_server_latencies(tc_server *srv, double *out, size_t cap, size_t *n_out)
{
    if (!srv || !n_out || (cap && !out))
        return sfail(TC_EINVAL, "tc_server_latencies: bad arguments");
    std::lock_guard<std::mutex> lq(srv->mu_queue);
    const size_t n = std::min(cap, srv->lat.size());
    if (n)
        std::memcpy(out, srv->lat.data(), n * sizeof(double));
    srv->lat.erase(srv->lat.begin(), srv->lat.begin() + (long)n);
    *n_out = n;
    return TC_OK;
}

tc_status tc_server_step(tc_server *srv, size_t *blocks_done)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_step: server is NULL");
    if (srv->run.load())
        return sfail(TC_ESTATE, "tc_server_step: the worker thread is running");
    std::lock_guard<std::mutex> lk(srv->mu_state);
    S_CU(cudaSetDevice(srv->device));
    size_t n = 0;
    tc_status st = step_locked(srv, &n);
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
    std::lock_guard<std::mutex> lk(srv->mu_state);
    SStream *s = find(srv, id);
    if (!s)
        return sfail(TC_EINVAL, "tc_server_flush: unknown stream");
    const long long tail = s->L - 1;
    if ((long long)cap < tail)
        return sfail(TC_EINVAL, "tc_server_flush: cap < L - 1");
    if (s->flushed)
        return sfail(TC_ESTATE, "tc_server_flush: already flushed");
    S_CU(cudaSetDevice(srv->device));
    // The tail is the output of L - 1 zero samples (the accumulator drained,
    // Sec. 4.2): zero blocks of `block` samples run through ordinary steps
    // (other streams' pending blocks ride along).
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        s->tail_out.clear();
        for (long long off = 0; off < tail; off += s->block) {
            Block b;
            b.x.assign((size_t)std::min<long long>(s->block, tail - off), 0.f);
            b.t_submit = now_s();
            b.tail = true;
            s->pending.push_back(std::move(b));
        }
        s->ended = true;
        s->flushed = true;
    }
    for (;;) {
        {
            std::lock_guard<std::mutex> lq(srv->mu_queue);
            if (s->pending.empty())
                break;
        }
        size_t nb = 0;
        S_TRY(step_locked(srv, &nb));
        if (nb == 0)
            return sfail(TC_ESTATE, "tc_server_flush: internal: a step made no progress");
    }
    if ((long long)s->tail_out.size() != tail)
        return sfail(TC_ESTATE, "tc_server_flush: internal: tail length");
    if (tail > 0)
        std::memcpy(y, s->tail_out.data(), (size_t)tail * sizeof(float));
    s->tail_out.clear();
    s->tail_out.shrink_to_fit();
    if (n_out)
        *n_out = (size_t)tail;
    return TC_OK;
}

tc_status tc_server_remove(tc_server *srv, uint64_t id)
{
    if (!srv)
        return sfail(TC_EINVAL, "tc_server_remove: server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu_state);
    std::unique_ptr<SStream> s;
    {
        std::lock_guard<std::mutex> lq(srv->mu_queue);
        auto it = srv->streams.find(id);
        if (it == srv->streams.end())
            return sfail(TC_EINVAL, "tc_server_remove: unknown stream");
        if (!it->second->pending.empty())
            return sfail(TC_ESTATE, "tc_server_remove: the stream still has blocks queued");
        s = std::move(it->second);
        srv->streams.erase(it);
    }
    cudaSetDevice(srv->device);
    cudaStreamSynchronize(srv->cs);
    free_stream(s.get());
    srv->used -= s->bytes;
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
    return TC_OK;
}

double tc_server_clock(void) { return now_s(); }

}  // extern "C"
