// capi.cu -- implementation of the C ABI in include/taches.h (host code).
//
// Device state of a stream:
//   hist     input history, one row per input channel, float32, row pitch
//            `cap`. Sample n of a row lives at column n - base. The row keeps at
//            least `keep` samples behind the next push, which is L plus one tap
//            chunk. When a push would run past the row end, the kept tail is
//            copied to the row start (one 2-D copy, source and destination
//            disjoint) and base moves.
//   ir       IR slots [slot][set][4 shifted copies][Lpad] for K1.
//   vt       version table: (first sample, slot) per live IR version
//            (abstract, Sec. 6: a new IR is used for the next samples).
//   partial  K1 scratch for tap-chunk partial sums, plus ticket counters.
//   hist_hi/lo, Toeplitz tiles, K-part partials: the tensor-core paths (K2 for
//            shared-IR groups and mono BF16 streams, K3 for MIMO).
// The kernels run on one CUDA stream per tc_stream, in call order, so a slot
// or table entry is never overwritten while an earlier kernel may read it.
// Asynchronous pushes from page-locked host buffers add a copy stream (and an
// IR-upload stream), ordered against the kernels with events.
#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/taches.h"
#include "tc_internal.h"

namespace {

thread_local std::string g_err;

tc_status fail(tc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define TC_CU(call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA, "%s: %s", #call,     \
                        cudaGetErrorString(e_));                                                      \
    } while (0)

// Stream-ordered allocations back TMA tensor maps and 16-byte stores; the
// kernels need at least 16-byte alignment, and 256 is what is checked.
#define TC_ALIGNED(ptr)                                                                     \
    do {                                                                                    \
        if ((reinterpret_cast<uintptr_t>(ptr) & 255u) != 0)                                 \
            return fail(TC_ECUDA, "internal: a stream-ordered allocation is not 256-byte aligned"); \
    } while (0)

#define TC_TRY(expr)                 \
    do {                             \
        tc_status st_ = (expr);      \
        if (st_ != TC_OK)            \
            return st_;              \
    } while (0)

long long round_up(long long a, long long m) { return (a + m - 1) / m * m; }
long long floor8(long long a) { return a >= 0 ? (a & ~7LL) : -(((-a) + 7) & ~7LL); }

constexpr int kMaxVersions = 16;

struct Version {
    long long start;
    int slot;
    long long ramp;  // crossfade from the previous version over this many samples (1: hard switch)
};

// Device copy of the version table.
struct DevTable {
    long long vstart[kMaxVersions];
    int vslot[kMaxVersions];
    int vramp[kMaxVersions];
    int nver;
};

enum Kind { KIND_GROUP = 0, KIND_MIMO = 1 };
enum State { ST_OPEN = 0, ST_ENDED = 1, ST_FLUSHED = 2 };

}  // namespace

namespace tc {
// Lets other translation units of the library report through tc_last_error().
void set_last_error(const char *msg) { g_err = msg ? msg : ""; }
}  // namespace tc

struct tc_stream {
    // Shape.
    int kind = KIND_GROUP;
    size_t rows = 1;   // history rows (channels, or MIMO inputs)
    size_t items = 1;  // output rows (channels, or MIMO outputs)
    size_t nin = 1;    // inputs summed per output row
    size_t nsets = 1;  // IR rows per version
    size_t L = 0, block = 0, max_push = 0;
    int shared_ir = 0;
    tc_precision prec = TC_FP32;
    int device = 0;

    cudaStream_t own_cs = nullptr;
    cudaStream_t cs = nullptr;

    // Stream state.
    long long pos = 0;
    long long base = 0;
    int state = ST_OPEN;
    long long pos_end_hint = -1;  // number of real input samples (set at flush), for MAC counting

    // History.
    float *hist = nullptr;
    long long cap = 0;
    long long keep = 0;

    // IR slots.
    int nslots = 4;
    long long Lpad = 0;
    float *ir = nullptr;
    float *ir_stage = nullptr;  // device staging for host IR uploads [nsets][L]
    float *pin_ir = nullptr;    // pinned staging [nsets][L]
    cudaEvent_t ev_ir = nullptr;
    bool ir_ever_set = false;

    // Versions.
    std::vector<Version> vt;
    std::vector<char> slot_used;
    DevTable *d_vt = nullptr;
    DevTable *pin_vt = nullptr;
    cudaEvent_t ev_vt = nullptr;
    bool vt_dirty = false;
    long long next_ramp = 1;  // crossfade length of the next IR switches (tc_set_crossfade)

    // Host-pointer staging.
    float *pin_x = nullptr;   // [rows][max_push]
    float *pin_y = nullptr;   // [items][max_push]
    float *d_y = nullptr;     // [items][max_push]
    cudaEvent_t ev_x = nullptr;
    int *pin_err = nullptr;

    // Asynchronous pushes from page-locked host buffers (tc_push mode 2): a
    // copy stream moves the inputs into two device staging slots and the
    // outputs back, so the copies of one push overlap the kernels of its
    // neighbours. Created on the first such push.
    cudaStream_t ccs = nullptr;
    cudaStream_t ics = nullptr;         // page-locked IR uploads beside the asynchronous pushes
    cudaEvent_t ev_ir_prep = nullptr;   // the last IR prep (last reader of the IR staging rows) ran
    float *d_xs[2] = {nullptr, nullptr};
    float *d_ys[2] = {nullptr, nullptr};
    cudaEvent_t ev_xs_ready[2] = {}, ev_xs_free[2] = {}, ev_ys_ready[2] = {}, ev_ys_free[2] = {};
    int aslot = 0;

    // K1 scratch: chunk sums of every tile and one ticket per tile.
    float *partial = nullptr;
    size_t partial_floats = 0;
    unsigned *counter = nullptr;
    size_t counter_n = 0;
    int *d_err = nullptr;
    int k1_variant_fixed = -1;  // -1: chosen per launch
    long long k2_range = -1;    // K blocks per tensor-core CTA range (-1: by precision)
    int k2_nsplit = -1;         // K parts per K2 tile (-1: planned from the waves)
    bool k2_fold = true;        // K parts added inside K2 (false: a k2_reduce launch)
    int k2_order = 2;           // unit order of the persistent CTA pairs (K2Params::order)
    int k2_mode = 2;  // plain BF16: 0 one channel tile per CTA, 1 two per CTA, 2 persistent CTA pairs,
                      // 3 CTA pairs launched per unit (tuning knob)
    bool zero_skip = false;      // K1 zero gating (tuning knob)

    // BF16 tensor-core path (shared-IR groups): bf16 hi/lo histories and, per
    // IR slot and alignment shift delta, the materialised Toeplitz tiles.
    void *hist_hi = nullptr;
    void *hist_lo = nullptr;
    CUtensorMap mx_hi{}, mx_lo{};
    struct TSet {
        bool ready = false;
        long long nkb = 0;
        void *thi = nullptr, *tlo = nullptr;
        CUtensorMap mt_hi{}, mt_lo{};
        CUtensorMap mt2_hi{}, mt2_lo{};  // the same tiles in boxes of 128 rows (half a tile: CTA pairs)
    };
    std::vector<std::array<TSet, 8>> tsets;  // [slot][delta]
    float *k2_partial = nullptr;
    size_t k2_partial_floats = 0;
    unsigned *k2_ticket = nullptr;  // after the partials in the same allocation: K-part tickets
    size_t k2_ticket_n = 0;
    long long k2_launches = 0, k1_fallbacks = 0;

    // BF16 tensor-core path for MIMO (K3): reversed bf16 hi/lo inputs of a
    // launch and, per IR slot, the phase-shifted IR tiles of every pair.
    void *xr_hi = nullptr, *xr_lo = nullptr;
    long long xr_pitch = 0;
    int k3_nkbp = 0;
    struct K3Set {
        bool ready = false;
        void *bh = nullptr, *bl = nullptr;
        CUtensorMap mb_hi{}, mb_lo{};
    };
    std::vector<K3Set> k3sets;  // [slot]
    float *k3_partial = nullptr;
    size_t k3_partial_floats = 0;

    // Kernel timing (tc_profile).
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;   // pairs (start, stop)
    size_t ev_used = 0;                 // events in use, even
    double prof_macs = 0.0;
    uint64_t prof_launches = 0;
};

namespace {

tc_status check_stream(const tc_stream *s)
{
    if (!s)
        return fail(TC_EINVAL, "stream is NULL");
    return TC_OK;
}

tc_status use_device(const tc_stream *s)
{
    int cur = -1;
    TC_CU(cudaGetDevice(&cur));
    if (cur != s->device)
        TC_CU(cudaSetDevice(s->device));
    return TC_OK;
}

void free_all(tc_stream *s)
{
    if (s->ccs) {
        cudaStreamSynchronize(s->ccs);
        for (int k = 0; k < 2; ++k) {
            cudaFree(s->d_xs[k]);
            cudaFree(s->d_ys[k]);
            for (cudaEvent_t e : {s->ev_xs_ready[k], s->ev_xs_free[k], s->ev_ys_ready[k], s->ev_ys_free[k]})
                if (e)
                    cudaEventDestroy(e);
        }
        cudaStreamDestroy(s->ccs);
        s->ccs = nullptr;
    }
    if (s->ics) {
        cudaStreamSynchronize(s->ics);
        cudaStreamDestroy(s->ics);
        s->ics = nullptr;
    }
    if (s->ev_ir_prep) {
        cudaEventDestroy(s->ev_ir_prep);
        s->ev_ir_prep = nullptr;
    }
    if (s->cs)
        cudaStreamSynchronize(s->cs);
    cudaFree(s->hist);
    cudaFree(s->ir);
    cudaFree(s->ir_stage);
    cudaFree(s->d_vt);
    cudaFree(s->d_y);
    cudaFree(s->partial);
    cudaFree(s->hist_hi);
    cudaFree(s->hist_lo);
    cudaFree(s->k2_partial);
    for (auto &arr : s->tsets)
        for (auto &t : arr) {
            cudaFree(t.thi);
            cudaFree(t.tlo);
        }
    cudaFree(s->xr_hi);
    cudaFree(s->xr_lo);
    for (auto &k : s->k3sets) {
        cudaFree(k.bh);
        cudaFree(k.bl);
    }
    cudaFree(s->k3_partial);
    cudaFree(s->counter);
    cudaFree(s->d_err);
    cudaFreeHost(s->pin_ir);
    cudaFreeHost(s->pin_vt);
    cudaFreeHost(s->pin_x);
    cudaFreeHost(s->pin_y);
    cudaFreeHost(s->pin_err);
    if (s->ev_ir)
        cudaEventDestroy(s->ev_ir);
    if (s->ev_vt)
        cudaEventDestroy(s->ev_vt);
    if (s->ev_x)
        cudaEventDestroy(s->ev_x);
    for (cudaEvent_t e : s->ev_pool)
        cudaEventDestroy(e);
    if (s->own_cs)
        cudaStreamDestroy(s->own_cs);
}

// True when p is page-locked host memory (cudaHostAlloc, cudaHostRegister, or
// a pinned torch tensor): the copy engines read and write it directly, so the
// host-pointer calls skip their staging copy through the stream's own pinned
// buffers.
bool pinned_host(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // pageable memory on older drivers: clear the error
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

tc_status alloc_ir(tc_stream *s)
{
    if (s->ir) {
        TC_CU(cudaStreamSynchronize(s->cs));
        TC_CU(cudaFree(s->ir));
        s->ir = nullptr;
    }
    const size_t floats = (size_t)s->nslots * s->nsets * 4 * (size_t)s->Lpad;
    TC_CU(cudaMalloc(&s->ir, floats * sizeof(float)));
    TC_CU(cudaMemsetAsync(s->ir, 0, floats * sizeof(float), s->cs));
    s->slot_used.assign((size_t)s->nslots, 0);
    for (auto &arr : s->tsets)
        for (auto &t : arr) {
            cudaFree(t.thi);
            cudaFree(t.tlo);
        }
    s->tsets.assign((size_t)s->nslots, std::array<tc_stream::TSet, 8>{});
    return TC_OK;
}

tc_status clear_state(tc_stream *s)
{
    s->pos = 0;
    s->base = -s->keep;
    s->state = ST_OPEN;
    s->pos_end_hint = -1;
    s->vt.clear();
    std::fill(s->slot_used.begin(), s->slot_used.end(), 0);
    s->vt_dirty = true;
    s->next_ramp = 1;
    s->ir_ever_set = false;
    TC_CU(cudaMemsetAsync(s->hist, 0, (size_t)s->rows * s->cap * sizeof(float), s->cs));
    if (s->hist_hi) {
        TC_CU(cudaMemsetAsync(s->hist_hi, 0, (size_t)s->rows * s->cap * 2, s->cs));
        TC_CU(cudaMemsetAsync(s->hist_lo, 0, (size_t)s->rows * s->cap * 2, s->cs));
    }
    for (auto &arr : s->tsets)
        for (auto &t : arr)
            t.ready = false;
    for (auto &k : s->k3sets)
        k.ready = false;
    TC_CU(cudaMemsetAsync(s->counter, 0, s->counter_n * sizeof(unsigned), s->cs));
    if (s->k2_ticket)
        TC_CU(cudaMemsetAsync(s->k2_ticket, 0, s->k2_ticket_n * sizeof(unsigned), s->cs));
    TC_CU(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->cs));
    return TC_OK;
}

tc_status open_common(tc_stream *s)
{
    TC_CU(cudaGetDevice(&s->device));
    TC_CU(cudaStreamCreateWithFlags(&s->own_cs, cudaStreamNonBlocking));
    s->cs = s->own_cs;
    TC_CU(cudaEventCreateWithFlags(&s->ev_ir, cudaEventDisableTiming));
    TC_CU(cudaEventCreateWithFlags(&s->ev_vt, cudaEventDisableTiming));
    TC_CU(cudaEventCreateWithFlags(&s->ev_x, cudaEventDisableTiming));

    // History row: `keep` samples behind the next push (L taps plus the
    // largest tap chunk and alignment), the push itself, and one output tile
    // of overrun. Doubled so that a compaction copy never overlaps itself.
    s->keep = round_up((long long)s->L + tc::K1_KC_MAX + 16, 8);
    s->cap = round_up(2 * s->keep + (long long)s->max_push + 512 + 160, 64);
    TC_CU(cudaMalloc(&s->hist, (size_t)s->rows * s->cap * sizeof(float)));

    s->Lpad = round_up((long long)s->L + 4 + tc::K1_KC_MAX, 4);
    TC_TRY(alloc_ir(s));
    TC_CU(cudaMalloc(&s->ir_stage, s->nsets * s->L * sizeof(float)));
    TC_CU(cudaHostAlloc(&s->pin_ir, s->nsets * s->L * sizeof(float), cudaHostAllocDefault));

    TC_CU(cudaMalloc(&s->d_vt, sizeof(DevTable)));
    TC_CU(cudaHostAlloc(&s->pin_vt, sizeof(DevTable), cudaHostAllocDefault));
    std::memset(s->pin_vt, 0, sizeof(DevTable));

    TC_CU(cudaHostAlloc(&s->pin_x, s->rows * s->max_push * sizeof(float), cudaHostAllocDefault));
    TC_CU(cudaHostAlloc(&s->pin_y, s->items * s->max_push * sizeof(float), cudaHostAllocDefault));
    TC_CU(cudaMalloc(&s->d_y, s->items * s->max_push * sizeof(float)));
    TC_CU(cudaHostAlloc(&s->pin_err, sizeof(int), cudaHostAllocDefault));
    *s->pin_err = 0;

    // Chunk sums of every tile of the largest launch, one ticket per tile.
    const long long max_tiles = (long long)s->items * (((long long)s->max_push + tc::K1_MO - 1) / tc::K1_MO);
    s->counter_n = (size_t)max_tiles;
    s->partial_floats = (size_t)tc::k1_partial_floats_max((long long)s->L, (int)s->nin, max_tiles);
    TC_CU(cudaMalloc(&s->partial, s->partial_floats * sizeof(float)));
    TC_CU(cudaMalloc(&s->counter, s->counter_n * sizeof(unsigned)));
    TC_CU(cudaMalloc(&s->d_err, sizeof(int)));
    if (s->prec != TC_FP32 && s->kind == KIND_MIMO) {
        // K3 reads reversed bf16 copies of the inputs, made per launch.
        s->k3_nkbp = tc::k3_kblocks_per_input((long long)s->L);
        const int tp = tc::k3_tiles_per_cta();
        const int ntile_max = (int)((s->max_push + 1023) / 1024 + tp - 1) / tp * tp;
        s->xr_pitch = round_up(tc::k3_xr_span(ntile_max, s->k3_nkbp), 64);
        TC_CU(cudaMalloc(&s->xr_hi, (size_t)s->nin * s->xr_pitch * 2));
        TC_CU(cudaMalloc(&s->xr_lo, (size_t)s->nin * s->xr_pitch * 2));
        s->k3sets.assign((size_t)s->nslots, tc_stream::K3Set{});
    } else if (s->prec != TC_FP32) {
        TC_CU(cudaMalloc(&s->hist_hi, (size_t)s->rows * s->cap * 2));
        TC_CU(cudaMalloc(&s->hist_lo, (size_t)s->rows * s->cap * 2));
        const int kbs = tc::k2_kblock(s->prec == TC_BF16 ? 1 : 3);
        TC_CU(tc::encode_bf16_2d(&s->mx_hi, s->hist_hi, (unsigned long long)s->cap, s->rows,
                                 (unsigned long long)s->cap * 2, kbs, tc::k2_tile_m()));
        TC_CU(tc::encode_bf16_2d(&s->mx_lo, s->hist_lo, (unsigned long long)s->cap, s->rows,
                                 (unsigned long long)s->cap * 2, kbs, tc::k2_tile_m()));
    }
    TC_TRY(clear_state(s));
    TC_CU(cudaStreamSynchronize(s->cs));
    return TC_OK;
}

tc_status open_any(int kind, size_t rows, size_t items, size_t nin, size_t nsets, size_t L, size_t block,
                   int shared_ir, tc_precision prec, size_t max_push, tc_stream **out)
{
    if (!out)
        return fail(TC_EINVAL, "out is NULL");
    *out = nullptr;
    if (L == 0 || block == 0 || rows == 0 || items == 0)
        return fail(TC_EINVAL, "L, block and channel counts must be > 0");
    if (max_push == 0)
        max_push = block;
    if (max_push < block)
        return fail(TC_EINVAL, "max_push (%zu) < block (%zu)", max_push, block);
    if (L > (size_t)1 << 30 || max_push > (size_t)1 << 28 || rows > (size_t)1 << 20)
        return fail(TC_EINVAL, "size out of range");
    if (prec != TC_FP32 && prec != TC_BF16 && prec != TC_BF16_SPLIT)
        return fail(TC_EINVAL, "unknown precision %d", (int)prec);
    if (prec != TC_FP32 && kind == KIND_GROUP && !shared_ir)
        return fail(TC_EUNSUPPORTED, "the BF16 tensor-core path needs one IR shared by all channels");
    if (prec != TC_FP32 && kind == KIND_MIMO && items > 16)
        return fail(TC_EUNSUPPORTED, "the BF16 tensor-core MIMO path takes at most 16 outputs");
    tc_stream *s = new (std::nothrow) tc_stream();
    if (!s)
        return fail(TC_ENOMEM, "host allocation failed");
    s->kind = kind;
    s->rows = rows;
    s->items = items;
    s->nin = nin;
    s->nsets = nsets;
    s->L = L;
    s->block = block;
    s->max_push = max_push;
    s->shared_ir = shared_ir;
    s->prec = prec;
    tc_status st = open_common(s);
    if (st != TC_OK) {
        std::string msg = g_err;
        free_all(s);
        delete s;
        g_err = msg;
        return st;
    }
    *out = s;
    return TC_OK;
}

// Drops versions whose samples can no longer reach a future output: version v
// is dead once the next version starts at or before pos - L + 1.
void retire_versions(tc_stream *s)
{
    const long long oldest_needed = s->pos - (long long)s->L + 1;
    size_t drop = 0;
    // Version i is dead once version i + 1 has fully taken over (its ramp
    // ended) before the oldest sample a future output reads.
    while (drop + 1 < s->vt.size() && s->vt[drop + 1].start + s->vt[drop + 1].ramp - 1 <= oldest_needed)
        ++drop;
    for (size_t i = 0; i < drop; ++i)
        s->slot_used[(size_t)s->vt[i].slot] = 0;
    if (drop) {
        s->vt.erase(s->vt.begin(), s->vt.begin() + (long)drop);
        s->vt_dirty = true;
    }
}

tc_status upload_table(tc_stream *s)
{
    if (!s->vt_dirty)
        return TC_OK;
    TC_CU(cudaEventSynchronize(s->ev_vt));  // the previous upload has read the mirror
    DevTable &t = *s->pin_vt;
    std::memset(&t, 0, sizeof t);
    t.nver = (int)s->vt.size();
    for (size_t i = 0; i < s->vt.size(); ++i) {
        t.vstart[i] = s->vt[i].start;
        t.vslot[i] = s->vt[i].slot;
        t.vramp[i] = (int)s->vt[i].ramp;
    }
    TC_CU(cudaMemcpyAsync(s->d_vt, &t, sizeof t, cudaMemcpyHostToDevice, s->cs));
    TC_CU(cudaEventRecord(s->ev_vt, s->cs));
    s->vt_dirty = false;
    return TC_OK;
}

tc_status set_ir_impl(tc_stream *s, const float *h, size_t n, long long sample, bool rows_given,
                      bool on_device)
{
    tc::Range nvtx_range("tc set_ir");
    TC_TRY(check_stream(s));
    if (!h)
        return fail(TC_EINVAL, "h is NULL");
    if (n == 0 || n > s->L)
        return fail(TC_EINVAL, "IR length %zu not in [1, L=%zu]", n, s->L);
    if (s->state != ST_OPEN)
        return fail(TC_ESTATE, "stream has ended; reset it first");
    if (sample < s->pos)
        return fail(TC_EINVAL, "IR switch at sample %lld is before the next sample to push (%lld)", sample,
                    s->pos);
    if (!s->vt.empty() && sample < s->vt.back().start)
        return fail(TC_EINVAL, "IR switch at sample %lld is before the latest version (%lld)", sample,
                    s->vt.back().start);
    if (!s->vt.empty() && sample != s->vt.back().start && s->vt.size() > 1 &&
        sample < s->vt.back().start + s->vt.back().ramp - 1)
        return fail(TC_EINVAL, "IR switch at sample %lld starts before the crossfade to the latest version ends (%lld)",
                    sample, s->vt.back().start + s->vt.back().ramp - 1);
    TC_TRY(use_device(s));
    retire_versions(s);

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
            return fail(TC_ENOMEM,
                        "all %d IR slots hold live versions (a version stays live until L-1 samples after the "
                        "next one starts); raise tc_set_max_versions",
                        s->nslots);
    }

    // Source rows: [nsets][n]. A single host IR is replicated to every set.
    const size_t sets = s->nsets;
    const float *src = h;
    long long src_pitch = (long long)n;
    if (!on_device && pinned_host(h)) {
        // Page-locked h: one copy straight into the staging rows, waited for so
        // that h is free when the call returns.
        const size_t cnt = (rows_given ? sets : 1) * n * sizeof(float);
        if (s->ics) {
            // Beside asynchronous pushes: the copy waits only for the previous
            // IR's prep (the last reader of the staging rows), not for the
            // pushes enqueued since, and the prep waits for the copy.
            TC_CU(cudaStreamWaitEvent(s->ics, s->ev_ir_prep, 0));
            TC_CU(cudaMemcpyAsync(s->ir_stage, h, cnt, cudaMemcpyHostToDevice, s->ics));
            TC_CU(cudaEventRecord(s->ev_ir, s->ics));
            TC_CU(cudaEventSynchronize(s->ev_ir));
            TC_CU(cudaStreamWaitEvent(s->cs, s->ev_ir, 0));
        } else {
            TC_CU(cudaMemcpyAsync(s->ir_stage, h, cnt, cudaMemcpyHostToDevice, s->cs));
            TC_CU(cudaEventRecord(s->ev_ir, s->cs));
            TC_CU(cudaEventSynchronize(s->ev_ir));
        }
        if (!rows_given)
            src_pitch = 0;
        src = s->ir_stage;
    } else if (!on_device) {
        TC_CU(cudaEventSynchronize(s->ev_ir));
        if (rows_given) {
            std::memcpy(s->pin_ir, h, sets * n * sizeof(float));
            TC_CU(cudaMemcpyAsync(s->ir_stage, s->pin_ir, sets * n * sizeof(float), cudaMemcpyHostToDevice,
                                  s->cs));
        } else {
            std::memcpy(s->pin_ir, h, n * sizeof(float));
            TC_CU(cudaMemcpyAsync(s->ir_stage, s->pin_ir, n * sizeof(float), cudaMemcpyHostToDevice, s->cs));
            src_pitch = 0;  // every set reads row 0
        }
        TC_CU(cudaEventRecord(s->ev_ir, s->cs));
        src = s->ir_stage;
    }
    for (auto &t : s->tsets[(size_t)slot])
        t.ready = false;  // the slot gets a new IR: its Toeplitz tiles are stale
    if ((size_t)slot < s->k3sets.size())
        s->k3sets[(size_t)slot].ready = false;
    float *dst = s->ir + (size_t)slot * sets * 4 * (size_t)s->Lpad;
    TC_CU(tc::ir_prep_launch(src, src_pitch, (long long)n, (int)sets, dst, 4 * s->Lpad, s->Lpad, s->Lpad, s->cs));
    if (s->ev_ir_prep)
        TC_CU(cudaEventRecord(s->ev_ir_prep, s->cs));

    if (!replace) {
        s->vt.push_back(Version{sample, slot, s->vt.empty() ? 1 : s->next_ramp});
        s->slot_used[(size_t)slot] = 1;
    } else if (s->vt.size() > 1) {
        s->vt.back().ramp = s->next_ramp;
    }
    s->vt_dirty = true;
    s->ir_ever_set = true;
    return TC_OK;
}

// Makes room in the history rows for n more samples (plus tile overrun).
// Mono tensor-core streams read up to 256 + 31 samples past a push (the last
// 256-sample row of K2's row view): keep that much more room after it.
long long room_extra(const tc_stream *s) { return (s->rows == 1 && s->prec != TC_FP32) ? 512 : 0; }

tc_status ensure_room(tc_stream *s, long long n)
{
    if (s->pos + n + tc::K1_MO + 8 <= s->base + s->cap)
        return TC_OK;
    const long long nb = floor8(s->pos - s->keep);
    const long long len = s->pos - nb;
    const long long shift = nb - s->base;
    if (shift < len || len + n + tc::K1_MO + 8 > s->cap)
        return fail(TC_EINVAL, "internal: history compaction would overlap");
    TC_CU(cudaMemcpy2DAsync(s->hist, (size_t)s->cap * sizeof(float), s->hist + shift,
                            (size_t)s->cap * sizeof(float), (size_t)len * sizeof(float), s->rows,
                            cudaMemcpyDeviceToDevice, s->cs));
    if (s->hist_hi) {
        for (void *hb : {s->hist_hi, s->hist_lo}) {
            if (hb == s->hist_lo && s->prec == TC_BF16)
                continue;  // plain BF16 never reads the lo history
            char *b = static_cast<char *>(hb);
            TC_CU(cudaMemcpy2DAsync(b, (size_t)s->cap * 2, b + shift * 2, (size_t)s->cap * 2, (size_t)len * 2,
                                    s->rows, cudaMemcpyDeviceToDevice, s->cs));
        }
    }
    s->base = nb;
    return TC_OK;
}

// bf16 hi/lo split of history columns [col0, col0 + n) (BF16 streams only).
tc_status split_new(tc_stream *s, long long col0, long long n)
{
    if (!s->hist_hi)
        return TC_OK;
    TC_CU(tc::k2_split_launch(s->hist, s->cap, (int)s->rows, col0, n, s->hist_hi,
                              s->prec == TC_BF16 ? nullptr : s->hist_lo, s->cs));  // plain BF16 reads hi only
    return TC_OK;
}

tc_status prof_begin(tc_stream *s)
{
    if (!s->profile)
        return TC_OK;
    while (s->ev_pool.size() < s->ev_used + 2) {
        cudaEvent_t e;
        TC_CU(cudaEventCreate(&e));
        s->ev_pool.push_back(e);
    }
    TC_CU(cudaEventRecord(s->ev_pool[s->ev_used], s->cs));
    return TC_OK;
}

tc_status prof_end(tc_stream *s, long long t0, long long nout)
{
    if (!s->profile)
        return TC_OK;
    TC_CU(cudaEventRecord(s->ev_pool[s->ev_used + 1], s->cs));
    s->ev_used += 2;
    // Useful multiply-adds: output m sees the taps k < L with 0 <= m - k < n_end,
    // where n_end is the number of real input samples (all pushed samples
    // before a flush, the end of the input during one).
    const long long n_end = s->pos_end_hint >= 0 ? s->pos_end_hint : t0 + nout;
    double macs = 0.0;
    for (long long m = t0; m < t0 + nout; ++m) {
        const long long hi = std::min<long long>(m, (long long)s->L - 1);
        const long long lo = std::max<long long>(0, m - n_end + 1);
        if (hi >= lo)
            macs += (double)(hi - lo + 1);
    }
    s->prof_macs += macs * (double)s->items * (double)s->nin;
    s->prof_launches += 1;
    return TC_OK;
}

// TC_CHECK_LAUNCH=1 in the environment (read per launch): before each K1
// launch, the host checks the ranges the kernel will touch against the
// stream's buffers, and a launch that would leave them returns TC_EINVAL
// instead of running. The staged window of output tile i and tap chunk c
// starts at n_lo = t0 + 128 i - (KC c - e) - KC + 1 and holds KC + 128
// samples; it grows with i and shrinks with c, so the extreme windows are
// (tile 0, last chunk) and (last tile, chunk 0).
bool check_launches()
{
    const char *e = std::getenv("TC_CHECK_LAUNCH");
    return e && e[0] == '1';
}

tc_status check_k1_launch(const tc_stream *s, const tc::K1Params &p, const tc::K1Plan &plan)
{
    const long long KC = tc::k1_chunk_taps(plan.variant);
    const long long first = p.t0 - ((long long)(plan.nchunk - 1) * KC - p.e) - KC + 1;
    const long long last_end = p.t0 + (long long)(p.ntile - 1) * tc::K1_MO + p.e + 1 + tc::K1_MO;
    if ((first - p.base) % 4 != 0)
        return fail(TC_EINVAL, "launch check: staged window at %lld is not 16-byte aligned (base %lld)", first,
                    p.base);
    if (first < p.base || last_end > p.base + p.pitch)
        return fail(TC_EINVAL, "launch check: windows [%lld, %lld) leave the history [%lld, %lld)", first, last_end,
                    p.base, p.base + p.pitch);
    if ((long long)plan.nchunk * KC > s->Lpad || p.e < 0 || p.e > 3)
        return fail(TC_EINVAL, "launch check: %d chunks of %lld taps leave the IR slot of %lld", plan.nchunk, KC,
                    s->Lpad);
    const long long rows = (long long)(p.nitems - 1) * p.x_item_rows + (long long)(p.nin - 1) * p.x_in_rows + 1;
    if (rows > (long long)s->rows)
        return fail(TC_EINVAL, "launch check: %lld history rows of %zu", rows, s->rows);
    if ((long long)p.nout > p.y_pitch && p.nitems > 1)
        return fail(TC_EINVAL, "launch check: output rows of %d samples at pitch %lld", p.nout, p.y_pitch);
    for (const Version &v : s->vt)
        if (v.slot < 0 || v.slot >= s->nslots)
            return fail(TC_EINVAL, "launch check: version slot %d of %d", v.slot, s->nslots);
    if ((size_t)p.nitems * p.ntile > s->counter_n || (size_t)plan.ctas * tc::K1_MO > s->partial_floats)
        return fail(TC_EINVAL, "launch check: K1 scratch too small");
    return TC_OK;
}

tc_status launch_k1(tc_stream *s, long long t0, long long nout, float *y, long long y_pitch)
{
    tc::K1Params p{};
    p.hist = s->hist;
    p.pitch = s->cap;
    p.base = s->base;
    const bool mimo = s->kind == KIND_MIMO;
    p.x_item_rows = mimo ? 0 : 1;
    p.x_in_rows = mimo ? 1 : 0;
    p.ir = s->ir;
    p.ir_slot = (long long)s->nsets * 4 * s->Lpad;
    p.ir_item = s->shared_ir ? 0 : (mimo ? (long long)s->nin * 4 * s->Lpad : 4 * s->Lpad);
    p.ir_in = mimo ? 4 * s->Lpad : 0;
    p.ir_phase = s->Lpad;
    p.L = (int)s->L;
    p.vstart = s->d_vt->vstart;
    p.vslot = s->d_vt->vslot;
    p.nver = &s->d_vt->nver;
    // The ramp table only when a live version crossfades (hard switches read
    // no ramps on the device).
    bool ramps = false;
    for (const Version &v : s->vt)
        ramps = ramps || v.ramp > 1;
    p.vramp = ramps ? s->d_vt->vramp : nullptr;
    p.vt_item = 0;
    p.nitems = (int)s->items;
    p.nin = (int)s->nin;
    p.t0 = t0;
    p.nout = (int)nout;
    p.ntile = (int)((nout + tc::K1_MO - 1) / tc::K1_MO);
    p.e = tc::k1_shift_e(t0, s->base);
    tc::K1Plan plan{};
    TC_CU(tc::k1_plan((long long)s->L, p.e, p.nin, p.nitems, p.ntile, s->k1_variant_fixed, &plan));
    p.y = y;
    p.y_pitch = y_pitch;
    p.partial = s->partial;
    p.counter = s->counter;
    p.err = s->d_err;
    p.zero_skip = s->zero_skip ? 1 : 0;
    if (s->pos_end_hint >= 0) {  // a flush: the input ended at pos_end_hint
        p.has_end = 1;
        p.x_end = s->pos_end_hint;
    }
    if ((size_t)p.nitems * p.ntile > s->counter_n ||
        (size_t)plan.ctas * tc::K1_MO > s->partial_floats)
        return fail(TC_EINVAL, "internal: K1 scratch too small");
    if (check_launches())
        TC_TRY(check_k1_launch(s, p, plan));
    TC_TRY(prof_begin(s));
    TC_CU(tc::k1_launch(p, plan, s->cs));
    return prof_end(s, t0, nout);
}

// K parts per K2 tile: the fewest (up to 64, k2_reduce's tree, each at least
// 16 K blocks long) that fill the GPU's waves to >= 90 %, so that a small
// launch (one serving step of one group) spreads over the GPU.
long long k2_plan_nsplit(long long tiles, long long nkb, int sms)
{
    long long nsplit = 1;
    double best = 0.0;
    for (long long ns = 1; ns <= 64 && ns <= nkb && (ns == 1 || nkb / ns >= 16); ++ns) {
        const long long units = tiles * ns;
        const double eff = (double)units / (double)(((units + sms - 1) / sms) * sms);
        if (eff > best + 1e-9) {
            best = eff;
            nsplit = ns;
        }
        if (eff >= 0.9)
            break;
    }
    const long long kb_per = (nkb + nsplit - 1) / nsplit;
    return (nkb + kb_per - 1) / kb_per;
}

// K-part partials of `floats` floats, followed by the tickets of the parts
// folded inside the kernel (one per 128 x 256 tile and warp slice: at most
// floats / 4096), zeroed in stream order.
tc_status k2_partial_alloc(tc_stream *s, size_t floats)
{
    const size_t tickets = floats / 4096 + 8;
    if (s->k2_partial)
        cudaFreeAsync(s->k2_partial, s->cs);  // after the launches that used it
    s->k2_partial = nullptr;
    s->k2_ticket = nullptr;
    s->k2_partial_floats = s->k2_ticket_n = 0;
    TC_CU(tc::pool_alloc(reinterpret_cast<void **>(&s->k2_partial), floats * sizeof(float) + tickets * sizeof(unsigned),
                         s->cs));
    TC_ALIGNED(s->k2_partial);
    s->k2_ticket = reinterpret_cast<unsigned *>(s->k2_partial + floats);
    TC_CU(cudaMemsetAsync(s->k2_ticket, 0, tickets * sizeof(unsigned), s->cs));
    s->k2_partial_floats = floats;
    s->k2_ticket_n = tickets;
    return TC_OK;
}

// K2 on the tensor cores when every input sample of the launch's window
// spawned its tache with the same IR version; false in *used otherwise.
// Buffers (and tensor maps) of the Toeplitz tiles of IR slot `slot` at shift
// `delta`, with room for nkb K blocks; allocated once (stream-ordered: no host
// or device-wide synchronisation while pushes are in flight).
tc_status ensure_tset_mem(tc_stream *s, int slot, int delta, long long nkb)
{
    const int TN = tc::k2_tile_n(), KB = tc::k2_kblock(s->prec == TC_BF16 ? 1 : 3);
    tc_stream::TSet &ts = s->tsets[(size_t)slot][(size_t)delta];
    if (ts.thi && ts.nkb >= nkb)
        return TC_OK;
    if (ts.thi)
        cudaFreeAsync(ts.thi, s->cs);
    if (ts.tlo)
        cudaFreeAsync(ts.tlo, s->cs);
    ts.thi = ts.tlo = nullptr;
    ts.ready = false;
    const size_t bytes = (size_t)nkb * TN * KB * 2;
    TC_CU(tc::pool_alloc(&ts.thi, bytes, s->cs));
    TC_ALIGNED(ts.thi);
    ts.nkb = nkb;
    TC_CU(tc::encode_bf16_2d(&ts.mt_hi, ts.thi, (unsigned long long)KB, (unsigned long long)nkb * TN,
                             (unsigned long long)KB * 2, KB, TN));
    if (s->prec != TC_BF16) {  // plain BF16 reads only the hi tiles
        TC_CU(tc::pool_alloc(&ts.tlo, bytes, s->cs));
        TC_ALIGNED(ts.tlo);
        TC_CU(tc::encode_bf16_2d(&ts.mt_lo, ts.tlo, (unsigned long long)KB, (unsigned long long)nkb * TN,
                                 (unsigned long long)KB * 2, KB, TN));
        TC_CU(tc::encode_bf16_2d(&ts.mt2_lo, ts.tlo, (unsigned long long)KB, (unsigned long long)nkb * TN,
                                 (unsigned long long)KB * 2, KB, TN / 2));
    }
    TC_CU(tc::encode_bf16_2d(&ts.mt2_hi, ts.thi, (unsigned long long)KB, (unsigned long long)nkb * TN,
                             (unsigned long long)KB * 2, KB, TN / 2));
    return TC_OK;
}

tc_status launch_k2(tc_stream *s, long long t0, long long nout, float *y, long long y_pitch, bool *used)
{
    *used = false;
    const long long L = (long long)s->L;
    const int delta = (int)((((t0 - L + 1 - s->base) % 8) + 8) % 8);
    const long long w0 = t0 - L + 1 - delta;
    const int TN = tc::k2_tile_n(), TM = tc::k2_tile_m(), KB = tc::k2_kblock(s->prec == TC_BF16 ? 1 : 3);
    const long long nkb = tc::k2_nkb(L, delta, KB);
    const long long ntile_o = (nout + TN - 1) / TN;
    const long long hi = w0 + (ntile_o - 1) * TN + nkb * KB;  // past the last sample read
    // Single version over [max(w0, first start), hi)?
    int v = -1;
    for (size_t i = 0; i < s->vt.size(); ++i)
        if (s->vt[i].start <= std::max(w0, s->vt.front().start))
            v = (int)i;
    if (v < 0)
        return TC_OK;
    if ((size_t)v + 1 < s->vt.size() && s->vt[(size_t)v + 1].start < hi)
        return TC_OK;
    if (v > 0 && s->vt[(size_t)v].start + s->vt[(size_t)v].ramp - 1 > w0)
        return TC_OK;  // the window reads samples of a crossfade
    const int slot = s->vt[(size_t)v].slot;
    tc_stream::TSet &ts = s->tsets[(size_t)slot][(size_t)delta];
    if (!ts.ready) {
        TC_TRY(ensure_tset_mem(s, slot, delta, nkb));
        // The slot's unshifted fp32 copy (shift e = 0) holds h[k] at index k.
        const float *h = s->ir + (size_t)slot * s->nsets * 4 * (size_t)s->Lpad;
        TC_CU(tc::k2_tprep_launch(h, (int)L, delta, (int)nkb, KB, ts.thi, s->prec == TC_BF16 ? nullptr : ts.tlo,
                                  s->cs));
        ts.ready = true;
    }
    tc::K2Params p{};
    p.C = (int)s->rows;
    p.nout = (int)nout;
    p.ntile_o = (int)ntile_o;
    p.x_col0 = w0 - s->base;
    p.nkb = (int)nkb;
    // A mono stream cuts the push's output into rows of 256 samples and runs
    // them as K2's channels: row r's history is the window from w0 + 256 r, so
    // the X tensor map is one strided view of the history (row stride 512
    // bytes) and 128 rows fill a tile. The rows are written straight into y
    // (row-major, pitch 256), the last one cut at the push's end.
    CUtensorMap mxr_hi{}, mxr_lo{};
    const bool rowview = s->rows == 1 && nout >= TN &&
                         (w0 - s->base) + (ntile_o - 1) * TN + nkb * KB <= s->cap;
    if (rowview) {
        const long long col = w0 - s->base;  // a multiple of 8: 16-byte aligned
        TC_CU(tc::encode_bf16_2d(&mxr_hi, static_cast<char *>(s->hist_hi) + col * 2, (unsigned long long)nkb * KB,
                                 (unsigned long long)ntile_o, (unsigned long long)TN * 2, KB, TM));
        TC_CU(tc::encode_bf16_2d(&mxr_lo, static_cast<char *>(s->hist_lo) + col * 2, (unsigned long long)nkb * KB,
                                 (unsigned long long)ntile_o, (unsigned long long)TN * 2, KB, TM));
        p.C = (int)ntile_o;
        p.nout = TN;
        p.ntile_o = 1;
        p.x_col0 = 0;
    }
    // Plain BF16 runs two channel tiles per CTA (one T stage feeds both), as
    // long as a unit's K range fits one TMEM run.
    const long long ntile_c1 = ((long long)p.C + TM - 1) / TM;
    // The persistent CTA pairs take two channel tiles of one output tile; a
    // group of one channel tile pairs two adjacent output tiles instead (the
    // same IR tile serves both), so that neither SM of a pair computes empty
    // rows. The BF16 split takes the pairs when it has two tiles of either kind.
    const bool pair_o = s->k2_mode == 2 && ntile_c1 == 1 && p.ntile_o >= 2;
    const bool spair = s->prec == TC_BF16_SPLIT && s->k2_mode == 2 && (ntile_c1 >= 2 || pair_o);
    bool pair = (s->prec == TC_BF16 && s->k2_mode != 0) || spair;
    const bool cta_pair = pair && s->k2_mode >= 2;
    p.pair_o = pair_o ? 1 : 0;
    p.ntile_c = (int)(pair && !pair_o ? (ntile_c1 + 1) / 2 : ntile_c1);
    const long long tiles = (long long)p.ntile_c * (pair_o ? (p.ntile_o + 1) / 2 : p.ntile_o);
    // TMEM runs of `range` K blocks before each drain into FP32 registers.
    // The BF16 split's error grows with the run (measured at L = 96000:
    // 4.4e-6 at 16, 6.2e-6 at 48, 7.4e-6 at 64 relative L2), and draining
    // every 16 blocks is hidden behind the MMAs of the other TMEM buffer.
    // Plain BF16 is limited by its operands, not by the run. K parts per
    // tile: the fewest that fill the GPU's waves to >= 90 %.
    p.range = (int)(s->k2_range > 0 ? s->k2_range : (s->prec == TC_BF16_SPLIT ? 16 : 4096));
    p.range += p.range & 1;  // the split's CTA pairs run whole pipeline stages of 2 K blocks
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    long long nsplit = k2_plan_nsplit(tiles, nkb, cta_pair ? sms / 2 : sms);  // a CTA pair takes two SMs
    if (s->k2_nsplit > 0)
        nsplit = std::min<long long>(s->k2_nsplit, nkb);
    const long long kb_per = (nkb + nsplit - 1) / nsplit;
    nsplit = (nkb + kb_per - 1) / kb_per;
    p.nsplit = (int)nsplit;
    p.kb_per = (int)kb_per;
    if (pair && !spair && p.range < p.kb_per) {
        // One TMEM run cannot hold this unit's K range: single tiles, same K split.
        pair = false;
        p.pair_o = 0;
        p.ntile_c = (int)ntile_c1;
    }
    p.order = s->k2_order;
    p.y = y;
    p.y_pitch = rowview ? TN : y_pitch;
    p.y_total = rowview ? nout : 0;
    p.err = s->d_err;
    if (nsplit > 1) {
        // Partials per 128-channel tile (the pair kernel writes that layout too).
        const size_t need = (size_t)(2 * ((ntile_c1 + 1) / 2) * p.ntile_o * nsplit) * TM * TN;
        if (need > s->k2_partial_floats)
            TC_TRY(k2_partial_alloc(s, need));
        p.partial = s->k2_partial;
        // The persistent CTA pairs and the one-tile kernel fold the parts
        // themselves (tickets per warp slice).
        if (s->k2_fold && (!pair || (cta_pair && s->k2_mode == 2)) && nsplit <= 16 &&
            (size_t)(2 * ((ntile_c1 + 1) / 2) * p.ntile_o * 8) <= s->k2_ticket_n)
            p.ticket = s->k2_ticket;
    }
    tc_stream::TSet &t = ts;
    TC_TRY(prof_begin(s));
    const CUtensorMap &mxh = rowview ? mxr_hi : s->mx_hi;
    const CUtensorMap &mxl = rowview ? mxr_lo : s->mx_lo;
    if (spair)
        TC_CU(tc::k2_launch_c2s(mxh, mxl, t.mt2_hi, t.mt2_lo, p, s->cs));
    else if (pair && cta_pair && s->k2_mode == 2)
        TC_CU(tc::k2_launch_c2p(mxh, t.mt2_hi, p, s->cs));
    else if (pair && cta_pair)
        TC_CU(tc::k2_launch_c2(mxh, t.mt2_hi, p, s->cs));
    else if (pair)
        TC_CU(tc::k2_launch_pair(mxh, t.mt_hi, p, s->cs));
    else
        TC_CU(tc::k2_launch(mxh, mxl, t.mt_hi, t.mt_lo, p, s->prec == TC_BF16 ? 1 : 3, s->cs));
    TC_TRY(prof_end(s, t0, nout));
    s->k2_launches++;
    *used = true;
    return TC_OK;
}

// K3 (MIMO on the tensor cores) when every input sample the launch reads
// spawned its tache with the same IR version; false in *used otherwise.
tc_status launch_k3(tc_stream *s, long long t0, long long nout, float *y, long long y_pitch, bool *used)
{
    *used = false;
    const long long L = (long long)s->L;
    const int nkbp = s->k3_nkbp;
    const int tp = tc::k3_tiles_per_cta();
    const int ntile = (int)(((nout + 1023) / 1024 + tp - 1) / tp * tp);  // padded tiles compute zeros
    // Samples read: [t0 + 8 - 32 nkbp, t0 + nout) (later ones are zeroed).
    const long long lo = t0 + 8 - 32LL * nkbp, hi = t0 + nout;
    int v = -1;
    for (size_t i = 0; i < s->vt.size(); ++i)
        if (s->vt[i].start <= std::max(lo, s->vt.front().start))
            v = (int)i;
    if (v < 0)
        return TC_OK;
    if ((size_t)v + 1 < s->vt.size() && s->vt[(size_t)v + 1].start < hi)
        return TC_OK;
    if (v > 0 && s->vt[(size_t)v].start + s->vt[(size_t)v].ramp - 1 > lo)
        return TC_OK;  // the window reads samples of a crossfade
    // k3_rev copies samples [R - span + 1, R], R = t0 + 1024 ntile - 1.
    if (t0 + 1024LL * ntile - tc::k3_xr_span(ntile, nkbp) < s->base)
        return fail(TC_EINVAL, "internal: K3 window starts before the kept history");
    const int slot = s->vt[(size_t)v].slot;
    tc_stream::K3Set &ks = s->k3sets[(size_t)slot];
    if (!ks.ready) {
        const unsigned long long rows = (unsigned long long)s->nin * nkbp * 128;
        if (!ks.bh) {
            TC_CU(tc::pool_alloc(&ks.bh, rows * 32 * 2, s->cs));
            TC_CU(tc::pool_alloc(&ks.bl, rows * 32 * 2, s->cs));
            TC_ALIGNED(ks.bh);
            TC_ALIGNED(ks.bl);
            TC_CU(tc::encode_bf16_2d(&ks.mb_hi, ks.bh, 32, rows, 64, 32, 128));
            TC_CU(tc::encode_bf16_2d(&ks.mb_lo, ks.bl, 32, rows, 64, 32, 128));
        }
        const float *ir = s->ir + (size_t)slot * s->nsets * 4 * (size_t)s->Lpad;
        TC_CU(tc::k3_tprep_launch(ir, 4 * s->Lpad, (int)s->nin, (int)s->items, (int)L, nkbp, ks.bh, ks.bl, s->cs));
        ks.ready = true;
    }
    TC_CU(tc::k3_rev_launch(s->hist, s->cap, s->base, (int)s->nin, t0 + 1024LL * ntile - 1, t0 + nout,
                            tc::k3_xr_span(ntile, nkbp), s->xr_hi, s->xr_lo, s->xr_pitch, s->cs));
    tc::K3Params p{};
    p.nin = (int)s->nin;
    p.ntile = ntile;
    p.nkbp = nkbp;
    p.range = (int)(s->k2_range > 0 ? s->k2_range : (s->prec == TC_BF16_SPLIT ? 16 : 4096));
    p.range = (p.range + 7) / 8 * 8;  // K3 runs hold whole stages of K blocks (8 in BF16, 4 in the split)
    // K parts per tile: the fewest (<= 64) that fill the GPU's waves to >= 90 %,
    // each a whole number of A chunks.
    const long long gtot = (long long)s->nin * nkbp;
    const int kbc = tc::k3_chunk_blocks();
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    long long nsplit = 1;
    double best = 0.0;
    for (long long ns = 1; ns <= 64 && ns * kbc <= gtot; ++ns) {
        const long long units = (long long)(ntile / tp) * ns;
        const double eff = (double)units / (double)(((units + sms - 1) / sms) * sms);
        if (eff > best + 1e-9) {
            best = eff;
            nsplit = ns;
        }
        if (eff >= 0.9)
            break;
    }
    const long long per = (gtot + nsplit - 1) / nsplit;
    const long long kb_per = (per + kbc - 1) / kbc * kbc;
    nsplit = (gtot + kb_per - 1) / kb_per;
    p.nsplit = (int)nsplit;
    p.kb_per = (int)kb_per;
    p.xr_hi = s->xr_hi;
    p.xr_lo = s->xr_lo;
    p.xr_pitch = s->xr_pitch;
    p.err = s->d_err;
    const size_t need = (size_t)ntile * nsplit * 128 * 128;
    if (need > s->k3_partial_floats) {
        if (s->k3_partial)
            cudaFreeAsync(s->k3_partial, s->cs);  // after the launches that used it
        s->k3_partial = nullptr;
        s->k3_partial_floats = 0;
        TC_CU(tc::pool_alloc(reinterpret_cast<void **>(&s->k3_partial), need * sizeof(float), s->cs));
        TC_ALIGNED(s->k3_partial);
        s->k3_partial_floats = need;
    }
    p.partial = s->k3_partial;
    TC_TRY(prof_begin(s));
    TC_CU(tc::k3_launch(ks.mb_hi, ks.mb_lo, p, s->prec == TC_BF16 ? 1 : 3, y, y_pitch, (int)s->items, (int)nout,
                        s->cs));
    TC_TRY(prof_end(s, t0, nout));
    s->k2_launches++;
    *used = true;
    return TC_OK;
}

// One convolution launch for outputs [t0, t0 + nout) of every row.
tc_status launch_conv(tc_stream *s, long long t0, long long nout, float *y, long long y_pitch)
{
    if (s->prec != TC_FP32 && s->kind == KIND_MIMO) {
        bool used = false;
        TC_TRY(launch_k3(s, t0, nout, y, y_pitch, &used));
        if (used)
            return TC_OK;
        s->k1_fallbacks++;
        return launch_k1(s, t0, nout, y, y_pitch);
    }
    if (s->prec != TC_FP32) {
        bool used = false;
        TC_TRY(launch_k2(s, t0, nout, y, y_pitch, &used));
        if (used)
            return TC_OK;
        s->k1_fallbacks++;  // a window that straddles an IR switch runs on the FP32 gather
    }
    return launch_k1(s, t0, nout, y, y_pitch);
}

tc_status check_err_word(tc_stream *s)
{
    if (*s->pin_err) {
        const int w = *s->pin_err;
        *s->pin_err = 0;
        cudaMemsetAsync(s->d_err, 0, sizeof(int), s->cs);
        cudaMemsetAsync(s->counter, 0, s->counter_n * sizeof(unsigned), s->cs);
        if (s->k2_ticket)
            cudaMemsetAsync(s->k2_ticket, 0, s->k2_ticket_n * sizeof(unsigned), s->cs);
        return fail(TC_ETIMEOUT, "a kernel's bounded wait gave up (device error word 0x%x)", w);
    }
    return TC_OK;
}

tc_status async_init(tc_stream *s)
{
    if (s->ccs)
        return TC_OK;
    TC_CU(cudaStreamCreateWithFlags(&s->ccs, cudaStreamNonBlocking));
    TC_CU(cudaStreamCreateWithFlags(&s->ics, cudaStreamNonBlocking));
    TC_CU(cudaEventCreateWithFlags(&s->ev_ir_prep, cudaEventDisableTiming));
    TC_CU(cudaEventRecord(s->ev_ir_prep, s->cs));  // every IR prep enqueued so far
    for (int k = 0; k < 2; ++k) {
        TC_CU(cudaMalloc(&s->d_xs[k], s->rows * s->max_push * sizeof(float)));
        TC_CU(cudaMalloc(&s->d_ys[k], s->items * s->max_push * sizeof(float)));
        for (cudaEvent_t *e : {&s->ev_xs_ready[k], &s->ev_xs_free[k], &s->ev_ys_ready[k], &s->ev_ys_free[k]})
            TC_CU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    return TC_OK;
}

// mode: PUSH_HOST (synchronous, host buffers), PUSH_DEVICE (device pointers,
// enqueued), PUSH_PINNED_ASYNC (page-locked host buffers, enqueued).
enum { PUSH_HOST = 0, PUSH_DEVICE = 1, PUSH_PINNED_ASYNC = 2 };

tc_status push_impl(tc_stream *s, const float *x, size_t n, float *y, int mode, size_t limit)
{
    tc::Range nvtx_range("tc push");
    TC_TRY(check_stream(s));
    if (!x || !y)
        return fail(TC_EINVAL, "x or y is NULL");
    if (n == 0 || n > limit)
        return fail(TC_EINVAL, "n = %zu not in [1, %zu]", n, limit);
    if (s->state != ST_OPEN)
        return fail(TC_ESTATE, "stream has ended (short last block or flush); reset it first");
    if (s->vt.empty() || s->vt.front().start > s->pos)
        return fail(TC_ESTATE, "no IR covers input sample %lld; call tc_set_ir first", s->pos);
    TC_TRY(use_device(s));
    retire_versions(s);
    TC_TRY(ensure_room(s, (long long)n + room_extra(s)));

    if (tc::inject_take(TC_INJECT_PUSH_COPY))
        return fail(TC_ECUDA, "injected failure of the push's input copy (tc_test_inject)");

    float *hist_at = s->hist + (s->pos - s->base);
    const size_t pitch_b = (size_t)s->cap * sizeof(float);
    const size_t row_b = n * sizeof(float);
    const bool on_device = mode == PUSH_DEVICE;
    int k = 0;
    if (mode == PUSH_PINNED_ASYNC) {
        if (!pinned_host(x) || !pinned_host(y))
            return fail(TC_EINVAL, "asynchronous pushes take page-locked host buffers for x and y");
        TC_TRY(async_init(s));
        k = s->aslot;
        s->aslot ^= 1;
        // Input: into staging slot k on the copy stream, once the slot's last
        // contents are in the history; then into the history on the stream.
        TC_CU(cudaStreamWaitEvent(s->ccs, s->ev_xs_free[k], 0));
        TC_CU(cudaMemcpyAsync(s->d_xs[k], x, s->rows * row_b, cudaMemcpyHostToDevice, s->ccs));
        TC_CU(cudaEventRecord(s->ev_xs_ready[k], s->ccs));
        TC_CU(cudaStreamWaitEvent(s->cs, s->ev_xs_ready[k], 0));
        TC_CU(cudaMemcpy2DAsync(hist_at, pitch_b, s->d_xs[k], row_b, row_b, s->rows, cudaMemcpyDeviceToDevice,
                                s->cs));
        TC_CU(cudaEventRecord(s->ev_xs_free[k], s->cs));
    } else if (on_device) {
        TC_CU(cudaMemcpy2DAsync(hist_at, pitch_b, x, row_b, row_b, s->rows, cudaMemcpyDeviceToDevice, s->cs));
    } else if (pinned_host(x)) {
        TC_CU(cudaMemcpy2DAsync(hist_at, pitch_b, x, row_b, row_b, s->rows, cudaMemcpyHostToDevice, s->cs));
    } else {
        TC_CU(cudaEventSynchronize(s->ev_x));
        std::memcpy(s->pin_x, x, s->rows * row_b);
        TC_CU(cudaMemcpy2DAsync(hist_at, pitch_b, s->pin_x, row_b, row_b, s->rows, cudaMemcpyHostToDevice, s->cs));
        TC_CU(cudaEventRecord(s->ev_x, s->cs));
    }
    TC_TRY(split_new(s, s->pos - s->base, (long long)n));
    TC_TRY(upload_table(s));
    float *ydst = on_device ? y : s->d_y;
    if (mode == PUSH_PINNED_ASYNC) {
        TC_CU(cudaStreamWaitEvent(s->cs, s->ev_ys_free[k], 0));  // slot k's last output is on the host
        ydst = s->d_ys[k];
    }
    TC_TRY(launch_conv(s, s->pos, (long long)n, ydst, (long long)n));
    s->pos += (long long)n;
    if (n % s->block != 0)
        s->state = ST_ENDED;
    if (mode == PUSH_PINNED_ASYNC) {
        // Output: back to y on the copy stream once the kernels are done.
        TC_CU(cudaEventRecord(s->ev_ys_ready[k], s->cs));
        TC_CU(cudaStreamWaitEvent(s->ccs, s->ev_ys_ready[k], 0));
        TC_CU(cudaMemcpyAsync(y, s->d_ys[k], s->items * row_b, cudaMemcpyDeviceToHost, s->ccs));
        TC_CU(cudaEventRecord(s->ev_ys_free[k], s->ccs));
    } else if (!on_device) {
        const bool direct = pinned_host(y);
        TC_CU(cudaMemcpyAsync(direct ? y : s->pin_y, s->d_y, s->items * row_b, cudaMemcpyDeviceToHost, s->cs));
        TC_CU(cudaMemcpyAsync(s->pin_err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->cs));
        TC_CU(cudaStreamSynchronize(s->cs));
        TC_TRY(check_err_word(s));
        if (!direct)
            std::memcpy(y, s->pin_y, s->items * row_b);
    }
    return TC_OK;
}

// Emits the L-1 tail into device rows y (pitch y_pitch floats) by pushing
// zeros through the gather in pieces of at most max_push samples.
tc_status flush_to_device(tc_stream *s, float *y, long long y_pitch)
{
    tc::Range nvtx_range("tc flush");
    const long long tail = (long long)s->L - 1;
    s->pos_end_hint = s->pos;
    for (long long off = 0; off < tail;) {
        const long long piece = std::min<long long>(tail - off, (long long)s->max_push);
        TC_TRY(ensure_room(s, piece + room_extra(s)));
        TC_CU(cudaMemset2DAsync(s->hist + (s->pos - s->base), (size_t)s->cap * sizeof(float), 0,
                                (size_t)piece * sizeof(float), s->rows, s->cs));
        TC_TRY(split_new(s, s->pos - s->base, piece));
        TC_TRY(upload_table(s));
        TC_TRY(launch_conv(s, s->pos, piece, y + off, y_pitch));
        s->pos += piece;
        off += piece;
    }
    s->state = ST_FLUSHED;
    return TC_OK;
}

tc_status flush_checks(tc_stream *s)
{
    TC_TRY(check_stream(s));
    if (s->state == ST_FLUSHED)
        return fail(TC_ESTATE, "stream already flushed; reset it first");
    if (!s->ir_ever_set)
        return fail(TC_ESTATE, "no IR was set");
    return TC_OK;
}

}  // namespace

namespace tc {

// A shared-IR group stream driven by the server's worker: pushes of up to
// max_push samples per channel, any length (block 1: a push never ends the
// stream), device pointers, on the group's own CUDA stream (the server orders
// it against its steps with events, so groups run concurrently).
tc_status group_open(size_t channels, size_t L, size_t max_push, int precision, tc_stream **out, size_t *bytes)
{
    TC_TRY(open_any(KIND_GROUP, channels, channels, 1, 1, L, 1, 1, (tc_precision)precision, max_push, out));
    tc_stream *s = *out;
    if (s->prec != TC_FP32) {
        // K-part partials for the largest push, now: growing them while
        // serving would map memory in the middle of a step.
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        const long long TM = tc::k2_tile_m(), TN = tc::k2_tile_n();
        const long long ntile_c1 = ((long long)s->rows + TM - 1) / TM;
        const long long nkb = tc::k2_nkb((long long)L, 7, tc::k2_kblock(s->prec == TC_BF16 ? 1 : 3));
        size_t need = 0;
        for (long long no = 1; no <= ((long long)max_push + TN - 1) / TN; ++no) {
            // Single tiles over all SMs; tile pairs (plain BF16, and the split on
            // CTA pairs) over all SMs or over half of them.
            for (const long long tcno : {ntile_c1 * no, (ntile_c1 + 1) / 2 * no, ntile_c1 * ((no + 1) / 2)})
                for (int slots : {sms, sms / 2}) {
                    const long long ns = k2_plan_nsplit(tcno, nkb, slots);
                    if (ns > 1)
                        need = std::max(need, (size_t)(2 * ((ntile_c1 + 1) / 2) * no * ns * TM * TN));
                }
        }
        if (need > 0) {
            tc_status st = k2_partial_alloc(s, need);
            if (st != TC_OK) {
                tc_close(s);
                *out = nullptr;
                return st;
            }
        }
    }
    if (s->prec != TC_FP32) {
        // The Toeplitz tiles of the first IR version (slot 0) at the shift of
        // pushes from sample 0 (pushes at multiples of 8 samples keep it), now:
        // allocating them at the first push would map memory while other
        // streams' steps run. Later versions' slots still allocate at their
        // first push.
        const int delta0 = (int)((((0 - (long long)L + 1 - s->base) % 8) + 8) % 8);
        tc_status st =
            ensure_tset_mem(s, 0, delta0, tc::k2_nkb((long long)L, delta0, tc::k2_kblock(s->prec == TC_BF16 ? 1 : 3)));
        if (st != TC_OK) {
            tc_close(s);
            *out = nullptr;
            return st;
        }
    }
    // Device footprint: what open allocated, plus what the tensor-core
    // launches allocate in steady use (Toeplitz tiles of two live IR versions
    // at one alignment shift: pushes at multiples of 8 samples keep the
    // shift; K-part partials of the largest push).
    size_t b = s->rows * (size_t)s->cap * sizeof(float) + (size_t)s->nslots * 4 * (size_t)s->Lpad * sizeof(float) +
               s->L * sizeof(float) + s->items * s->max_push * sizeof(float) + s->partial_floats * sizeof(float) +
               s->counter_n * sizeof(unsigned) + sizeof(DevTable) + sizeof(int);
    if (s->prec != TC_FP32) {
        b += s->rows * (size_t)s->cap * 4;  // bf16 hi and lo histories
        const size_t kbs = (size_t)tc::k2_kblock(s->prec == TC_BF16 ? 1 : 3);
        const size_t nkb = (size_t)tc::k2_nkb((long long)s->L, 7, (int)kbs);
        b += (size_t)2 * (s->prec == TC_BF16 ? 1 : 2) * nkb * 256 * kbs * 2;  // hi (and lo) tiles, two versions
        const size_t tiles = ((s->rows + 255) / 256 * 2) * ((s->max_push + 255) / 256);
        const size_t parts = std::max<size_t>(1, std::min<size_t>(64, 2 * 152 / std::max<size_t>(tiles, 1)));
        b += tiles * parts * 128 * 256 * sizeof(float);
    }
    *bytes = b;
    return TC_OK;
}

tc_status group_push(tc_stream *s, const float *x, size_t n, float *y)
{
    return push_impl(s, x, n, y, PUSH_DEVICE, s->max_push);
}

int *group_err(tc_stream *s) { return s->d_err; }

void *group_stream(tc_stream *s) { return s->cs; }

}  // namespace tc

extern "C" {

tc_status tc_open_stream(size_t L, size_t block, tc_stream **out)
{
    return open_any(KIND_GROUP, 1, 1, 1, 1, L, block, 1, TC_FP32, block, out);
}

tc_status tc_open_stream_ex(size_t L, size_t block, tc_precision precision, int device, size_t max_push,
                            tc_stream **out)
{
    int ndev = 0, cur = 0;
    TC_CU(cudaGetDeviceCount(&ndev));
    if (device < -1 || device >= ndev)
        return fail(TC_EINVAL, "device %d not in [-1, %d)", device, ndev);
    if (precision != TC_FP32 && precision != TC_BF16 && precision != TC_BF16_SPLIT)
        return fail(TC_EINVAL, "unknown precision");
    TC_CU(cudaGetDevice(&cur));
    if (device >= 0 && device != cur)
        TC_CU(cudaSetDevice(device));
    // A mono stream is a one-channel group; its IR is shared by that channel.
    const tc_status st = open_any(KIND_GROUP, 1, 1, 1, 1, L, block, 1, precision, max_push, out);
    if (device >= 0 && device != cur)
        cudaSetDevice(cur);
    return st;
}

tc_status tc_open_group(size_t channels, size_t L, size_t block, int shared_ir, tc_precision precision,
                        size_t max_push, tc_stream **out)
{
    const size_t sets = shared_ir ? 1 : channels;
    return open_any(KIND_GROUP, channels, channels, 1, sets, L, block, shared_ir ? 1 : 0, precision, max_push,
                    out);
}

tc_status tc_open_mimo(size_t nin, size_t nout, size_t L, size_t block, tc_precision precision, size_t max_push,
                       tc_stream **out)
{
    return open_any(KIND_MIMO, nin, nout, nin, nin * nout, L, block, 0, precision, max_push, out);
}

tc_status tc_close(tc_stream *s)
{
    if (!s)
        return TC_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    const int dev = s->device;
    if (cur != dev)
        cudaSetDevice(dev);
    free_all(s);
    delete s;
    tc::pool_trim();
    if (cur >= 0 && cur != dev)
        cudaSetDevice(cur);
    return TC_OK;
}

tc_status tc_reset(tc_stream *s)
{
    TC_TRY(check_stream(s));
    TC_TRY(use_device(s));
    // Stream-ordered: the memsets run after the stream's earlier work.
    TC_TRY(clear_state(s));
    return TC_OK;
}

tc_status tc_set_max_versions(tc_stream *s, int max_versions)
{
    TC_TRY(check_stream(s));
    if (max_versions < 2 || max_versions > kMaxVersions)
        return fail(TC_EINVAL, "max_versions must be in [2, %d]", kMaxVersions);
    if (s->ir_ever_set)
        return fail(TC_ESTATE, "max_versions can only change before the first IR is set");
    TC_TRY(use_device(s));
    s->nslots = max_versions;
    return alloc_ir(s);
}

tc_status tc_set_cuda_stream(tc_stream *s, void *cuda_stream)
{
    TC_TRY(check_stream(s));
    TC_TRY(use_device(s));
    cudaStream_t next = cuda_stream ? (cudaStream_t)cuda_stream : s->own_cs;
    if (next != s->cs) {
        // Order the new stream after everything already enqueued on the old one.
        TC_CU(cudaStreamSynchronize(s->cs));
        s->cs = next;
    }
    return TC_OK;
}

tc_status tc_get_info(const tc_stream *s, tc_info *info)
{
    TC_TRY(check_stream(s));
    if (!info)
        return fail(TC_EINVAL, "info is NULL");
    info->channels = s->rows;
    info->outputs = s->items;
    info->L = s->L;
    info->block = s->block;
    info->max_push = s->max_push;
    info->pushed = (uint64_t)s->pos;
    info->shared_ir = s->shared_ir;
    info->precision = (int)s->prec;
    info->state = s->state;
    info->max_versions = s->nslots;
    info->tensor_launches = (uint64_t)s->k2_launches;
    info->fp32_fallbacks = (uint64_t)s->k1_fallbacks;
    return TC_OK;
}

tc_status tc_set_crossfade(tc_stream *s, size_t ramp)
{
    TC_TRY(check_stream(s));
    if (ramp < 1 || ramp > ((size_t)1 << 24))
        return fail(TC_EINVAL, "crossfade ramp %zu not in [1, 2^24] samples", ramp);
    s->next_ramp = (long long)ramp;
    return TC_OK;
}

tc_status tc_set_ir(tc_stream *s, const float *h, size_t n)
{
    if (!s)
        return fail(TC_EINVAL, "stream is NULL");
    return set_ir_impl(s, h, n, s->pos, false, false);
}

tc_status tc_set_ir_at(tc_stream *s, const float *h, size_t n, uint64_t sample)
{
    if (sample > (uint64_t)1 << 62)
        return fail(TC_EINVAL, "sample out of range");
    return set_ir_impl(s, h, n, (long long)sample, false, false);
}

tc_status tc_set_ir_rows(tc_stream *s, const float *h, size_t n, uint64_t sample, int h_on_device)
{
    if (sample > (uint64_t)1 << 62)
        return fail(TC_EINVAL, "sample out of range");
    return set_ir_impl(s, h, n, (long long)sample, true, h_on_device != 0);
}

tc_status tc_push_block(tc_stream *s, const float *x, size_t n, float *y)
{
    if (!s)
        return fail(TC_EINVAL, "stream is NULL");
    return push_impl(s, x, n, y, PUSH_HOST, s->block);
}

tc_status tc_push(tc_stream *s, const float *x, size_t n, float *y, int on_device)
{
    if (!s)
        return fail(TC_EINVAL, "stream is NULL");
    if (on_device < 0 || on_device > 2)
        return fail(TC_EINVAL, "on_device must be 0 (host), 1 (device) or 2 (page-locked host, asynchronous)");
    return push_impl(s, x, n, y, on_device, s->max_push);
}

tc_status tc_flush(tc_stream *s, float *y, size_t cap, size_t *n_out)
{
    TC_TRY(flush_checks(s));
    if (!y)
        return fail(TC_EINVAL, "y is NULL");
    const size_t tail = s->L - 1;
    if (cap < tail)
        return fail(TC_EINVAL, "cap %zu < L-1 = %zu", cap, tail);
    TC_TRY(use_device(s));
    if (n_out)
        *n_out = tail;
    if (tail == 0) {
        s->state = ST_FLUSHED;
        return TC_OK;
    }
    float *d = nullptr;
    TC_CU(tc::pool_alloc(reinterpret_cast<void **>(&d), s->items * tail * sizeof(float), s->cs));
    tc_status st = flush_to_device(s, d, (long long)tail);
    if (st == TC_OK) {
        cudaError_t e = cudaMemcpy2DAsync(y, cap * sizeof(float), d, tail * sizeof(float), tail * sizeof(float),
                                          s->items, cudaMemcpyDeviceToHost, s->cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->pin_err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->cs);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s->cs);
        if (e != cudaSuccess)
            st = fail(TC_ECUDA, "flush copy: %s", cudaGetErrorString(e));
        else
            st = check_err_word(s);
    }
    if (st == TC_OK && s->ccs && cudaStreamSynchronize(s->ccs) != cudaSuccess)
        st = fail(TC_ECUDA, "flush: copy stream");  // outputs of asynchronous pushes are on the host
    cudaFreeAsync(d, s->cs);
    return st;
}

tc_status tc_flush_dev(tc_stream *s, float *y, size_t *n_out)
{
    TC_TRY(flush_checks(s));
    if (!y)
        return fail(TC_EINVAL, "y is NULL");
    TC_TRY(use_device(s));
    const size_t tail = s->L - 1;
    if (n_out)
        *n_out = tail;
    if (tail == 0) {
        s->state = ST_FLUSHED;
        return TC_OK;
    }
    return flush_to_device(s, y, (long long)tail);
}

tc_status tc_sync(tc_stream *s)
{
    TC_TRY(check_stream(s));
    TC_TRY(use_device(s));
    TC_CU(cudaMemcpyAsync(s->pin_err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->cs));
    TC_CU(cudaStreamSynchronize(s->cs));
    if (s->ccs)
        TC_CU(cudaStreamSynchronize(s->ccs));  // outputs of asynchronous pushes are on the host
    return check_err_word(s);
}

tc_status tc_convolve(const float *x, size_t N, const float *h, size_t L, float *y, void *cuda_stream)
{
    return tc::oneshot_alloc(x, N, h, L, y, cuda_stream);
}

const char *tc_last_error(void) { return g_err.c_str(); }

const char *tc_status_str(tc_status st)
{
    switch (st) {
    case TC_OK: return "TC_OK";
    case TC_EINVAL: return "TC_EINVAL";
    case TC_ENOMEM: return "TC_ENOMEM";
    case TC_ESTATE: return "TC_ESTATE";
    case TC_ECUDA: return "TC_ECUDA";
    case TC_ETIMEOUT: return "TC_ETIMEOUT";
    case TC_EUNSUPPORTED: return "TC_EUNSUPPORTED";
    default: return "TC_UNKNOWN";
    }
}

uint64_t tc_kernel_launches(void) { return tc::launches(); }

tc_status tc_test_inject(int site, int nth)
{
    if (site != TC_INJECT_PUSH_COPY && site != TC_INJECT_SERVER_STEP)
        return fail(TC_EINVAL, "tc_test_inject: unknown site %d", site);
    if (nth < 0)
        return fail(TC_EINVAL, "tc_test_inject: nth must be >= 0");
    tc::inject_arm(site, nth);
    return TC_OK;
}

tc_status tc_set_tuning(tc_stream *s, int knob, long long value)
{
    TC_TRY(check_stream(s));
    switch (knob) {
    case TC_TUNE_K1_CHUNK:
        if (value < -1 || value >= tc::K1_NVARIANTS)
            return fail(TC_EINVAL, "TC_TUNE_K1_CHUNK must be -1 or in [0, %d)", tc::K1_NVARIANTS);
        s->k1_variant_fixed = (int)value;
        return TC_OK;
    case TC_TUNE_K2_RANGE:
        if (value == -1) {
            s->k2_range = -1;
            return TC_OK;
        }
        if (value < 1 || value > 4096)
            return fail(TC_EINVAL, "TC_TUNE_K2_RANGE must be -1 or in [1, 4096]");
        s->k2_range = value;
        return TC_OK;
    case TC_TUNE_K2_PAIR:
        if (value < -1 || value > 3)
            return fail(TC_EINVAL, "TC_TUNE_K2_PAIR must be -1, 0, 1, 2 or 3");
        s->k2_mode = value == -1 ? 2 : (int)value;
        return TC_OK;
    case TC_TUNE_K2_SPLIT:
        if (value != -1 && (value < 1 || value > 64))
            return fail(TC_EINVAL, "TC_TUNE_K2_SPLIT must be -1 or in [1, 64]");
        s->k2_nsplit = (int)value;
        return TC_OK;
    case TC_TUNE_K2_FOLD:
        if (value != -1 && value != 0 && value != 1)
            return fail(TC_EINVAL, "TC_TUNE_K2_FOLD must be -1, 0 or 1");
        s->k2_fold = value != 0;
        return TC_OK;
    case TC_TUNE_K2_ORDER:
        if (value < -1 || value > 2)
            return fail(TC_EINVAL, "TC_TUNE_K2_ORDER must be -1, 0, 1 or 2");
        s->k2_order = value == -1 ? 2 : (int)value;
        return TC_OK;
    case TC_TUNE_ZERO_SKIP:
        if (value != -1 && value != 0 && value != 1)
            return fail(TC_EINVAL, "TC_TUNE_ZERO_SKIP must be -1, 0 or 1");
        s->zero_skip = value == 1;
        return TC_OK;
    default:
        return fail(TC_EINVAL, "unknown tuning knob %d", knob);
    }
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: the whole state a stream's future outputs depend on.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kBlobMagic = 0x31534354u;  // "TCS1"

struct BlobHeader {
    uint32_t magic, version;
    int32_t kind, prec, shared_ir, state;
    uint64_t rows, items, nin, nsets, L, block, max_push;
    int64_t pos, base, next_ramp, nver, hist_len;
    int32_t k1_variant_fixed, k2_mode, zero_skip, pad;
    int64_t k2_range;
};

size_t blob_size(const tc_stream *s)
{
    const size_t nver = s->vt.size();
    const size_t hist_len = (size_t)std::max<long long>(0, s->pos - s->base);
    return sizeof(BlobHeader) + nver * 2 * sizeof(int64_t) + nver * s->nsets * s->L * sizeof(float) +
           s->rows * hist_len * sizeof(float);
}

}  // namespace

tc_status tc_stream_export(tc_stream *s, void *buf, size_t cap, size_t *size)
{
    TC_TRY(check_stream(s));
    if (!size)
        return fail(TC_EINVAL, "size is NULL");
    TC_TRY(use_device(s));
    const size_t need = blob_size(s);
    *size = need;
    if (!buf)
        return TC_OK;
    if (cap < need)
        return fail(TC_EINVAL, "buffer of %zu bytes < %zu needed", cap, need);
    TC_CU(cudaStreamSynchronize(s->cs));
    char *out = static_cast<char *>(buf);
    BlobHeader hd{};
    hd.magic = kBlobMagic;
    hd.version = 1;
    hd.kind = s->kind;
    hd.prec = (int32_t)s->prec;
    hd.shared_ir = s->shared_ir;
    hd.state = s->state;
    hd.rows = s->rows;
    hd.items = s->items;
    hd.nin = s->nin;
    hd.nsets = s->nsets;
    hd.L = s->L;
    hd.block = s->block;
    hd.max_push = s->max_push;
    hd.pos = s->pos;
    hd.base = s->base;
    hd.next_ramp = s->next_ramp;
    hd.nver = (int64_t)s->vt.size();
    hd.hist_len = std::max<long long>(0, s->pos - s->base);
    hd.k1_variant_fixed = s->k1_variant_fixed;
    hd.k2_mode = s->k2_mode;
    hd.zero_skip = s->zero_skip ? 1 : 0;
    hd.k2_range = s->k2_range;
    std::memcpy(out, &hd, sizeof hd);
    out += sizeof hd;
    for (const Version &v : s->vt) {
        const int64_t sv[2] = {v.start, v.ramp};
        std::memcpy(out, sv, sizeof sv);
        out += sizeof sv;
    }
    // IR rows of each live version: the slot's unshifted copy holds h[k] at k.
    for (const Version &v : s->vt)
        for (size_t set = 0; set < s->nsets; ++set) {
            const float *src = s->ir + ((size_t)v.slot * s->nsets + set) * 4 * (size_t)s->Lpad;
            TC_CU(cudaMemcpy(out, src, s->L * sizeof(float), cudaMemcpyDeviceToHost));
            out += s->L * sizeof(float);
        }
    // History rows from base to pos (the stream's layout is kept, so the
    // kernels' tap-chunk alignment and the results resume bit for bit).
    if (hd.hist_len > 0)
        TC_CU(cudaMemcpy2D(out, (size_t)hd.hist_len * sizeof(float), s->hist, (size_t)s->cap * sizeof(float),
                           (size_t)hd.hist_len * sizeof(float), s->rows, cudaMemcpyDeviceToHost));
    return TC_OK;
}

tc_status tc_stream_import(tc_stream *s, const void *buf, size_t size)
{
    TC_TRY(check_stream(s));
    if (!buf || size < sizeof(BlobHeader))
        return fail(TC_EINVAL, "buffer is NULL or too short");
    BlobHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kBlobMagic || hd.version != 1)
        return fail(TC_EINVAL, "not a stream checkpoint of this library");
    if (hd.kind != s->kind || hd.prec != (int32_t)s->prec || hd.shared_ir != s->shared_ir || hd.rows != s->rows ||
        hd.items != s->items || hd.nin != s->nin || hd.nsets != s->nsets || hd.L != s->L ||
        hd.block != s->block || hd.max_push != s->max_push)
        return fail(TC_EINVAL, "the checkpoint is of a stream of another shape (kind, precision, channels, L, "
                               "block, max_push must match)");
    if (hd.nver < 1 || hd.nver > s->nslots || hd.hist_len < 0 || hd.hist_len > s->cap ||
        hd.pos - hd.base != hd.hist_len)
        return fail(TC_EINVAL, "inconsistent checkpoint (versions or history length)");
    const size_t need = sizeof hd + (size_t)hd.nver * 2 * sizeof(int64_t) +
                        (size_t)hd.nver * s->nsets * s->L * sizeof(float) + s->rows * (size_t)hd.hist_len * 4;
    if (size < need)
        return fail(TC_EINVAL, "checkpoint of %zu bytes < %zu expected", size, need);
    TC_TRY(use_device(s));
    TC_TRY(clear_state(s));  // also marks every Toeplitz / MIMO tile cache stale
    const char *in = static_cast<const char *>(buf) + sizeof hd;
    std::vector<Version> vt;
    for (int64_t i = 0; i < hd.nver; ++i) {
        int64_t sv[2];
        std::memcpy(sv, in, sizeof sv);
        in += sizeof sv;
        vt.push_back(Version{sv[0], (int)i, sv[1]});
    }
    for (int64_t i = 0; i < hd.nver; ++i) {
        // IR rows to the staging area, then the four shifted copies of slot i.
        TC_CU(cudaMemcpy(s->ir_stage, in, s->nsets * s->L * sizeof(float), cudaMemcpyHostToDevice));
        in += s->nsets * s->L * sizeof(float);
        float *dst = s->ir + (size_t)i * s->nsets * 4 * (size_t)s->Lpad;
        TC_CU(tc::ir_prep_launch(s->ir_stage, (long long)s->L, (long long)s->L, (int)s->nsets, dst, 4 * s->Lpad,
                                 s->Lpad, s->Lpad, s->cs));
        TC_CU(cudaStreamSynchronize(s->cs));  // the staging area is reused by the next version
        s->slot_used[(size_t)i] = 1;
    }
    if (hd.hist_len > 0) {
        TC_CU(cudaMemcpy2DAsync(s->hist, (size_t)s->cap * sizeof(float), in, (size_t)hd.hist_len * sizeof(float),
                                (size_t)hd.hist_len * sizeof(float), s->rows, cudaMemcpyHostToDevice, s->cs));
    }
    s->vt = vt;
    s->vt_dirty = true;
    s->ir_ever_set = true;
    s->pos = hd.pos;
    s->base = hd.base;
    s->state = hd.state;
    s->next_ramp = hd.next_ramp;
    s->k1_variant_fixed = hd.k1_variant_fixed;
    s->k2_mode = (hd.k2_mode >= 0 && hd.k2_mode <= 3) ? hd.k2_mode : 2;
    s->zero_skip = hd.zero_skip != 0;
    s->k2_range = hd.k2_range;
    if (hd.hist_len > 0)
        TC_TRY(split_new(s, 0, hd.hist_len));  // bf16 hi/lo copies of the history (tensor-core streams)
    TC_CU(cudaStreamSynchronize(s->cs));
    return TC_OK;
}

tc_status tc_profile(tc_stream *s, int enable)
{
    TC_TRY(check_stream(s));
    s->profile = enable != 0;
    return TC_OK;
}

tc_status tc_profile_read(tc_stream *s, double *ms, uint64_t *launches, double *useful_macs)
{
    TC_TRY(check_stream(s));
    TC_TRY(use_device(s));
    TC_CU(cudaStreamSynchronize(s->cs));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < s->ev_used; i += 2) {
        float e = 0.f;
        TC_CU(cudaEventElapsedTime(&e, s->ev_pool[i], s->ev_pool[i + 1]));
        tot += e;
    }
    if (ms)
        *ms = tot;
    if (launches)
        *launches = s->prof_launches;
    if (useful_macs)
        *useful_macs = s->prof_macs;
    s->ev_used = 0;
    s->prof_launches = 0;
    s->prof_macs = 0.0;
    return TC_OK;
}

}  // extern "C"
