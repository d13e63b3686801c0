// oneshot.cu -- the one-shot FP32 convolutions y = x * h (Sec. 3.2, Eq. 4
// with one IR version): tc_convolve and tc_convolve_noalloc.
//
// Both run K1 over the whole signal from one scratch area laid out as
//   [error word][IR: 4 shifted copies][history row: zeros, x, zeros]
//   [tickets][split-sum partials],
// in as few launches as the partials allow. They differ only in where the
// scratch comes from:
//   - tc_convolve takes it from the library's stream-ordered pool
//     (allocated and freed in order on the caller's stream; the pool keeps
//     freed memory for the next call), sized so that one launch covers the
//     whole output;
//   - tc_convolve_noalloc uses one fixed 32 MiB file-scope device array and
//     never allocates. Who needs it: callers that cannot call cudaMalloc at
//     the point of use (a real-time audio callback, where an allocation can
//     block for an unbounded time; a host whose own allocator owns all device
//     memory).
//
// The fixed array is part of this library's device image. Every GPU on which
// the library's kernels are loaded holds it until the process exits. Its
// device address is looked up once per device, with that device current, on
// the first call made on that device. Make that first call outside any CUDA
// stream capture. The looked-up addresses are kept for the life of the
// process: do not use this library across cudaDeviceReset (the module, and
// with it the array, is loaded again at a new address). All calls share it,
// and it keeps the last call's contents,
// so each call first clears what must start at zero: the zero margins of the
// input history, the split-sum tickets and the error word. Calls that overlap
// on the GPU race on the array and give wrong results. Serialise them.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <utility>

#include "../../include/taches.h"
#include "tc_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;             // 32 MiB
constexpr long long kScratchFloats = (long long)(kNoAllocScratchBytes / sizeof(float));
constexpr long long kMinPieceTiles = 32;  // smallest K1 launch accepted: 32 tiles of 128 outputs
constexpr int kMaxDev = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float)];

// The single IR version of a one-shot convolution: starts at sample 0, slot 0.
// Read-only for the kernels.
static __device__ long long g_noalloc_vstart[1] = {0};
static __device__ int g_noalloc_vslot[1] = {0};
static __device__ int g_noalloc_nver = 1;

struct DevPtrs {
    float *scratch = nullptr;
    long long *vstart = nullptr;
    int *vslot = nullptr;
    int *nver = nullptr;
    bool ready = false;
};

DevPtrs g_ptrs[kMaxDev];
std::mutex g_ptrs_mu;

long long ru(long long a, long long m) { return (a + m - 1) / m * m; }

tc_status na_fail(tc_status st, const std::string &msg)
{
    tc::set_last_error(msg.c_str());
    return st;
}

// Looks up the device addresses of the file-scope arrays once per device.
tc_status setup(int dev, DevPtrs *out)
{
    std::lock_guard<std::mutex> lk(g_ptrs_mu);
    DevPtrs &p = g_ptrs[dev];
    if (!p.ready) {
        cudaError_t e = cudaGetSymbolAddress((void **)&p.scratch, g_noalloc_scratch);
        if (e == cudaSuccess)
            e = cudaGetSymbolAddress((void **)&p.vstart, g_noalloc_vstart);
        if (e == cudaSuccess)
            e = cudaGetSymbolAddress((void **)&p.vslot, g_noalloc_vslot);
        if (e == cudaSuccess)
            e = cudaGetSymbolAddress((void **)&p.nver, g_noalloc_nver);
        if (e != cudaSuccess)
            return na_fail(TC_ECUDA, std::string("one-shot convolution: cudaGetSymbolAddress: ") +
                                         cudaGetErrorString(e));
        p.ready = true;
    }
    *out = p;
    return TC_OK;
}

// Offsets (floats, 64-float aligned segments) of the scratch of one call:
//   [error word][IR: 4 shifted copies of Lpad][history row][tickets][split-sum partials].
// One K1 launch covers a piece of the output: as many 128-output tiles as the
// space left holds chunk sums for (with the most chunks any variant may use)
// and one ticket each; at least kMinPieceTiles, at most all of y (and 2^20).
// scratch_floats < 0: size the scratch for pieces of up to 64 Mi floats of
// partials (about 900000 outputs at L = 48000: dozens of waves per launch).
struct Layout {
    long long keep, Lpad, cap, off_err, off_ir, off_hist, off_ctr, off_part, piece_tiles, need, total;
    bool fits;
};

Layout layout(long long N, long long L, long long scratch_floats)
{
    Layout l{};
    l.keep = ru(L + tc::K1_KC_MAX + 8, 4);  // zero samples before x[0]
    l.Lpad = ru(L + 4 + tc::K1_KC_MAX, 4);
    const long long ny = N + L - 1;
    l.cap = ru(l.keep + ny + tc::K1_MO + 160, 64);  // history row: zeros, x, zeros
    l.off_err = 0;
    l.off_ir = 64;
    l.off_hist = l.off_ir + ru(4 * l.Lpad, 64);
    l.off_ctr = l.off_hist + l.cap;
    const long long per_tile = tc::k1_partial_floats_max(L, 1, 1);  // chunk sums of one tile
    const long long tiles_all = (ny + tc::K1_MO - 1) / tc::K1_MO;
    const long long most = std::min(tiles_all, 1LL << 20);
    l.piece_tiles = scratch_floats < 0
                        ? std::min(most, std::max(kMinPieceTiles, (64LL << 20) / per_tile))
                        : std::min(most, (scratch_floats - l.off_ctr - 64) / (per_tile + 1));
    l.off_part = l.off_ctr + ru(std::max(l.piece_tiles, 1LL), 64);
    l.total = l.off_part + std::max(l.piece_tiles, 1LL) * per_tile;
    l.need = l.off_ctr + 64 + std::min(kMinPieceTiles, tiles_all) * (per_tile + 1);
    l.fits = scratch_floats < 0 || (l.need <= scratch_floats && l.piece_tiles >= std::min(kMinPieceTiles, tiles_all));
    return l;
}

// Runs the convolution from `scratch` (scratch_floats floats). who names the
// entry point in error messages.
tc_status run_oneshot(const char *who, const float *x, size_t N, const float *h, size_t L, float *y,
                      cudaStream_t cs, float *scratch, long long scratch_floats, const DevPtrs &P)
{
    tc::Range nvtx_range(who);
    const long long Ll = (long long)L, Nl = (long long)N;
    const Layout lay = layout(Nl, Ll, scratch_floats);
    float *base = scratch;
    unsigned *counters = reinterpret_cast<unsigned *>(base + lay.off_ctr);  // [piece_tiles]
    int *err = reinterpret_cast<int *>(base + lay.off_err);
    float *ir = base + lay.off_ir;
    float *hist = base + lay.off_hist;
    float *part = base + lay.off_part;

#define NA_CU(call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return na_fail(TC_ECUDA, std::string(who) + ": " #call ": " + cudaGetErrorString(e_));   \
    } while (0)

    // Clear what must start at zero: the error word, the tickets, and the
    // history's zero margins before x[0] and after x[N-1].
    NA_CU(cudaMemsetAsync(err, 0, sizeof(int), cs));
    NA_CU(cudaMemsetAsync(counters, 0, (size_t)(lay.off_part - lay.off_ctr) * sizeof(float), cs));
    NA_CU(cudaMemsetAsync(hist, 0, (size_t)lay.keep * sizeof(float), cs));
    NA_CU(cudaMemsetAsync(hist + lay.keep + Nl, 0, (size_t)(lay.cap - lay.keep - Nl) * sizeof(float), cs));
    NA_CU(cudaMemcpyAsync(hist + lay.keep, x, (size_t)Nl * sizeof(float), cudaMemcpyDeviceToDevice, cs));
    NA_CU(tc::ir_prep_launch(h, Ll, Ll, 1, ir, 4 * lay.Lpad, lay.Lpad, lay.Lpad, cs));

    tc::K1Params p{};
    p.hist = hist;
    p.pitch = lay.cap;
    p.base = -lay.keep;
    p.x_item_rows = 1;
    p.x_in_rows = 0;
    p.ir = ir;
    p.ir_slot = 4 * lay.Lpad;
    p.ir_item = 0;
    p.ir_in = 0;
    p.ir_phase = lay.Lpad;
    p.L = (int)Ll;
    p.vstart = P.vstart;
    p.vslot = P.vslot;
    p.nver = P.nver;
    p.vt_item = 0;
    p.nitems = 1;
    p.nin = 1;
    p.partial = part;
    p.counter = counters;
    p.err = err;
    p.has_end = 1;  // x ends at N: the taps past it are skipped
    p.x_end = Nl;
    const long long ny = Nl + Ll - 1;
    const long long piece = lay.piece_tiles * tc::K1_MO;
    for (long long t0 = 0; t0 < ny; t0 += piece) {
        const long long n = (ny - t0 < piece) ? ny - t0 : piece;
        p.t0 = t0;
        p.nout = (int)n;
        p.ntile = (int)((n + tc::K1_MO - 1) / tc::K1_MO);
        p.e = tc::k1_shift_e(t0, p.base);
        p.y = y + t0;
        p.y_pitch = n;
        tc::K1Plan plan{};
        NA_CU(tc::k1_plan(Ll, p.e, 1, 1, p.ntile, -1, &plan));
        if (plan.ctas * tc::K1_MO > tc::k1_partial_floats_max(Ll, 1, lay.piece_tiles))
            return na_fail(TC_EINVAL, std::string(who) + ": internal: chunk-sum scratch too small");
        NA_CU(tc::k1_launch(p, plan, cs));
    }
    int herr = 0;
    NA_CU(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, cs));
    NA_CU(cudaStreamSynchronize(cs));
#undef NA_CU
    if (herr)
        return na_fail(TC_ETIMEOUT, std::string(who) + ": a kernel's bounded wait gave up");
    return TC_OK;
}

}  // namespace

namespace tc {

tc_status oneshot_alloc(const float *x, size_t N, const float *h, size_t L, float *y, void *cuda_stream)
{
    if (!x || !h || !y)
        return na_fail(TC_EINVAL, "tc_convolve: x, h or y is NULL");
    if (N == 0 || L == 0)
        return na_fail(TC_EINVAL, "tc_convolve: N and L must be > 0");
    // Role swap (Sec. 3.2: x * h = h * x). The gather computes every output
    // over all L taps, (N + L - 1) L multiply-adds, so the shorter operand
    // takes the IR role: a short sound through a long IR costs about N L.
    if (N < L && !no_role_swap()) {
        std::swap(x, h);
        std::swap(N, L);
    }
    if (L > ((size_t)1 << 30) || N > ((size_t)1 << 40))
        return na_fail(TC_EINVAL, "tc_convolve: L must be <= 2^30 and N <= 2^40");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return na_fail(TC_ECUDA, std::string("tc_convolve: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDev)
        return na_fail(TC_EINVAL, "tc_convolve: device index out of range");
    DevPtrs P;
    const tc_status sst = setup(dev, &P);
    if (sst != TC_OK)
        return sst;
    // Scratch: the history row, the IR copies and the partials of one piece.
    const long long Ll = (long long)L, Nl = (long long)N;
    const Layout full = layout(Nl, Ll, -1);
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    float *scratch = nullptr;
    e = tc::pool_alloc(reinterpret_cast<void **>(&scratch), (size_t)full.total * sizeof(float), cs);
    if (e != cudaSuccess)
        return na_fail(e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA,
                       std::string("tc_convolve: pool allocation: ") + cudaGetErrorString(e));
    if ((reinterpret_cast<uintptr_t>(scratch) & 255u) != 0) {
        cudaFreeAsync(scratch, cs);
        return na_fail(TC_ECUDA, "tc_convolve: the stream-ordered allocation is not 256-byte aligned");
    }
    const tc_status st = run_oneshot("tc_convolve", x, N, h, L, y, cs, scratch, full.total, P);
    cudaFreeAsync(scratch, cs);
    return st;
}

}  // namespace tc

extern "C" tc_status tc_convolve_noalloc(const float *x, size_t N, const float *h, size_t L, float *y,
                                         void *cuda_stream)
{
    if (!x || !h || !y)
        return na_fail(TC_EINVAL, "tc_convolve_noalloc: x, h or y is NULL");
    if (N == 0 || L == 0)
        return na_fail(TC_EINVAL, "tc_convolve_noalloc: N and L must be > 0");
    // Neither operand can be longer than the fixed array: reject such sizes
    // before any arithmetic on them (a size_t near 2^64, e.g. a -1 passed
    // through an unsigned argument, would wrap when converted to long long).
    if (N > (size_t)kScratchFloats || L > (size_t)kScratchFloats) {
        char buf[192];
        snprintf(buf, sizeof buf,
                 "tc_convolve_noalloc: N=%zu or L=%zu exceeds the fixed array of %.0f MiB (use tc_convolve)", N, L,
                 kNoAllocScratchBytes / double(1 << 20));
        return na_fail(TC_EINVAL, buf);
    }
    // Role swap as in tc_convolve (Sec. 3.2): the shorter operand is the IR.
    if (N < L && !tc::no_role_swap()) {
        std::swap(x, h);
        std::swap(N, L);
    }
    const Layout lay = layout((long long)N, (long long)L, kScratchFloats);
    if (!lay.fits) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "tc_convolve_noalloc: N=%zu, L=%zu need %.1f MiB of scratch; the fixed array holds %.0f MiB "
                 "(use tc_convolve, which allocates)",
                 N, L, lay.need * 4.0 / (1 << 20), kNoAllocScratchBytes / double(1 << 20));
        return na_fail(TC_EINVAL, buf);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return na_fail(TC_ECUDA, std::string("tc_convolve_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDev)
        return na_fail(TC_EINVAL, "tc_convolve_noalloc: device index out of range");
    DevPtrs P;
    tc_status st = setup(dev, &P);
    if (st != TC_OK)
        return st;
    return run_oneshot("tc_convolve_noalloc", x, N, h, L, y, (cudaStream_t)cuda_stream, P.scratch, kScratchFloats, P);
}

// ---------------------------------------------------------------------------
// One signal on the tensor cores: the output reshaped into rows of 256
// samples, each row a "channel" of the shared-IR contraction K2.
//
// With xs the input delayed by L - 1 (zeros before and after it), row r of the
// output is y[256 r + i] = sum_j T[i][j] xs[256 r + j], i < 256, j < KB nkb,
// T[i][j] = h[L - 1 + i - j]: exactly K2's product for a group whose channel
// r has the history xs[256 r + .] (K blocks of KB = 64 samples in plain BF16,
// 32 in the split). Those histories overlap, so K2's X tensor map is one
// strided view of xs: row stride 256 samples (512 bytes), row length KB nkb.
// The Toeplitz tiles of h are built once per call; the rows are written
// straight into y, the last one cut at its end.
// ---------------------------------------------------------------------------
extern "C" tc_status tc_convolve_tc(const float *x, size_t N, const float *h, size_t L, float *y, int precision,
                                    void *cuda_stream)
{
    if (!x || !h || !y)
        return na_fail(TC_EINVAL, "tc_convolve_tc: x, h or y is NULL");
    if (N == 0 || L == 0)
        return na_fail(TC_EINVAL, "tc_convolve_tc: N and L must be > 0");
    if (precision == TC_FP32)
        return tc::oneshot_alloc(x, N, h, L, y, cuda_stream);
    if (precision != TC_BF16 && precision != TC_BF16_SPLIT)
        return na_fail(TC_EINVAL, "tc_convolve_tc: unknown precision");
    tc::Range nvtx_range("tc_convolve_tc");
    if (N < L && !tc::no_role_swap()) {  // Sec. 3.2: the shorter operand is the IR
        std::swap(x, h);
        std::swap(N, L);
    }
    if (L > ((size_t)1 << 26) || N > ((size_t)1 << 34))
        return na_fail(TC_EINVAL, "tc_convolve_tc: L must be <= 2^26 and N <= 2^34");
    const int TM = tc::k2_tile_m(), TN = tc::k2_tile_n(), KB = tc::k2_kblock(precision == TC_BF16 ? 1 : 3);
    const long long Ll = (long long)L, Nl = (long long)N;
    const long long ny = Nl + Ll - 1;
    const long long R = (ny + TN - 1) / TN;              // output rows of 256 samples
    const long long nkb = tc::k2_nkb(Ll, 0, KB);         // K blocks per row window
    const long long off = Ll - 1;                        // xs[m] = x[m - off]
    const long long npad = ru((R - 1) * TN + nkb * KB + 64, 64);
    if (R > (1LL << 24))
        return na_fail(TC_EINVAL, "tc_convolve_tc: output too long");
    const int nprod = precision == TC_BF16 ? 1 : 3;
    cudaStream_t cs = (cudaStream_t)cuda_stream;

    // Scratch: padded fp32 input, its bf16 hi/lo, Toeplitz tiles hi/lo, the
    // row-major output and the K-part partials.
    const long long ntile_c1 = (R + TM - 1) / TM;
    // Plain BF16 on persistent CTA pairs; the split too when there are two row tiles to pair.
    const bool spair = precision == TC_BF16_SPLIT && ntile_c1 >= 2;
    bool pair = precision == TC_BF16 || spair;
    tc::K2Params p{};
    p.C = (int)R;
    p.nout = TN;
    p.ntile_o = 1;
    p.x_col0 = 0;
    p.nkb = (int)nkb;
    p.range = precision == TC_BF16_SPLIT ? 16 : 4096;
    p.order = 2;  // persistent pairs: row tiles fastest, K parts slowest
    p.ntile_c = (int)(pair ? (ntile_c1 + 1) / 2 : ntile_c1);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long nsplit = 1;
    double best = 0.0;
    const int slots = pair ? sms / 2 : sms;  // plain BF16 runs on CTA pairs: two SMs per unit
    for (long long ns = 1; ns <= 64 && ns <= nkb && (ns == 1 || nkb / ns >= 16); ++ns) {
        const long long units = (long long)p.ntile_c * ns;
        const double eff = (double)units / (double)(((units + slots - 1) / slots) * slots);
        if (eff > best + 1e-9) {
            best = eff;
            nsplit = ns;
        }
        if (eff >= 0.9)
            break;
    }
    const long long kb_per = (nkb + nsplit - 1) / nsplit;
    nsplit = (nkb + kb_per - 1) / kb_per;
    p.nsplit = (int)nsplit;
    p.kb_per = (int)kb_per;
    if (pair && !spair && p.range < p.kb_per) {
        pair = false;
        p.ntile_c = (int)ntile_c1;
    }
    // The bf16 input rows are split straight from x into the padded buffers (zero margins before and after).
    // Plain BF16 reads only the hi input and tiles; the rows are written straight into y.
    const size_t b_xs = 0, b_xb = (size_t)npad * 2, b_t = (size_t)nkb * TN * KB * 2;
    const size_t b_xl = nprod == 1 ? 0 : b_xb, b_tl = nprod == 1 ? 0 : b_t;
    const size_t b_part = nsplit > 1 ? (size_t)2 * ((ntile_c1 + 1) / 2) * nsplit * TM * TN * 4 : 0;
    // K-part tickets of the in-kernel fold (one per 128-row tile and warp slice).
    const bool fold = nsplit > 1 && nsplit <= 16;
    const size_t b_tk = fold ? (size_t)2 * ((ntile_c1 + 1) / 2) * 8 * 4 : 0;
    const size_t o_xs = 0, o_hi = o_xs + ru(b_xs, 256), o_lo = o_hi + ru(b_xb, 256), o_th = o_lo + ru(b_xl, 256);
    const size_t o_tl = o_th + ru(b_t, 256), o_part = o_tl + ru(b_tl, 256);
    const size_t o_tk = o_part + ru(b_part, 256), o_err = o_tk + ru(b_tk, 256), total = o_err + 256;
    char *mem = nullptr;
    cudaError_t e = tc::pool_alloc(reinterpret_cast<void **>(&mem), total, cs);
    if (e != cudaSuccess)
        return na_fail(e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA,
                       std::string("tc_convolve_tc: pool allocation: ") + cudaGetErrorString(e));
    if ((reinterpret_cast<uintptr_t>(mem) & 255u) != 0) {
        cudaFreeAsync(mem, cs);
        return na_fail(TC_ECUDA, "tc_convolve_tc: the stream-ordered allocation is not 256-byte aligned");
    }
    void *xhi = mem + o_hi, *xlo = mem + o_lo, *thi = mem + o_th, *tlo = mem + o_tl;
    int *err = reinterpret_cast<int *>(mem + o_err);
    p.y = y;
    p.y_pitch = TN;
    p.y_total = ny;  // the last row stops at the end of y
    p.partial = nsplit > 1 ? reinterpret_cast<float *>(mem + o_part) : nullptr;
    p.ticket = fold ? reinterpret_cast<unsigned *>(mem + o_tk) : nullptr;
    p.err = err;
    // One launch prepares the bf16 input rows (with their zero margins), the
    // Toeplitz tiles and the zeroed tickets and error word; the tensor maps
    // are encoded on the host while it runs.
    e = tc::k2_oneshot_prep_launch(x, Nl, off, npad, xhi, nprod == 1 ? nullptr : xlo, h, (int)Ll, (int)nkb, KB, thi,
                                   nprod == 1 ? nullptr : tlo, reinterpret_cast<unsigned *>(mem + o_tk),
                                   (long long)(total - o_tk) / 4, cs);
    CUtensorMap mx_hi{}, mx_lo{}, mt_hi{}, mt_lo{}, mt2_hi{}, mt2_lo{};
    // The error word comes back through a pinned word of this thread (a
    // true asynchronous copy); pageable memory where that cannot be had.
    struct PinnedWord {
        int *p = nullptr;
        PinnedWord()
        {
            if (cudaHostAlloc(reinterpret_cast<void **>(&p), sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
                p = nullptr;
                cudaGetLastError();
            }
        }
        ~PinnedWord()
        {
            if (p)
                cudaFreeHost(p);
        }
    };
    static thread_local PinnedWord pinned;
    int herr_pageable = 0;
    int *const herr_p = pinned.p ? pinned.p : &herr_pageable;
    *herr_p = 0;
    // Rows of the X view overlap: row r starts 256 samples after row r - 1.
    if (e == cudaSuccess)
        e = tc::encode_bf16_2d(&mx_hi, xhi, (unsigned long long)nkb * KB, (unsigned long long)R,
                               (unsigned long long)TN * 2, KB, TM);
    if (e == cudaSuccess && nprod == 3)
        e = tc::encode_bf16_2d(&mx_lo, xlo, (unsigned long long)nkb * KB, (unsigned long long)R,
                               (unsigned long long)TN * 2, KB, TM);
    if (e == cudaSuccess)
        e = tc::encode_bf16_2d(&mt_hi, thi, KB, (unsigned long long)nkb * TN, KB * 2, KB, TN);
    if (e == cudaSuccess && nprod == 3)
        e = tc::encode_bf16_2d(&mt_lo, tlo, KB, (unsigned long long)nkb * TN, KB * 2, KB, TN);
    if (e == cudaSuccess)
        e = tc::encode_bf16_2d(&mt2_hi, thi, KB, (unsigned long long)nkb * TN, KB * 2, KB, TN / 2);
    if (e == cudaSuccess && nprod == 3)
        e = tc::encode_bf16_2d(&mt2_lo, tlo, KB, (unsigned long long)nkb * TN, KB * 2, KB, TN / 2);
    if (e == cudaSuccess)
        e = spair  ? tc::k2_launch_c2s(mx_hi, mx_lo, mt2_hi, mt2_lo, p, cs)
            : pair ? tc::k2_launch_c2p(mx_hi, mt2_hi, p, cs)
                   : tc::k2_launch(mx_hi, mx_lo, mt_hi, mt_lo, p, nprod, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(herr_p, err, sizeof(int), cudaMemcpyDeviceToHost, cs);
    cudaFreeAsync(mem, cs);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess)
        return na_fail(TC_ECUDA, std::string("tc_convolve_tc: ") + cudaGetErrorString(e));
    if (*herr_p)
        return na_fail(TC_ETIMEOUT, "tc_convolve_tc: a kernel's bounded wait gave up");
    return TC_OK;
}
