// noalloc.cu -- tc_convolve_noalloc: the one-shot FP32 convolution of
// tc_convolve without any device or host allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point of use. For
// example, code running inside a real-time audio callback, where an
// allocation can block for an unbounded time and break the deadline. Or a
// host whose own allocator owns all device memory and forbids outside
// allocations. tc_convolve opens a temporary stream and allocates its history,
// IR copies and split-sum scratch on every call. This entry point instead puts
// all of that in one file-scope device array of fixed size.
//
// The array (kNoAllocScratchBytes, 32 MiB) is part of this library's device
// image. Every GPU on which the library's kernels are loaded holds it until
// the process exits. Its device address is looked up once per device, with
// that device current, on the first call made on that device. Make that first
// call outside any CUDA stream capture.
//
// All calls share the array, and it keeps the last call's contents. So each
// call first clears what must start at zero: the zero margins of the input
// history, the split-sum ticket counters and the error word. Calls that
// overlap on the GPU (two streams, or two host threads without ordering)
// race on the array and give wrong results. Serialise them.
#include <cstdio>
#include <mutex>
#include <string>
#include <utility>

#include "../../include/taches.h"
#include "tc_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;             // 32 MiB
constexpr long long kScratchFloats = (long long)(kNoAllocScratchBytes / sizeof(float));
constexpr long long kPiece = 4096;                              // outputs per K1 launch
constexpr long long kPieceTiles = kPiece / tc::K1_MO;  // tickets needed per launch
static_assert(kPieceTiles <= 64, "the ticket area holds 64 counters");
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
            return na_fail(TC_ECUDA, std::string("tc_convolve_noalloc: cudaGetSymbolAddress: ") +
                                         cudaGetErrorString(e));
        p.ready = true;
    }
    *out = p;
    return TC_OK;
}

}  // namespace

extern "C" tc_status tc_convolve_noalloc(const float *x, size_t N, const float *h, size_t L, float *y,
                                         void *cuda_stream)
{
    if (!x || !h || !y)
        return na_fail(TC_EINVAL, "tc_convolve_noalloc: x, h or y is NULL");
    if (N == 0 || L == 0)
        return na_fail(TC_EINVAL, "tc_convolve_noalloc: N and L must be > 0");
    // Role swap as in tc_convolve (Sec. 3.2): the shorter operand is the IR.
    if (N < L && !tc::no_role_swap()) {
        std::swap(x, h);
        std::swap(N, L);
    }

    // Scratch layout (floats, 64-float aligned segments):
    //   [counters + error word][IR: 4 shifted copies of Lpad][history row][split-sum partials]
    const long long Ll = (long long)L, Nl = (long long)N;
    const long long keep = ru(Ll + tc::K1_KC_MAX + 8, 4);          // zero samples before x[0]
    const long long Lpad = ru(Ll + 4 + tc::K1_KC_MAX, 4);
    const long long ny = Nl + Ll - 1;
    const long long cap = ru(keep + ny + tc::K1_MO + 160, 64);       // history row: zeros, x, zeros
    // Chunk sums: every tile of one piece (4096 outputs) with the most chunks
    // any variant may use; one ticket per tile.
    const long long off_ctr = 0;                                    // tickets, error word
    const long long off_ir = 128;
    const long long off_hist = off_ir + ru(4 * Lpad, 64);
    const long long off_part = off_hist + cap;
    const long long need = off_part + tc::k1_partial_floats_max(Ll, 1, kPieceTiles);
    if (need > kScratchFloats) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "tc_convolve_noalloc: N=%zu, L=%zu need %.1f MiB of scratch; the fixed array holds %.0f MiB "
                 "(use tc_convolve, which allocates)",
                 N, L, need * 4.0 / (1 << 20), kNoAllocScratchBytes / double(1 << 20));
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

    cudaStream_t cs = (cudaStream_t)cuda_stream;
    float *base = P.scratch;
    unsigned *counters = reinterpret_cast<unsigned *>(base + off_ctr);  // [kPieceTiles]
    int *err = reinterpret_cast<int *>(base + off_ctr + 64);
    float *ir = base + off_ir;
    float *hist = base + off_hist;
    float *part = base + off_part;

#define NA_CU(call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return na_fail(TC_ECUDA, std::string("tc_convolve_noalloc: " #call ": ") + cudaGetErrorString(e_)); \
    } while (0)

    // Clear what must start at zero: counters and error word, and the
    // history's zero margins before x[0] and after x[N-1].
    NA_CU(cudaMemsetAsync(counters, 0, 128 * sizeof(float), cs));
    NA_CU(cudaMemsetAsync(hist, 0, (size_t)keep * sizeof(float), cs));
    NA_CU(cudaMemsetAsync(hist + keep + Nl, 0, (size_t)(cap - keep - Nl) * sizeof(float), cs));
    NA_CU(cudaMemcpyAsync(hist + keep, x, (size_t)Nl * sizeof(float), cudaMemcpyDeviceToDevice, cs));
    NA_CU(tc::ir_prep_launch(h, Ll, Ll, 1, ir, 4 * Lpad, Lpad, Lpad, cs));

    tc::K1Params p{};
    p.hist = hist;
    p.pitch = cap;
    p.base = -keep;
    p.x_item_rows = 1;
    p.x_in_rows = 0;
    p.ir = ir;
    p.ir_slot = 4 * Lpad;
    p.ir_item = 0;
    p.ir_in = 0;
    p.ir_phase = Lpad;
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
    for (long long t0 = 0; t0 < ny; t0 += kPiece) {
        const long long n = (ny - t0 < kPiece) ? ny - t0 : kPiece;
        p.t0 = t0;
        p.nout = (int)n;
        p.ntile = (int)((n + tc::K1_MO - 1) / tc::K1_MO);
        p.e = tc::k1_shift_e(t0, p.base);
        p.y = y + t0;
        p.y_pitch = n;
        tc::K1Plan plan{};
        NA_CU(tc::k1_plan(Ll, p.e, 1, 1, p.ntile, -1, &plan));
        if (plan.ctas * tc::K1_MO > tc::k1_partial_floats_max(Ll, 1, kPieceTiles))
            return na_fail(TC_EINVAL, "tc_convolve_noalloc: internal: chunk-sum scratch too small");
        NA_CU(tc::k1_launch(p, plan, cs));
    }
    int herr = 0;
    NA_CU(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, cs));
    NA_CU(cudaStreamSynchronize(cs));
#undef NA_CU
    if (herr)
        return na_fail(TC_ETIMEOUT, "tc_convolve_noalloc: a kernel's bounded wait gave up");
    return TC_OK;
}
