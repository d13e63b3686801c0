// k1_gather.cu -- K1, the FP32 output-side gather of the taches-algorithm.
//
// The paper scatters each input sample's tache e(n)*h into a ring of
// partial outputs (Sec. 4.2, the two wrapped loops). Scattering from many
// threads races. K1 computes the same sums from the output side instead:
//     y[m] = sum_k h_{v(m-k)}[k] * x[m-k]              (Eq. 4, per-sample IR)
// Each output is then written by exactly one thread, with no atomics on the
// data. The per-sample IR version v(n) is kept as a version table. A CTA whose
// input window straddles a version boundary runs once per version over a
// masked copy of its window. This is the superposition of the taches of each
// version.
//
// CTA tile: 128 outputs x KC taps, 256 threads = 8 output groups (16
// consecutive outputs each) x 32 tap sub-segments (S consecutive taps each,
// KC = 32*S).
//   * The input window (KC+128 samples) and the IR chunk (KC taps) are
//     staged in shared memory by 1-D TMA bulk copies (cp.async.bulk) that
//     complete on an mbarrier.
//   * Each thread keeps 16 accumulators and a 20-register sliding window of
//     the input. Per 4 taps it does one 128-bit load of h, one 128-bit load of
//     the next 4 input samples and 64 FMAs. The window rotates through
//     registers by compile-time renaming over 5 steps, so S is a multiple of
//     20. S/4 is odd, which makes the 128-bit shared loads conflict-free.
//   * Sub-segment sums are combined by a pairwise tree: warp shuffles, then
//     shared memory. Chunk partials go to a scratch buffer. The last CTA of
//     the tile (a ticket counter) adds them in a fixed pairwise tree and
//     writes y. The result does not depend on CTA scheduling.
#include <climits>

#include "ptx.cuh"
#include "tc_internal.h"

namespace tc {

namespace {

template <int S>
struct K1Cfg {
    static_assert(S % 20 == 0 && (S / 4) % 2 == 1, "S must be a multiple of 20 with S/4 odd");
    static constexpr int R = 16;            // outputs per thread
    static constexpr int MO = K1_MO;        // outputs per CTA
    static constexpr int KC = 32 * S;       // taps per CTA
    static constexpr int XS = KC + MO;      // staged input samples
    static constexpr int PAD = 8;           // floats before xs[0]: the last prefetches read xs[-8..-1]
    static constexpr int TAIL = 4;          // floats after hs: the last prefetch of h reads hs[KC..KC+3]
    static constexpr int STAGE = PAD + XS + KC + TAIL;
    static constexpr int RED = 32 * MO;     // floats for one piece of the chunk reduction
    static constexpr int SMEM_FLOATS = STAGE > RED ? STAGE : RED;
};

// The thread's S taps for its 16 outputs: acc[r] += h[j] * x[m0 + r - j].
// xp points at xs[ia], the lowest input sample needed by the first 4 taps.
// Logical window at step q is w_q[i] = xp[i - 4q], i in [0, 20); tap 4q+u of
// output r reads w_q[3 - u + r]. The physical register of w_q[i] is
// (i - 4q) mod 20, so the window slides without moves. The h and x loads of
// step q+1 are issued before the FMAs of step q. The prefetch after the
// last step reads padding.
template <int S>
__device__ __forceinline__ void k1_taps(const float *__restrict__ xp, const float *__restrict__ hp,
                                        float (&acc)[16])
{
    float w[20];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float4 t = reinterpret_cast<const float4 *>(xp)[i];
        w[4 * i + 0] = t.x;
        w[4 * i + 1] = t.y;
        w[4 * i + 2] = t.z;
        w[4 * i + 3] = t.w;
    }
    float4 h_nx = *reinterpret_cast<const float4 *>(hp);
    float4 x_nx = *reinterpret_cast<const float4 *>(xp - 4);
#pragma unroll 1
    for (int it = 0; it < S / 20; ++it) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int j = it * 20 + 4 * q;
            const float4 h4 = h_nx;
            const float4 xn = x_nx;
            h_nx = *reinterpret_cast<const float4 *>(hp + j + 4);
            x_nx = *reinterpret_cast<const float4 *>(xp - j - 8);
            const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int r = 0; r < 16; ++r)
                    acc[r] = fmaf(hv[u], w[(3 - u + r - 4 * q + 40) % 20], acc[r]);
            }
            w[(16 - 4 * q + 40) % 20] = xn.x;
            w[(17 - 4 * q + 40) % 20] = xn.y;
            w[(18 - 4 * q + 40) % 20] = xn.z;
            w[(19 - 4 * q + 40) % 20] = xn.w;
        }
    }
}

template <int S>
__global__ void __launch_bounds__(K1_THREADS, 3) k1_gather(const K1Params p)
{
    using C = K1Cfg<S>;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_last;
    float *xs = smem + C::PAD;
    float *hs = smem + C::PAD + C::XS;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // Block -> (item, tile, input, chunk); chunks fastest.
    const int ctot = p.nin * p.nchunk;
    long long bid = blockIdx.x;
    const int cidx = (int)(bid % ctot);
    bid /= ctot;
    const int tile = (int)(bid % p.ntile);
    const int item = (int)(bid / p.ntile);
    const int inp = cidx / p.nchunk;
    const int chunk = cidx % p.nchunk;

    const long long t0 = p.t0 + (long long)tile * C::MO;
    const int kc0 = chunk * C::KC - p.e;             // first tap of the chunk; kc0 = t0 + 1 - base (mod 4)
    const long long n_lo = t0 - kc0 - C::KC + 1;      // first staged input sample; n_lo = base (mod 4)
    const long long n_end = n_lo + C::XS;

    const float *xsrc = p.hist + ((long long)item * p.x_item_rows + (long long)inp * p.x_in_rows) * p.pitch +
                        (n_lo - p.base);
    const float *hsrc = p.ir + (long long)item * p.ir_item + (long long)inp * p.ir_in +
                        (long long)p.e * p.ir_phase + (long long)chunk * C::KC;

    const long long *vst = p.vstart + (long long)item * p.vt_item;
    const int *vsl = p.vslot + (long long)item * p.vt_item;
    const int nv = p.nver[p.vt_item ? item : 0];

    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Thread roles: lane bits 0-1 pick the sub-segment within the warp, bit 2
    // and bits 3-4 the output group, so each quarter-warp spans 2 groups x 4
    // sub-segments (conflict-free 128-bit loads for S/4 odd).
    const int s_lo = lane & 3;
    const int g = ((lane >> 2) & 1) | ((lane >> 3) << 1);
    const int s = warp * 4 + s_lo;
    const int ia = g * C::R - s * S + C::KC - 4;
    // Input samples this thread reads (inclusive): outputs t0+16g .. +15, taps kc0+sS .. +S-1.
    const long long th_hi = t0 + 16 * g + 15 - (kc0 + (long long)s * S);
    const long long th_lo = th_hi - 15 - (S - 1);

    float acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
        acc[r] = 0.f;

    uint32_t parity = 0;
    bool failed = false;
    for (int v = 0; v < nv; ++v) {
        const long long a = vst[v];
        const long long b = (v + 1 < nv) ? vst[v + 1] : LLONG_MAX;
        if (b <= n_lo || a >= n_end)
            continue;  // this version spawned no tache that reaches the tile through this chunk
        if (tid == 0) {
            mbar_arrive_expect_tx(&bar, (uint32_t)((C::XS + C::KC) * sizeof(float)));
            bulk_g2s(xs, xsrc, (uint32_t)(C::XS * sizeof(float)), &bar);
            bulk_g2s(hs, hsrc + (long long)vsl[v] * p.ir_slot, (uint32_t)(C::KC * sizeof(float)), &bar);
        }
        const bool ok = mbar_wait_bounded(&bar, parity, p.err, ERR_TIMEOUT_TMA);
        parity ^= 1u;
        if (!__syncthreads_and(ok)) {
            // Give the copies in flight a bounded chance to land before the CTA exits.
            mbar_wait_bounded(&bar, parity ^ 1u, nullptr, 0);
            failed = true;
            break;
        }
        if (a > n_lo || b < n_end) {
            // Keep only the samples that spawned their tache with version v.
            for (int i = tid; i < C::XS; i += K1_THREADS) {
                const long long n = n_lo + i;
                if (n < a || n >= b)
                    xs[i] = 0.f;
            }
            __syncthreads();
        }
        if (th_hi >= a && th_lo < b)  // only threads that see a tache of version v
            k1_taps<S>(xs + ia, hs + s * S, acc);
        fence_proxy_async_smem();
        __syncthreads();
    }
    if (failed)
        return;

    // Pairwise tree over the 32 sub-segments: lanes (s, s^1), then (s, s^2)
    // inside the warp, then warps (0,1),(2,3).. through shared memory.
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        float v = acc[r];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        acc[r] = v;
    }
    float *red = smem;  // [8 warps][128 outputs]; the stage is no longer read
    if (s_lo == 0) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
            red[warp * C::MO + g * 16 + r] = acc[r];
    }
    __syncthreads();
    float tot = 0.f;
    if (tid < C::MO) {
        const float w01 = red[0 * C::MO + tid] + red[1 * C::MO + tid];
        const float w23 = red[2 * C::MO + tid] + red[3 * C::MO + tid];
        const float w45 = red[4 * C::MO + tid] + red[5 * C::MO + tid];
        const float w67 = red[6 * C::MO + tid] + red[7 * C::MO + tid];
        tot = (w01 + w23) + (w45 + w67);
    }

    const int valid = min(C::MO, p.nout - tile * C::MO);
    float *yrow = p.y + (long long)item * p.y_pitch + (long long)tile * C::MO;
    if (ctot == 1) {
        if (tid < valid)
            yrow[tid] = tot;
        return;
    }

    // Chunk partial -> scratch; the last CTA of the tile reduces.
    float *part = p.partial + (((long long)item * p.ntile + tile) * ctot) * C::MO;
    if (tid < C::MO) {
        __stcg(part + (long long)cidx * C::MO + tid, tot);
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(p.counter + (long long)item * p.ntile + tile, 1u);
        s_last = (prev == (unsigned)(ctot - 1));
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();

    // Fixed pairwise tree over the ctot partials: pieces of 32 (adjacent
    // pairs, zero-padded), then the piece sums (adjacent pairs).
    const int npieces = (ctot + 31) / 32;  // <= 8 (ctot <= K1_MAX_CHUNKS)
    float ps[8];
#pragma unroll
    for (int pc = 0; pc < 8; ++pc) {
        ps[pc] = 0.f;
        if (pc < npieces) {
            __syncthreads();
            const int c0 = pc * 32;
            const int cn = min(32, ctot - c0);
            for (int i = tid; i < 32 * C::MO; i += K1_THREADS) {
                const int c = i / C::MO;
                const int o = i % C::MO;
                red[i] = (c < cn) ? __ldcg(part + (long long)(c0 + c) * C::MO + o) : 0.f;
            }
            __syncthreads();
            if (tid < C::MO) {
                float v[32];
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    v[c] = red[c * C::MO + tid];
#pragma unroll
                for (int wdt = 16; wdt >= 1; wdt >>= 1) {
#pragma unroll
                    for (int c = 0; c < wdt; ++c)
                        v[c] = v[2 * c] + v[2 * c + 1];
                }
                ps[pc] = v[0];
            }
        }
    }
    if (tid < C::MO) {
        const float t = ((ps[0] + ps[1]) + (ps[2] + ps[3])) + ((ps[4] + ps[5]) + (ps[6] + ps[7]));
        if (tid < valid)
            yrow[tid] = t;
    }
    if (tid == 0)
        p.counter[(long long)item * p.ntile + tile] = 0u;
}

constexpr int kMaxDevices = 64;

template <int S>
cudaError_t launch_variant(const K1Params &p, cudaStream_t st)
{
    using C = K1Cfg<S>;
    static bool attr_set[kMaxDevices] = {};
    const size_t smem = (size_t)C::SMEM_FLOATS * sizeof(float);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k1_gather<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        attr_set[dev] = true;
    }
    const long long grid = (long long)p.nitems * p.ntile * p.nin * p.nchunk;
    if (grid <= 0)
        return cudaSuccess;
    if (grid > 0x7fffffffLL)
        return cudaErrorInvalidConfiguration;
    k1_gather<S><<<(unsigned)grid, K1_THREADS, smem, st>>>(p);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

int k1_taps_per_thread(int variant)
{
    switch (variant) {
    case K1_S20: return 20;
    case K1_S60: return 60;
    case K1_S100: return 100;
    case K1_S260: return 260;
    default: return 0;
    }
}

int k1_chunk_taps(int variant) { return 32 * k1_taps_per_thread(variant); }

size_t k1_smem_bytes(int variant)
{
    switch (variant) {
    case K1_S20: return sizeof(float) * K1Cfg<20>::SMEM_FLOATS;
    case K1_S60: return sizeof(float) * K1Cfg<60>::SMEM_FLOATS;
    case K1_S100: return sizeof(float) * K1Cfg<100>::SMEM_FLOATS;
    case K1_S260: return sizeof(float) * K1Cfg<260>::SMEM_FLOATS;
    default: return 0;
    }
}

cudaError_t k1_launch(const K1Params &p, int variant, cudaStream_t st)
{
    if (p.nin * p.nchunk > K1_MAX_CHUNKS || p.nin < 1 || p.nchunk < 1 || p.e < 0 || p.e > 3 ||
        (p.base & 3) != 0 || (p.pitch & 3) != 0)
        return cudaErrorInvalidValue;
    switch (variant) {
    case K1_S20: return launch_variant<20>(p, st);
    case K1_S60: return launch_variant<60>(p, st);
    case K1_S100: return launch_variant<100>(p, st);
    case K1_S260: return launch_variant<260>(p, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc
