// k1_gather.cu -- K1, the FP32 output-side gather of the taches-algorithm.
//
// The paper scatters each input sample's tache e(n)*h into a ring of
// partial outputs (Sec. 4.2, the two wrapped loops). Scattering from many
// threads races. K1 computes the same sums from the output side instead:
//     y[m] = sum_k h_{v(m-k)}[k] * x[m-k]              (Eq. 4, per-sample IR)
// Each output is then written by exactly one thread, with no atomics on the
// data. The per-sample IR version v(n) is kept as a version table. A chunk
// whose input window straddles a version boundary is computed once per
// version over the samples that spawned their tache with that version: the
// superposition of the taches of each version.
//
// CTA = one output tile (128 samples of one item) x one tap chunk-task (KC =
// 640 P taps of one input). 256 threads = 8 output groups (16 consecutive
// outputs) x 32 tap sub-segments.
//   * For each IR version that reaches the tile through the chunk, one thread
//     issues two 1-D TMA bulk copies (cp.async.bulk) into shared memory: the
//     input window (KC+128 samples) and the IR chunk (KC taps, from the
//     shifted copy that makes it 16-byte aligned). They complete on an
//     mbarrier, which that thread waits on (bounded); the others wait at the
//     CTA barrier, which costs no issue slots.
//   * In pass p a thread covers taps [20(32p+s), +20) of the chunk with 16
//     accumulators and a 20-register input window. The window rotates by
//     compile-time renaming inside the fully unrolled 20-tap pass, with
//     128-bit shared loads (conflict-free: 20/4 is odd). When the window
//     straddles a version boundary, the samples of other versions are zeroed
//     in shared memory first; threads with no sample of the version skip the
//     pass.
//   * Epilogue: pairwise tree over the 32 sub-segments (warp shuffles, then
//     shared memory). The chunk sum goes to scratch, then a ticket counter
//     picks the tile's last CTA, which adds the chunk sums by a pairwise
//     binary-counter stack per output column and writes y. The order is fixed
//     by the decomposition, not by scheduling.
#include <algorithm>
#include <climits>

#include "ptx.cuh"
#include "tc_internal.h"

namespace tc {

namespace {

// Crossfade share alpha(n) of a version starting at s with a ramp of R
// samples: clamp((n - s + 1) / R, 0, 1). mode 1: the first version (always
// 1); mode -1: no next version (always 0).
__device__ __forceinline__ float ramp_alpha(long long n, long long s, int R, int mode)
{
    if (mode > 0)
        return 1.f;
    if (mode < 0)
        return 0.f;
    const long long d = n - s + 1;
    if (d <= 0)
        return 0.f;
    if (d >= R)
        return 1.f;
    return (float)d / (float)R;
}

// True if any of xs[lo, hi) is nonzero (+0 and -0 count as zero); a CTA-wide
// barrier: every thread of the block calls it.
__device__ __forceinline__ bool any_nonzero(const float *xs, int lo, int hi)
{
    bool nz = false;
    for (int i = lo + (int)threadIdx.x; i < hi; i += K1_THREADS)
        nz |= (__float_as_uint(xs[i]) << 1) != 0u;
    return __syncthreads_or(nz) != 0;
}

// Floor division by a positive divisor.
__device__ __forceinline__ long long floor_div(long long x, long long d)
{
    const long long q = x / d;
    return (x % d < 0) ? q - 1 : q;
}

template <int P>
struct K1Cfg {
    static constexpr int MO = K1_MO;          // outputs per tile
    static constexpr int SEG = K1_SEG;        // taps per thread per pass
    static constexpr int KC = 32 * SEG * P;   // taps per chunk
    static constexpr int XS = KC + MO;        // staged input samples
    static constexpr int STAGE = XS + KC;     // window, then IR chunk
    static constexpr int LEVELS = 12;         // pairwise stack depth: chunk-tasks per tile < 4096
    static constexpr int RED = 8 * MO;
    static constexpr int TAIL = RED + LEVELS * MO;  // reduction area, overlays the finished stage
    static constexpr int SMEM_FLOATS = STAGE > TAIL ? STAGE : TAIL;
};

// One pass: 20 taps for 16 outputs, fully unrolled. xp = xs + ia, the lowest
// input sample read by the first 4 taps. Logical window w_q[i] = xp[i - 4q];
// tap 4q+u of output r reads w_q[3-u+r]. Physical register of w_q[i] is
// (i - 4q) mod 20, so the window slides without moves.
__device__ __forceinline__ void k1_pass(const float *__restrict__ xp, const float *__restrict__ hp,
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
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const float4 h4 = *reinterpret_cast<const float4 *>(hp + 4 * q);
        float4 xn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < 4)
            xn = *reinterpret_cast<const float4 *>(xp - 4 * q - 4);
        const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                acc[r] = fmaf(hv[u], w[(3 - u + r - 4 * q + 40) % 20], acc[r]);
        }
        if (q < 4) {
            w[(16 - 4 * q + 40) % 20] = xn.x;
            w[(17 - 4 * q + 40) % 20] = xn.y;
            w[(18 - 4 * q + 40) % 20] = xn.z;
            w[(19 - 4 * q + 40) % 20] = xn.w;
        }
    }
}

// LIST = false: one uniform launch described by p0.
// LIST = true: a work list (continuous batching of independent streams).
// CTA b belongs to item i with cta_begin[i] <= b < cta_begin[i+1]; the item's
// parameters are copied to shared memory, then the CTA runs as in a uniform
// launch over that item alone.
template <int P, bool LIST, bool EXT = false>
__global__ void __launch_bounds__(K1_THREADS, 4)
    k1_gather(const K1Params p0, const K1Params *__restrict__ items, const long long *__restrict__ cta_begin,
              int nlist)
{
    using C = K1Cfg<P>;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_last;
    __shared__ __align__(16) K1Params s_item;
    __shared__ long long s_first;
    if (LIST) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = nlist - 1;  // last item whose first CTA is <= blockIdx.x
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cta_begin[mid] <= (long long)blockIdx.x)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            s_first = cta_begin[lo];
            s_last = lo;
        }
        __syncthreads();
        constexpr int W = (int)(sizeof(K1Params) / sizeof(int));
        static_assert(sizeof(K1Params) % sizeof(int) == 0, "K1Params copies as ints");
        const int *src = reinterpret_cast<const int *>(items + s_last);
        int *dst = reinterpret_cast<int *>(&s_item);
        for (int i = threadIdx.x; i < W; i += K1_THREADS)
            dst[i] = src[i];
        __syncthreads();
    }
    const K1Params &p = LIST ? s_item : p0;
    float *const xs = smem;
    float *const hs = smem + C::XS;
    float *const red = smem;                  // [8 warps][16 r][8 g], after the last pass
    float *const lv = red + C::RED;           // [LEVELS][128] pairwise stack of the last CTA

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // Block -> (item, tile, input, chunk); chunks fastest.
    const int ctot = p.nin * p.nchunk;
    long long bid = LIST ? (long long)blockIdx.x - s_first : (long long)blockIdx.x;
    const int cidx = (int)(bid % ctot);
    bid /= ctot;
    const int tile = (int)(bid % p.ntile);
    const int item = (int)(bid / p.ntile);
    const int inp = cidx / p.nchunk;
    const int chunk = cidx % p.nchunk;

    const long long t0 = p.t0 + (long long)tile * C::MO;
    const int kc0 = chunk * C::KC - p.e;             // first tap; kc0 = t0 + 1 - base (mod 4)
    const long long n_lo = t0 - kc0 - C::KC + 1;      // first staged sample; n_lo = base (mod 4)
    const long long n_end = n_lo + C::XS;

    const float *xsrc = p.hist + ((long long)item * p.x_item_rows + (long long)inp * p.x_in_rows) * p.pitch +
                        (n_lo - p.base);
    const float *hsrc = p.ir + (long long)item * p.ir_item + (long long)inp * p.ir_in +
                        (long long)p.e * p.ir_phase + (long long)chunk * C::KC;

    const long long *vst = p.vstart + (long long)item * p.vt_item;
    const int *vsl = p.vslot + (long long)item * p.vt_item;
    // Crossfade ramps (EXT instances only; the others compile without them).
    const int *vrm = (EXT && p.vramp) ? p.vramp + (long long)item * p.vt_item : nullptr;
    const int nv = p.nver[p.vt_item ? item : 0];
    // After the last input sample every sample is zero (a flush): nothing past x_end spawns a tache.
    const long long x_end = p.has_end ? p.x_end : LLONG_MAX;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Lane bits 0-1: sub-segment within the warp; bit 2 and bits 3-4: output
    // group. Each quarter-warp spans 2 groups x 4 sub-segments.
    const int s_lo = lane & 3;
    const int g = ((lane >> 2) & 1) | ((lane >> 3) << 1);
    const int s = warp * 4 + s_lo;
    const long long out_hi = t0 + 16 * g + 15;  // last output of this thread

    float acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
        acc[r] = 0.f;

    constexpr int PA = (P >= 4) ? (P + 2) / 3 : P;  // passes fed by part A
    constexpr bool SPLIT = PA < P;
    constexpr int HA = 32 * C::SEG * PA;            // IR taps of part A
    constexpr int XA = C::KC - HA;                  // first staged sample of part A
    static_assert(XA % 4 == 0 && HA % 4 == 0, "parts start on 16-byte boundaries");

    uint32_t parity = 0;
    for (int v = 0; v < nv; ++v) {
        // Version v's samples: [a, b). With crossfades, version v takes over
        // over ra samples from a on and hands over to v + 1 over rb samples
        // from bn on; weight w(n) = alpha_v(n) - alpha_{v+1}(n).
        const long long a = vst[v];
        const long long bn = (v + 1 < nv) ? vst[v + 1] : LLONG_MAX;
        const int ra = (EXT && vrm && v > 0) ? vrm[v] : 1;
        const int rb = (EXT && vrm && v + 1 < nv) ? vrm[v + 1] : 1;
        const long long b = (bn == LLONG_MAX) ? LLONG_MAX : bn + rb - 1;
        const long long be = b < x_end ? b : x_end;  // samples of this version that can be nonzero: [a, be)
        if (be <= n_lo || a >= n_end)
            continue;  // this version spawned no tache that reaches the tile through this chunk
        // Two parts on two mbarriers (chunks of 4 passes or more): part A =
        // the IR taps of passes [0, PA) and the input samples they read,
        // xs[XA, XS); part B = the rest. Passes [0, PA) start once part A has
        // landed, while part B is still in flight.
        const float *hv = hsrc + (long long)vsl[v] * p.ir_slot;
        bool ok = true;
        if (tid == 0) {
            if (SPLIT) {
                mbar_arrive_expect_tx(&bar[0], (uint32_t)((C::XS - XA + HA) * sizeof(float)));
                bulk_g2s(xs + XA, xsrc + XA, (uint32_t)((C::XS - XA) * sizeof(float)), &bar[0]);
                bulk_g2s(hs, hv, (uint32_t)(HA * sizeof(float)), &bar[0]);
                mbar_arrive_expect_tx(&bar[1], (uint32_t)((XA + C::KC - HA) * sizeof(float)));
                bulk_g2s(xs, xsrc, (uint32_t)(XA * sizeof(float)), &bar[1]);
                bulk_g2s(hs + HA, hv + HA, (uint32_t)((C::KC - HA) * sizeof(float)), &bar[1]);
            } else {
                mbar_arrive_expect_tx(&bar[0], (uint32_t)(C::STAGE * sizeof(float)));
                bulk_g2s(xs, xsrc, (uint32_t)(C::XS * sizeof(float)), &bar[0]);
                bulk_g2s(hs, hv, (uint32_t)(C::KC * sizeof(float)), &bar[0]);
            }
            ok = mbar_wait_bounded(&bar[0], parity, p.err, ERR_TIMEOUT_TMA);
        }
        if (!__syncthreads_and(ok)) {
            // Give the copies in flight a bounded chance to land before the CTA exits.
            if (tid == 0) {
                mbar_wait_bounded(&bar[0], parity, nullptr, 0);
                if (SPLIT)
                    mbar_wait_bounded(&bar[1], parity, nullptr, 0);
            }
            __syncthreads();
            return;
        }
        // A window that straddles a version boundary keeps only the samples
        // that spawned their tache with this version: [n_lo, a) and
        // [b, n_end) of the staged window are zeroed, in each part once it
        // has landed.
        const bool straddle = (a > n_lo || b < n_end);
        // A ramp inside the window: weight the staged samples instead of masking.
        const bool ramped = EXT && ((ra > 1 && a + ra - 1 > n_lo) || (rb > 1 && bn < n_end));
        const long long za = a - n_lo, zb = b - n_lo;
        const int z0 = (za > 0) ? (za < C::XS ? (int)za : C::XS) : 0;
        const int z1 = (b < n_end) ? (zb > 0 ? (int)zb : 0) : C::XS;
        auto weigh = [&](int lo, int hi) {  // xs[i] *= w(n_lo + i), i in [lo, hi)
            for (int i = lo + tid; i < hi; i += K1_THREADS) {
                const long long n = n_lo + i;
                const float w = ramp_alpha(n, a, ra, v == 0) - ramp_alpha(n, bn, rb, bn == LLONG_MAX ? -1 : 0);
                xs[i] = (w == 0.f) ? 0.f : xs[i] * w;
            }
        };
        if (ramped) {
            weigh(SPLIT ? XA : 0, C::XS);
            __syncthreads();
        } else if (straddle) {
            constexpr int r0 = SPLIT ? XA : 0;
            for (int i = r0 + tid; i < z0; i += K1_THREADS)
                xs[i] = 0.f;
            for (int i = max(z1, r0) + tid; i < C::XS; i += K1_THREADS)
                xs[i] = 0.f;
            __syncthreads();
        }
        // Passes this thread runs for this version: pass p covers sub-segment
        // seg = 32 p + s, i.e. taps kc0 + 20 seg + [0, 19], and reads samples
        // out_hi - kc0 - 20 seg - [0, 34]. It is needed iff
        //   that range meets [a, be): 20 seg <= out_hi - kc0 - a  and
        //                             20 seg >  out_hi - kc0 - 34 - be,
        //   and its first tap is inside the IR: kc0 + 20 seg <= L - 1.
        // Those bounds are solved once here instead of tested per pass.
        const long long seg_hi = min(floor_div(out_hi - kc0 - a, C::SEG), floor_div((long long)p.L - 1 - kc0, C::SEG));
        const long long seg_lo =
            (be == LLONG_MAX) ? -(1LL << 40) : floor_div(out_hi - kc0 - (15 + C::SEG - 1) - be, C::SEG) + 1;
        const int p_lo = (int)max(0LL, min((long long)P, -floor_div(s - seg_lo, 32)));
        const int p_hi = (int)max(-1LL, min((long long)P - 1, floor_div(seg_hi - s, 32)));
        int pass = p_lo;
        int ia = g * 16 - (p_lo * 32 + s) * C::SEG + C::KC - 4;
        const float *hp = hs + (p_lo * 32 + s) * C::SEG;
        // Pass p reads xs[KC - 640 (p + 1), KC - 640 p + 128) and hs[640 p, 640 (p + 1)):
        // passes below PA touch part A only.
        const int pa_end = min(p_hi, PA - 1);
        // Zero gating (exact): passes whose staged input is all zero add
        // nothing, so they are skipped. Passes below PA read xs[XA, XS); the
        // rest read xs[0, XA + 128).
        if (EXT && p.zero_skip && !any_nonzero(xs, SPLIT ? XA : 0, C::XS)) {
            const int k = max(0, pa_end - pass + 1);
            pass += k;
            ia -= k * 32 * C::SEG;
            hp += k * 32 * C::SEG;
        }
#pragma unroll 1
        for (; pass <= pa_end; ++pass, ia -= 32 * C::SEG, hp += 32 * C::SEG)
            k1_pass(xs + ia, hp, acc);
        if (SPLIT) {
            bool okb = true;
            if (tid == 0)
                okb = mbar_wait_bounded(&bar[1], parity, p.err, ERR_TIMEOUT_TMA);
            if (!__syncthreads_and(okb)) {
                if (tid == 0)
                    mbar_wait_bounded(&bar[1], parity, nullptr, 0);
                __syncthreads();
                return;
            }
            if (ramped) {
                weigh(0, XA);
                __syncthreads();
            } else if (straddle) {
                for (int i = tid; i < min(z0, XA); i += K1_THREADS)
                    xs[i] = 0.f;
                for (int i = z1 + tid; i < XA; i += K1_THREADS)
                    xs[i] = 0.f;
                __syncthreads();
            }
            if (EXT && p.zero_skip && !any_nonzero(xs, 0, XA + 128))
                pass = p_hi + 1;
#pragma unroll 1
            for (; pass <= p_hi; ++pass, ia -= 32 * C::SEG, hp += 32 * C::SEG)
                k1_pass(xs + ia, hp, acc);
        }
        parity ^= 1u;
        fence_proxy_async_smem();
        __syncthreads();
    }

    // Pairwise tree over the 32 sub-segments: lanes (s, s^1), then (s, s^2)
    // inside the warp, then warps (0,1),(2,3).. through shared memory.
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        float v = acc[r];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (s_lo == 0)
            red[warp * C::MO + r * 8 + g] = v;  // the 8 writing lanes hit 8 banks
    }
    __syncthreads();
    float tot = 0.f;
    const int o = tid;                        // output within the tile (threads < 128)
    if (tid < C::MO) {
        const int ti = (o % 16) * 8 + o / 16;
        const float w01 = red[0 * C::MO + ti] + red[1 * C::MO + ti];
        const float w23 = red[2 * C::MO + ti] + red[3 * C::MO + ti];
        const float w45 = red[4 * C::MO + ti] + red[5 * C::MO + ti];
        const float w67 = red[6 * C::MO + ti] + red[7 * C::MO + ti];
        tot = (w01 + w23) + (w45 + w67);
    }

    const int valid = min(C::MO, p.nout - tile * C::MO);
    float *yrow = p.y + (long long)item * p.y_pitch + (long long)tile * C::MO;
    if (ctot == 1) {
        if (tid < valid)
            yrow[tid] = tot;
        return;
    }

    // Chunk sum -> scratch; the last CTA of the tile reduces.
    float *part = p.partial + (((long long)item * p.ntile + tile) * ctot) * C::MO;
    if (tid < C::MO) {
        __stcg(part + (long long)cidx * C::MO + o, tot);
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
    if (tid < C::MO) {
        // Fixed pairwise tree over the chunk sums, per output column: a
        // binary-counter stack in this thread's column (older block on the left).
        // The sums are loaded eight at a time, so that a tile with hundreds of
        // chunk-tasks (long IRs, small chunks) waits for one L2 round trip per
        // eight sums instead of one per sum; the order of the adds is unchanged.
        for (int cb = 0; cb < ctot; cb += 8) {
            float v8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                v8[j] = (cb + j < ctot) ? __ldcg(part + (long long)(cb + j) * C::MO + o) : 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (cb + j >= ctot)
                    break;
                float carry = v8[j];
                int cc = cb + j, l = 0;
                while (cc & 1) {
                    carry = lv[l * C::MO + o] + carry;
                    cc >>= 1;
                    ++l;
                }
                lv[l * C::MO + o] = carry;
            }
        }
        float y = 0.f;
        bool first = true;
        for (int l = 0; l < C::LEVELS; ++l) {
            if ((ctot >> l) & 1) {
                const float v = lv[l * C::MO + o];
                y = first ? v : v + y;
                first = false;
            }
        }
        if (tid < valid)
            yrow[tid] = y;
    }
    if (tid == 0)
        p.counter[(long long)item * p.ntile + tile] = 0u;
}

constexpr int kMaxDevices = 64;

struct DevInfo {
    bool ready = false;
    int sms = 0;
    int blocks_per_sm[K1_NVARIANTS] = {};
};
DevInfo g_dev[kMaxDevices];

template <int P>
size_t smem_bytes()
{
    return (size_t)K1Cfg<P>::SMEM_FLOATS * sizeof(float);
}

template <int P>
cudaError_t prepare_variant(int dev, int variant)
{
    const size_t smem = smem_bytes<P>();
    cudaError_t e = cudaFuncSetAttribute(k1_gather<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_gather<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_gather<P, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // All of the unified L1/shared storage as shared memory: four CTAs of the
    // largest chunk need almost all of it.
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_gather<P, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_gather<P, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_gather<P, false, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k1_gather<P, false>, K1_THREADS, smem);
    if (e != cudaSuccess)
        return e;
    g_dev[dev].blocks_per_sm[variant] = n > 0 ? n : 1;
    return cudaSuccess;
}

cudaError_t device_info(DevInfo **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    DevInfo &d = g_dev[dev];
    if (!d.ready) {
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = prepare_variant<1>(dev, K1_P1);
        if (e == cudaSuccess)
            e = prepare_variant<4>(dev, K1_P4);
        if (e == cudaSuccess)
            e = prepare_variant<K1_PBIG>(dev, K1_P11);
        if (e != cudaSuccess)
            return e;
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

}  // namespace

int k1_chunk_taps(int variant)
{
    switch (variant) {
    case K1_P1: return 32 * K1_SEG * 1;
    case K1_P4: return 32 * K1_SEG * 4;
    case K1_P11: return 32 * K1_SEG * K1_PBIG;
    default: return 0;
    }
}

cudaError_t k1_plan(long long L, int e, int nin, int nitems, int ntile, int forced_variant, K1Plan *plan)
{
    DevInfo *d = nullptr;
    cudaError_t err = device_info(&d);
    if (err != cudaSuccess)
        return err;
    if (L < 1 || nin < 1 || nitems < 1 || ntile < 1 || e < 0 || e > 3)
        return cudaErrorInvalidValue;
    const long long tiles = (long long)nitems * ntile;
    int chosen = -1;
    if (forced_variant >= 0 && forced_variant < K1_NVARIANTS) {
        chosen = forced_variant;
    } else {
        // The largest chunk that still gives about four waves of CTAs and
        // wastes < 10 % on the padded last chunk; otherwise the smallest chunk
        // whose chunk-task count fits the tile's pairwise stack.
        static const int order[] = {K1_P11, K1_P4, K1_P1};
        for (int v : order) {
            const long long kc = k1_chunk_taps(v);
            const long long nchunk = (L + e + kc - 1) / kc;
            const long long ctas = tiles * nchunk * nin;
            const long long waves = ctas / ((long long)d->blocks_per_sm[v] * d->sms);
            const bool tight = nchunk * kc <= L + L / 10 + 64;
            if (nchunk * nin <= K1_MAX_CHUNK_TASKS && waves >= 4 && tight) {
                chosen = v;
                break;
            }
        }
        if (chosen < 0) {
            static const int small_first[] = {K1_P1, K1_P4, K1_P11};
            for (int v : small_first) {
                const long long kc = k1_chunk_taps(v);
                if ((L + e + kc - 1) / kc * nin <= K1_MAX_CHUNK_TASKS) {
                    chosen = v;
                    break;
                }
            }
        }
        if (chosen < 0)
            return cudaErrorInvalidValue;
    }
    const long long kc = k1_chunk_taps(chosen);
    const long long nchunk = (L + e + kc - 1) / kc;
    if (nchunk * nin > K1_MAX_CHUNK_TASKS)
        return cudaErrorInvalidValue;
    plan->variant = chosen;
    plan->nchunk = (int)nchunk;
    plan->ctas = tiles * nchunk * nin;
    return cudaSuccess;
}

long long k1_partial_floats_max(long long L, int nin, long long tiles)
{
    const long long kc = k1_chunk_taps(K1_P1);
    const long long ctot = (L + 3 + kc - 1) / kc * nin;
    return std::max<long long>(1, tiles * std::min<long long>(ctot, K1_MAX_CHUNK_TASKS)) * K1_MO;
}

cudaError_t k1_launch(K1Params &p, const K1Plan &plan, cudaStream_t st)
{
    if ((p.base & 3) != 0 || (p.pitch & 3) != 0 || p.e < 0 || p.e > 3)
        return cudaErrorInvalidValue;
    DevInfo *d = nullptr;
    cudaError_t e = device_info(&d);
    if (e != cudaSuccess)
        return e;
    p.nchunk = plan.nchunk;
    if (plan.ctas <= 0)
        return cudaSuccess;
    if (plan.ctas > 0x7fffffffLL)
        return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)plan.ctas;
    // Crossfades and zero gating run in separate kernel instances, so that
    // the plain instances compile exactly as without them.
    const bool ext = p.vramp != nullptr || p.zero_skip != 0;
    switch (plan.variant) {
    case K1_P1:
        if (ext)
            k1_gather<1, false, true><<<grid, K1_THREADS, smem_bytes<1>(), st>>>(p, nullptr, nullptr, 0);
        else
            k1_gather<1, false><<<grid, K1_THREADS, smem_bytes<1>(), st>>>(p, nullptr, nullptr, 0);
        break;
    case K1_P4:
        if (ext)
            k1_gather<4, false, true><<<grid, K1_THREADS, smem_bytes<4>(), st>>>(p, nullptr, nullptr, 0);
        else
            k1_gather<4, false><<<grid, K1_THREADS, smem_bytes<4>(), st>>>(p, nullptr, nullptr, 0);
        break;
    case K1_P11:
        if (ext)
            k1_gather<K1_PBIG, false, true><<<grid, K1_THREADS, smem_bytes<K1_PBIG>(), st>>>(p, nullptr, nullptr, 0);
        else
            k1_gather<K1_PBIG, false><<<grid, K1_THREADS, smem_bytes<K1_PBIG>(), st>>>(p, nullptr, nullptr, 0);
        break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

const void *k1_list_kernel(int variant, size_t *smem)
{
    DevInfo *d = nullptr;
    if (device_info(&d) != cudaSuccess)
        return nullptr;
    switch (variant) {
    case K1_P1: *smem = smem_bytes<1>(); return reinterpret_cast<const void *>(&k1_gather<1, true>);
    case K1_P4: *smem = smem_bytes<4>(); return reinterpret_cast<const void *>(&k1_gather<4, true>);
    case K1_P11: *smem = smem_bytes<K1_PBIG>(); return reinterpret_cast<const void *>(&k1_gather<K1_PBIG, true>);
    default: return nullptr;
    }
}

cudaError_t k1_launch_list(const K1Params *d_items, const long long *d_cta_begin, int nitems, long long total_ctas,
                           int variant, cudaStream_t st)
{
    DevInfo *d = nullptr;
    cudaError_t e = device_info(&d);
    if (e != cudaSuccess)
        return e;
    if (nitems < 1 || total_ctas <= 0)
        return cudaSuccess;
    if (total_ctas > 0x7fffffffLL)
        return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)total_ctas;
    const K1Params none{};
    switch (variant) {
    case K1_P1: k1_gather<1, true><<<grid, K1_THREADS, smem_bytes<1>(), st>>>(none, d_items, d_cta_begin, nitems); break;
    case K1_P4: k1_gather<4, true><<<grid, K1_THREADS, smem_bytes<4>(), st>>>(none, d_items, d_cta_begin, nitems); break;
    case K1_P11:
        k1_gather<K1_PBIG, true><<<grid, K1_THREADS, smem_bytes<K1_PBIG>(), st>>>(none, d_items, d_cta_begin, nitems);
        break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace tc
