// k3_mimo_tc.cu -- K3: the MIMO contraction on the tcgen05 tensor cores.
//
// MIMO (multichannel use, Sec. 6): output o is the sum over the inputs i of
// the convolutions x_i * h_{o,i} (Eq. 4 per pair). For a tile of 1024
// consecutive output times, write t = Tb - 8 r - p (row r < 128, phase
// p < 8). Then, with k' = k + p,
//     y_o[t] = sum_i sum_k' x_i[Tb - 8 r - k'] * h_{o,i}[k' - p],
// a product D[r][(p, o)] = sum_i sum_k' A_i[r][k'] B_i[k'][(p, o)] with
//     A_i[r][k'] = x_i[Tb - 8 r - k'],   B_i[k'][(p, o)] = h_{o,i}[k' - p].
// M = 128 rows, N = 8 phases x 16 outputs = 128 columns, K = inputs x taps.
//
// A needs no materialised matrix. With the input stored reversed,
// xr_i[j] = x_i[R - j], row r of A is xr_i[s0 + 8 r + k'], so in the K-major
// no-swizzle layout (8-row x 16-byte core matrices) consecutive rows are 16
// bytes apart and the core matrix that follows along K starts 16 bytes later:
// one contiguous stretch of xr in shared memory is A for every K block of a
// chunk, each block just moves the descriptor's start by 64 bytes. A CTA
// computes two adjacent tiles (2048 outputs) from one stretch, so that every
// B tile loaded from L2 feeds both.
// B (the phase-shifted IR tiles, 128 x 32 per K block) is materialised once
// per IR version by k3_tprep and loaded by 2-D TMA with a 64-byte swizzle.
// The phase shift sits in B so that every A start stays 16-byte aligned.
//
// Roles as in K2: warp 0 lane 0 loads A chunks (1-D bulk copies) and B tiles
// (2-D TMA), warp 1 lane 0 issues tcgen05.mma (kind::f16, BF16 in, FP32 in
// TMEM) into interleaved accumulator chains (consecutive K blocks into
// different chains: a 128 x 128 x 16 MMA is short, and back-to-back MMAs into
// one accumulator wait on each other), warp 2 owns TMEM, eight epilogue warps
// drain TMEM runs of `range` K blocks (all chains) into FP32 register sums. A tile's K range (inputs x taps)
// is split over `nsplit` CTAs; k3_reduce adds their partials in a fixed
// pairwise tree and writes y. Precision: plain BF16 or the hi/lo split
// (A_hi B_hi + A_hi B_lo + A_lo B_hi). Every wait is bounded.
#include <algorithm>
#include <cuda_bf16.h>

#include "tc5.cuh"
#include "tc_internal.h"

namespace tc {

namespace {

constexpr int K3_M = 128;                 // rows (output times of one phase)
constexpr int K3_N = 128;                 // 8 phases x 16 outputs
constexpr int K3_KB = 32;                 // taps per K block
constexpr int K3_KBC = 64;                // K blocks per A chunk
constexpr int K3_TP = 2;                  // output tiles per CTA (they share every B tile)
constexpr int K3_SPAN = K3_KB * K3_KBC + 1024 * K3_TP;  // xr elements of one A chunk (both tiles' rows)
constexpr int K3_BBYTES = K3_N * K3_KB * 2;     // 8 KB per B tile
constexpr int K3_ABYTES = K3_SPAN * 2;          // 8 KB per A chunk part
constexpr int K3_ROLE_WARPS = 4;
constexpr int K3_EPI_WARPS = 8;
constexpr int K3_THREADS = 32 * (K3_ROLE_WARPS + K3_EPI_WARPS);

template <int NPROD>
struct K3Cfg {
    // Tiles x chains x TMEM buffers = 4 blocks of 128 columns. Independent
    // accumulators keep the tensor pipe busy: plain BF16 (2 MMAs per K block
    // and tile) uses 2 chains per tile and, having at most a few TMEM runs per
    // unit, drains without a second buffer; the split (6 MMAs per block and
    // tile) uses 1 chain per tile, double-buffered.
    static constexpr int CH = NPROD == 1 ? 2 : 1;
    static constexpr int NB = 4 / (K3_TP * CH);
    // A B stage holds the B tiles of one group of GS K blocks (one full and
    // one empty barrier per group; block j of a group goes to chain j % CH);
    // 192 KB of B tiles in flight, in 3 stages. Every stage costs a barrier
    // round trip and a commit whatever its size, so the stages are as large
    // as three of them fit: 8 (BF16) or 4 (split) K blocks. Measured on the
    // 16 x 16 MIMO workload against 4 / 2 blocks in 5 stages of 160 KB:
    // BF16 70.5 % -> 84.6 %, split 83.3 % -> 92.9 % of the sustained peak.
    static constexpr int GS = NPROD == 1 ? 8 : 4;
    static constexpr int BBLK = NPROD == 1 ? K3_BBYTES : 2 * K3_BBYTES;  // one K block (hi[, lo])
    static constexpr int BSTAGE = GS * BBLK;
    static constexpr int NS = 192 * 1024 / BSTAGE;
    static constexpr int ASLOT = NPROD == 1 ? K3_ABYTES : 2 * K3_ABYTES;
    static constexpr int AOFF = NS * BSTAGE;                           // A slots after the B ring
    static constexpr int SMEM = AOFF + 2 * ASLOT + 1024;               // + alignment slack
};

template <int NPROD>
__global__ void __launch_bounds__(K3_THREADS, 1)
    k3_mimo(const __grid_constant__ CUtensorMap mb_hi, const __grid_constant__ CUtensorMap mb_lo, const K3Params p)
{
    using C = K3Cfg<NPROD>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[C::NS];
    __shared__ __align__(8) uint64_t empty[C::NS];
    __shared__ __align__(8) uint64_t afull[2];
    __shared__ __align__(8) uint64_t aempty[2];
    __shared__ __align__(8) uint64_t accfull[2];
    __shared__ __align__(8) uint64_t accfree[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;

    uint8_t *const smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    // Unit = (pair of output tiles, K part). K blocks are numbered g = input * nkbp + kb.
    const int part = (int)(blockIdx.x % p.nsplit);
    const int pair = (int)(blockIdx.x / p.nsplit);  // tiles 2 pair and 2 pair + 1 (ntile is even)
    const long long gtot = (long long)p.nin * p.nkbp;
    const long long gbeg = (long long)part * p.kb_per;
    const long long gend = min(gbeg + (long long)p.kb_per, gtot);
    const int nk = (int)max(gend - gbeg, 0LL);           // a multiple of K3_KBC
    const int nchunk = nk / K3_KBC;
    const int nr = (nk + p.range - 1) / p.range;         // TMEM runs
    // xr offset of row 0 of tile 2 pair + 1; tile 2 pair starts 1024 later.
    const long long s0 = (long long)(p.ntile - 2 - 2 * pair) * 1024;

    if (tid == 0) {
        for (int i = 0; i < C::NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&afull[i], 1);
            mbar_init(&aempty[i], 1);
            mbar_init(&accfull[i], 1);
            mbar_init(&accfree[i], K3_EPI_WARPS);
        }
        s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 2)
        tmem_alloc(&tmem_base, 4 * K3_N);  // buffers x tiles x chains
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: A chunks and B tiles ----
            const char *xh = static_cast<const char *>(p.xr_hi);
            const char *xl = static_cast<const char *>(p.xr_lo);
            int i = 0;
            for (int c = 0; c < nchunk && !s_fail; ++c) {
                const long long g0 = gbeg + (long long)c * K3_KBC;
                const int inp = (int)(g0 / p.nkbp);
                const int kb0 = (int)(g0 % p.nkbp);
                const int slot = c & 1;
                const int use = c >> 1;
                if (use > 0 && !mbar_wait_bounded(&aempty[slot], (uint32_t)((use - 1) & 1), p.err, ERR_TIMEOUT_TMA)) {
                    s_fail = 1;
                    break;
                }
                uint8_t *as = smem + C::AOFF + slot * C::ASLOT;
                const long long off = ((long long)inp * p.xr_pitch + s0 + (long long)kb0 * K3_KB) * 2;
                mbar_arrive_expect_tx(&afull[slot], (uint32_t)C::ASLOT);
                bulk_g2s(as, xh + off, (uint32_t)K3_ABYTES, &afull[slot]);
                if (NPROD == 3)
                    bulk_g2s(as + K3_ABYTES, xl + off, (uint32_t)K3_ABYTES, &afull[slot]);
                for (int b = 0; b < K3_KBC; b += C::GS, ++i) {  // i counts groups
                    const int st = i % C::NS;
                    const int ub = i / C::NS;
                    if (ub > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((ub - 1) & 1), p.err, ERR_TIMEOUT_TMA)) {
                        s_fail = 1;
                        break;
                    }
                    uint8_t *bs = smem + st * C::BSTAGE;
                    const int row = (int)(((long long)inp * p.nkbp + kb0 + b) * K3_N);
                    mbar_arrive_expect_tx(&full[st], (uint32_t)C::BSTAGE);
#pragma unroll
                    for (int j = 0; j < C::GS; ++j) {
                        tma_load_2d(bs + j * C::BBLK, &mb_hi, 0, row + j * K3_N, &full[st]);
                        if (NPROD == 3)
                            tma_load_2d(bs + j * C::BBLK + K3_BBYTES, &mb_lo, 0, row + j * K3_N, &full[st]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            // CH accumulator chains: K blocks go in groups of CH, block j of a
            // group into chain j, with the chains' MMAs interleaved, so that
            // consecutive MMAs never wait on one another's accumulator. A run
            // (range K blocks, a multiple of CH) fills the CH chains of TMEM
            // buffer run % NB; the epilogue adds the chains.
            const uint32_t idesc = umma_idesc_bf16(K3_M, K3_N);
            int i = 0, g = 0, run = 0;  // K blocks, groups, runs
            uint32_t acc = tmem;
            bool first = true;
            // Descriptors advance by adding byte offsets >> 4 to their start
            // field (shared-memory addresses stay below 2^18 bytes).
            const uint64_t bdesc0 = umma_desc_sw64(smem_u32(smem));
            for (int c = 0; c < nchunk && !s_fail; ++c) {
                const int slot = c & 1;
                if (!mbar_wait_bounded(&afull[slot], (uint32_t)((c >> 1) & 1), p.err, ERR_TIMEOUT_MMA)) {
                    s_fail = 1;
                    break;
                }
                tc_fence_after_sync();
                const uint64_t adesc0 = umma_desc_noswz(smem_u32(smem + C::AOFF + slot * C::ASLOT), 16, 128);
                for (int b = 0; b < K3_KBC; b += C::GS, i += C::GS, ++g) {
                    if (i % p.range == 0) {
                        // A new TMEM run in buffer run % NB, once its previous drain is done.
                        const int buf = run % C::NB;
                        const int reuse = run / C::NB;
                        if (reuse > 0 &&
                            !mbar_wait_bounded(&accfree[buf], (uint32_t)((reuse - 1) & 1), p.err, ERR_TIMEOUT_MMA)) {
                            s_fail = 1;
                            break;
                        }
                        tc_fence_after_sync();
                        acc = tmem + (uint32_t)(buf * K3_TP * C::CH * K3_N);
                        first = true;
                    }
                    const int st = g % C::NS;
                    if (!mbar_wait_bounded(&full[st], (uint32_t)((g / C::NS) & 1), p.err, ERR_TIMEOUT_MMA)) {
                        s_fail = 1;
                        break;
                    }
                    tc_fence_after_sync();
                    const uint64_t bst = bdesc0 + (uint64_t)((st * C::BSTAGE) >> 4);
#pragma unroll
                    for (int kk = 0; kk < K3_KB / 16; ++kk) {
                        // A rows: 16 bytes apart inside a core matrix; core
                        // matrices 16 bytes apart along K, 128 bytes along M.
                        // K block b + j starts 64 bytes after block b + j - 1;
                        // tile 2 pair (t = 0) reads 2048 bytes further on.
                        const uint64_t a = adesc0 + (uint64_t)((2 * (b * K3_KB + kk * 16)) >> 4);
#pragma unroll
                        for (int j = 0; j < C::GS; ++j) {
                            // The first MMA of a chain in a run starts its accumulator.
                            const uint32_t accum = (first && kk == 0 && j < C::CH) ? 0u : 1u;
                            const int ch = j % C::CH;
#pragma unroll
                            for (int t = 0; t < K3_TP; ++t)
                                umma_bf16(acc + (t * C::CH + ch) * K3_N, a + (uint64_t)(j * 4 + (1 - t) * 128),
                                          bst + (uint64_t)((j * C::BBLK + kk * 32) >> 4), idesc, accum);
                        }
                        if (NPROD == 3) {
#pragma unroll
                            for (int j = 0; j < C::GS; ++j)
#pragma unroll
                                for (int t = 0; t < K3_TP; ++t)
                                    umma_bf16(acc + (t * C::CH + j % C::CH) * K3_N, a + (uint64_t)(j * 4 + (1 - t) * 128),
                                              bst + (uint64_t)((j * C::BBLK + K3_BBYTES + kk * 32) >> 4), idesc, 1u);
#pragma unroll
                            for (int j = 0; j < C::GS; ++j)
#pragma unroll
                                for (int t = 0; t < K3_TP; ++t)
                                    umma_bf16(acc + (t * C::CH + j % C::CH) * K3_N,
                                              a + (uint64_t)(j * 4 + (1 - t) * 128 + (K3_ABYTES >> 4)),
                                              bst + (uint64_t)((j * C::BBLK + kk * 32) >> 4), idesc, 1u);
                        }
                    }
                    first = false;
                    umma_commit(&empty[st]);
                    if ((i + C::GS) % p.range == 0 || i + C::GS == nk) {
                        umma_commit(&accfull[run % C::NB]);  // the run is complete in TMEM
                        ++run;
                    }
                }
                if (s_fail)
                    break;
                umma_commit(&aempty[slot]);  // the A chunk is free once its MMAs are done
            }
        }
    } else if (warp >= K3_ROLE_WARPS) {
        // ---- epilogue: drain each run into FP32 register sums ----
        const int ew = warp - K3_ROLE_WARPS;
        const int q = warp & 3;    // TMEM lane quarter this warp may access
        const int half = ew >> 2;  // columns [64 half, 64 half + 64)
        float sum[K3_TP][64];
#pragma unroll
        for (int t = 0; t < K3_TP; ++t)
#pragma unroll
            for (int j = 0; j < 64; ++j)
                sum[t][j] = 0.f;
        bool ok = true;
        for (int r = 0; r < nr; ++r) {
            const int buf = r % C::NB;
            const uint32_t par = (uint32_t)((r / C::NB) & 1);
            bool got = true;
            if (lane == 0)  // bounded, and abandoned early if another role has failed
                got = mbar_wait_limited(&accfull[buf], par, p.err, ERR_TIMEOUT_MMA, kWaitLimitNs, &s_fail);
            got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
            if (!got) {
                ok = false;
                break;
            }
            mbar_try_wait(&accfull[buf], par);
            tc_fence_after_sync();
            const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * K3_TP * C::CH * K3_N + half * 64);
#pragma unroll
            for (int t = 0; t < K3_TP; ++t) {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    float v0[16];
                    tmem_ld_32x16(src + (t * C::CH) * K3_N + cc * 16, v0);
                    if (C::CH == 2) {
                        float v1[16];
                        tmem_ld_32x16(src + (t * C::CH + 1) * K3_N + cc * 16, v1);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            sum[t][cc * 16 + j] += v0[j] + v1[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            sum[t][cc * 16 + j] += v0[j];
                    }
                }
            }
            tc_fence_before_sync();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&accfree[buf]);
        }
        if (ok && !s_fail) {
            const int row = q * 32 + lane;
#pragma unroll
            for (int t = 0; t < K3_TP; ++t) {
                const int tile = 2 * pair + t;
                float *dst = p.partial + (((long long)tile * p.nsplit + part) * K3_M + row) * K3_N + half * 64;
#pragma unroll
                for (int j = 0; j < 64; j += 4)
                    *reinterpret_cast<float4 *>(dst + j) =
                        make_float4(sum[t][j], sum[t][j + 1], sum[t][j + 2], sum[t][j + 3]);
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 4 * K3_N);
    }
}

// Adds the nsplit partials of each (tile, row, column) by a fixed pairwise
// tree (adjacent pairs, zero-padded to 64 leaves) and writes y_o[t] for the
// outputs inside [t0, t0 + nout): column = 16 p + o, t = Tb - 8 r - p.
__global__ void k3_reduce(const float *__restrict__ partial, int ntile, int nsplit, int nout_ch, int nout,
                          float *y, long long y_pitch)
{
    const long long total = (long long)ntile * K3_M * K3_N;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(q % K3_N);
        const int row = (int)((q / K3_N) % K3_M);
        const int tile = (int)(q / ((long long)K3_N * K3_M));
        const int ph = col >> 4, o = col & 15;
        const long long t = (long long)tile * 1024 + 1023 - 8 * row - ph;  // relative to t0
        if (o >= nout_ch || t >= nout)
            continue;
        const float *src = partial + (((long long)tile * nsplit) * K3_M + row) * K3_N + col;
        float v[64];
#pragma unroll
        for (int s = 0; s < 64; ++s)
            v[s] = (s < nsplit) ? src[(long long)s * K3_M * K3_N] : 0.f;
#pragma unroll
        for (int w = 32; w >= 1; w >>= 1) {
#pragma unroll
            for (int s = 0; s < w; ++s)
                v[s] = v[2 * s] + v[2 * s + 1];
        }
        y[(long long)o * y_pitch + t] = v[0];
    }
}

// Reversed bf16 hi/lo copies of the inputs for one launch:
//   xr_i[j] = x_i[R - j], x_i[n] = hist[i * pitch + n - base] for n < n_end, 0 beyond,
// hi = bf16(x), lo = bf16(x - hi), for j < span.
__global__ void k3_rev(const float *__restrict__ hist, long long pitch, long long base, int nin, long long R,
                       long long n_end, long long span, __nv_bfloat16 *xh, __nv_bfloat16 *xl, long long xr_pitch)
{
    const long long total = (long long)nin * span;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / span);
        const long long j = q % span;
        const long long n = R - j;
        const float v = (n < n_end) ? hist[(long long)i * pitch + (n - base)] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        xh[(long long)i * xr_pitch + j] = hi;
        xl[(long long)i * xr_pitch + j] = lo;
    }
}

// Phase-shifted IR tiles of one IR version, bf16 hi/lo, [nin][nkbp][128][32]:
//   B[i][kb][16 p + o][j] = h_{o,i}[32 kb + j - p]  (0 outside [0, L) and for o >= nout),
// reading h_{o,i}[k] = ir[(o * nin + i) * set_stride + k] (the unshifted copy).
__global__ void k3_tprep(const float *__restrict__ ir, long long set_stride, int nin, int nout, int L, int nkbp,
                         __nv_bfloat16 *bh, __nv_bfloat16 *bl)
{
    const long long total = (long long)nin * nkbp * K3_N * K3_KB;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q % K3_KB);
        const int col = (int)((q / K3_KB) % K3_N);
        const long long kb = (q / ((long long)K3_KB * K3_N)) % nkbp;
        const int i = (int)(q / ((long long)K3_KB * K3_N * nkbp));
        const int ph = col >> 4, o = col & 15;
        const long long k = kb * K3_KB + j - ph;
        float v = 0.f;
        if (o < nout && k >= 0 && k < L)
            v = ir[((long long)o * nin + i) * set_stride + k];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        bh[q] = hi;
        bl[q] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

unsigned k3_grid(long long work)
{
    long long b = (work + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min<long long>(b, 16384));
}

}  // namespace

int k3_kblocks_per_input(long long L) { return (int)((L + 7 + K3_KB * K3_KBC - 1) / (K3_KB * K3_KBC)) * K3_KBC; }
int k3_chunk_blocks() { return K3_KBC; }
int k3_tiles_per_cta() { return K3_TP; }
long long k3_xr_span(int ntile, int nkbp) { return (long long)ntile * 1024 + (long long)nkbp * K3_KB + 1024; }

cudaError_t k3_tprep_launch(const float *ir, long long set_stride, int nin, int nout, int L, int nkbp, void *bh,
                            void *bl, cudaStream_t st)
{
    const long long work = (long long)nin * nkbp * K3_N * K3_KB;
    k3_tprep<<<k3_grid(work), 256, 0, st>>>(ir, set_stride, nin, nout, L, nkbp, (__nv_bfloat16 *)bh,
                                            (__nv_bfloat16 *)bl);
    count_launch();
    return cudaGetLastError();
}

cudaError_t k3_rev_launch(const float *hist, long long pitch, long long base, int nin, long long R, long long n_end,
                          long long span, void *xh, void *xl, long long xr_pitch, cudaStream_t st)
{
    k3_rev<<<k3_grid((long long)nin * span), 256, 0, st>>>(hist, pitch, base, nin, R, n_end, span,
                                                           (__nv_bfloat16 *)xh, (__nv_bfloat16 *)xl, xr_pitch);
    count_launch();
    return cudaGetLastError();
}

size_t k3_smem_bytes(int nprod) { return nprod == 1 ? K3Cfg<1>::SMEM : K3Cfg<3>::SMEM; }

cudaError_t k3_launch(const CUtensorMap &mb_hi, const CUtensorMap &mb_lo, const K3Params &p, int nprod, float *y,
                      long long y_pitch, int nout_ch, int nout, cudaStream_t st)
{
    static bool attr[64][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64 || (nprod != 1 && nprod != 3) || p.nsplit < 1 || p.nsplit > 64 || p.range < 1 ||
        p.kb_per % K3_KBC != 0 || p.nkbp % K3_KBC != 0 || nout_ch < 1 || nout_ch > 16 ||
        p.range % (nprod == 1 ? K3Cfg<1>::GS : K3Cfg<3>::GS) != 0)
        return cudaErrorInvalidValue;
    const int vi = nprod == 1 ? 0 : 1;
    const size_t smem = k3_smem_bytes(nprod);
    if (!attr[dev][vi]) {
        e = nprod == 1 ? cudaFuncSetAttribute(k3_mimo<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(k3_mimo<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        attr[dev][vi] = true;
    }
    if (p.ntile % K3_TP != 0)
        return cudaErrorInvalidValue;
    const long long units = (long long)(p.ntile / K3_TP) * p.nsplit;
    if (units <= 0)
        return cudaSuccess;
    if (nprod == 1)
        k3_mimo<1><<<(unsigned)units, K3_THREADS, smem, st>>>(mb_hi, mb_lo, p);
    else
        k3_mimo<3><<<(unsigned)units, K3_THREADS, smem, st>>>(mb_hi, mb_lo, p);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const long long work = (long long)p.ntile * K3_M * K3_N;
    k3_reduce<<<k3_grid(work), 256, 0, st>>>(p.partial, p.ntile, p.nsplit, nout_ch, nout, y, y_pitch);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tc
