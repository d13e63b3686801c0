// k2_toeplitz_tc.cu -- K2: the shared-IR contraction on the tcgen05 tensor cores.
//
// When C channels share one IR h, a block of outputs of every channel is one
// dense product (Sec. 4.2 suggests organising a channel's data "as a part of
// a matrix" for GPUs):
//     Y[c][t0+i] = sum_j X[c][w0+j] * T[i][j],   T[i][j] = h[t0 + i - w0 - j],
// with X the input history and T a Toeplitz matrix of the IR. With the
// window start w0 = t0 - L + 1 - delta on an 8-sample grid, T depends only on
// delta and on j's block, not on t0. So its tiles are materialised once per IR
// version (k2_tprep) and shared by every output tile of every push.
//
// Tile: M = 128 channels (TMEM lanes) x N = 256 outputs (TMEM columns) per CTA
// (the default kernels pair two CTAs into M = 256, tcgen05 cta_group::2), K in
// blocks of 64 samples for plain BF16 (128-byte swizzled rows) and 32 for the
// split (64-byte swizzled rows). Warp roles: warp 0 lane 0 issues
// TMA tensor loads of the X tile (bf16 history) and the T tile into a stage
// ring; warp 1 lane 0 issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulate
// in TMEM) and commits each stage back to the producer; warp 2 owns the TMEM
// allocation; eight epilogue warps read the accumulators out (tcgen05.ld).
// Precision modes: plain BF16 (X_hi T_hi) and the hi/lo split (X_hi T_hi +
// X_hi T_lo + X_lo T_hi), all into the same FP32 accumulator.
//
// FP32 accumulation in TMEM loses accuracy with the length of a serial run
// (measured at L = 96000: BF16-split error 4.4e-6 at 16 K blocks, 6.2e-6 at
// 48, 2e-5 at 256). So the MMA
// thread accumulates a tile's K blocks in runs of `range` blocks, alternating
// between two TMEM accumulators. Eight epilogue warps drain each finished run
// into FP32 running sums in registers (round-to-nearest adds), which overlaps
// the next run's MMAs; the tensor core never waits for the drain. A tile's K
// range may also be split over `nsplit` CTAs (wave balance). Their sums are
// added in a fixed pairwise tree: inside the kernel, by the warp that stores
// the last part of its slice, or by k2_reduce. Every wait is an mbarrier wait
// bounded by %globaltimer, and a failing role raises a shared flag so the
// others stop early.
#include <algorithm>
#include <cuda_bf16.h>

#include "tc5.cuh"
#include "tc_internal.h"

namespace tc {

namespace {

constexpr int K2_M = 128;
constexpr int K2_N = 256;
constexpr int K2_KB = 32;   // K block of the BF16 split: rows of 64 bytes (64-byte swizzle)
constexpr int K2_KB1 = 64;  // K block of plain BF16: rows of 128 bytes (128-byte swizzle)
constexpr int K2_ROLE_WARPS = 4;   // producer, MMA, TMEM owner, spare
constexpr int K2_EPI_WARPS = 8;    // two per TMEM lane quarter (column halves)
constexpr int K2_THREADS = 32 * (K2_ROLE_WARPS + K2_EPI_WARPS);
constexpr int K2_XBYTES1 = K2_M * K2_KB1 * 2;  // 16 KB
constexpr int K2_TBYTES1 = K2_N * K2_KB1 * 2;  // 32 KB

template <int NPROD>
struct K2Cfg {
    static constexpr int KB = NPROD == 1 ? K2_KB1 : K2_KB;  // samples per K block
    static constexpr int XB = K2_M * KB * 2, TB = K2_N * KB * 2;
    static constexpr int XOFF_LO = XB;  // X_lo after X_hi (split only)
    static constexpr int TOFF = NPROD == 1 ? XB : 2 * XB;
    static constexpr int BLK = NPROD == 1 ? XB + TB : 2 * (XB + TB);  // one K block
    // A pipeline stage holds GS consecutive K blocks (one full and one empty
    // barrier per stage). A K block of a 128 x 256 tile already carries 4
    // (plain) or 6 (split) MMAs of 128 x 256 x 16, and a deeper ring of
    // one-block stages measured faster here than fewer two-block stages (the
    // split: 72 % vs 58 % of peak).
    static constexpr int GS = 1;
    static constexpr int STAGE = GS * BLK;
    static constexpr int NS = 4;                    // stages
    static constexpr int SMEM = NS * STAGE + 1024;  // + alignment slack
};

// Outputs of row c from column col on that may be written: lim, and with a
// flat destination of y_total elements (a row view writing the caller's
// output directly) no further than its end.
__device__ __forceinline__ long long k2_ylim(const K2Params &p, long long lim, long long c, long long col)
{
    return p.y_total > 0 ? min(lim, p.y_total - c * p.y_pitch - col) : lim;
}

// K parts folded inside the kernel (no k2_reduce launch): every epilogue warp
// owns a slice of its CTA's tile (32 channels x 128 outputs). After a warp has
// stored its slice of one K part's sums, it takes a ticket for that slice; the
// warp that takes the last ticket reads all the parts back from L2 and adds
// them by the same fixed pairwise tree as k2_reduce (adjacent pairs, zero
// padded), so the result does not depend on which part finished last, and
// writes y. Nothing waits: a slice whose tickets are not all taken is simply
// not folded. Up to K2_FOLD_MAX parts.
constexpr int K2_FOLD_MAX = 16;

__device__ __forceinline__ float4 k2_add4(float4 a, float4 b)
{
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// NS parts of RG = 16 / NS rows at a time (at most 16 loads of 16 bytes in
// flight per lane). The tree adds adjacent pairs level by level and carries
// an odd last element up unchanged, which gives the same sums as the zero
// padded tree of k2_reduce (x + 0 = x).
template <int NS>
__device__ __forceinline__ void k2_fold_rows(const K2Params &p, const float *src, float *dst, long long lim,
                                             long long col, int c, int nrow)
{
    constexpr int RG = NS >= 16 ? 1 : 16 / NS;
    const long long part_stride = (long long)K2_M * K2_N;
    for (int r0 = 0; r0 < nrow; r0 += RG) {
        float4 v[RG][NS];
#pragma unroll
        for (int g = 0; g < RG; ++g)
#pragma unroll
            for (int s = 0; s < NS; ++s)
                v[g][s] = r0 + g < nrow
                              ? __ldcg(reinterpret_cast<const float4 *>(src + s * part_stride + (r0 + g) * K2_N))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int g = 0; g < RG; ++g) {
#pragma unroll
            for (int n = NS; n > 1; n = (n + 1) / 2) {
#pragma unroll
                for (int s = 0; s < n / 2; ++s)
                    v[g][s] = k2_add4(v[g][2 * s], v[g][2 * s + 1]);
                if (n & 1)
                    v[g][n / 2] = v[g][n - 1];
            }
            if (r0 + g >= nrow)
                continue;
            const long long lr = k2_ylim(p, lim, c + r0 + g, col);
            if (lr <= 0)
                continue;
            float *d = dst + (long long)(c + r0 + g) * p.y_pitch;
            if (lr >= 4 && (reinterpret_cast<uintptr_t>(d) & 15) == 0) {
                *reinterpret_cast<float4 *>(d) = v[g][0];
            } else {
                d[0] = v[g][0].x;
                if (lr > 1)
                    d[1] = v[g][0].y;
                if (lr > 2)
                    d[2] = v[g][0].z;
                if (lr > 3)
                    d[3] = v[g][0].w;
            }
        }
    }
}

// Folds slice (q, half) of 128-channel tile tc1, output tile tile_o: rows
// q*32 .. q*32+31, this lane's four outputs 128 half + 4 lane .. + 3.
__device__ __forceinline__ void k2_fold_slice(const K2Params &p, int tc1, int tile_o, int q, int half, int lane)
{
    const int c = tc1 * K2_M + q * 32;  // first channel of the slice
    const int nrow = min(32, p.C - c);
    if (nrow <= 0)
        return;
    const float *src = p.partial + ((long long)tc1 * p.ntile_o + tile_o) * p.nsplit * K2_M * K2_N +
                       (long long)(q * 32) * K2_N + half * 128 + lane * 4;
    const long long col = (long long)tile_o * K2_N + half * 128 + lane * 4;  // this lane's first output
    float *dst = p.y + col;
    const long long lim = (long long)p.nout - col;
    switch (p.nsplit) {
#define K2_FOLD_CASE(n)                                    \
    case n:                                                \
        k2_fold_rows<n>(p, src, dst, lim, col, c, nrow); \
        break;
        K2_FOLD_CASE(2) K2_FOLD_CASE(3) K2_FOLD_CASE(4) K2_FOLD_CASE(5) K2_FOLD_CASE(6) K2_FOLD_CASE(7)
        K2_FOLD_CASE(8) K2_FOLD_CASE(9) K2_FOLD_CASE(10) K2_FOLD_CASE(11) K2_FOLD_CASE(12) K2_FOLD_CASE(13)
        K2_FOLD_CASE(14) K2_FOLD_CASE(15) K2_FOLD_CASE(16)
#undef K2_FOLD_CASE
    default:
        break;  // 1 part needs no fold; more than K2_FOLD_MAX parts go to k2_reduce
    }
}

template <int NPROD>
__global__ void __launch_bounds__(K2_THREADS, 1)
    k2_toeplitz(const __grid_constant__ CUtensorMap mx_hi, const __grid_constant__ CUtensorMap mx_lo,
                const __grid_constant__ CUtensorMap mt_hi, const __grid_constant__ CUtensorMap mt_lo, const K2Params p)
{
    using C = K2Cfg<NPROD>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[C::NS];
    __shared__ __align__(8) uint64_t empty[C::NS];
    __shared__ __align__(8) uint64_t accfull[2];
    __shared__ __align__(8) uint64_t accfree[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;

    // Swizzled tiles need 512-byte aligned stages.
    uint8_t *const smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    // Unit = (channel tile, output tile, K part).
    long long u = blockIdx.x;
    const int part = (int)(u % p.nsplit);
    u /= p.nsplit;
    const int tile_o = (int)(u % p.ntile_o);
    const int tile_c = (int)(u / p.ntile_o);
    const int kb0 = part * p.kb_per;
    const int kb1 = min(kb0 + p.kb_per, p.nkb);
    const int nk = max(kb1 - kb0, 0);
    const int nr = (nk + p.range - 1) / p.range;  // TMEM runs of this unit
    const int c0 = tile_c * K2_M;
    const long long xcol0 = p.x_col0 + (long long)tile_o * K2_N;  // history column of the tile's window start

    if (tid == 0) {
        for (int i = 0; i < C::NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accfree[i], K2_EPI_WARPS);
        }
        s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 2)
        tmem_alloc(&tmem_base, 2 * K2_N);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer ----
            for (int gi = 0; gi * C::GS < nk && !s_fail; ++gi) {
                const int st = gi % C::NS;
                const int use = gi / C::NS;
                if (use > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((use - 1) & 1), p.err, ERR_TIMEOUT_TMA)) {
                    s_fail = 1;
                    break;
                }
                const int nb = min(C::GS, nk - gi * C::GS);  // K blocks in this stage
                mbar_arrive_expect_tx(&full[st], (uint32_t)(nb * C::BLK));
                for (int j = 0; j < nb; ++j) {
                    uint8_t *sb = smem + st * C::STAGE + j * C::BLK;
                    const int kb = kb0 + gi * C::GS + j;
                    const int xc = (int)(xcol0 + (long long)kb * C::KB);
                    tma_load_2d(sb, &mx_hi, xc, c0, &full[st]);
                    if (NPROD == 3)
                        tma_load_2d(sb + C::XOFF_LO, &mx_lo, xc, c0, &full[st]);
                    tma_load_2d(sb + C::TOFF, &mt_hi, 0, kb * K2_N, &full[st]);
                    if (NPROD == 3)
                        tma_load_2d(sb + C::TOFF + C::TB, &mt_lo, 0, kb * K2_N, &full[st]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            // Runs are whole stages (range is a multiple of GS).
            const uint32_t idesc = umma_idesc_bf16(K2_M, K2_N);
            // Descriptors advance by adding byte offsets >> 4 to the start field.
            const uint64_t d0 = NPROD == 1 ? umma_desc_sw128(smem_u32(smem)) : umma_desc_sw64(smem_u32(smem));
            int gi = 0;
            for (int r = 0; r < nr && !s_fail; ++r) {
                const int buf = r & 1;
                const int reuse = r >> 1;  // earlier runs in this buffer
                if (reuse > 0 &&
                    !mbar_wait_bounded(&accfree[buf], (uint32_t)((reuse - 1) & 1), p.err, ERR_TIMEOUT_MMA)) {
                    s_fail = 1;
                    break;
                }
                tc_fence_after_sync();
                const uint32_t acc = tmem + (uint32_t)(buf * K2_N);
                const int iend = min(nk, (r + 1) * p.range);
                for (bool first = true; gi * C::GS < iend; ++gi) {
                    const int st = gi % C::NS;
                    if (!mbar_wait_bounded(&full[st], (uint32_t)((gi / C::NS) & 1), p.err, ERR_TIMEOUT_MMA)) {
                        s_fail = 1;
                        break;
                    }
                    tc_fence_after_sync();
                    const int nb = min(C::GS, nk - gi * C::GS);
                    for (int j = 0; j < nb; ++j, first = false) {
                        const uint64_t sd = d0 + (uint64_t)((st * C::STAGE + j * C::BLK) >> 4);
#pragma unroll
                        for (int kk = 0; kk < C::KB / 16; ++kk) {
                            // 16 bf16 = 32 bytes along the swizzled row.
                            const uint64_t xh = sd + (uint64_t)(kk * 2);
                            const uint64_t th = sd + (uint64_t)((C::TOFF + kk * 32) >> 4);
                            umma_bf16(acc, xh, th, idesc, (first && kk == 0) ? 0u : 1u);
                            if (NPROD == 3) {
                                const uint64_t xl = sd + (uint64_t)((C::XOFF_LO + kk * 32) >> 4);
                                const uint64_t tl = sd + (uint64_t)((C::TOFF + C::TB + kk * 32) >> 4);
                                umma_bf16(acc, xh, tl, idesc, 1u);
                                umma_bf16(acc, xl, th, idesc, 1u);
                            }
                        }
                    }
                    umma_commit(&empty[st]);  // the stage is free once these MMAs are done
                }
                if (s_fail)
                    break;
                umma_commit(&accfull[buf]);  // the run is complete in TMEM
            }
        }
    } else if (warp >= K2_ROLE_WARPS) {
        // ---- epilogue: drain each run into FP32 register sums ----
        const int ew = warp - K2_ROLE_WARPS;
        const int q = warp & 3;          // TMEM lane quarter this warp may access
        const int half = ew >> 2;        // column half: outputs [128 half, 128 half + 128)
        float sum[128];
#pragma unroll
        for (int j = 0; j < 128; ++j)
            sum[j] = 0.f;
        bool ok = true;
        for (int r = 0; r < nr; ++r) {
            const int buf = r & 1;
            const uint32_t par = (uint32_t)((r >> 1) & 1);
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
            const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * K2_N + half * 128);
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                float v[16];
                tmem_ld_32x16(src + cc * 16, v);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    sum[cc * 16 + j] += v[j];
            }
            tc_fence_before_sync();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&accfree[buf]);
        }
        const int ch = q * 32 + lane;  // channel within the tile
        const int c = c0 + ch;
        if (ok && !s_fail && c < p.C) {
            float *dst;
            long long lim;
            if (p.nsplit == 1) {
                dst = p.y + (long long)c * p.y_pitch + (long long)tile_o * K2_N + half * 128;
                lim = k2_ylim(p, p.nout - (long long)tile_o * K2_N - half * 128, c,
                              (long long)tile_o * K2_N + half * 128);
            } else {
                dst = p.partial + ((((long long)tile_c * p.ntile_o + tile_o) * p.nsplit + part) * K2_M + ch) * K2_N +
                      half * 128;
                lim = 128;
            }
            // 16-byte stores only where the row is 16-byte aligned: a y row of
            // pitch n starts at c n floats (n = L - 1 in a flush is often odd).
            if (lim >= 128 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                for (int j = 0; j < 128; j += 4)
                    *reinterpret_cast<float4 *>(dst + j) = make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 128; ++j)
                    if (j < lim)
                        dst[j] = sum[j];
            }
        }
        // K parts folded here: the warp that takes this slice's last ticket adds them.
        const bool go = __shfl_sync(0xffffffffu, (ok && !s_fail) ? 1 : 0, 0) != 0;
        if (go && p.nsplit > 1 && p.nsplit <= K2_FOLD_MAX && p.ticket != nullptr) {
            unsigned *tk = p.ticket + ((long long)tile_c * p.ntile_o + tile_o) * K2_EPI_WARPS + ew;
            __threadfence();  // this lane's part sums before the ticket
            __syncwarp();
            unsigned prev = 0;
            if (lane == 0)
                prev = atomicAdd(tk, 1u);
            prev = __shfl_sync(0xffffffffu, prev, 0);
            if (prev == (unsigned)(p.nsplit - 1)) {
                __threadfence();  // the other parts' sums after their tickets
                k2_fold_slice(p, tile_c, tile_o, q, half, lane);
                if (lane == 0)
                    *tk = 0u;  // zero again for the next launch
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 2 * K2_N);
    }
}

// Plain BF16 with two channel tiles per CTA: both 128-channel X tiles of a
// K block are multiplied by the same T stage, so each T tile loaded from L2
// feeds two MMAs (T is 2/3 of a single-tile stage's bytes). One TMEM run per
// unit (the K range fits one FP32 accumulation, as plain BF16 is limited by
// its operands, not by the run length); two accumulators of 256 columns. The
// epilogue writes TMEM straight to y (or to the K-part partials).
constexpr int K2P_BLK = 2 * K2_XBYTES1 + K2_TBYTES1;  // one K block: X tile a, X tile b, T
constexpr int K2P_GS = 1;                             // K blocks per pipeline stage
constexpr int K2P_STAGE = K2P_GS * K2P_BLK;
constexpr int K2P_NS = 3;
constexpr int K2P_SMEM = K2P_NS * K2P_STAGE + 1024;

__global__ void __launch_bounds__(K2_THREADS, 1)
    k2_toeplitz_pair(const __grid_constant__ CUtensorMap mx_hi, const __grid_constant__ CUtensorMap mt_hi,
                     const K2Params p)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[K2P_NS];
    __shared__ __align__(8) uint64_t empty[K2P_NS];
    __shared__ __align__(8) uint64_t accfull;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;

    uint8_t *const smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    // Unit = (channel-tile pair, output tile, K part).
    long long u = blockIdx.x;
    const int part = (int)(u % p.nsplit);
    u /= p.nsplit;
    const int tile_o = (int)(u % p.ntile_o);
    const int tile_c = (int)(u / p.ntile_o);  // pair index
    const int kb0 = part * p.kb_per;
    const int kb1 = min(kb0 + p.kb_per, p.nkb);
    const int nk = max(kb1 - kb0, 0);
    const int c0 = tile_c * 2 * K2_M;
    const long long xcol0 = p.x_col0 + (long long)tile_o * K2_N;

    if (tid == 0) {
        for (int i = 0; i < K2P_NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&accfull, 1);
        s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 2)
        tmem_alloc(&tmem_base, 2 * K2_N);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer ----
            for (int gi = 0; gi * K2P_GS < nk && !s_fail; ++gi) {
                const int st = gi % K2P_NS;
                const int use = gi / K2P_NS;
                if (use > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((use - 1) & 1), p.err, ERR_TIMEOUT_TMA)) {
                    s_fail = 1;
                    break;
                }
                const int nb = min(K2P_GS, nk - gi * K2P_GS);
                mbar_arrive_expect_tx(&full[st], (uint32_t)(nb * K2P_BLK));
                for (int j = 0; j < nb; ++j) {
                    uint8_t *sb = smem + st * K2P_STAGE + j * K2P_BLK;
                    const int kb = kb0 + gi * K2P_GS + j;
                    const int xc = (int)(xcol0 + (long long)kb * K2_KB1);
                    tma_load_2d(sb, &mx_hi, xc, c0, &full[st]);
                    tma_load_2d(sb + K2_XBYTES1, &mx_hi, xc, c0 + K2_M, &full[st]);
                    tma_load_2d(sb + 2 * K2_XBYTES1, &mt_hi, 0, kb * K2_N, &full[st]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            const uint32_t idesc = umma_idesc_bf16(K2_M, K2_N);
            const uint64_t d0 = umma_desc_sw128(smem_u32(smem));
            for (int gi = 0; gi * K2P_GS < nk; ++gi) {
                const int st = gi % K2P_NS;
                if (!mbar_wait_bounded(&full[st], (uint32_t)((gi / K2P_NS) & 1), p.err, ERR_TIMEOUT_MMA)) {
                    s_fail = 1;
                    break;
                }
                tc_fence_after_sync();
                const int nb = min(K2P_GS, nk - gi * K2P_GS);
                for (int j = 0; j < nb; ++j) {
                    const uint64_t sd = d0 + (uint64_t)((st * K2P_STAGE + j * K2P_BLK) >> 4);
#pragma unroll
                    for (int kk = 0; kk < K2_KB1 / 16; ++kk) {
                        const uint64_t th = sd + (uint64_t)((2 * K2_XBYTES1 + kk * 32) >> 4);
                        const uint32_t accum = (gi == 0 && j == 0 && kk == 0) ? 0u : 1u;
                        umma_bf16(tmem, sd + (uint64_t)(kk * 2), th, idesc, accum);
                        umma_bf16(tmem + K2_N, sd + (uint64_t)((K2_XBYTES1 + kk * 32) >> 4), th, idesc, accum);
                    }
                }
                umma_commit(&empty[st]);
            }
            if (!s_fail)
                umma_commit(&accfull);
        }
    } else if (warp >= K2_ROLE_WARPS) {
        // ---- epilogue: TMEM -> y / partials ----
        const int ew = warp - K2_ROLE_WARPS;
        const int q = warp & 3;    // TMEM lane quarter this warp may access
        const int half = ew >> 2;  // column half
        bool got = true;
        if (lane == 0)  // bounded, and abandoned early if another role has failed
            got = mbar_wait_limited(&accfull, 0, p.err, ERR_TIMEOUT_MMA, kWaitLimitNs, &s_fail);
        got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (got && nk > 0) {
            mbar_try_wait(&accfull, 0);
            tc_fence_after_sync();
#pragma unroll 1
            for (int a = 0; a < 2; ++a) {
                const int ch = a * K2_M + q * 32 + lane;  // channel within the pair
                const int c = c0 + ch;
                float *dst;
                long long lim;
                if (p.nsplit == 1) {
                    dst = p.y + (long long)c * p.y_pitch + (long long)tile_o * K2_N + half * 128;
                    lim = k2_ylim(p, p.nout - (long long)tile_o * K2_N - half * 128, c,
                                  (long long)tile_o * K2_N + half * 128);
                } else {
                    // Partials are laid out per 128-channel tile, as k2_reduce reads them.
                    const int tc1 = tile_c * 2 + a;
                    dst = p.partial + ((((long long)tc1 * p.ntile_o + tile_o) * p.nsplit + part) * K2_M +
                                       (q * 32 + lane)) * K2_N + half * 128;
                    lim = 128;
                }
                const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * K2_N + half * 128);
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    float v[16];
                    tmem_ld_32x16(src + cc * 16, v);
                    if (c >= p.C)
                        continue;
                    const long long j0 = cc * 16;
                    if (lim >= j0 + 16 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4 *>(dst + j0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j0 + j < lim)
                                dst[j0 + j] = v[j];
                    }
                }
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 2 * K2_N);
    }
}

// Plain BF16 on a CTA pair (cluster of two, tcgen05 cta_group::2): a unit of
// 256 channels x 256 outputs is one M = 256, N = 256 accumulation. Each CTA
// stages its own 128 channels of X and its half (128 outputs) of the T tile,
// so a CTA's shared memory feeds 8 KB of operands per 128 x 256 x 16 of its
// accumulator, against 12 KB when one CTA holds a whole 128 x 256 tile; the
// tensor cores read the peer's T half over the pair. The even CTA's producer
// arms the stage barrier for both CTAs' bytes, and the odd CTA's loads count
// on it. The even CTA's MMA thread issues the pair MMAs and commits each
// stage to both CTAs' free barriers, the last one also to both accumulator
// barriers; each CTA's eight epilogue warps then read its own TMEM (128
// lanes = its channels, 256 columns = the outputs). One TMEM run per unit.
// K blocks of 64 samples: 128-byte rows take half the L2 requests per byte
// of the 64-byte rows that K blocks of 32 would give. Each pipeline stage
// has a fixed cost (its barrier round trip and commit), so a stage holds two
// K blocks (8 MMAs): measured on the 1024-stream shared-IR workload, 2 blocks
// x 3 stages 75-77 % of the sustained BF16 peak against 72-73 % for 1 x 6 and
// 1 x 7 (with K blocks of 32 the same trade gave 39 % for 1 x 10 and 64 % for
// 3 x 4).
constexpr int K2C_BLK = 2 * K2_XBYTES1;  // one K block per CTA: X (128 x 64) and T half (128 x 64)
constexpr int K2C_GS = 2;               // K blocks per pipeline stage
constexpr int K2C_STAGE = K2C_GS * K2C_BLK;
constexpr int K2C_NS = 3;
constexpr int K2C_SMEM = K2C_NS * K2C_STAGE + 1024;

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(K2_THREADS, 1)
    k2_toeplitz_c2(const __grid_constant__ CUtensorMap mx_hi, const __grid_constant__ CUtensorMap mt2_hi,
                   const K2Params p)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[K2C_NS];
    __shared__ __align__(8) uint64_t empty[K2C_NS];
    __shared__ __align__(8) uint64_t accfull;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;

    uint8_t *const smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const uint32_t rank = cluster_ctarank();  // 0: issues the MMAs; 1: its pair peer

    // Unit = (channel-tile pair, output tile, K part), one cluster each.
    long long u = blockIdx.x >> 1;
    const int part = (int)(u % p.nsplit);
    u /= p.nsplit;
    const int tile_o = (int)(u % p.ntile_o);
    const int tile_c = (int)(u / p.ntile_o);  // pair index
    const int kb0 = part * p.kb_per;
    const int kb1 = min(kb0 + p.kb_per, p.nkb);
    const int nk = max(kb1 - kb0, 0);
    const int c0 = tile_c * 2 * K2_M + (int)rank * K2_M;  // this CTA's 128 channels
    const long long xcol0 = p.x_col0 + (long long)tile_o * K2_N;

    if (tid == 0) {
        for (int i = 0; i < K2C_NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&accfull, 1);
        s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 2)
        tmem_alloc_pair(&tmem_base, K2_N);
    tc_fence_before_sync();
    cluster_sync();  // both CTAs' barriers exist before either CTA signals the other's
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer (each CTA loads its own halves) ----
            for (int gi = 0; gi * K2C_GS < nk && !s_fail; ++gi) {
                const int st = gi % K2C_NS;
                const int use = gi / K2C_NS;
                if (use > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((use - 1) & 1), p.err, ERR_TIMEOUT_TMA)) {
                    s_fail = 1;
                    break;
                }
                const int nb = min(K2C_GS, nk - gi * K2C_GS);  // K blocks in this stage
                if (rank == 0)
                    mbar_arrive_expect_tx(&full[st], (uint32_t)(2 * nb * K2C_BLK));  // both CTAs' bytes
                const uint32_t bar = mapa_shared(smem_u32(&full[st]), 0);
                for (int j = 0; j < nb; ++j) {
                    uint8_t *sb = smem + st * K2C_STAGE + j * K2C_BLK;
                    const int kb = kb0 + gi * K2C_GS + j;
                    tma_load_2d_pair(sb, &mx_hi, (int)(xcol0 + (long long)kb * K2_KB1), c0, bar);
                    tma_load_2d_pair(sb + K2_XBYTES1, &mt2_hi, 0, kb * K2_N + (int)rank * (K2_N / 2), bar);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---- MMA issuer (even CTA) ----
            const uint32_t idesc = umma_idesc_bf16(2 * K2_M, K2_N);
            const uint64_t d0 = umma_desc_sw128(smem_u32(smem));
            bool ok = true;
            for (int gi = 0; gi * K2C_GS < nk; ++gi) {
                const int st = gi % K2C_NS;
                if (!mbar_wait_bounded(&full[st], (uint32_t)((gi / K2C_NS) & 1), p.err, ERR_TIMEOUT_MMA)) {
                    s_fail = 1;
                    ok = false;
                    break;
                }
                tc_fence_after_sync();
                const int nb = min(K2C_GS, nk - gi * K2C_GS);
                for (int j = 0; j < nb; ++j) {
                    const uint64_t sd = d0 + (uint64_t)((st * K2C_STAGE + j * K2C_BLK) >> 4);
#pragma unroll
                    for (int kk = 0; kk < K2_KB1 / 16; ++kk) {
                        const uint64_t xa = sd + (uint64_t)(kk * 2);
                        const uint64_t tb = sd + (uint64_t)((K2_XBYTES1 + kk * 32) >> 4);
                        umma_bf16_pair(tmem, xa, tb, idesc, (gi == 0 && j == 0 && kk == 0) ? 0u : 1u);
                    }
                }
                umma_commit_pair(&empty[st], 0x3);
            }
            if (ok && nk > 0)
                umma_commit_pair(&accfull, 0x3);
        }
    } else if (warp >= K2_ROLE_WARPS) {
        // ---- epilogue (each CTA: its TMEM lanes = its 128 channels) ----
        const int ew = warp - K2_ROLE_WARPS;
        const int q = warp & 3;
        const int half = ew >> 2;
        bool got = nk > 0;
        if (got && lane == 0)
            got = mbar_wait_limited(&accfull, 0, p.err, ERR_TIMEOUT_MMA, kWaitLimitNs, &s_fail);
        got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (got) {
            mbar_try_wait(&accfull, 0);
            tc_fence_after_sync();
            const int ch = q * 32 + lane;
            const int c = c0 + ch;
            float *dst;
            long long lim;
            if (p.nsplit == 1) {
                dst = p.y + (long long)c * p.y_pitch + (long long)tile_o * K2_N + half * 128;
                lim = k2_ylim(p, p.nout - (long long)tile_o * K2_N - half * 128, c,
                              (long long)tile_o * K2_N + half * 128);
            } else {
                // Partials per 128-channel tile, as k2_reduce reads them.
                const int tc1 = tile_c * 2 + (int)rank;
                dst = p.partial + ((((long long)tc1 * p.ntile_o + tile_o) * p.nsplit + part) * K2_M + ch) * K2_N +
                      half * 128;
                lim = 128;
            }
            const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 128);
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                float v[16];
                tmem_ld_32x16(src + cc * 16, v);
                if (c >= p.C)
                    continue;
                const long long j0 = cc * 16;
                if (lim >= j0 + 16 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(dst + j0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j0 + j < lim)
                            dst[j0 + j] = v[j];
                }
            }
        }
    }
    // Neither CTA leaves while the other may still signal its barriers or
    // read its shared memory (the pair MMAs read both CTAs' operands).
    tc_fence_before_sync();
    cluster_sync();
    if (warp == 2) {
        tc_fence_after_sync();
        tmem_dealloc_pair(tmem, K2_N);
    }
}

// The CTA-pair kernel made persistent: one cluster per SM pair walks the
// units u = cluster, cluster + clusters, ... The producers run ahead into the
// next unit's K blocks (the stage ring never drains between units), and the
// accumulators alternate between two TMEM buffers of 256 columns, so the
// epilogue of one unit runs under the MMAs of the next. Each CTA's eight
// epilogue warps release a buffer on the even CTA's `accfree` barrier (16
// arrivals: eight local, eight from the odd CTA at cluster scope); the MMA
// thread waits on it before it reuses the buffer.
struct K2Unit {
    int part, tile_o, tile_c, kb0, nk;
};

// What one CTA of a pair computes of unit w: its 128-channel tile and its
// output tile. Two channel tiles of one output tile (the usual pair), or,
// with pair_o (groups of one channel tile), two adjacent output tiles of the
// same channels: T does not depend on the output tile, so each CTA stages X
// from its own window and both multiply it by the shared T tile.
struct K2Cta {
    int tc1, ot;
};

__device__ __forceinline__ K2Cta k2_cta(const K2Params &p, const K2Unit &w, uint32_t rank)
{
    K2Cta m;
    m.tc1 = p.pair_o ? w.tile_c : w.tile_c * 2 + (int)rank;
    m.ot = p.pair_o ? w.tile_o * 2 + (int)rank : w.tile_o;
    return m;
}

// Output tiles of one unit row: all of them, or their pairs when the two
// CTAs of a pair take two adjacent output tiles of the same channels.
__device__ __forceinline__ int k2_unit_ntile_o(const K2Params &p)
{
    return p.pair_o ? (p.ntile_o + 1) / 2 : p.ntile_o;
}

__device__ __forceinline__ K2Unit k2_unit(const K2Params &p, long long u)
{
    K2Unit w;
    const int nto = k2_unit_ntile_o(p);
    if (p.order == 1) {  // output tile fastest, then K part
        w.tile_o = (int)(u % nto);
        u /= nto;
        w.part = (int)(u % p.nsplit);
        w.tile_c = (int)(u / p.nsplit);
    } else if (p.order == 2) {  // output tile fastest, then channel tile; K part slowest
        w.tile_o = (int)(u % nto);
        u /= nto;
        w.tile_c = (int)(u % p.ntile_c);
        w.part = (int)(u / p.ntile_c);
    } else {  // K part fastest, then output tile
        w.part = (int)(u % p.nsplit);
        u /= p.nsplit;
        w.tile_o = (int)(u % nto);
        w.tile_c = (int)(u / nto);
    }
    w.kb0 = w.part * p.kb_per;
    w.nk = max(min(w.kb0 + p.kb_per, p.nkb) - w.kb0, 0);
    return w;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(K2_THREADS, 1)
    k2_toeplitz_c2p(const __grid_constant__ CUtensorMap mx_hi, const __grid_constant__ CUtensorMap mt2_hi,
                    const K2Params p, long long units)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[K2C_NS];
    __shared__ __align__(8) uint64_t empty[K2C_NS];
    __shared__ __align__(8) uint64_t accfull[2];
    __shared__ __align__(8) uint64_t accfree[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;

    uint8_t *const smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const uint32_t rank = cluster_ctarank();
    const long long cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (tid == 0) {
        for (int i = 0; i < K2C_NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accfree[i], 2 * K2_EPI_WARPS);
        }
        s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 2)
        tmem_alloc_pair(&tmem_base, 2 * K2_N);
    tc_fence_before_sync();
    cluster_sync();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer (each CTA loads its own halves), across units ----
            // The IR tiles of a K range are read by every pair working in it: keep them in L2.
            const uint64_t pol = l2_policy_evict_last();
            long long gi = 0;  // stage fills so far
            for (long long u = cid; u < units && !s_fail; u += ncl) {
                const K2Unit w = k2_unit(p, u);
                const K2Cta m = k2_cta(p, w, rank);
                const int c0 = m.tc1 * K2_M;
                const long long xcol0 = p.x_col0 + (long long)m.ot * K2_N;
                for (int g = 0; g * K2C_GS < w.nk; ++g, ++gi) {
                    const int st = (int)(gi % K2C_NS);
                    const long long use = gi / K2C_NS;
                    if (use > 0 &&
                        !mbar_wait_bounded(&empty[st], (uint32_t)((use - 1) & 1), p.err, ERR_TIMEOUT_TMA)) {
                        s_fail = 1;
                        break;
                    }
                    const int nb = min(K2C_GS, w.nk - g * K2C_GS);
                    if (rank == 0)
                        mbar_arrive_expect_tx(&full[st], (uint32_t)(2 * nb * K2C_BLK));
                    const uint32_t bar = mapa_shared(smem_u32(&full[st]), 0);
                    for (int j = 0; j < nb; ++j) {
                        uint8_t *sb = smem + st * K2C_STAGE + j * K2C_BLK;
                        const int kb = w.kb0 + g * K2C_GS + j;
                        tma_load_2d_pair(sb, &mx_hi, (int)(xcol0 + (long long)kb * K2_KB1), c0, bar);
                        tma_load_2d_pair_hint(sb + K2_XBYTES1, &mt2_hi, 0, kb * K2_N + (int)rank * (K2_N / 2), bar,
                                              pol);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---- MMA issuer (even CTA), across units ----
            const uint32_t idesc = umma_idesc_bf16(2 * K2_M, K2_N);
            const uint64_t d0 = umma_desc_sw128(smem_u32(smem));
            long long gi = 0;
            long long k = 0;  // units done by this cluster
            for (long long u = cid; u < units && !s_fail; u += ncl, ++k) {
                const K2Unit w = k2_unit(p, u);
                const int buf = (int)(k & 1);
                const long long reuse = k >> 1;
                if (reuse > 0 &&
                    !mbar_wait_cluster_bounded(&accfree[buf], (uint32_t)((reuse - 1) & 1), p.err, ERR_TIMEOUT_MMA)) {
                    s_fail = 1;
                    break;
                }
                tc_fence_after_sync();
                const uint32_t acc = tmem + (uint32_t)(buf * K2_N);
                bool ok = true;
                for (int g = 0; g * K2C_GS < w.nk; ++g, ++gi) {
                    const int st = (int)(gi % K2C_NS);
                    if (!mbar_wait_bounded(&full[st], (uint32_t)((gi / K2C_NS) & 1), p.err, ERR_TIMEOUT_MMA)) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after_sync();
                    const int nb = min(K2C_GS, w.nk - g * K2C_GS);
                    for (int j = 0; j < nb; ++j) {
                        const uint64_t sd = d0 + (uint64_t)((st * K2C_STAGE + j * K2C_BLK) >> 4);
#pragma unroll
                        for (int kk = 0; kk < K2_KB1 / 16; ++kk) {
                            const uint64_t xa = sd + (uint64_t)(kk * 2);
                            const uint64_t tb = sd + (uint64_t)((K2_XBYTES1 + kk * 32) >> 4);
                            umma_bf16_pair(acc, xa, tb, idesc, (g == 0 && j == 0 && kk == 0) ? 0u : 1u);
                        }
                    }
                    umma_commit_pair(&empty[st], 0x3);
                }
                if (!ok)
                    break;
                umma_commit_pair(&accfull[buf], 0x3);
            }
        }
    } else if (warp >= K2_ROLE_WARPS) {
        // ---- epilogue (each CTA: its TMEM lanes = its 128 channels), across units ----
        const int ew = warp - K2_ROLE_WARPS;
        const int q = warp & 3;
        const int half = ew >> 2;
        const uint32_t free0 = mapa_shared(smem_u32(&accfree[0]), 0), free1 = mapa_shared(smem_u32(&accfree[1]), 0);
        const bool fold = p.nsplit > 1 && p.nsplit <= K2_FOLD_MAX && p.ticket != nullptr;
        long long k = 0;
        for (long long u = cid; u < units; u += ncl, ++k) {
            const K2Unit w = k2_unit(p, u);
            const int buf = (int)(k & 1);
            const uint32_t par = (uint32_t)((k >> 1) & 1);
            bool got = true;
            if (lane == 0)
                got = mbar_wait_limited(&accfull[buf], par, p.err, ERR_TIMEOUT_MMA, kWaitLimitNs, &s_fail);
            got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
            if (!got)
                break;
            mbar_try_wait(&accfull[buf], par);
            tc_fence_after_sync();
            const int ch = q * 32 + lane;
            const K2Cta m = k2_cta(p, w, rank);
            const bool live = m.ot < p.ntile_o;  // the odd last output tile of a pair_o row has no partner
            const int c = m.tc1 * K2_M + ch;
            float *dst;
            long long lim;
            if (p.nsplit == 1) {
                dst = p.y + (long long)c * p.y_pitch + (long long)m.ot * K2_N + half * 128;
                lim = k2_ylim(p, p.nout - (long long)m.ot * K2_N - half * 128, c, (long long)m.ot * K2_N + half * 128);
            } else {
                dst = p.partial +
                      ((((long long)m.tc1 * p.ntile_o + m.ot) * p.nsplit + w.part) * K2_M + ch) * K2_N + half * 128;
                lim = 128;
            }
            const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * K2_N + half * 128);
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                float v[16];
                tmem_ld_32x16(src + cc * 16, v);
                if (c >= p.C || !live)
                    continue;
                const long long j0 = cc * 16;
                if (lim >= j0 + 16 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(dst + j0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j0 + j < lim)
                            dst[j0 + j] = v[j];
                }
            }
            tc_fence_before_sync();
            __syncwarp();
            if (lane == 0)
                mbar_arrive_cluster(buf ? free1 : free0);  // this buffer may take the next unit's MMAs
            if (fold && live) {
                unsigned *tk = p.ticket + ((long long)m.tc1 * p.ntile_o + m.ot) * K2_EPI_WARPS + ew;
                __threadfence();  // this lane's part sums before the ticket
                __syncwarp();
                unsigned prev = 0;
                if (lane == 0)
                    prev = atomicAdd(tk, 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev == (unsigned)(p.nsplit - 1)) {
                    __threadfence();  // the other parts' sums after their tickets
                    k2_fold_slice(p, m.tc1, m.ot, q, half, lane);
                    if (lane == 0)
                        *tk = 0u;  // every part has its ticket: zero again for the next launch
                }
            }
        }
    }
    // Neither CTA leaves while the other may still signal its barriers or
    // read its shared memory.
    tc_fence_before_sync();
    cluster_sync();
    if (warp == 2) {
        tc_fence_after_sync();
        tmem_dealloc_pair(tmem, 2 * K2_N);
    }
}

// The BF16 hi/lo split on persistent CTA pairs. As k2_toeplitz_c2p, each
// CTA of a pair stages its 128 channels of X (hi and lo) and its 128-output
// half of T (hi and lo), so a K block costs each SM 32 KB instead of the
// single-tile kernel's 48 KB; the three products of a K block go into one
// M = 256 accumulator. As k2_toeplitz<3>, a unit's K blocks are accumulated
// in TMEM runs of `range` blocks, alternating between two accumulators, and
// the eight epilogue warps of each CTA drain every finished run into FP32
// register sums (round-to-nearest adds) under the next run's MMAs. Runs are
// counted across units, so the MMAs of a unit's first run never wait for the
// previous unit's last drain. Two K blocks per stage (runs are whole stages:
// `range` even).
constexpr int K2S_BLK = 4 * K2_M * K2_KB * 2;  // one K block per CTA: X hi, X lo, T hi half, T lo half (8 KB each)
constexpr int K2S_GS = 2;                        // K blocks per pipeline stage
constexpr int K2S_STAGE = K2S_GS * K2S_BLK;
constexpr int K2S_NS = 3;
constexpr int K2S_SMEM = K2S_NS * K2S_STAGE + 1024;

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(K2_THREADS, 1)
    k2_toeplitz_c2s(const __grid_constant__ CUtensorMap mx_hi, const __grid_constant__ CUtensorMap mx_lo,
                    const __grid_constant__ CUtensorMap mt2_hi, const __grid_constant__ CUtensorMap mt2_lo,
                    const K2Params p, long long units)
{
    constexpr int XB = K2_M * K2_KB * 2;  // 8 KB
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[K2S_NS];
    __shared__ __align__(8) uint64_t empty[K2S_NS];
    __shared__ __align__(8) uint64_t accfull[2];
    __shared__ __align__(8) uint64_t accfree[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;

    uint8_t *const smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const uint32_t rank = cluster_ctarank();
    const long long cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
    const int range = p.range;

    if (tid == 0) {
        for (int i = 0; i < K2S_NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accfree[i], 2 * K2_EPI_WARPS);
        }
        s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 2)
        tmem_alloc_pair(&tmem_base, 2 * K2_N);
    tc_fence_before_sync();
    cluster_sync();
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer (each CTA loads its own halves), across units ----
            // The IR tiles of a K range are read by every pair working in it: keep them in L2.
            const uint64_t pol = l2_policy_evict_last();
            long long gi = 0;
            for (long long u = cid; u < units && !s_fail; u += ncl) {
                const K2Unit w = k2_unit(p, u);
                const K2Cta m = k2_cta(p, w, rank);
                const int c0 = m.tc1 * K2_M;
                const long long xcol0 = p.x_col0 + (long long)m.ot * K2_N;
                for (int g = 0; g * K2S_GS < w.nk; ++g, ++gi) {
                    const int st = (int)(gi % K2S_NS);
                    const long long use = gi / K2S_NS;
                    if (use > 0 &&
                        !mbar_wait_bounded(&empty[st], (uint32_t)((use - 1) & 1), p.err, ERR_TIMEOUT_TMA)) {
                        s_fail = 1;
                        break;
                    }
                    const int nb = min(K2S_GS, w.nk - g * K2S_GS);
                    if (rank == 0)
                        mbar_arrive_expect_tx(&full[st], (uint32_t)(2 * nb * K2S_BLK));
                    const uint32_t bar = mapa_shared(smem_u32(&full[st]), 0);
                    for (int j = 0; j < nb; ++j) {
                        uint8_t *sb = smem + st * K2S_STAGE + j * K2S_BLK;
                        const int kb = w.kb0 + g * K2S_GS + j;
                        const int xc = (int)(xcol0 + (long long)kb * K2_KB);
                        const int tr = kb * K2_N + (int)rank * (K2_N / 2);
                        tma_load_2d_pair(sb, &mx_hi, xc, c0, bar);
                        tma_load_2d_pair(sb + XB, &mx_lo, xc, c0, bar);
                        tma_load_2d_pair_hint(sb + 2 * XB, &mt2_hi, 0, tr, bar, pol);
                        tma_load_2d_pair_hint(sb + 3 * XB, &mt2_lo, 0, tr, bar, pol);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---- MMA issuer (even CTA): runs of `range` K blocks, across units ----
            const uint32_t idesc = umma_idesc_bf16(2 * K2_M, K2_N);
            const uint64_t d0 = umma_desc_sw64(smem_u32(smem));
            long long gi = 0, run = 0;
            for (long long u = cid; u < units && !s_fail; u += ncl) {
                const K2Unit w = k2_unit(p, u);
                for (int k0 = 0; k0 < w.nk && !s_fail; k0 += range, ++run) {
                    const int buf = (int)(run & 1);
                    const long long reuse = run >> 1;
                    if (reuse > 0 && !mbar_wait_cluster_bounded(&accfree[buf], (uint32_t)((reuse - 1) & 1), p.err,
                                                                ERR_TIMEOUT_MMA)) {
                        s_fail = 1;
                        break;
                    }
                    tc_fence_after_sync();
                    const uint32_t acc = tmem + (uint32_t)(buf * K2_N);
                    const int k1 = min(w.nk, k0 + range);
                    // range is a multiple of K2S_GS: the run's stages are the producer's stages.
                    for (int g = k0 / K2S_GS; g * K2S_GS < k1; ++g, ++gi) {
                        const int st = (int)(gi % K2S_NS);
                        if (!mbar_wait_bounded(&full[st], (uint32_t)((gi / K2S_NS) & 1), p.err, ERR_TIMEOUT_MMA)) {
                            s_fail = 1;
                            break;
                        }
                        tc_fence_after_sync();
                        const int nb = min(K2S_GS, k1 - g * K2S_GS);
                        for (int j = 0; j < nb; ++j) {
                            const uint64_t sd = d0 + (uint64_t)((st * K2S_STAGE + j * K2S_BLK) >> 4);
#pragma unroll
                            for (int kk = 0; kk < K2_KB / 16; ++kk) {
                                const uint64_t xh = sd + (uint64_t)(kk * 2);
                                const uint64_t xl = sd + (uint64_t)((XB + kk * 32) >> 4);
                                const uint64_t th = sd + (uint64_t)((2 * XB + kk * 32) >> 4);
                                const uint64_t tl = sd + (uint64_t)((3 * XB + kk * 32) >> 4);
                                const bool first = g * K2S_GS + j == k0 && kk == 0;
                                umma_bf16_pair(acc, xh, th, idesc, first ? 0u : 1u);
                                umma_bf16_pair(acc, xh, tl, idesc, 1u);
                                umma_bf16_pair(acc, xl, th, idesc, 1u);
                            }
                        }
                        umma_commit_pair(&empty[st], 0x3);
                    }
                    if (s_fail)
                        break;
                    umma_commit_pair(&accfull[buf], 0x3);  // the run is complete in both CTAs' TMEM
                }
            }
        }
    } else if (warp >= K2_ROLE_WARPS) {
        // ---- epilogue: drain each run into FP32 register sums, across units ----
        const int ew = warp - K2_ROLE_WARPS;
        const int q = warp & 3;
        const int half = ew >> 2;
        const uint32_t free0 = mapa_shared(smem_u32(&accfree[0]), 0), free1 = mapa_shared(smem_u32(&accfree[1]), 0);
        const bool fold = p.nsplit > 1 && p.nsplit <= K2_FOLD_MAX && p.ticket != nullptr;
        long long run = 0;
        bool ok = true;
        for (long long u = cid; u < units && ok; u += ncl) {
            const K2Unit w = k2_unit(p, u);
            float sum[128];
#pragma unroll
            for (int j = 0; j < 128; ++j)
                sum[j] = 0.f;
            for (int k0 = 0; k0 < w.nk; k0 += range, ++run) {
                const int buf = (int)(run & 1);
                const uint32_t par = (uint32_t)((run >> 1) & 1);
                bool got = true;
                if (lane == 0)
                    got = mbar_wait_limited(&accfull[buf], par, p.err, ERR_TIMEOUT_MMA, kWaitLimitNs, &s_fail);
                got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                if (!got) {
                    ok = false;
                    break;
                }
                mbar_try_wait(&accfull[buf], par);
                tc_fence_after_sync();
                const uint32_t src = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * K2_N + half * 128);
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    float v[16];
                    tmem_ld_32x16(src + cc * 16, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        sum[cc * 16 + j] += v[j];
                }
                tc_fence_before_sync();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive_cluster(buf ? free1 : free0);  // this accumulator may take the next run
            }
            if (!ok)
                break;
            const int ch = q * 32 + lane;
            const K2Cta m = k2_cta(p, w, rank);
            const bool live = m.ot < p.ntile_o;  // the odd last output tile of a pair_o row has no partner
            const int c = m.tc1 * K2_M + ch;
            if (c < p.C && live) {
                float *dst;
                long long lim;
                if (p.nsplit == 1) {
                    dst = p.y + (long long)c * p.y_pitch + (long long)m.ot * K2_N + half * 128;
                    lim = k2_ylim(p, p.nout - (long long)m.ot * K2_N - half * 128, c,
                                  (long long)m.ot * K2_N + half * 128);
                } else {
                    dst = p.partial +
                          ((((long long)m.tc1 * p.ntile_o + m.ot) * p.nsplit + w.part) * K2_M + ch) * K2_N +
                          half * 128;
                    lim = 128;
                }
                if (lim >= 128 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                    for (int j = 0; j < 128; j += 4)
                        *reinterpret_cast<float4 *>(dst + j) =
                            make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 128; ++j)
                        if (j < lim)
                            dst[j] = sum[j];
                }
            }
            if (fold && live) {
                unsigned *tk = p.ticket + ((long long)m.tc1 * p.ntile_o + m.ot) * K2_EPI_WARPS + ew;
                __threadfence();  // this lane's part sums before the ticket
                __syncwarp();
                unsigned prev = 0;
                if (lane == 0)
                    prev = atomicAdd(tk, 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev == (unsigned)(p.nsplit - 1)) {
                    __threadfence();  // the other parts' sums after their tickets
                    k2_fold_slice(p, m.tc1, m.ot, q, half, lane);
                    if (lane == 0)
                        *tk = 0u;  // zero again for the next launch
                }
            }
        }
    }
    tc_fence_before_sync();
    cluster_sync();
    if (warp == 2) {
        tc_fence_after_sync();
        tmem_dealloc_pair(tmem, 2 * K2_N);
    }
}

// Adds the nsplit K-range partials of each (channel, output) by a fixed
// pairwise tree (adjacent pairs, zero-padded to 64 leaves) and writes y.
__global__ void k2_reduce(const float *__restrict__ partial, int nsplit, int C, int ntile_o, int nout, float *y,
                          long long y_pitch, long long y_total)
{
    const long long total = (long long)C * nout;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / nout);
        const int o = (int)(q % nout);
        const int tc_ = c / K2_M, ch = c % K2_M, to = o / K2_N, oo = o % K2_N;
        const float *src = partial + ((((long long)tc_ * ntile_o + to) * nsplit) * K2_M + ch) * K2_N + oo;
        float v[64];
#pragma unroll
        for (int s = 0; s < 64; ++s)
            v[s] = (s < nsplit) ? src[(long long)s * K2_M * K2_N] : 0.f;
#pragma unroll
        for (int w = 32; w >= 1; w >>= 1) {
#pragma unroll
            for (int s = 0; s < w; ++s)
                v[s] = v[2 * s] + v[2 * s + 1];
        }
        if (y_total <= 0 || (long long)c * y_pitch + o < y_total)
            y[(long long)c * y_pitch + o] = v[0];
    }
}

// Materialises the Toeplitz tiles of one IR for alignment shift delta, in
// K blocks of kbs samples (32 or 64):
//   T[kb][i][j] = h[L - 1 + delta + i - kbs kb - j]  (0 outside [0, L)),
// as bf16 hi = bf16(h) and lo = bf16(h - hi), row-major [kb][256][kbs]
// (tlo may be null: plain BF16). One thread writes eight consecutive j of a
// row (one 16-byte store per tile).
__device__ __forceinline__ uint32_t k2_pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Group q (eight consecutive j of one row) of the Toeplitz tiles; sh = log2
// of the groups per row (kbs / 8).
__device__ __forceinline__ void k2_tprep_group(const float *__restrict__ h, int L, int delta, int kbs, int sh,
                                               long long q, __nv_bfloat16 *thi, __nv_bfloat16 *tlo)
{
    const int jg = (int)(q & ((1 << sh) - 1));
    const long long r = q >> sh;  // kb * 256 + i
    const int i = (int)(r & (K2_N - 1));
    const long long kb = r >> 8;
    const long long k0 = (long long)L - 1 + delta + i - (long long)kbs * kb - 8 * jg;  // tap of j = 8 jg
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        const long long ka = k0 - e, kb2 = k0 - e - 1;
        const float va = (ka >= 0 && ka < L) ? h[ka] : 0.f;
        const float vb = (kb2 >= 0 && kb2 < L) ? h[kb2] : 0.f;
        const __nv_bfloat16 ha = __float2bfloat16_rn(va), hb = __float2bfloat16_rn(vb);
        hw[e / 2] = k2_pack_bf16(ha, hb);
        lw[e / 2] = k2_pack_bf16(__float2bfloat16_rn(va - __bfloat162float(ha)),
                                 __float2bfloat16_rn(vb - __bfloat162float(hb)));
    }
    const long long o = r * kbs + 8 * jg;
    *reinterpret_cast<uint4 *>(thi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    if (tlo)  // plain BF16 reads only the hi tiles
        *reinterpret_cast<uint4 *>(tlo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

__global__ void k2_tprep(const float *__restrict__ h, int L, int delta, int nkb, int kbs, __nv_bfloat16 *thi,
                         __nv_bfloat16 *tlo)
{
    const int sh = kbs == 64 ? 3 : 2;
    const long long total = ((long long)nkb * K2_N) << sh;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x)
        k2_tprep_group(h, L, delta, kbs, sh, q, thi, tlo);
}

// bf16 hi = bf16(v) and lo = bf16(v - hi) of four values, as two 8-byte words.
__device__ __forceinline__ void k2_split4(const float v[4], uint2 &hi, uint2 &lo)
{
    __nv_bfloat16 b[4];
    float r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        b[e] = __float2bfloat16_rn(v[e]);
        r[e] = v[e] - __bfloat162float(b[e]);
    }
    hi = make_uint2(k2_pack_bf16(b[0], b[1]), k2_pack_bf16(b[2], b[3]));
    lo = make_uint2(k2_pack_bf16(__float2bfloat16_rn(r[0]), __float2bfloat16_rn(r[1])),
                    k2_pack_bf16(__float2bfloat16_rn(r[2]), __float2bfloat16_rn(r[3])));
}

// Splits new history samples into bf16 hi = bf16(x) and lo = bf16(x - hi):
// rows r < rows, columns [col0, col0 + n) of pitch-`pitch` histories (hlo
// may be null: plain BF16). One thread takes four consecutive elements of the
// flat history, on a four-element boundary (16-byte loads, 8-byte stores
// where all four are in the range).
__global__ void k2_split(const float *__restrict__ hist, long long pitch, int rows, long long col0, long long n,
                         __nv_bfloat16 *hhi, __nv_bfloat16 *hlo)
{
    const long long lead = col0 & 3;               // elements of the first group before col0 (pitch % 4 == 0)
    const long long gpr = (lead + n + 3) >> 2;     // groups per row
    const long long total = (long long)rows * gpr;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = q / gpr;
        const long long c = (col0 - lead) + ((q - r * gpr) << 2);  // first column of the group
        const long long idx = r * pitch + c;
        if (c >= col0 && c + 4 <= col0 + n) {
            const float4 f = *reinterpret_cast<const float4 *>(hist + idx);
            const float v[4] = {f.x, f.y, f.z, f.w};
            uint2 hi, lo;
            k2_split4(v, hi, lo);
            *reinterpret_cast<uint2 *>(hhi + idx) = hi;
            if (hlo)  // plain BF16 reads only the hi history
                *reinterpret_cast<uint2 *>(hlo + idx) = lo;
        } else {
            for (int e = 0; e < 4; ++e) {
                if (c + e < col0 || c + e >= col0 + n)
                    continue;
                const float v = hist[idx + e];
                const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                hhi[idx + e] = hi;
                if (hlo)
                    hlo[idx + e] = __float2bfloat16_rn(v - __bfloat162float(hi));
            }
        }
    }
}

// Everything a one-shot call prepares, in one launch: the padded input as
// bf16 hi (and lo) rows, xs[d] = x[d - off] for d in [off, off + N) and 0 on
// the rest of [0, npad) (groups of four, 8-byte stores); the Toeplitz tiles
// of h at shift 0 (as k2_tprep); and nzero zero words (tickets, error word).
__global__ void k2_oneshot_prep(const float *__restrict__ x, long long N, long long off, long long npad,
                                __nv_bfloat16 *xhi, __nv_bfloat16 *xlo, const float *__restrict__ h, int L, int nkb,
                                int kbs, __nv_bfloat16 *thi, __nv_bfloat16 *tlo, unsigned *zero, long long nzero)
{
    const long long gx = npad >> 2;
    const int sh = kbs == 64 ? 3 : 2;
    const long long gt = ((long long)nkb * K2_N) << sh;
    const long long total = gx + gt + nzero;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        if (q < gx) {
            const long long d = q << 2;
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                v[e] = (d + e >= off && d + e < off + N) ? x[d + e - off] : 0.f;
            uint2 hi, lo;
            k2_split4(v, hi, lo);
            *reinterpret_cast<uint2 *>(xhi + d) = hi;
            if (xlo)
                *reinterpret_cast<uint2 *>(xlo + d) = lo;
        } else if (q < gx + gt) {
            k2_tprep_group(h, L, 0, kbs, sh, q - gx, thi, tlo);
        } else {
            zero[q - gx - gt] = 0u;
        }
    }
}

unsigned grid_for(long long work)
{
    long long b = (work + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min<long long>(b, 8192));
}

}  // namespace

int k2_tile_m() { return K2_M; }
int k2_tile_n() { return K2_N; }
int k2_kblock(int nprod) { return nprod == 1 ? K2_KB1 : K2_KB; }

long long k2_nkb(long long L, int delta, int kbs) { return (L - 1 + delta + K2_N + kbs - 1) / kbs; }

cudaError_t k2_tprep_launch(const float *h, int L, int delta, int nkb, int kbs, void *thi, void *tlo,
                            cudaStream_t st)
{
    if (kbs != K2_KB && kbs != K2_KB1)
        return cudaErrorInvalidValue;
    const long long work = (long long)nkb * K2_N * (kbs / 8);
    k2_tprep<<<grid_for(work), 256, 0, st>>>(h, L, delta, nkb, kbs, (__nv_bfloat16 *)thi, (__nv_bfloat16 *)tlo);
    count_launch();
    return cudaGetLastError();
}

cudaError_t k2_split_launch(const float *hist, long long pitch, int rows, long long col0, long long n, void *hhi,
                            void *hlo, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    if (pitch % 4 != 0 || (reinterpret_cast<uintptr_t>(hist) & 15) != 0 || (reinterpret_cast<uintptr_t>(hhi) & 7) != 0 ||
        (reinterpret_cast<uintptr_t>(hlo) & 7) != 0)
        return cudaErrorInvalidValue;  // the four-element groups need these alignments
    k2_split<<<grid_for((long long)rows * ((n + 6) / 4)), 256, 0, st>>>(hist, pitch, rows, col0, n,
                                                                       (__nv_bfloat16 *)hhi, (__nv_bfloat16 *)hlo);
    count_launch();
    return cudaGetLastError();
}

cudaError_t k2_oneshot_prep_launch(const float *x, long long N, long long off, long long npad, void *xhi, void *xlo,
                                   const float *h, int L, int nkb, int kbs, void *thi, void *tlo, unsigned *zero,
                                   long long nzero, cudaStream_t st)
{
    if ((kbs != K2_KB && kbs != K2_KB1) || npad % 4 != 0 || (reinterpret_cast<uintptr_t>(xhi) & 7) != 0 ||
        (reinterpret_cast<uintptr_t>(xlo) & 7) != 0 || (reinterpret_cast<uintptr_t>(thi) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(tlo) & 15) != 0)
        return cudaErrorInvalidValue;
    const long long work = npad / 4 + (long long)nkb * K2_N * (kbs / 8) + nzero;
    k2_oneshot_prep<<<grid_for(work), 256, 0, st>>>(x, N, off, npad, (__nv_bfloat16 *)xhi, (__nv_bfloat16 *)xlo, h,
                                                    L, nkb, kbs, (__nv_bfloat16 *)thi, (__nv_bfloat16 *)tlo, zero,
                                                    nzero);
    count_launch();
    return cudaGetLastError();
}

size_t k2_smem_bytes(int nprod) { return nprod == 1 ? K2Cfg<1>::SMEM : K2Cfg<3>::SMEM; }

cudaError_t k2_launch_pair(const CUtensorMap &mx_hi, const CUtensorMap &mt_hi, const K2Params &p, cudaStream_t st)
{
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64 || p.nsplit < 1 || p.nsplit > 64 || p.range < p.kb_per)
        return cudaErrorInvalidValue;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(k2_toeplitz_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, K2P_SMEM);
        if (e != cudaSuccess)
            return e;
        attr[dev] = true;
    }
    const long long units = (long long)p.ntile_c * p.ntile_o * p.nsplit;  // ntile_c counts tile pairs here
    if (units <= 0)
        return cudaSuccess;
    k2_toeplitz_pair<<<(unsigned)units, K2_THREADS, K2P_SMEM, st>>>(mx_hi, mt_hi, p);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess || p.nsplit == 1)
        return e;
    const long long work = (long long)p.C * p.nout;
    k2_reduce<<<grid_for(work), 256, 0, st>>>(p.partial, p.nsplit, p.C, (p.nout + K2_N - 1) / K2_N, p.nout, p.y,
                                              p.y_pitch, p.y_total);
    count_launch();
    return cudaGetLastError();
}

cudaError_t k2_launch_c2p(const CUtensorMap &mx_hi, const CUtensorMap &mt2_hi, const K2Params &p, cudaStream_t st)
{
    static bool attr[64] = {};
    static int clusters[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64 || p.nsplit < 1 || p.nsplit > 64)
        return cudaErrorInvalidValue;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(k2_toeplitz_c2p, cudaFuncAttributeMaxDynamicSharedMemorySize, K2C_SMEM);
        if (e != cudaSuccess)
            return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
        clusters[dev] = std::max(1, sms / 2);  // one CTA per SM, two per cluster
        attr[dev] = true;
    }
    // ntile_c counts tile pairs here (or channel tiles, with pair_o taking output-tile pairs).
    const long long nto = p.pair_o ? (p.ntile_o + 1) / 2 : p.ntile_o;
    const long long units = (long long)p.ntile_c * nto * p.nsplit;
    if (units <= 0)
        return cudaSuccess;
    const long long ncl = std::min<long long>(units, clusters[dev]);
    k2_toeplitz_c2p<<<(unsigned)(2 * ncl), K2_THREADS, K2C_SMEM, st>>>(mx_hi, mt2_hi, p, units);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess || p.nsplit == 1 || (p.ticket != nullptr && p.nsplit <= K2_FOLD_MAX))
        return e;  // no parts, or folded in the kernel
    const long long work = (long long)p.C * p.nout;
    k2_reduce<<<grid_for(work), 256, 0, st>>>(p.partial, p.nsplit, p.C, (p.nout + K2_N - 1) / K2_N, p.nout, p.y,
                                              p.y_pitch, p.y_total);
    count_launch();
    return cudaGetLastError();
}

cudaError_t k2_launch_c2s(const CUtensorMap &mx_hi, const CUtensorMap &mx_lo, const CUtensorMap &mt2_hi,
                          const CUtensorMap &mt2_lo, const K2Params &p, cudaStream_t st)
{
    static bool attr[64] = {};
    static int clusters[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64 || p.nsplit < 1 || p.nsplit > 64 || p.range < 1 || p.range % K2S_GS != 0)
        return cudaErrorInvalidValue;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(k2_toeplitz_c2s, cudaFuncAttributeMaxDynamicSharedMemorySize, K2S_SMEM);
        if (e != cudaSuccess)
            return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
        clusters[dev] = std::max(1, sms / 2);
        attr[dev] = true;
    }
    // ntile_c counts tile pairs here (or channel tiles, with pair_o taking output-tile pairs).
    const long long nto = p.pair_o ? (p.ntile_o + 1) / 2 : p.ntile_o;
    const long long units = (long long)p.ntile_c * nto * p.nsplit;
    if (units <= 0)
        return cudaSuccess;
    const long long ncl = std::min<long long>(units, clusters[dev]);
    k2_toeplitz_c2s<<<(unsigned)(2 * ncl), K2_THREADS, K2S_SMEM, st>>>(mx_hi, mx_lo, mt2_hi, mt2_lo, p, units);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess || p.nsplit == 1 || (p.ticket != nullptr && p.nsplit <= K2_FOLD_MAX))
        return e;  // no parts, or folded in the kernel
    const long long work = (long long)p.C * p.nout;
    k2_reduce<<<grid_for(work), 256, 0, st>>>(p.partial, p.nsplit, p.C, (p.nout + K2_N - 1) / K2_N, p.nout, p.y,
                                              p.y_pitch, p.y_total);
    count_launch();
    return cudaGetLastError();
}

cudaError_t k2_launch_c2(const CUtensorMap &mx_hi, const CUtensorMap &mt2_hi, const K2Params &p, cudaStream_t st)
{
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64 || p.nsplit < 1 || p.nsplit > 64)
        return cudaErrorInvalidValue;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(k2_toeplitz_c2, cudaFuncAttributeMaxDynamicSharedMemorySize, K2C_SMEM);
        if (e != cudaSuccess)
            return e;
        attr[dev] = true;
    }
    const long long units = (long long)p.ntile_c * p.ntile_o * p.nsplit;  // ntile_c counts tile pairs here
    if (units <= 0)
        return cudaSuccess;
    if (2 * units > 0x7fffffffLL)
        return cudaErrorInvalidConfiguration;
    k2_toeplitz_c2<<<(unsigned)(2 * units), K2_THREADS, K2C_SMEM, st>>>(mx_hi, mt2_hi, p);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess || p.nsplit == 1)
        return e;
    const long long work = (long long)p.C * p.nout;
    k2_reduce<<<grid_for(work), 256, 0, st>>>(p.partial, p.nsplit, p.C, (p.nout + K2_N - 1) / K2_N, p.nout, p.y,
                                              p.y_pitch, p.y_total);
    count_launch();
    return cudaGetLastError();
}

cudaError_t k2_launch(const CUtensorMap &mx_hi, const CUtensorMap &mx_lo, const CUtensorMap &mt_hi,
                      const CUtensorMap &mt_lo, const K2Params &p, int nprod, cudaStream_t st)
{
    static bool attr[64][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64 || (nprod != 1 && nprod != 3) || p.nsplit < 1 || p.nsplit > 64 || p.range < 1 ||
        p.range % K2Cfg<1>::GS != 0)
        return cudaErrorInvalidValue;
    const int vi = nprod == 1 ? 0 : 1;
    const size_t smem = k2_smem_bytes(nprod);
    if (!attr[dev][vi]) {
        e = nprod == 1 ? cudaFuncSetAttribute(k2_toeplitz<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(k2_toeplitz<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        attr[dev][vi] = true;
    }
    const long long units = (long long)p.ntile_c * p.ntile_o * p.nsplit;
    if (units <= 0)
        return cudaSuccess;
    if (nprod == 1)
        k2_toeplitz<1><<<(unsigned)units, K2_THREADS, smem, st>>>(mx_hi, mx_lo, mt_hi, mt_lo, p);
    else
        k2_toeplitz<3><<<(unsigned)units, K2_THREADS, smem, st>>>(mx_hi, mx_lo, mt_hi, mt_lo, p);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess || p.nsplit == 1 || (p.ticket != nullptr && p.nsplit <= K2_FOLD_MAX))
        return e;  // no parts, or folded in the kernel
    const long long work = (long long)p.C * p.nout;
    k2_reduce<<<grid_for(work), 256, 0, st>>>(p.partial, p.nsplit, p.C, p.ntile_o, p.nout, p.y,
                                              p.y_pitch, p.y_total);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tc
