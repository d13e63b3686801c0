// k4_q15.cu -- K4: exact fixed-point convolution with one requantization.
//
// Sec. 5.4 ("ideal requantization"): with an accumulator of unlimited range
// an output sample is requantized once, after all of its products are summed.
// Here input and taps are Q15 (int16); each product is exact in 32 bits and
// each output's sum is kept exactly in 64 bits (|sum| <= L * 2^30 < 2^49 for
// L <= 2^19), then requantized once to Q15: round half to even of
// sum / 2^15, saturated to int16.
//
// Integer addition is associative, so the result does not depend on how the
// work is split: CTA = 1024 outputs (128 threads x 8 consecutive outputs) x a
// chunk of 2048 taps; each thread keeps 8 int64 sums in registers and the
// chunk sums meet by 64-bit atomic adds, exact in any order. The input window
// and the IR chunk are staged in shared memory as int16 (zero outside the
// signal and the IR); per 8 taps a thread loads 16 inputs and 8 taps with
// three 16-byte shared loads and does 64 exact multiply-adds.
#include <cstdint>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>

#include "../../include/taches.h"
#include "tc_internal.h"

namespace tc {
namespace {

constexpr int K4_T = 128;              // threads per CTA
constexpr int K4_R = 8;                // consecutive outputs per thread
constexpr int K4_MO = K4_T * K4_R;     // outputs per CTA
constexpr int K4_KC = 2048;            // taps per chunk
constexpr int K4_XS = K4_KC + K4_MO;   // staged input samples

__device__ __forceinline__ void unpack8(const int4 v, int (&o)[8])
{
    const uint32_t w[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = (int)(int16_t)(w[i] & 0xFFFFu);
        o[2 * i + 1] = (int)(int16_t)(w[i] >> 16);
    }
}

// Inner-loop forms, both exact:
//   K4_IMAD: each product x * h (int16 x int16, exact in 32 bits) is added to an
//            int64 sum with one widening multiply-add.
//   K4_DP2A: h = 256 hh + hl with hh = h >> 8 (signed byte) and hl = h & 255
//            (unsigned byte); one dp2a adds two 16 x 8-bit products into an int32
//            sum, one sum for hh and one for hl, folded into int64 as
//            256 S_hh + S_hl every 256 taps (|S_hh| <= 2^30, |S_hl| < 2^31).
enum { K4_IMAD = 0, K4_DP2A = 1 };

__device__ __forceinline__ int dp2a_lo_ss(int a, unsigned b, int c)
{
    int d;
    asm("dp2a.lo.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ int dp2a_hi_su(int a, unsigned b, int c)
{
    int d;
    asm("dp2a.hi.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <int INNER>
__global__ void __launch_bounds__(K4_T) k4_q15(const int16_t *__restrict__ x, long long N,
                                                const int16_t *__restrict__ h, long long L,
                                                unsigned long long *__restrict__ acc, long long ny)
{
    __shared__ __align__(16) int16_t xs[K4_XS];
    // K4_IMAD: taps as int16. K4_DP2A: one word per tap pair (k, k+1), bytes
    // (hh[k+1], hh[k], hl[k+1], hl[k]) from the low byte up.
    __shared__ __align__(16) uint32_t hsw[K4_KC / 2];
    const int tid = threadIdx.x;
    const long long m_base = (long long)blockIdx.x * K4_MO;
    const long long k0 = (long long)blockIdx.y * K4_KC;
    // xs[i] = x[n_lo + i]: every x[m - k] for m in the tile, k in the chunk.
    const long long n_lo = m_base - k0 - K4_KC + 1;
    for (int i = tid; i < K4_XS; i += K4_T) {
        const long long n = n_lo + i;
        xs[i] = (n >= 0 && n < N) ? x[n] : (int16_t)0;
    }
    for (int p = tid; p < K4_KC / 2; p += K4_T) {
        const long long k = k0 + 2 * p;
        const uint32_t a = (k < L) ? (uint32_t)(uint16_t)h[k] : 0u;
        const uint32_t b = (k + 1 < L) ? (uint32_t)(uint16_t)h[k + 1] : 0u;
        if (INNER == K4_IMAD)
            hsw[p] = a | (b << 16);
        else
            hsw[p] = (b >> 8) | (a & 0xFF00u) | ((b & 0xFFu) << 16) | ((a & 0xFFu) << 24);
    }
    __syncthreads();

    // Thread outputs m0 + r, r < 8; tap k0 + kk + j reads xs[base + r - j + 7]
    // with base = 8 tid - kk + KC - 8, a multiple of 8 (16-byte aligned).
    long long sum[K4_R];
#pragma unroll
    for (int r = 0; r < K4_R; ++r)
        sum[r] = 0;
    if (INNER == K4_IMAD) {
        const int16_t *hs = reinterpret_cast<const int16_t *>(hsw);
#pragma unroll 2
        for (int kk = 0; kk < K4_KC; kk += 8) {
            const int4 *xp = reinterpret_cast<const int4 *>(xs + 8 * tid - kk + K4_KC - 8);
            int lo[8], hi[8], hv[8];
            unpack8(xp[0], lo);
            unpack8(xp[1], hi);
            unpack8(*reinterpret_cast<const int4 *>(hs + kk), hv);
            int xv[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                xv[i] = lo[i];
                xv[8 + i] = hi[i];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int r = 0; r < K4_R; ++r)
                    sum[r] += (long long)xv[r - j + 7] * (long long)hv[j];
        }
    } else {
        for (int kb = 0; kb < K4_KC; kb += 256) {
            int sh[K4_R], sl[K4_R];
#pragma unroll
            for (int r = 0; r < K4_R; ++r)
                sh[r] = sl[r] = 0;
#pragma unroll 2
            for (int kk = kb; kk < kb + 256; kk += 8) {
                const int4 *xp = reinterpret_cast<const int4 *>(xs + 8 * tid - kk + K4_KC - 8);
                const int4 x0 = xp[0], x1 = xp[1];
                const int w[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                // w[i] = (xv[2i], xv[2i+1]); o[i] = (xv[2i+1], xv[2i+2]).
                int o[7];
#pragma unroll
                for (int i = 0; i < 7; ++i)
                    o[i] = (int)__byte_perm((unsigned)w[i], (unsigned)w[i + 1], 0x5432);
                const uint4 hq = *reinterpret_cast<const uint4 *>(hsw + kk / 2);
                const unsigned hp[4] = {hq.x, hq.y, hq.z, hq.w};
                // Taps (2q, 2q+1) of output r read (xv[u], xv[u+1]), u = r - 2q + 6.
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int r = 0; r < K4_R; ++r) {
                        const int u = r - 2 * q + 6;
                        const int a = (u & 1) ? o[u >> 1] : w[u >> 1];
                        sh[r] = dp2a_lo_ss(a, hp[q], sh[r]);
                        sl[r] = dp2a_hi_su(a, hp[q], sl[r]);
                    }
            }
#pragma unroll
            for (int r = 0; r < K4_R; ++r)
                sum[r] += (long long)sh[r] * 256 + (long long)sl[r];
        }
    }
    const long long m0 = m_base + (long long)K4_R * tid;
#pragma unroll
    for (int r = 0; r < K4_R; ++r)
        if (m0 + r < ny && sum[r] != 0)
            atomicAdd(acc + m0 + r, (unsigned long long)sum[r]);
}

// y[m] = sat16(round half to even(acc[m] / 2^15)).
__global__ void k4_requant(const long long *__restrict__ acc, long long ny, int16_t *__restrict__ y)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < ny;
         m += (long long)gridDim.x * blockDim.x) {
        const long long a = acc[m];
        long long q = a >> 15;                 // floor(a / 2^15) (arithmetic shift)
        const long long rem = a - q * 32768;   // in [0, 2^15)
        if (rem > 16384 || (rem == 16384 && (q & 1)))
            ++q;
        q = q > 32767 ? 32767 : (q < -32768 ? -32768 : q);
        y[m] = (int16_t)q;
    }
}

// Inner-loop form: TC_Q15_INNER=imad or dp2a in the environment, read at each
// call; dp2a by default. Both give the same, exact, result.
int q15_inner()
{
    const char *e = std::getenv("TC_Q15_INNER");
    return (e && std::strcmp(e, "imad") == 0) ? (int)K4_IMAD : (int)K4_DP2A;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_convolve_q15(const int16_t *x, size_t N, const int16_t *h, size_t L, int16_t *y,
                                     int64_t *acc, void *cuda_stream)
{
    tc::Range nvtx_range("tc_convolve_q15");
    if (!x || !h || (!y && !acc))
        return (tc::set_last_error("tc_convolve_q15: x, h or both outputs are NULL"), TC_EINVAL);
    if (N == 0 || L == 0 || L > ((size_t)1 << 19) || N > ((size_t)1 << 40))
        return (tc::set_last_error("tc_convolve_q15: N must be > 0 and L in [1, 2^19]"), TC_EINVAL);
    // Role swap (Sec. 3.2): the kernel's work is (N + L - 1) L, so the shorter
    // operand takes the IR role. Integer sums make the result bit-identical.
    if (N < L && !tc::no_role_swap()) {
        std::swap(x, h);
        std::swap(N, L);
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long ny = (long long)N + (long long)L - 1;
    long long *a = reinterpret_cast<long long *>(acc);
    cudaError_t e = cudaSuccess;
    if (!a)
        e = tc::pool_alloc(reinterpret_cast<void **>(&a), (size_t)ny * sizeof(long long), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(a, 0, (size_t)ny * sizeof(long long), st);
    if (e == cudaSuccess) {
        const dim3 grid((unsigned)((ny + tc::K4_MO - 1) / tc::K4_MO), (unsigned)(((long long)L + tc::K4_KC - 1) / tc::K4_KC));
        if ((long long)grid.x * tc::K4_MO < ny)
            e = cudaErrorInvalidConfiguration;
        else {
            auto kern = tc::q15_inner() == tc::K4_DP2A ? tc::k4_q15<tc::K4_DP2A> : tc::k4_q15<tc::K4_IMAD>;
            kern<<<grid, tc::K4_T, 0, st>>>(x, (long long)N, h, (long long)L,
                                           reinterpret_cast<unsigned long long *>(a), ny);
            tc::count_launch();
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && y) {
        const long long blocks = std::min<long long>((ny + 255) / 256, 65535);
        tc::k4_requant<<<(unsigned)blocks, 256, 0, st>>>(a, ny, y);
        tc::count_launch();
        e = cudaGetLastError();
    }
    if (!acc && a)
        cudaFreeAsync(a, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        tc::set_last_error((std::string("tc_convolve_q15: ") + cudaGetErrorString(e)).c_str());
        return e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA;
    }
    return TC_OK;
}
