// k_prep.cu -- IR preparation for K1: four copies of each IR row, shifted by
// e = 0..3 taps and zero-padded, so that every tap chunk that K1 stages
// starts on a 16-byte boundary whatever the output alignment.
#include <cstdlib>
#include <atomic>
#include <mutex>

#include "tc_internal.h"

namespace tc {

namespace {

std::atomic<uint64_t> g_launches{0};

__global__ void ir_prep_kernel(const float *__restrict__ src, long long src_pitch, long long n, int rows,
                               float *__restrict__ dst, long long row_stride, long long phase, long long Lpad)
{
    // One float4 of one shifted copy per thread iteration: Lpad / 4 float4s
    // per copy, 4 copies per row.
    const long long per_row = Lpad / 4;
    const long long total = (long long)rows * 4 * per_row;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = q / (4 * per_row);
        const long long rem = q % (4 * per_row);
        const int e = (int)(rem / per_row);
        const long long j0 = 4 * (rem % per_row);
        const float *s = src + r * src_pitch;
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long k = j0 + u - e;
            v[u] = (k >= 0 && k < n) ? s[k] : 0.f;
        }
        *reinterpret_cast<float4 *>(dst + r * row_stride + e * phase + j0) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

}  // namespace

cudaError_t ir_prep_launch(const float *src, long long src_pitch, long long n, int rows, float *dst,
                           long long row_stride, long long phase, long long Lpad, cudaStream_t st)
{
    if ((Lpad & 3) || (phase & 3) || (row_stride & 3) || rows < 1 || n < 1 || n > Lpad)
        return cudaErrorInvalidValue;
    const long long work = (long long)rows * Lpad;  // float4 items
    long long blocks = (work + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    ir_prep_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, src_pitch, n, rows, dst, row_stride, phase, Lpad);
    count_launch();
    return cudaGetLastError();
}

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

namespace {
std::atomic<int> g_inject[3];  // per site: passes left before the armed failure (0: disarmed)
}  // namespace

void inject_arm(int site, int nth) { g_inject[site].store(nth); }

bool inject_take(int site)
{
    int v = g_inject[site].load(std::memory_order_relaxed);
    while (v > 0) {
        if (g_inject[site].compare_exchange_weak(v, v - 1))
            return v == 1;
    }
    return false;
}
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

// The library's stream-ordered memory pool on each device, for the scratch of
// one-shot calls. It keeps up to 2 GiB of freed memory mapped, so that calls
// in a row do not map and unmap their scratch each time (the device's default
// pool returns freed memory at every synchronisation). Created on first use.
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
constexpr uint64_t kPoolKeep = 2ull << 30;
}  // namespace

cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pools[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pools[dev], &props);
            if (e != cudaSuccess)
                return e;
            uint64_t keep = kPoolKeep;
            e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess)
                return e;
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

// Memory freed into the pool above its 2 GiB is otherwise released at the
// next synchronisation on the device, whoever makes it: after a large close
// (a server with a hundred groups frees tens of GB) that unmapping can stall
// the next user's steps. Closing trims the pool itself instead.
void pool_trim()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        pool = g_pools[dev];
    }
    if (pool)
        cudaMemPoolTrimTo(pool, kPoolKeep);
}

bool no_role_swap()
{
    const char *e = std::getenv("TC_NO_ROLE_SWAP");
    return e && e[0] == '1';
}

}  // namespace tc
