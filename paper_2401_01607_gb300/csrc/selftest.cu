// selftest.cu -- check of failure detection: a device-side wait that nothing
// will ever satisfy must run out, report, and leave the context usable.
//
// Every wait in the kernels (TMA completion, MMA completion, accumulator
// hand-over) is an mbarrier poll bounded by %globaltimer and by a poll count.
// When a bound is reached the waiting thread ORs an error bit into the
// launch's error word and the kernel returns; the host turns the word into
// TC_ETIMEOUT. tc_selftest_wait exercises exactly that path on an mbarrier
// that no thread or copy ever completes.
#include "../../include/taches.h"
#include "ptx.cuh"
#include "tc_internal.h"

#include <string>

namespace tc {
namespace {

__global__ void wait_selftest_kernel(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        // Phase 0 of `bar` never completes: the wait gives up after limit_ns.
        mbar_wait_limited(&bar, 0, err, ERR_TIMEOUT_TMA, limit_ns);
    }
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_selftest_wait(unsigned long long limit_ns, void *cuda_stream)
{
    if (limit_ns == 0 || limit_ns > 10000000000ull) {
        tc::set_last_error("tc_selftest_wait: limit_ns must be in [1, 1e10]");
        return TC_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int *d_err = nullptr;
    int h_err = 0;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_err), sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        tc::wait_selftest_kernel<<<1, 32, 0, st>>>(d_err, limit_ns);
        tc::count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (d_err)
        cudaFreeAsync(d_err, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        tc::set_last_error((std::string("tc_selftest_wait: ") + cudaGetErrorString(e)).c_str());
        return TC_ECUDA;
    }
    if (h_err & tc::ERR_TIMEOUT_TMA) {
        tc::set_last_error("tc_selftest_wait: the bounded wait ran out and reported, as it must");
        return TC_ETIMEOUT;
    }
    tc::set_last_error("tc_selftest_wait: the wait returned without reporting a timeout");
    return TC_ECUDA;
}
