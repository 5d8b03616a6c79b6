// Self-test of the bounded waits every pipelined kernel of this library uses:
// one warp initialises an mbarrier that nothing ever arrives on and waits on
// it through the same bounded wait; the wait gives up after its time limit,
// the kernel records the timeout in a status word and returns, and the host
// reports it.  Nothing is in flight (no copies, no MMAs, no tensor memory),
// so the context stays usable.
#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

__global__ void k_wait_without_arrival(int* status, unsigned long long* waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        mbar_fence_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        const uint64_t t0 = global_timer();
        const bool ok = mbar_wait_bounded(b, 0);   // phase 0 never completes
        *waited_ns = global_timer() - t0;
        *status = ok ? 0 : kStatusTimeout;
    }
}

}  // namespace
}  // namespace lmmew

using namespace lmmew;

extern "C" int lm_selftest_wait_timeout(double* waited_ms) {
    if (!waited_ms) return set_error(LMMEW_ERR_INVALID_ARG, "waited_ms is NULL");
    int* d_status = nullptr;
    unsigned long long* d_ns = nullptr;
    if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_ns, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_status);
        return set_error(LMMEW_ERR_OOM, "self-test buffers");
    }
    k_wait_without_arrival<<<1, 32>>>(d_status, d_ns);
    int status = 0;
    unsigned long long ns = 0;
    int rc = LMMEW_OK;
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = set_error(LMMEW_ERR_CUDA, "self-test kernel");
    cudaFree(d_status);
    cudaFree(d_ns);
    if (rc != LMMEW_OK) return rc;
    *waited_ms = ns / 1e6;
    if (status & kStatusTimeout)
        return set_error(LMMEW_ERR_TIMEOUT, "bounded wait ran out as intended");
    return set_error(LMMEW_ERR_CUDA, "the wait completed although nothing arrived");
}
