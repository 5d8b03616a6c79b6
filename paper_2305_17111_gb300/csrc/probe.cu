// Exponential throughput of the GPU: the peak of the row kernel's roofline
// measured on the device itself.  Each thread runs four independent chains of
// exponentials (enough to keep the unit busy); the rate is results per clock
// per SM at the device's maximum SM clock.
#include <algorithm>

#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

constexpr int kProbeIters = 4096;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_f32(float* out) {
    float a = threadIdx.x * 1e-3f, b = a + 0.1f, c = a + 0.2f, d = a + 0.3f;
    for (int i = 0; i < kProbeIters; ++i) {
        asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a));
        asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(b));
        asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(c));
        asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(d));
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a + b + c + d;
}
template <int KIND>   // 1: f16x2, 2: bf16x2
__global__ void __launch_bounds__(kProbeThreads) k_probe_x2(float* out) {
    uint32_t a = (KIND == 1 ? 0x3c003c00u : 0x3f803f80u) ^ threadIdx.x, b = a ^ 1u, c = a ^ 2u,
             d = a ^ 3u;
    for (int i = 0; i < kProbeIters; ++i) {
        if (KIND == 1) {
            asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(a));
            asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(b));
            asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(c));
            asm volatile("ex2.approx.f16x2 %0, %0;" : "+r"(d));
        } else {
            asm volatile("ex2.approx.ftz.bf16x2 %0, %0;" : "+r"(a));
            asm volatile("ex2.approx.ftz.bf16x2 %0, %0;" : "+r"(b));
            asm volatile("ex2.approx.ftz.bf16x2 %0, %0;" : "+r"(c));
            asm volatile("ex2.approx.ftz.bf16x2 %0, %0;" : "+r"(d));
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)(a ^ b ^ c ^ d);
}

}  // namespace
}  // namespace lmmew

using namespace lmmew;

extern "C" int lm_probe_ex2_rate(lm_stream stream, double* out4) {
    if (!out4) return set_error(LMMEW_ERR_INVALID_ARG, "out4 is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, khz = 0;
    LMMEW_CUDA(cudaGetDevice(&dev));
    LMMEW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LMMEW_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const int blocks = sms * 8;
    float* buf = nullptr;
    LMMEW_CUDA(cudaMalloc(&buf, sizeof(float) * (size_t)blocks * kProbeThreads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LMMEW_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = set_error(LMMEW_ERR_CUDA, "event creation");
    for (int kind = 0; kind < 3 && rc == LMMEW_OK; ++kind) {
        float best = 3.0e38f;
        for (int rep = 0; rep < 3 && rc == LMMEW_OK; ++rep) {   // the first launch warms up
            cudaEventRecord(e0, st);
            if (kind == 0) k_probe_f32<<<blocks, kProbeThreads, 0, st>>>(buf);
            else if (kind == 1) k_probe_x2<1><<<blocks, kProbeThreads, 0, st>>>(buf);
            else k_probe_x2<2><<<blocks, kProbeThreads, 0, st>>>(buf);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = set_error(LMMEW_ERR_CUDA, "ex2 probe");
            else if (rep > 0)
                best = std::min(best, ms);
        }
        if (rc != LMMEW_OK) break;
        const double results = (double)blocks * kProbeThreads * kProbeIters * 4 * (kind == 0 ? 1 : 2);
        out4[kind] = results / (best * 1e-3) / sms / (khz * 1e3);
    }
    out4[3] = khz / 1e3;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    return rc;
}
