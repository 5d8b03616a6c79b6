// lm_forward_noalloc: the forward projection of lm_forward for callers that
// cannot allocate device memory while they run.  Its scratch (the sort's
// group arrays, sorted events, tiles, the image on the voxel list, the
// per-tile partial sums and the row-block ranges) lives in one statically
// sized device array of this file instead of memory the library would
// otherwise cudaMalloc; it runs the same kernels, in the same order, as
// lm_forward.
#include <mutex>

#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kNoAllocBytes = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the static array on the current device, looked up once
// per device (host code must not use the symbol itself as an address).  The
// address stays cached for the life of the process: after a device reset
// (cudaDeviceReset) it would be stale, so the library must not be used
// across one.
int scratch_address(void** out) {
    int dev = 0;
    LMMEW_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(LMMEW_ERR_INVALID_ARG, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LMMEW_OK;
}

}  // namespace
}  // namespace lmmew

using namespace lmmew;

extern "C" int lm_forward_noalloc(lm_handle* h, const lm_events* ev, const float* image,
                                  float* out_y, lm_stream stream) {
    if (!h || !ev) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    if (ev->n < 0) return set_error(LMMEW_ERR_INVALID_ARG, "negative event count");
    // the surrogate models keep a row block of the whole event list: refused
    // before anything is queued
    if (h->scatter_model == LMMEW_SCATTER_SURROGATE ||
        h->scatter_model == LMMEW_SCATTER_SURROGATE_COARSE)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED,
                         "lm_forward_noalloc runs the exact and the scatter-free models; use "
                         "lm_forward with a surrogate scatter model");
    if (ev->n == 0) return LMMEW_OK;
    if (!ev->angle || !ev->bin || !ev->energy_keV || !image || !out_y)
        return set_error(LMMEW_ERR_INVALID_ARG, "NULL event, image or output pointer");
    const ModelConst& m = h->mc;
    const int64_t n = ev->n;
    if (n >= (int64_t(1) << 31))
        return set_error(LMMEW_ERR_INVALID_ARG, "at most 2^31 - 1 events per call");
    // one row block of every event; every word of the region is written
    // before it is read within a call, so nothing has to start at zero
    const ForwardPlan fp = forward_plan(h, n, int64_t(1) << 40);
    const int G = sort_groups(h, m.A);
    const size_t need = bump_bytes(sizeof(int) * m.A) + 2 * bump_bytes(sizeof(int) * G) +
                        forward_region_bytes(h, fp);
    if (need > kNoAllocBytes)
        return set_error(LMMEW_ERR_INVALID_ARG,
                         "lm_forward_noalloc: " + std::to_string(n) + " events need " +
                             std::to_string(need) + " bytes of scratch, more than its fixed " +
                             std::to_string(kNoAllocBytes) + " bytes; use lm_forward");
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != LMMEW_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char* arena = (char*)base;
    const GroupArrays ga = group_arrays_into(h, arena, st);
    LMMEW_CUDA(cudaGetLastError());
    return forward_async(h, ev, image, out_y, ga, fp, arena, st);
}
