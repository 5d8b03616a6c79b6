// lm_forward_noalloc: the forward projection of lm_forward for callers that
// cannot allocate device memory while they run.  Its scratch (sorted events,
// tiles, the image on the voxel list and the per-tile partial sums) lives in
// one statically sized device array of this file instead of memory the
// library would otherwise cudaMalloc.
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
// per device (host code must not use the symbol itself as an address).
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
    if (ev->n == 0) return LMMEW_OK;
    if (!ev->angle || !ev->bin || !ev->energy_keV || !image || !out_y)
        return set_error(LMMEW_ERR_INVALID_ARG, "NULL event, image or output pointer");
    const ModelConst& m = h->mc;
    const int64_t n = ev->n;
    // every word of the region below is written before it is read within a
    // call, so nothing has to start at zero
    const size_t need = sort_fixed_bytes(n, sort_groups(h, m.A)) + bump_bytes(sizeof(float) * m.nq) +
                        bump_bytes(sizeof(float) * (size_t)m.nqt * n);
    if (n >= (int64_t(1) << 31) || need > kNoAllocBytes)
        return set_error(LMMEW_ERR_INVALID_ARG,
                         "lm_forward_noalloc: " + std::to_string(n) + " events need " +
                             std::to_string(need) + " bytes of scratch, more than its fixed " +
                             std::to_string(kNoAllocBytes) + " bytes; use lm_forward");
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != LMMEW_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char* arena = (char*)base;
    SortedFixed se;
    rc = sort_events_fixed(h, ev, arena, &se, st);
    if (rc != LMMEW_OK) return rc;
    float* lam_v = bump<float>(arena, m.nq);
    float* ypart = bump<float>(arena, (size_t)m.nqt * n);
    rc = launch_gather_image(h, image, lam_v, st);
    if (rc != LMMEW_OK) return rc;
    RowLaunch L{se.tiles, 0, se.n_tiles, se.bin, se.energy, lam_v, nullptr, 0, 0, ypart, n,
                se.n_valid};
    L.tile_ev = se.tile_ev;
    rc = launch_row(h, L, st);
    if (rc != LMMEW_OK) return rc;
    return launch_forward_out(h, ypart, n, 0, se.n_valid, se.perm, out_y, st);
}
