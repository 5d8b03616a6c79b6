// The rest of an LM-OSEM sub-iteration (Eq. os-lm-mlem with z_bar_update_os):
// the per-event ratio 1/y_j, the back projection sum_j a_j[q] / y_j by voxel
// ownership (every voxel's sum is owned by one thread, no global atomics),
// the FP64 log-likelihood of Eq. (lll_med) and the multiplicative update.
// All sums run in a fixed order, so an OSEM run is bit-reproducible.
#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

constexpr int kBpEvents = kBpChunkEvents;   // events per back-projection partial
constexpr int kBpVoxels = 256;    // voxels per back-projection block

// FP64 sums of a voxel's partials in a fixed order: within each run of
// partials (one row block, or one realisation's chunks), partial i goes to
// strand i mod 8, each strand in order of i; the strands are added pairwise
// at the end.  Eight independent chains keep eight loads and adds in flight
// in the one thread that owns the voxel, and the order is the same in every
// reduction, so the one-realisation and batched paths still agree bit for bit.
__device__ __forceinline__ void strand_add(double (&s)[8], const float* bpart, int64_t first,
                                           int64_t n, int nq, int q) {
    int64_t i = 0;
    for (; i + 8 <= n; i += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) s[u] += (double)bpart[(size_t)(first + i + u) * nq + q];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
        if (i + u < n) s[u] += (double)bpart[(size_t)(first + i + u) * nq + q];
}
__device__ __forceinline__ double strand_total(const double (&s)[8]) {
    return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

__global__ void k_forward_out(const float* ypart, int64_t stride, int nqt, int64_t count,
                              const uint32_t* perm, float* out_y) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    float y = 0.f;
    for (int t = 0; t < nqt; ++t) y += ypart[(size_t)t * stride + j];
    out_y[perm[j]] = y;
}

// One block per (chunk of 128 events, 256 voxels).  The block first forms
// the events' weights: r_j = 1 / y_j from the per-q-tile partial forward
// sums (0 when y_j <= 0), or the caller's weights.  Blocks of the first voxel
// column also write the chunk's sum of log y_j (FP64).
__global__ void __launch_bounds__(kBpVoxels) k_bp_partial(
    const float* rows, int row_stride, const float* ypart, int64_t ypart_stride, int nqt,
    int64_t count, const uint32_t* perm, const float* weight, int nq, float* bpart, int64_t row0,
    double* llpart) {
    __shared__ float r[kBpEvents];
    __shared__ double ll[kBpEvents];
    const int t = threadIdx.x;
    // the log-likelihood terms, wanted from one voxel column when asked for
    const bool want_ll = llpart != nullptr && blockIdx.y == 0;
    const int64_t j0 = (int64_t)blockIdx.x * kBpEvents;
    if (t < kBpEvents) {
        const int64_t j = j0 + t;
        float rv = 0.f;
        double lv = 0.0;
        if (j < count) {
            if (weight) {
                rv = weight[perm[j]];
            } else {
                float y = 0.f;
                for (int k = 0; k < nqt; ++k) y += ypart[(size_t)k * ypart_stride + j];
                if (y > 0.f) {
                    rv = 1.0f / y;
                    if (want_ll) lv = log((double)y);   // FP64: slow on this GPU, so only where used
                }
            }
        }
        r[t] = rv;
        ll[t] = lv;
    }
    __syncthreads();
    if (llpart && blockIdx.y == 0) {
        for (int off = kBpEvents / 2; off > 0; off >>= 1) {
            if (t < off) ll[t] += ll[t + off];
            __syncthreads();
        }
        if (t == 0) llpart[row0 + blockIdx.x] = ll[0];
    }
    const int q = blockIdx.y * kBpVoxels + t;
    if (q >= nq) return;
    const int64_t rem = count - j0;
    const int n_here = rem < kBpEvents ? (int)rem : kBpEvents;
    const float* rp = rows + (size_t)j0 * row_stride + q;
    float acc = 0.f;
    for (int e = 0; e < n_here; ++e) acc = fmaf(r[e], rp[(size_t)e * row_stride], acc);
    bpart[(size_t)(row0 + blockIdx.x) * nq + q] = acc;
}

// The same with the chunk's size on the device (range: sorted events
// [z, w)); rows, ypart and weights are indexed from z, blocks past the
// chunk's events return at once.
__global__ void __launch_bounds__(kBpVoxels) k_bp_partial_range(
    const float* rows, int row_stride, const float* ypart, int64_t ypart_stride, int nqt,
    const ChunkRange* range, const uint32_t* perm, const float* weight, int nq, float* bpart,
    int64_t slot0, double* llpart) {
    __shared__ float r[kBpEvents];
    __shared__ double ll[kBpEvents];
    const ChunkRange R = *range;
    const int64_t count = (int64_t)R.w - R.z;
    const int t = threadIdx.x;
    // the log-likelihood terms, wanted from one voxel column when asked for
    const bool want_ll = llpart != nullptr && blockIdx.y == 0;
    const int64_t j0 = (int64_t)blockIdx.x * kBpEvents;
    if (j0 >= count) return;
    if (t < kBpEvents) {
        const int64_t j = j0 + t;
        float rv = 0.f;
        double lv = 0.0;
        if (j < count) {
            if (weight) {
                rv = weight[perm[R.z + j]];
            } else {
                float y = 0.f;
                for (int k = 0; k < nqt; ++k) y += ypart[(size_t)k * ypart_stride + j];
                if (y > 0.f) {
                    rv = 1.0f / y;
                    if (want_ll) lv = log((double)y);   // FP64: slow on this GPU, so only where used
                }
            }
        }
        r[t] = rv;
        ll[t] = lv;
    }
    __syncthreads();
    if (llpart && blockIdx.y == 0) {
        for (int off = kBpEvents / 2; off > 0; off >>= 1) {
            if (t < off) ll[t] += ll[t + off];
            __syncthreads();
        }
        if (t == 0) llpart[slot0 + blockIdx.x] = ll[0];
    }
    const int q = blockIdx.y * kBpVoxels + t;
    if (q >= nq) return;
    const int64_t rem = count - j0;
    const int n_here = rem < kBpEvents ? (int)rem : kBpEvents;
    const float* rp = rows + (size_t)j0 * row_stride + q;
    float acc = 0.f;
    for (int e = 0; e < n_here; ++e) acc = fmaf(r[e], rp[(size_t)e * row_stride], acc);
    bpart[(size_t)(slot0 + blockIdx.x) * nq + q] = acc;
}

__device__ __forceinline__ int64_t parts_of(const ChunkRange& R) {
    return ((int64_t)R.w - R.z + kBpEvents - 1) / kBpEvents;
}

// Voxel sums over the partials of n_blocks row blocks, block k's at slots
// [k ppc, k ppc + its parts), in slot order.
__global__ void k_voxel_reduce_ranges(const float* bpart, const ChunkRange* ranges, int n_blocks,
                                      int64_t ppc, int nq, double* num) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < n_blocks; ++k) strand_add(s, bpart, k * ppc, parts_of(ranges[k]), nq, q);
    num[q] = strand_total(s);
}

__global__ void k_forward_out_range(const float* ypart, int64_t stride, int nqt,
                                    const ChunkRange* range, const uint32_t* perm, float* out_y) {
    const ChunkRange R = *range;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (int64_t)R.w - R.z) return;
    float y = 0.f;
    for (int t = 0; t < nqt; ++t) y += ypart[(size_t)t * stride + j];
    out_y[perm[R.z + j]] = y;
}

// Events that failed validation sort after the valid ones: their outputs
// are NaN (the status word tells the next synchronising call).
__global__ void k_invalid_out(const int* n_valid, int64_t n, const uint32_t* perm, float* out_y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && i >= *n_valid) out_y[perm[i]] = __int_as_float(0x7fc00000);
}

__global__ void k_voxel_reduce(const float* bpart, int64_t n_parts, int nq, double* num) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    strand_add(s, bpart, 0, n_parts, nq, q);
    num[q] = strand_total(s);
}

// Single block: log-likelihood at the incoming image, then the update.  The
// log terms are the n_ll partials at llpart, or (ranges set) the partials of
// n_ll row blocks, block k's at slots [k ppc, k ppc + its parts).
__global__ void __launch_bounds__(1024) k_update(float* lam, const double* num, const double* sens,
                                                 int nq, const double* llpart, int64_t n_ll,
                                                 double* loglik, const ChunkRange* ranges = nullptr,
                                                 int64_t ppc = 0) {
    __shared__ double red[1024];
    const int t = threadIdx.x;
    if (loglik) {
        double s = 0.0;
        if (ranges) {
            for (int64_t k = 0; k < n_ll; ++k) {
                const int64_t parts = parts_of(ranges[k]);
                for (int64_t i = t; i < parts; i += 1024) s += llpart[k * ppc + i];
            }
        } else {
            for (int64_t i = t; i < n_ll; i += 1024) s += llpart[i];
        }
        for (int q = t; q < nq; q += 1024) s -= (double)lam[q] * sens[q];
        red[t] = s;
        __syncthreads();
        for (int off = 512; off > 0; off >>= 1) {
            if (t < off) red[t] += red[t + off];
            __syncthreads();
        }
        if (t == 0) *loglik = red[0];
        __syncthreads();
    }
    for (int q = t; q < nq; q += 1024)
        lam[q] = sens[q] > 0.0 ? (float)((double)lam[q] * num[q] / sens[q]) : 0.f;
}

__global__ void k_gather(const float* image, const int* q_pix, int nq, float* lam) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nq) lam[q] = image[q_pix[q]];
}

__global__ void k_scatter_f(const float* v, const int* q_pix, int nq, float* image) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nq) image[q_pix[q]] = v[q];
}

__global__ void k_scatter_d(const double* v, const int* q_pix, int nq, double* image) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nq) image[q_pix[q]] = v[q];
}

__global__ void k_scatter_df(const double* v, const int* q_pix, int nq, float* image) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nq) image[q_pix[q]] = (float)v[q];
}

}  // namespace

int launch_forward_out(lm_handle* h, const float* ypart, int64_t ypart_stride, int64_t begin,
                       int64_t count, const uint32_t* perm, float* out_y, cudaStream_t st) {
    if (count <= 0) return LMMEW_OK;
    k_forward_out<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(ypart, ypart_stride, h->mc.nqt,
                                                                   count, perm + begin, out_y);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_bp_partial(lm_handle* h, const float* rows, int row_stride, const float* ypart,
                      int64_t ypart_stride, int64_t count, const uint32_t* perm,
                      const float* weight, float* bpart, int64_t bpart_row0, double* llpart,
                      cudaStream_t st) {
    if (count <= 0) return LMMEW_OK;
    const int nq = h->mc.nq;
    dim3 g((unsigned)((count + kBpEvents - 1) / kBpEvents), (nq + kBpVoxels - 1) / kBpVoxels);
    k_bp_partial<<<g, kBpVoxels, 0, st>>>(rows, row_stride, ypart, ypart_stride, h->mc.nqt, count,
                                          perm, weight, nq, bpart, bpart_row0, llpart);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int64_t bp_parts(int64_t count) { return (count + kBpEvents - 1) / kBpEvents; }

int launch_voxel_reduce(lm_handle* h, const float* bpart, int64_t n_parts, double* num,
                        cudaStream_t st) {
    k_voxel_reduce<<<(h->mc.nq + 255) / 256, 256, 0, st>>>(bpart, n_parts, h->mc.nq, num);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_update(lm_handle* h, float* lam_v, const double* num, const double* sens,
                  const double* llpart, int64_t n_ll, double* loglik_out, cudaStream_t st) {
    k_update<<<1, 1024, 0, st>>>(lam_v, num, sens, h->mc.nq, llpart, n_ll, loglik_out);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_forward_out_range(lm_handle* h, const float* ypart, int64_t ypart_stride,
                             int64_t capacity, const ChunkRange* range, const uint32_t* perm,
                             float* out_y, cudaStream_t st) {
    if (capacity <= 0) return LMMEW_OK;
    k_forward_out_range<<<(unsigned)((capacity + 255) / 256), 256, 0, st>>>(
        ypart, ypart_stride, h->mc.nqt, range, perm, out_y);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_invalid_out(lm_handle* h, const int* n_valid, int64_t n, const uint32_t* perm,
                       float* out_y, cudaStream_t st) {
    if (n <= 0) return LMMEW_OK;
    k_invalid_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_valid, n, perm, out_y);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_bp_partial_range(lm_handle* h, const float* rows, int row_stride, const float* ypart,
                            int64_t ypart_stride, int64_t capacity, const ChunkRange* range,
                            const uint32_t* perm, const float* weight, float* bpart,
                            int64_t slot0, double* llpart, cudaStream_t st) {
    if (capacity <= 0) return LMMEW_OK;
    const int nq = h->mc.nq;
    dim3 g((unsigned)((capacity + kBpEvents - 1) / kBpEvents), (nq + kBpVoxels - 1) / kBpVoxels);
    k_bp_partial_range<<<g, kBpVoxels, 0, st>>>(rows, row_stride, ypart, ypart_stride, h->mc.nqt,
                                                range, perm, weight, nq, bpart, slot0, llpart);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_voxel_reduce_ranges(lm_handle* h, const float* bpart, const ChunkRange* ranges,
                               int n_blocks, int64_t ppc, double* num, cudaStream_t st) {
    k_voxel_reduce_ranges<<<(h->mc.nq + 255) / 256, 256, 0, st>>>(bpart, ranges, n_blocks, ppc,
                                                                  h->mc.nq, num);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_update_ranges(lm_handle* h, float* lam_v, const double* num, const double* sens,
                         const double* llpart, const ChunkRange* ranges, int n_blocks,
                         int64_t ppc, double* loglik_out, cudaStream_t st) {
    k_update<<<1, 1024, 0, st>>>(lam_v, num, sens, h->mc.nq, llpart, n_blocks, loglik_out, ranges,
                                 ppc);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_gather_image(lm_handle* h, const float* image, float* lam_v, cudaStream_t st) {
    k_gather<<<(h->mc.nq + 255) / 256, 256, 0, st>>>(image, h->d_q_pix, h->mc.nq, lam_v);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_scatter_image(lm_handle* h, const float* lam_v, float* image, cudaStream_t st) {
    LMMEW_CUDA(cudaMemsetAsync(image, 0, sizeof(float) * h->mc.n * h->mc.n, st));
    k_scatter_f<<<(h->mc.nq + 255) / 256, 256, 0, st>>>(lam_v, h->d_q_pix, h->mc.nq, image);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_scatter_image_d(lm_handle* h, const double* v, double* image, cudaStream_t st) {
    LMMEW_CUDA(cudaMemsetAsync(image, 0, sizeof(double) * h->mc.n * h->mc.n, st));
    k_scatter_d<<<(h->mc.nq + 255) / 256, 256, 0, st>>>(v, h->d_q_pix, h->mc.nq, image);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_num_to_image(lm_handle* h, const double* num, float* image, cudaStream_t st) {
    LMMEW_CUDA(cudaMemsetAsync(image, 0, sizeof(float) * h->mc.n * h->mc.n, st));
    k_scatter_df<<<(h->mc.nq + 255) / 256, 256, 0, st>>>(num, h->d_q_pix, h->mc.nq, image);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

// ---------------------------------------------------------------------------
// Batched realisations: the same steps with every back-projection chunk
// holding one realisation's events, voxel sums and updates per realisation.
namespace {

// One block per (chunk, 256 voxels).  A chunk is up to 128 events of one
// realisation inside one row block, listed by the back-projection order
// (sorted positions); the block owns its voxels' partial sums in the chunk's
// slot.
__global__ void __launch_bounds__(kBpVoxels) k_bp_batch(
    const float* rows, int row_stride, const float* ypart, int64_t ypart_stride, int nqt,
    const uint32_t* bp_idx, int64_t row_base, const BpChunk* chunks, int nq, float* bpart,
    double* llpart) {
    __shared__ float r[kBpEvents];
    __shared__ int64_t idx[kBpEvents];
    __shared__ double ll[kBpEvents];
    const int t = threadIdx.x;
    // the log-likelihood terms, wanted from one voxel column when asked for
    const bool want_ll = llpart != nullptr && blockIdx.y == 0;
    const BpChunk C = chunks[blockIdx.x];
    if (t < kBpEvents) {
        float rv = 0.f;
        double lv = 0.0;
        int64_t j = 0;
        if (t < C.count) {
            j = (int64_t)bp_idx[C.begin + t] - row_base;
            float y = 0.f;
            for (int k = 0; k < nqt; ++k) y += ypart[(size_t)k * ypart_stride + j];
            if (y > 0.f) {
                rv = 1.0f / y;
                if (want_ll) lv = log((double)y);   // FP64: slow on this GPU, so only where used
            }
        }
        r[t] = rv;
        idx[t] = j;
        ll[t] = lv;
    }
    __syncthreads();
    if (llpart && blockIdx.y == 0) {
        for (int off = kBpEvents / 2; off > 0; off >>= 1) {
            if (t < off) ll[t] += ll[t + off];
            __syncthreads();
        }
        if (t == 0) llpart[C.slot] = ll[0];
    }
    const int q = blockIdx.y * kBpVoxels + t;
    if (q >= nq) return;
    float acc = 0.f;
    for (int e = 0; e < C.count; ++e) acc = fmaf(r[e], rows[(size_t)idx[e] * row_stride + q], acc);
    bpart[(size_t)C.slot * nq + q] = acc;
}

__global__ void k_voxel_reduce_batch(const float* bpart, const int* part_start, int nq,
                                     double* num) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.y;
    if (q >= nq) return;
    double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    strand_add(s, bpart, part_start[rr], part_start[rr + 1] - part_start[rr], nq, q);
    num[(size_t)rr * nq + q] = strand_total(s);
}

__global__ void __launch_bounds__(1024) k_update_batch(float* lam, const double* num,
                                                       const double* sens, int nq,
                                                       const double* llpart,
                                                       const int* part_start, double* loglik,
                                                       int ll_stride) {
    __shared__ double red[1024];
    const int t = threadIdx.x, rr = blockIdx.x;
    float* l = lam + (size_t)rr * nq;
    const double* nm = num + (size_t)rr * nq;
    if (loglik) {
        double s = 0.0;
        for (int i = part_start[rr] + t; i < part_start[rr + 1]; i += 1024) s += llpart[i];
        for (int q = t; q < nq; q += 1024) s -= (double)l[q] * sens[q];
        red[t] = s;
        __syncthreads();
        for (int off = 512; off > 0; off >>= 1) {
            if (t < off) red[t] += red[t + off];
            __syncthreads();
        }
        if (t == 0) loglik[(size_t)rr * ll_stride] = red[0];
        __syncthreads();
    }
    for (int q = t; q < nq; q += 1024)
        l[q] = sens[q] > 0.0 ? (float)((double)l[q] * nm[q] / sens[q]) : 0.f;
}

__global__ void k_gather_batch(const float* images, int npix, const int* q_pix, int nq,
                               float* lam) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nq) lam[(size_t)blockIdx.y * nq + q] = images[(size_t)blockIdx.y * npix + q_pix[q]];
}

__global__ void k_scatter_batch(const float* lam, const int* q_pix, int nq, float* images,
                                int npix) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nq) images[(size_t)blockIdx.y * npix + q_pix[q]] = lam[(size_t)blockIdx.y * nq + q];
}

}  // namespace

int launch_bp_batch(lm_handle* h, const float* rows, int row_stride, const float* ypart,
                    int64_t ypart_stride, const uint32_t* bp_idx, int64_t row_base,
                    const BpChunk* chunks, int n_chunks, float* bpart, double* llpart,
                    cudaStream_t st) {
    if (n_chunks <= 0) return LMMEW_OK;
    dim3 g(n_chunks, (h->mc.nq + kBpVoxels - 1) / kBpVoxels);
    k_bp_batch<<<g, kBpVoxels, 0, st>>>(rows, row_stride, ypart, ypart_stride, h->mc.nqt, bp_idx,
                                        row_base, chunks, h->mc.nq, bpart, llpart);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_reduce_update_batch(lm_handle* h, int R, const float* bpart, const int* part_start,
                               double* num, float* lam_v, const double* sens,
                               const double* llpart, double* loglik, int ll_stride,
                               cudaStream_t st) {
    dim3 g((h->mc.nq + 255) / 256, R);
    k_voxel_reduce_batch<<<g, 256, 0, st>>>(bpart, part_start, h->mc.nq, num);
    k_update_batch<<<R, 1024, 0, st>>>(lam_v, num, sens, h->mc.nq, llpart, part_start, loglik,
                                       ll_stride);
    h->launches += 2;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int launch_images_batch(lm_handle* h, int R, float* images, float* lam_v, bool to_voxels,
                        cudaStream_t st) {
    const int npix = h->mc.n * h->mc.n;
    dim3 g((h->mc.nq + 255) / 256, R);
    if (to_voxels) {
        k_gather_batch<<<g, 256, 0, st>>>(images, npix, h->d_q_pix, h->mc.nq, lam_v);
    } else {
        LMMEW_CUDA(cudaMemsetAsync(images, 0, sizeof(float) * (size_t)R * npix, st));
        k_scatter_batch<<<g, 256, 0, st>>>(lam_v, h->d_q_pix, h->mc.nq, images, npix);
    }
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

}  // namespace lmmew
