// Event validation and grouping (once per call that takes events): every
// event is checked against the model, keyed by (subset rank of its angle, bin)
// and stably sorted with an LSD radix sort written here (8-bit digits,
// per-block histograms, one global scan, stable per-block scatter by warp
// match).  The sorted order groups each angle's events contiguously, subsets
// in ascending order (subset(a) = a mod n_subsets, paper Sec. LM-OSEM), and
// cuts every angle's run into tiles of up to tile_ev events for the row kernel.
#include <algorithm>
#include <vector>

#include "lmmew_internal.cuh"

namespace lmmew {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortPerThread = 16;
constexpr int kSortChunk = kSortThreads * kSortPerThread;   // keys per block

__global__ void k_keys(const uint16_t* angle, const uint16_t* bin, const float* energy, int64_t n,
                       int A, int B, const int* rank_of_angle, int n_win,
                       float4 win01, float4 win23, float4 win45, float4 win67, uint32_t* keys,
                       uint32_t* vals, int* status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int a = angle[j], b = bin[j];
    const float e = energy[j];
    const float lo[8] = {win01.x, win01.z, win23.x, win23.z, win45.x, win45.z, win67.x, win67.z};
    const float hi[8] = {win01.y, win01.w, win23.y, win23.w, win45.y, win45.w, win67.y, win67.w};
    bool inwin = false;
    for (int k = 0; k < n_win; ++k) inwin |= (e >= lo[k] && e < hi[k]);
    const bool ok = a < A && b < B && isfinite(e) && inwin;
    keys[j] = ok ? (uint32_t)rank_of_angle[a] * (uint32_t)B + (uint32_t)b : (uint32_t)A * (uint32_t)B;
    vals[j] = (uint32_t)j;
    if (!ok) atomicOr(status, kStatusOutOfRange);
}

__global__ void __launch_bounds__(kSortThreads) k_hist(const uint32_t* keys, int64_t n, int shift,
                                                       uint32_t* hist, int nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortChunk;
    for (int i = 0; i < kSortPerThread; ++i) {
        const int64_t j = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `count` values in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan(uint32_t* v, int64_t count) {
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = (count + 1023) / 1024;
    const int64_t lo = t * per, hi = min(count, lo + per);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += v[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t x = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    uint32_t run = part[t] - s;
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t x = v[i];
        v[i] = run;
        run += x;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint32_t* keys, const uint32_t* vals,
                                                          int64_t n, int shift, const uint32_t* offs,
                                                          int nblk, uint32_t* okeys,
                                                          uint32_t* ovals) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kSortThreads / 32][257];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offs[(size_t)tid * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortChunk;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int it = 0; it < kSortPerThread; ++it) {
        for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t j = base + (int64_t)it * kSortThreads + tid;
        const bool valid = j < n;
        const uint32_t key = valid ? keys[j] : 0u;
        const uint32_t val = valid ? vals[j] : 0u;
        const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int lrank = __popc(peers & lt_mask);
        if (valid && lrank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t tot = 0;
        {
            uint32_t acc = 0;
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += c;
            }
            tot = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = run[d] + wcnt[warp][d] + lrank;
            okeys[pos] = key;
            ovals[pos] = val;
        }
        __syncthreads();
        run[tid] += tot;
        __syncthreads();
    }
}

__global__ void k_gather(const uint32_t* keys, const uint32_t* vals, const float* energy, int64_t n,
                         int B, uint32_t* perm, uint16_t* bin_s, float* e_s) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t v = vals[j], k = keys[j];
    perm[j] = v;
    bin_s[j] = (uint16_t)(k % (uint32_t)B);
    e_s[j] = energy[v];
}

__global__ void k_bounds(const uint32_t* keys, int64_t n, int A, int B, int* start) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > A) return;
    const uint32_t target = (uint32_t)r * (uint32_t)B;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < target) lo = mid + 1; else hi = mid;
    }
    start[r] = (int)lo;
}

// tile_start[r] = sum over ranks < r of ceil(count / tile_ev); one block.
__global__ void __launch_bounds__(1024) k_tile_scan(const int* start, int A, int tile_ev,
                                                    int* tile_start) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (A + 1023) / 1024;
    const int lo = t * per, hi = min(A, lo + per);
    int s = 0;
    for (int r = lo; r < hi; ++r) s += (start[r + 1] - start[r] + tile_ev - 1) / tile_ev;
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int x = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int r = lo; r < hi; ++r) {
        tile_start[r] = run;
        run += (start[r + 1] - start[r] + tile_ev - 1) / tile_ev;
    }
    if (t == 1023) tile_start[A] = part[1023];
}

__global__ void k_tiles(const int* start, const int* tile_start, const int* angle_of_rank, int A,
                        int tile_ev, const uint16_t* bin_s, Tile* tiles,
                        const int* real_of_rank = nullptr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A) return;
    const int b0 = start[r], b1 = start[r + 1];
    int t = tile_start[r];
    for (int e = b0; e < b1; e += tile_ev, ++t) {
        const int cnt = min(tile_ev, b1 - e);
        Tile T;
        T.a = angle_of_rank[r];
        T.begin = e;
        T.count = cnt;
        T.b_lo_hi = ((int)bin_s[e] << 16) | (int)bin_s[e + cnt - 1];
        T.r = real_of_rank ? real_of_rank[r] : 0;
        tiles[t] = T;
    }
}


}  // namespace

size_t sort_scratch_bytes(int64_t n, int A) {
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += ((bytes + 255) / 256) * 256 + 256; };
    add(4 * n); add(4 * n); add(4 * n); add(4 * n);    // keys/vals ping-pong
    add(4 * 256 * std::max<int64_t>(nblk, 1));         // histograms
    add(4 * n); add(2 * n); add(4 * n);                 // perm, bins, energies
    add(4 * (A + 1)); add(4 * (A + 1)); add(4 * A);     // angle_start, tile_start, angle_of_rank
    add(4 * A);                                         // rank_of_angle
    add(sizeof(Tile) * (size_t)(n / kETMin + A + 1));   // tiles (smallest tile size)
    return b;
}

int sort_events(lm_handle* h, const lm_events* ev, int n_subsets, SortedEvents* out, char*& arena,
                cudaStream_t st) {
    const ModelConst& m = h->mc;
    const int64_t n = ev->n;
    const int A = m.A, B = m.B;
    // angle order: subsets ascending, angles ascending inside a subset
    std::vector<int> rank_of_angle(A), angle_of_rank(A);
    {
        int r = 0;
        for (int s = 0; s < n_subsets; ++s)
            for (int a = s; a < A; a += n_subsets) { rank_of_angle[a] = r; angle_of_rank[r] = a; ++r; }
    }
    uint32_t* keys0 = bump<uint32_t>(arena, n);
    uint32_t* keys1 = bump<uint32_t>(arena, n);
    uint32_t* vals0 = bump<uint32_t>(arena, n);
    uint32_t* vals1 = bump<uint32_t>(arena, n);
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    uint32_t* hist = bump<uint32_t>(arena, 256 * std::max<int64_t>(nblk, 1));
    out->perm = bump<uint32_t>(arena, n);
    out->bin = bump<uint16_t>(arena, n);
    out->energy = bump<float>(arena, n);
    out->angle_start = bump<int>(arena, A + 1);
    out->tile_start = bump<int>(arena, A + 1);
    int* d_angle_of_rank = bump<int>(arena, A);
    int* d_rank_of_angle = bump<int>(arena, A);
    out->tiles = bump<Tile>(arena, n / kETMin + A + 1);
    out->tile_ev = h->tile_ev;
    out->n_groups = A;
    out->angle_of_group = d_angle_of_rank;

    LMMEW_CUDA(cudaMemcpyAsync(d_rank_of_angle, rank_of_angle.data(), sizeof(int) * A,
                               cudaMemcpyHostToDevice, st));
    LMMEW_CUDA(cudaMemcpyAsync(d_angle_of_rank, angle_of_rank.data(), sizeof(int) * A,
                               cudaMemcpyHostToDevice, st));
    if (n > 0) {
        float w[8][2] = {};
        for (int k = 0; k < m.n_win; ++k) { w[k][0] = (float)m.win_lo[k]; w[k][1] = (float)m.win_hi[k]; }
        const float4 w01 = make_float4(w[0][0], w[0][1], w[1][0], w[1][1]);
        const float4 w23 = make_float4(w[2][0], w[2][1], w[3][0], w[3][1]);
        const float4 w45 = make_float4(w[4][0], w[4][1], w[5][0], w[5][1]);
        const float4 w67 = make_float4(w[6][0], w[6][1], w[7][0], w[7][1]);
        k_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ev->angle, ev->bin, ev->energy_keV, n, A,
                                                            B, d_rank_of_angle, m.n_win, w01,
                                                            w23, w45, w67, keys0, vals0, h->d_status);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
        const uint64_t kmax = (uint64_t)A * (uint64_t)B;
        int bits = 1;
        while (bits < 32 && (kmax >> bits) != 0) ++bits;
        uint32_t *kin = keys0, *kout = keys1, *vin = vals0, *vout = vals1;
        for (int shift = 0; shift < bits; shift += 8) {
            k_hist<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, n, shift, hist, (int)nblk);
            ++h->launches;
            k_scan<<<1, 1024, 0, st>>>(hist, 256 * nblk);
            ++h->launches;
            k_scatter<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, vin, n, shift, hist, (int)nblk,
                                                              kout, vout);
            ++h->launches;
            LMMEW_CUDA(cudaGetLastError());
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kin, vin, ev->energy_keV, n, B,
                                                             out->perm, out->bin, out->energy);
        ++h->launches;
        k_bounds<<<(A + 1 + 127) / 128, 128, 0, st>>>(kin, n, A, B, out->angle_start);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
    } else {
        LMMEW_CUDA(cudaMemsetAsync(out->angle_start, 0, sizeof(int) * (A + 1), st));
    }
    k_tile_scan<<<1, 1024, 0, st>>>(out->angle_start, A, out->tile_ev, out->tile_start);
    ++h->launches;
    k_tiles<<<(A + 127) / 128, 128, 0, st>>>(out->angle_start, out->tile_start, d_angle_of_rank, A,
                                             out->tile_ev, out->bin, out->tiles);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    // one synchronisation: validation status and the work sizes
    out->h_angle_start.resize(A + 1);
    out->h_tile_start.resize(A + 1);
    out->h_rank_angle = angle_of_rank;
    int status = 0;
    LMMEW_CUDA(cudaMemcpyAsync(&out->h_angle_start[0], out->angle_start, sizeof(int) * (A + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&out->h_tile_start[0], out->tile_start, sizeof(int) * (A + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (status != 0) LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    if (status & kStatusTimeout)
        return set_error(LMMEW_ERR_TIMEOUT, "a kernel of an earlier call timed out in a pipeline wait");
    if (status & kStatusOutOfRange)
        return set_error(LMMEW_ERR_OUT_OF_RANGE,
                         "an event has an angle or bin outside the model or an energy outside "
                         "every window");
    out->n_valid = out->h_angle_start[A];
    return LMMEW_OK;
}

// ---------------------------------------------------------------------------
// Variant for callers that cannot allocate: every buffer comes from a
// caller-provided region, no host container is built, and the host reads
// back only three integers.  Angles keep their natural order (one subset).
namespace {
__global__ void k_identity(int* a, int* b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { a[i] = i; b[i] = i; }
}
}  // namespace

size_t sort_fixed_bytes(int64_t n, int A) { return sort_scratch_bytes(n, A); }

int sort_events_fixed(lm_handle* h, const lm_events* ev, char*& arena, SortedFixed* out,
                      cudaStream_t st) {
    const ModelConst& m = h->mc;
    const int64_t n = ev->n;
    const int A = m.A, B = m.B;
    uint32_t* keys0 = bump<uint32_t>(arena, n);
    uint32_t* keys1 = bump<uint32_t>(arena, n);
    uint32_t* vals0 = bump<uint32_t>(arena, n);
    uint32_t* vals1 = bump<uint32_t>(arena, n);
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    uint32_t* hist = bump<uint32_t>(arena, 256 * (nblk > 0 ? nblk : 1));
    out->perm = bump<uint32_t>(arena, n);
    out->bin = bump<uint16_t>(arena, n);
    out->energy = bump<float>(arena, n);
    int* angle_start = bump<int>(arena, A + 1);
    int* tile_start = bump<int>(arena, A + 1);
    int* d_angle_of_rank = bump<int>(arena, A);
    int* d_rank_of_angle = bump<int>(arena, A);
    out->tiles = bump<Tile>(arena, n / kETMin + A + 1);
    out->tile_ev = h->tile_ev;

    k_identity<<<(A + 255) / 256, 256, 0, st>>>(d_rank_of_angle, d_angle_of_rank, A);
    float w[8][2] = {};
    for (int k = 0; k < m.n_win; ++k) { w[k][0] = (float)m.win_lo[k]; w[k][1] = (float)m.win_hi[k]; }
    k_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        ev->angle, ev->bin, ev->energy_keV, n, A, B, d_rank_of_angle, m.n_win,
        make_float4(w[0][0], w[0][1], w[1][0], w[1][1]), make_float4(w[2][0], w[2][1], w[3][0], w[3][1]),
        make_float4(w[4][0], w[4][1], w[5][0], w[5][1]), make_float4(w[6][0], w[6][1], w[7][0], w[7][1]),
        keys0, vals0, h->d_status);
    LMMEW_CUDA(cudaGetLastError());
    const uint64_t kmax = (uint64_t)A * (uint64_t)B;
    int bits = 1;
    while (bits < 32 && (kmax >> bits) != 0) ++bits;
    uint32_t *kin = keys0, *kout = keys1, *vin = vals0, *vout = vals1;
    for (int shift = 0; shift < bits; shift += 8) {
        k_hist<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, n, shift, hist, (int)nblk);
        k_scan<<<1, 1024, 0, st>>>(hist, 256 * nblk);
        k_scatter<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, vin, n, shift, hist, (int)nblk, kout,
                                                          vout);
        LMMEW_CUDA(cudaGetLastError());
        uint32_t* t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
    }
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kin, vin, ev->energy_keV, n, B, out->perm,
                                                         out->bin, out->energy);
    k_bounds<<<(A + 1 + 127) / 128, 128, 0, st>>>(kin, n, A, B, angle_start);
    k_tile_scan<<<1, 1024, 0, st>>>(angle_start, A, out->tile_ev, tile_start);
    k_tiles<<<(A + 127) / 128, 128, 0, st>>>(angle_start, tile_start, d_angle_of_rank, A,
                                             out->tile_ev, out->bin, out->tiles);
    LMMEW_CUDA(cudaGetLastError());
    h->launches += 6 + 3 * ((bits + 7) / 8);
    int host3[3] = {0, 0, 0};   // tiles, valid events, status
    LMMEW_CUDA(cudaMemcpyAsync(&host3[0], tile_start + A, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&host3[1], angle_start + A, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&host3[2], h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (host3[2] != 0) {
        LMMEW_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), st));
        LMMEW_CUDA(cudaStreamSynchronize(st));
    }
    if (host3[2] & kStatusTimeout)
        return set_error(LMMEW_ERR_TIMEOUT, "a kernel of an earlier call timed out in a pipeline wait");
    if (host3[2] & kStatusOutOfRange)
        return set_error(LMMEW_ERR_OUT_OF_RANGE,
                         "an event has an angle or bin outside the model or an energy outside "
                         "every window");
    out->n_tiles = host3[0];
    out->n_valid = host3[1];
    return LMMEW_OK;
}

// ---------------------------------------------------------------------------
// Batched sort: R realisations' events concatenated and keyed by (subset,
// angle within the subset, bin) alone.  The radix sort is stable, so within
// one (angle, bin) the events keep realisation order and, inside a
// realisation, their input order: each realisation's events appear in the
// order lm_osem would sort them on their own.  An angle's run, and so every
// tile, holds the events of all realisations together, each with its
// realisation beside it: a sub-iteration's tiles are full whatever the
// realisations' event counts, and their bin ranges narrow as the
// realisations add up.
namespace {
__global__ void k_keys_batch(const uint16_t* angle, const uint16_t* bin, const float* energy,
                             int64_t n, int A, int B, int n_subsets, int A_s, int n_win,
                             float4 win01, float4 win23, float4 win45, float4 win67,
                             uint32_t* keys, uint32_t* vals, int* status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int a = angle[j], b = bin[j];
    const float e = energy[j];
    const float wl[8] = {win01.x, win01.z, win23.x, win23.z, win45.x, win45.z, win67.x, win67.z};
    const float wh[8] = {win01.y, win01.w, win23.y, win23.w, win45.y, win45.w, win67.y, win67.w};
    bool inwin = false;
    for (int k = 0; k < n_win; ++k) inwin |= (e >= wl[k] && e < wh[k]);
    const bool ok = a < A && b < B && isfinite(e) && inwin;
    const uint32_t V = (uint32_t)n_subsets * A_s;
    const uint32_t v = (uint32_t)(a % n_subsets) * A_s + a / n_subsets;
    keys[j] = ok ? v * (uint32_t)B + (uint32_t)b : V * (uint32_t)B;
    vals[j] = (uint32_t)j;
    if (!ok) atomicOr(status, kStatusOutOfRange);
}

// Realisation of every sorted event: off[r] <= perm[i] < off[r + 1].
__global__ void k_real_of(const uint32_t* perm, int64_t n, const int64_t* off, int R,
                          uint16_t* real) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
    int lo = 0, hi = R;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid;
    }
    real[i] = (uint16_t)lo;
}

// Back-projection key of sorted event i: (row block, realisation).
__global__ void k_bp_keys(const uint16_t* real, int64_t n, const int64_t* blk_start, int n_blk,
                          int R, uint32_t* keys, uint32_t* vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_blk;                   // block: blk_start[k] <= i < blk_start[k + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (blk_start[mid] <= i) lo = mid; else hi = mid;
    }
    keys[i] = (uint32_t)lo * (uint32_t)R + real[i];
    vals[i] = (uint32_t)i;
}

int key_bits(uint64_t kmax) {
    int bits = 1;
    while (bits < 32 && (kmax >> bits) != 0) ++bits;
    return bits;
}

// Stable LSD radix sort of (keys, vals) over the ping-pong buffers; the
// sorted pair ends in (kin, vin).
int radix_sort_pairs(lm_handle* h, int64_t n, int bits, uint32_t*& kin, uint32_t*& kout,
                     uint32_t*& vin, uint32_t*& vout, uint32_t* hist, cudaStream_t st) {
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    for (int shift = 0; shift < bits; shift += 8) {
        k_hist<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, n, shift, hist, (int)nblk);
        k_scan<<<1, 1024, 0, st>>>(hist, 256 * nblk);
        k_scatter<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, vin, n, shift, hist, (int)nblk, kout,
                                                          vout);
        LMMEW_CUDA(cudaGetLastError());
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    h->launches += 3 * ((bits + 7) / 8);
    return LMMEW_OK;
}
}  // namespace

size_t sort_batch_scratch_bytes(int64_t n, int64_t V, int R) {
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += bump_bytes(bytes); };
    add(4 * n); add(4 * n); add(4 * n); add(4 * n);    // keys/vals ping-pong (reused by bp_order)
    add(4 * 256 * (nblk > 0 ? nblk : 1));
    add(4 * n); add(2 * n); add(4 * n); add(2 * n);     // perm, bins, energies, realisations
    add(2 * n); add(2 * n); add(4 * n);                 // concatenated events
    add(4 * (V + 1)); add(4 * (V + 1)); add(4 * V);
    add(8 * (R + 1));
    add(sizeof(Tile) * (size_t)(n / kETMin + V + 1));
    return b;
}

int sort_events_batch(lm_handle* h, const lm_events* evs, int R, int n_subsets,
                      SortedEvents* out, char*& arena, cudaStream_t st) {
    const ModelConst& m = h->mc;
    const int A = m.A, B = m.B;
    const int A_s = (A + n_subsets - 1) / n_subsets;
    const int64_t V = (int64_t)n_subsets * A_s;
    std::vector<int64_t> off(R + 1, 0);
    for (int r = 0; r < R; ++r) off[r + 1] = off[r] + evs[r].n;
    const int64_t n = off[R];
    std::vector<int> angle_of_v(V);
    for (int64_t v = 0; v < V; ++v) {
        const int ai = (int)(v % A_s), s = (int)(v / A_s);
        const int a = ai * n_subsets + s;
        angle_of_v[v] = a < A ? a : 0;
    }
    out->tmp_keys0 = bump<uint32_t>(arena, n);
    out->tmp_keys1 = bump<uint32_t>(arena, n);
    out->tmp_vals0 = bump<uint32_t>(arena, n);
    out->tmp_vals1 = bump<uint32_t>(arena, n);
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    out->tmp_hist = bump<uint32_t>(arena, 256 * std::max<int64_t>(nblk, 1));
    out->perm = bump<uint32_t>(arena, n);
    out->bin = bump<uint16_t>(arena, n);
    out->energy = bump<float>(arena, n);
    out->real = bump<uint16_t>(arena, n);
    uint16_t* c_angle = bump<uint16_t>(arena, n);
    uint16_t* c_bin = bump<uint16_t>(arena, n);
    float* c_energy = bump<float>(arena, n);
    out->angle_start = bump<int>(arena, V + 1);
    out->tile_start = bump<int>(arena, V + 1);
    int* d_angle_of_v = bump<int>(arena, V);
    int64_t* d_off = bump<int64_t>(arena, R + 1);
    out->tiles = bump<Tile>(arena, n / kETMin + V + 1);
    out->tile_ev = h->tile_ev;
    out->n_groups = (int)V;
    out->angle_of_group = d_angle_of_v;

    for (int r = 0; r < R; ++r) {
        if (evs[r].n == 0) continue;
        LMMEW_CUDA(cudaMemcpyAsync(c_angle + off[r], evs[r].angle, 2 * evs[r].n,
                                   cudaMemcpyDeviceToDevice, st));
        LMMEW_CUDA(cudaMemcpyAsync(c_bin + off[r], evs[r].bin, 2 * evs[r].n,
                                   cudaMemcpyDeviceToDevice, st));
        LMMEW_CUDA(cudaMemcpyAsync(c_energy + off[r], evs[r].energy_keV, 4 * evs[r].n,
                                   cudaMemcpyDeviceToDevice, st));
    }
    LMMEW_CUDA(cudaMemcpyAsync(d_off, off.data(), 8 * (R + 1), cudaMemcpyHostToDevice, st));
    LMMEW_CUDA(cudaMemcpyAsync(d_angle_of_v, angle_of_v.data(), 4 * V, cudaMemcpyHostToDevice, st));
    if (n > 0) {
        float w[8][2] = {};
        for (int k = 0; k < m.n_win; ++k) { w[k][0] = (float)m.win_lo[k]; w[k][1] = (float)m.win_hi[k]; }
        uint32_t *kin = out->tmp_keys0, *kout = out->tmp_keys1;
        uint32_t *vin = out->tmp_vals0, *vout = out->tmp_vals1;
        k_keys_batch<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            c_angle, c_bin, c_energy, n, A, B, n_subsets, A_s, m.n_win,
            make_float4(w[0][0], w[0][1], w[1][0], w[1][1]), make_float4(w[2][0], w[2][1], w[3][0], w[3][1]),
            make_float4(w[4][0], w[4][1], w[5][0], w[5][1]), make_float4(w[6][0], w[6][1], w[7][0], w[7][1]),
            kin, vin, h->d_status);
        LMMEW_CUDA(cudaGetLastError());
        int rc = radix_sort_pairs(h, n, key_bits((uint64_t)V * (uint64_t)B), kin, kout, vin, vout,
                                  out->tmp_hist, st);
        if (rc != LMMEW_OK) return rc;
        k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kin, vin, c_energy, n, B, out->perm,
                                                             out->bin, out->energy);
        k_real_of<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out->perm, n, d_off, R, out->real);
        k_bounds<<<(unsigned)((V + 1 + 127) / 128), 128, 0, st>>>(kin, n, (int)V, B, out->angle_start);
        h->launches += 4;
        LMMEW_CUDA(cudaGetLastError());
    } else {
        LMMEW_CUDA(cudaMemsetAsync(out->angle_start, 0, sizeof(int) * (V + 1), st));
    }
    k_tile_scan<<<1, 1024, 0, st>>>(out->angle_start, (int)V, out->tile_ev, out->tile_start);
    k_tiles<<<(unsigned)((V + 127) / 128), 128, 0, st>>>(out->angle_start, out->tile_start,
                                                         d_angle_of_v, (int)V, out->tile_ev,
                                                         out->bin, out->tiles);
    h->launches += 2;
    LMMEW_CUDA(cudaGetLastError());
    out->h_angle_start.resize(V + 1);
    out->h_tile_start.resize(V + 1);
    int status = 0;
    LMMEW_CUDA(cudaMemcpyAsync(out->h_angle_start.data(), out->angle_start, 4 * (V + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(out->h_tile_start.data(), out->tile_start, 4 * (V + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (status != 0) LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    if (status & kStatusTimeout)
        return set_error(LMMEW_ERR_TIMEOUT, "a kernel of an earlier call timed out in a pipeline wait");
    if (status & kStatusOutOfRange)
        return set_error(LMMEW_ERR_OUT_OF_RANGE,
                         "an event has an angle or bin outside the model or an energy outside "
                         "every window");
    out->n_valid = out->h_angle_start[V];
    out->n_total = n;
    return LMMEW_OK;
}

// The back-projection order of a batch: sorted positions stably re-sorted by
// (row block, realisation), so that every realisation's events inside a row
// block form one run, in sorted order.  Reuses the batch sort's ping-pong
// buffers; blk_start [n_blk + 1] and grp_start [n_blk * R + 1] are device
// arrays the caller provides, grp_start also copied to the host.
int bp_order_batch(lm_handle* h, SortedEvents* se, int R, const int64_t* blk_start, int n_blk,
                   int* grp_start, std::vector<int>& h_grp_start, cudaStream_t st) {
    const int64_t n = se->n_total;
    const int64_t G = (int64_t)n_blk * R;
    h_grp_start.assign(G + 1, 0);
    if (n == 0) {
        se->bp_idx = se->tmp_vals0;
        return LMMEW_OK;
    }
    uint32_t *kin = se->tmp_keys0, *kout = se->tmp_keys1;
    uint32_t *vin = se->tmp_vals0, *vout = se->tmp_vals1;
    k_bp_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(se->real, n, blk_start, n_blk, R, kin,
                                                           vin);
    LMMEW_CUDA(cudaGetLastError());
    ++h->launches;
    int rc = radix_sort_pairs(h, n, key_bits((uint64_t)G), kin, kout, vin, vout, se->tmp_hist, st);
    if (rc != LMMEW_OK) return rc;
    k_bounds<<<(unsigned)((G + 1 + 127) / 128), 128, 0, st>>>(kin, n, (int)G, 1, grp_start);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    se->bp_idx = vin;
    LMMEW_CUDA(cudaMemcpyAsync(h_grp_start.data(), grp_start, 4 * (G + 1), cudaMemcpyDeviceToHost,
                               st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    return LMMEW_OK;
}

// Re-cut the sorted groups into tiles of tile_ev events: the tile array was
// sized for the smallest tile, so every size fits.
int recut_tiles(lm_handle* h, SortedEvents* se, int tile_ev, cudaStream_t st) {
    if (tile_ev != 32 && tile_ev != 64 && tile_ev != kET)
        return set_error(LMMEW_ERR_INVALID_ARG, "tile size must be 32, 64 or 128 events");
    if (se->tile_ev == tile_ev) return LMMEW_OK;
    const int G = se->n_groups;
    k_tile_scan<<<1, 1024, 0, st>>>(se->angle_start, G, tile_ev, se->tile_start);
    k_tiles<<<(unsigned)((G + 127) / 128), 128, 0, st>>>(se->angle_start, se->tile_start,
                                                         se->angle_of_group, G, tile_ev, se->bin,
                                                         se->tiles);
    h->launches += 2;
    LMMEW_CUDA(cudaGetLastError());
    se->h_tile_start.resize(G + 1);
    LMMEW_CUDA(cudaMemcpyAsync(se->h_tile_start.data(), se->tile_start, 4 * (size_t)(G + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    se->tile_ev = tile_ev;
    return LMMEW_OK;
}

}  // namespace lmmew
