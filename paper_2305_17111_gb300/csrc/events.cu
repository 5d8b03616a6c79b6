// Event validation and grouping (once per call that takes events): every
// event is checked against the model, keyed by (subset rank of its angle,
// energy class of its recorded energy, bin) and stably sorted with an LSD
// radix sort written here (8-bit digits, per-block histograms, one global
// scan, stable per-block scatter by warp match).  The sorted order groups each
// angle's events contiguously, subsets in ascending order (subset(a) = a mod
// n_subsets, paper Sec. LM-OSEM), inside an angle by energy class, and cuts
// every (angle, class) run into tiles of up to tile_ev events for the row
// kernel.  The class of a tile tells the row kernel which lines' single
// scatter can reach its recorded energies.
#include <math.h>

#include <algorithm>
#include <vector>

#include "lmmew_internal.cuh"

namespace lmmew {

// Reach of each line's single scatter in recorded energy, and the classes
// its ends cut the energy axis into (see EnergyClasses).  E' runs from the
// backscatter energy to E_w; E' -+ k sigma_E(E') is scanned in FP64 on a fine
// grid, widened by the largest change between neighbouring samples (the
// extremum between two samples lies within that of the nearer one), and
// rounded outward to FP32, the precision the recorded energies are compared
// in.  Classes are off (one class, every line) without scatter points, with
// more than 4 lines, when pruning is switched off, or when (angle rank,
// class, bin) keys would not fit 32 bits.
void build_energy_classes(lm_handle* h) {
    const ModelConst& m = h->mc;
    const int all = (1 << m.W) - 1;
    h->ecls.n_bnd = 0;
    h->n_classes = 1;
    for (int c = 0; c < 2 * LMMEW_MAX_LINES + 1; ++c) h->class_lines[c] = all;
    // the row kernels instantiate a stage per staged-line count up to 4 lines
    if (!h->prune_lines || m.np == 0 || m.W > 4) return;
    const double f2s = 1.0 / (2.0 * sqrt(2.0 * log(2.0)));
    auto sigma = [&](double e) { return m.fwhm_frac * e * pow(e / m.e_ref, m.expo) * f2s; };
    float lo[LMMEW_MAX_LINES], hi[LMMEW_MAX_LINES];
    std::vector<float> bnd;
    for (int w = 0; w < m.W; ++w) {
        const double ew = m.line_e[w];
        const double eb = ew / (1.0 + 2.0 * ew / 510.99895);
        constexpr int kSteps = 4096;
        double mn = 1e300, mx = -1e300, dl = 0.0, du = 0.0, pl = 0.0, pu = 0.0;
        for (int k = 0; k <= kSteps; ++k) {
            const double e = eb + (ew - eb) * k / kSteps;
            const double s = kScatterReachSigmas * sigma(e);
            const double l = e - s, u = e + s;
            if (k > 0) {
                dl = std::max(dl, fabs(l - pl));
                du = std::max(du, fabs(u - pu));
            }
            pl = l;
            pu = u;
            mn = std::min(mn, l);
            mx = std::max(mx, u);
        }
        lo[w] = nextafterf((float)(mn - dl), -INFINITY);
        hi[w] = nextafterf((float)(mx + du), INFINITY);
        bnd.push_back(lo[w]);
        bnd.push_back(hi[w]);
    }
    std::sort(bnd.begin(), bnd.end());
    bnd.erase(std::unique(bnd.begin(), bnd.end()), bnd.end());
    const int C = (int)bnd.size() + 1;
    // keys of the batched sort reach (2 A classes + 1) bins
    if ((2ull * (uint64_t)m.A * C + 1ull) * (uint64_t)m.B >= (1ull << 32)) return;
    h->ecls.n_bnd = (int)bnd.size();
    for (int k = 0; k < h->ecls.n_bnd; ++k) h->ecls.bnd[k] = bnd[k];
    h->n_classes = C;
    for (int c = 0; c < C; ++c) {
        // class c: bnd[c - 1] <= E_hat < bnd[c]; line w covers it or misses it
        int mask = 0;
        for (int w = 0; w < m.W; ++w) {
            const bool left_in = c > 0 && lo[w] <= bnd[c - 1];
            const bool right_in = c < C - 1 && bnd[c] <= hi[w];
            if (left_in && right_in) mask |= 1 << w;
        }
        h->class_lines[c] = mask;
    }
}

int sort_groups(const lm_handle* h, int A) { return A * h->n_classes; }

namespace {

__device__ __forceinline__ uint32_t energy_class(const EnergyClasses& ec, float e) {
    uint32_t c = 0;
    for (int k = 0; k < ec.n_bnd; ++k) c += ec.bnd[k] <= e ? 1u : 0u;
    return c;
}

constexpr int kSortThreads = 256;
constexpr int kSortPerThread = 16;
constexpr int kSortChunk = kSortThreads * kSortPerThread;   // keys per block

__global__ void k_keys(const uint16_t* angle, const uint16_t* bin, const float* energy, int64_t n,
                       int A, int B, const int* rank_of_angle, int n_win,
                       float4 win01, float4 win23, float4 win45, float4 win67,
                       const EnergyClasses ec, uint32_t* keys, uint32_t* vals, int* status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int a = angle[j], b = bin[j];
    const float e = energy[j];
    const float lo[8] = {win01.x, win01.z, win23.x, win23.z, win45.x, win45.z, win67.x, win67.z};
    const float hi[8] = {win01.y, win01.w, win23.y, win23.w, win45.y, win45.w, win67.y, win67.w};
    bool inwin = false;
    for (int k = 0; k < n_win; ++k) inwin |= (e >= lo[k] && e < hi[k]);
    const bool ok = a < A && b < B && isfinite(e) && inwin;
    const uint32_t C = (uint32_t)ec.n_bnd + 1u;
    keys[j] = ok ? ((uint32_t)rank_of_angle[a] * C + energy_class(ec, e)) * (uint32_t)B + (uint32_t)b
                 : (uint32_t)A * C * (uint32_t)B;
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
                        int tile_ev, const uint16_t* bin_s, const int* lines_of_group,
                        const int2* crange, int B, int np, Tile* tiles,
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
        const int b_lo = bin_s[e], b_hi = bin_s[e + cnt - 1];
        T.b_lo_hi = (b_lo << 16) | b_hi;
        T.r = real_of_rank ? real_of_rank[r] : 0;
        T.lines = lines_of_group[r];
        // the union of the tile's bins' collimator runs of scatter points
        int p_lo = np, p_hi = 0;
        for (int b = b_lo; b <= b_hi; ++b) {
            const int2 cr = crange[(size_t)T.a * B + b];
            if (cr.y > cr.x) {
                p_lo = min(p_lo, cr.x);
                p_hi = max(p_hi, cr.y);
            }
        }
        T.p_lo = p_lo;
        T.p_hi = p_hi;
        tiles[t] = T;
    }
}


}  // namespace

size_t sort_scratch_bytes(int64_t n, int G) {
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += bump_bytes(bytes); };
    add(4 * n); add(4 * n); add(4 * n); add(4 * n);    // keys/vals ping-pong
    add(4 * 256 * std::max<int64_t>(nblk, 1));         // histograms
    add(4 * n); add(2 * n); add(4 * n);                 // perm, bins, energies
    add(4 * (G + 1)); add(4 * (G + 1));                 // group_start, tile_start
    add(4 * G); add(4 * G); add(4 * G);                 // angle/lines of each group, rank of each angle
    add(sizeof(Tile) * (size_t)(n / kETMin + G + 1));   // tiles (smallest tile size)
    return b;
}

namespace {

int key_bits(uint64_t kmax) {
    int bits = 1;
    while (bits < 32 && (kmax >> bits) != 0) ++bits;
    return bits;
}

struct Windows {
    float4 w01, w23, w45, w67;
};
Windows windows_of(const ModelConst& m) {
    float w[8][2] = {};
    for (int k = 0; k < m.n_win; ++k) {
        w[k][0] = (float)m.win_lo[k];
        w[k][1] = (float)m.win_hi[k];
    }
    return Windows{make_float4(w[0][0], w[0][1], w[1][0], w[1][1]),
                   make_float4(w[2][0], w[2][1], w[3][0], w[3][1]),
                   make_float4(w[4][0], w[4][1], w[5][0], w[5][1]),
                   make_float4(w[6][0], w[6][1], w[7][0], w[7][1])};
}

// The sort shared by sort_events and sort_events_async: keys, radix passes,
// gather, group bounds and tiles of the G = A * n_classes groups, all on
// the caller's stream.  rank_of_angle [A], angle_of_group and lines_of_group
// [G] are device arrays already filled.
int sort_and_tile(lm_handle* h, const lm_events* ev, int G, const int* rank_of_angle,
                  const int* angle_of_group, const int* lines_of_group, uint32_t* keys0,
                  uint32_t* keys1, uint32_t* vals0, uint32_t* vals1, uint32_t* hist,
                  uint32_t* perm, uint16_t* bin_s, float* e_s, int* group_start, int* tile_start,
                  int tile_ev, Tile* tiles, cudaStream_t st) {
    const ModelConst& m = h->mc;
    const int64_t n = ev->n;
    const int B = m.B;
    if (n > 0) {
        const Windows wn = windows_of(m);
        k_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            ev->angle, ev->bin, ev->energy_keV, n, m.A, B, rank_of_angle, m.n_win, wn.w01, wn.w23,
            wn.w45, wn.w67, h->ecls, keys0, vals0, h->d_status);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
        const int bits = key_bits((uint64_t)G * (uint64_t)B);
        const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
        uint32_t *kin = keys0, *kout = keys1, *vin = vals0, *vout = vals1;
        for (int shift = 0; shift < bits; shift += 8) {
            k_hist<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, n, shift, hist, (int)nblk);
            k_scan<<<1, 1024, 0, st>>>(hist, 256 * nblk);
            k_scatter<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, vin, n, shift, hist, (int)nblk,
                                                              kout, vout);
            h->launches += 3;
            LMMEW_CUDA(cudaGetLastError());
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kin, vin, ev->energy_keV, n, B, perm,
                                                             bin_s, e_s);
        k_bounds<<<(G + 1 + 127) / 128, 128, 0, st>>>(kin, n, G, B, group_start);
        h->launches += 2;
        LMMEW_CUDA(cudaGetLastError());
    } else {
        LMMEW_CUDA(cudaMemsetAsync(group_start, 0, sizeof(int) * (G + 1), st));
    }
    k_tile_scan<<<1, 1024, 0, st>>>(group_start, G, tile_ev, tile_start);
    k_tiles<<<(G + 127) / 128, 128, 0, st>>>(group_start, tile_start, angle_of_group, G, tile_ev,
                                             bin_s, lines_of_group, h->d_crange, m.B, m.np,
                                             tiles);
    h->launches += 2;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

int status_error(int status) {
    if (status & kStatusTimeout)
        return set_error(LMMEW_ERR_TIMEOUT, "a kernel of an earlier call timed out in a pipeline wait");
    if (status & kStatusTables)
        return set_error(LMMEW_ERR_CUDA,
                         "a row launch needed path tables that were not resident (internal error)");
    if (status & kStatusOutOfRange)
        return set_error(LMMEW_ERR_OUT_OF_RANGE,
                         "an event has an angle or bin outside the model or an energy outside "
                         "every window");
    return LMMEW_OK;
}

}  // namespace

int sort_events(lm_handle* h, const lm_events* ev, int n_subsets, SortedEvents* out, char*& arena,
                cudaStream_t st) {
    const ModelConst& m = h->mc;
    const int64_t n = ev->n;
    const int A = m.A, C = h->n_classes, G = sort_groups(h, A);
    // angle order: subsets ascending, angles ascending inside a subset; a
    // rank's groups are its energy classes in ascending order
    std::vector<int> rank_of_angle(A), angle_of_group(G), lines_of_group(G);
    {
        int r = 0;
        for (int s = 0; s < n_subsets; ++s)
            for (int a = s; a < A; a += n_subsets) {
                rank_of_angle[a] = r;
                for (int c = 0; c < C; ++c) {
                    angle_of_group[r * C + c] = a;
                    lines_of_group[r * C + c] = h->class_lines[c];
                }
                ++r;
            }
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
    out->group_start = bump<int>(arena, G + 1);
    out->tile_start = bump<int>(arena, G + 1);
    int* d_angle_of_group = bump<int>(arena, G);
    int* d_lines_of_group = bump<int>(arena, G);
    int* d_rank_of_angle = bump<int>(arena, G);
    out->tiles = bump<Tile>(arena, n / kETMin + G + 1);
    out->tile_ev = h->tile_ev;
    out->n_groups = G;
    out->n_classes = C;
    out->angle_of_group = d_angle_of_group;
    out->lines_of_group = d_lines_of_group;

    LMMEW_CUDA(cudaMemcpyAsync(d_rank_of_angle, rank_of_angle.data(), sizeof(int) * A,
                               cudaMemcpyHostToDevice, st));
    LMMEW_CUDA(cudaMemcpyAsync(d_angle_of_group, angle_of_group.data(), sizeof(int) * G,
                               cudaMemcpyHostToDevice, st));
    LMMEW_CUDA(cudaMemcpyAsync(d_lines_of_group, lines_of_group.data(), sizeof(int) * G,
                               cudaMemcpyHostToDevice, st));
    int rc = sort_and_tile(h, ev, G, d_rank_of_angle, d_angle_of_group, d_lines_of_group, keys0,
                           keys1, vals0, vals1, hist, out->perm, out->bin, out->energy,
                           out->group_start, out->tile_start, out->tile_ev, out->tiles, st);
    if (rc != LMMEW_OK) return rc;
    // one synchronisation: validation status and the work sizes
    out->h_group_start.resize(G + 1);
    out->h_tile_start.resize(G + 1);
    int status = 0;
    LMMEW_CUDA(cudaMemcpyAsync(&out->h_group_start[0], out->group_start, sizeof(int) * (G + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&out->h_tile_start[0], out->tile_start, sizeof(int) * (G + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (status != 0) LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    rc = status_error(status);
    if (rc != LMMEW_OK) return rc;
    out->n_valid = out->h_group_start[G];
    out->n_total = n;
    return LMMEW_OK;
}

// ---------------------------------------------------------------------------
// The sort without host read-back (lm_forward, lm_backproject, lm_osem).

// Rank of each angle, angle and line mask of each group, for a partition into
// n_subsets: built on the host and copied once per partition and class set
// (set-up, like the subset sensitivities), then reused by every call.
int group_arrays(lm_handle* h, int n_subsets, GroupArrays* out) {
    const int A = h->mc.A, C = h->n_classes, G = A * C;
    if (h->grp_classes != C) {
        for (auto& kv : h->grp_cache) cudaFree(kv.second);
        h->grp_cache.clear();
        h->grp_classes = C;
    }
    auto it = h->grp_cache.find(n_subsets);
    if (it == h->grp_cache.end()) {
        std::vector<int> buf((size_t)A + 2 * (size_t)G);
        int* rank_of_angle = buf.data();
        int* angle_of_group = rank_of_angle + A;
        int* lines_of_group = angle_of_group + G;
        int r = 0;
        for (int s = 0; s < n_subsets; ++s)
            for (int a = s; a < A; a += n_subsets) {
                rank_of_angle[a] = r;
                for (int c = 0; c < C; ++c) {
                    angle_of_group[r * C + c] = a;
                    lines_of_group[r * C + c] = h->class_lines[c];
                }
                ++r;
            }
        int* d = nullptr;
        if (cudaMalloc(&d, sizeof(int) * buf.size()) != cudaSuccess) {
            cudaGetLastError();
            return set_error(LMMEW_ERR_OOM, "cannot allocate the sort's group arrays");
        }
        const cudaError_t e = cudaMemcpy(d, buf.data(), sizeof(int) * buf.size(),
                                         cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_error(e, "cudaMemcpy(group arrays)");
        }
        it = h->grp_cache.emplace(n_subsets, d).first;
    }
    out->rank_of_angle = it->second;
    out->angle_of_group = it->second + A;
    out->lines_of_group = it->second + A + G;
    return LMMEW_OK;
}

int sort_events_async(lm_handle* h, const lm_events* ev, const GroupArrays& ga, int G,
                      SortedEvents* out, char*& arena, cudaStream_t st) {
    const int64_t n = ev->n;
    uint32_t* keys0 = bump<uint32_t>(arena, n);
    uint32_t* keys1 = bump<uint32_t>(arena, n);
    uint32_t* vals0 = bump<uint32_t>(arena, n);
    uint32_t* vals1 = bump<uint32_t>(arena, n);
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    uint32_t* hist = bump<uint32_t>(arena, 256 * std::max<int64_t>(nblk, 1));
    out->perm = bump<uint32_t>(arena, n);
    out->bin = bump<uint16_t>(arena, n);
    out->energy = bump<float>(arena, n);
    out->group_start = bump<int>(arena, G + 1);
    out->tile_start = bump<int>(arena, G + 1);
    out->tiles = bump<Tile>(arena, n / kETMin + G + 1);
    out->tile_ev = h->tile_ev;
    out->n_groups = G;
    out->n_classes = h->n_classes;
    out->angle_of_group = ga.angle_of_group;
    out->lines_of_group = ga.lines_of_group;
    out->n_total = n;
    return sort_and_tile(h, ev, G, ga.rank_of_angle, ga.angle_of_group, ga.lines_of_group, keys0,
                         keys1, vals0, vals1, hist, out->perm, out->bin, out->energy,
                         out->group_start, out->tile_start, out->tile_ev, out->tiles, st);
}

int read_back_counts(lm_handle* h, SortedEvents* se, cudaStream_t st) {
    const int G = se->n_groups;
    se->h_group_start.resize(G + 1);
    se->h_tile_start.resize(G + 1);
    int status = 0;
    LMMEW_CUDA(cudaMemcpyAsync(se->h_group_start.data(), se->group_start, sizeof(int) * (G + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(se->h_tile_start.data(), se->tile_start, sizeof(int) * (G + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (status != 0) LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    const int rc = status_error(status);
    if (rc != LMMEW_OK) return rc;
    se->n_valid = se->h_group_start[G];
    return LMMEW_OK;
}

int take_status(lm_handle* h, cudaStream_t st) {
    int status = 0;
    LMMEW_CUDA(cudaStreamSynchronize(st));
    LMMEW_CUDA(cudaMemcpy(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    return status_error(status);
}

int recut_tiles_async(lm_handle* h, SortedEvents* se, int tile_ev, cudaStream_t st) {
    if (tile_ev != 32 && tile_ev != 64 && tile_ev != kET)
        return set_error(LMMEW_ERR_INVALID_ARG, "tile size must be 32, 64 or 128 events");
    if (se->tile_ev == tile_ev) return LMMEW_OK;
    const int G = se->n_groups;
    k_tile_scan<<<1, 1024, 0, st>>>(se->group_start, G, tile_ev, se->tile_start);
    k_tiles<<<(unsigned)((G + 127) / 128), 128, 0, st>>>(se->group_start, se->tile_start,
                                                         se->angle_of_group, G, tile_ev, se->bin,
                                                         se->lines_of_group, h->d_crange, h->mc.B,
                                                         h->mc.np, se->tiles);
    h->launches += 2;
    LMMEW_CUDA(cudaGetLastError());
    se->tile_ev = tile_ev;
    return LMMEW_OK;
}

namespace {
// One thread per (set, block): set s holds the ranks of subset s (ascending
// rank order: subset s has ceil((A - s) / n_subsets) of them), i.e. groups
// [r0 C, r1 C) and tiles [T0, T1) = [tile_start[r0 C], tile_start[r1 C]).
__global__ void k_plan(const int* group_start, const int* tile_start, const Tile* tiles, int A,
                       int C, int n_subsets, int blocks_per_set, int tpc, ChunkRange* ranges) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_subsets * blocks_per_set) return;
    const int s = i / blocks_per_set, k = i % blocks_per_set;
    int r0 = 0;
    for (int u = 0; u < s; ++u) r0 += (A - u + n_subsets - 1) / n_subsets;
    const int r1 = r0 + (A - s + n_subsets - 1) / n_subsets;
    const int T0 = tile_start[r0 * C], T1 = tile_start[r1 * C];
    const int t0 = min(T0 + k * tpc, T1), t1 = min(t0 + tpc, T1);
    ChunkRange R;
    R.x = t0;
    R.y = t1;
    if (t0 < t1) {
        R.z = tiles[t0].begin;
        R.w = tiles[t1 - 1].begin + tiles[t1 - 1].count;
    } else {
        R.z = R.w = group_start[r1 * C];
    }
    ranges[i] = R;
}
}  // namespace

int launch_plan(lm_handle* h, const SortedEvents& se, int n_subsets, int blocks_per_set,
                int tiles_per_block, ChunkRange* ranges, cudaStream_t st) {
    const int total = n_subsets * blocks_per_set;
    k_plan<<<(total + 127) / 128, 128, 0, st>>>(se.group_start, se.tile_start, se.tiles, h->mc.A,
                                                se.n_classes, n_subsets, blocks_per_set,
                                                tiles_per_block, ranges);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

namespace {
__global__ void k_clip_range(const ChunkRange* in, const int* tile_start, int g0, int g1,
                             ChunkRange* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ChunkRange R = *in;
    const int x = max(R.x, tile_start[g0]);
    R.y = max(x, min(R.y, tile_start[g1]));
    R.x = x;
    *out = R;
}
}  // namespace

int launch_clip_range(lm_handle* h, const ChunkRange* in, const SortedEvents& se, int g0, int g1,
                      ChunkRange* out, cudaStream_t st) {
    k_clip_range<<<1, 32, 0, st>>>(in, se.tile_start, g0, g1, out);
    ++h->launches;
    LMMEW_CUDA(cudaGetLastError());
    return LMMEW_OK;
}

// Group arrays of one subset built on the device into a caller's region.
namespace {
struct ClassLines {
    int v[2 * LMMEW_MAX_LINES + 1];
};
__global__ void k_identity_groups(int* rank_of_angle, int* angle_of_group, int* lines_of_group,
                                  int A, int C, const ClassLines cl) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < A) rank_of_angle[g] = g;
    if (g < A * C) {
        angle_of_group[g] = g / C;
        lines_of_group[g] = cl.v[g % C];
    }
}
}  // namespace

GroupArrays group_arrays_into(lm_handle* h, char*& arena, cudaStream_t st) {
    const int A = h->mc.A, C = h->n_classes, G = A * C;
    int* rank_of_angle = bump<int>(arena, A);
    int* angle_of_group = bump<int>(arena, G);
    int* lines_of_group = bump<int>(arena, G);
    ClassLines cl;
    for (int c = 0; c < 2 * LMMEW_MAX_LINES + 1; ++c) cl.v[c] = h->class_lines[c];
    k_identity_groups<<<(G + 255) / 256, 256, 0, st>>>(rank_of_angle, angle_of_group,
                                                       lines_of_group, A, C, cl);
    ++h->launches;
    return GroupArrays{rank_of_angle, angle_of_group, lines_of_group};
}

// ---------------------------------------------------------------------------
// Batched sort: R realisations' events concatenated and keyed by (subset,
// angle within the subset, energy class, bin) alone.  The radix sort is
// stable, so within one (angle, class, bin) the events keep realisation order
// and, inside a realisation, their input order: each realisation's events
// appear in the order lm_osem would sort them on their own.  An angle's run, and so every
// tile, holds the events of all realisations together, each with its
// realisation beside it: a sub-iteration's tiles are full whatever the
// realisations' event counts, and their bin ranges narrow as the
// realisations add up.
namespace {
__global__ void k_keys_batch(const uint16_t* angle, const uint16_t* bin, const float* energy,
                             int64_t n, int A, int B, int n_subsets, int A_s, int n_win,
                             float4 win01, float4 win23, float4 win45, float4 win67,
                             const EnergyClasses ec, uint32_t* keys, uint32_t* vals,
                             int* status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int a = angle[j], b = bin[j];
    const float e = energy[j];
    const float wl[8] = {win01.x, win01.z, win23.x, win23.z, win45.x, win45.z, win67.x, win67.z};
    const float wh[8] = {win01.y, win01.w, win23.y, win23.w, win45.y, win45.w, win67.y, win67.w};
    bool inwin = false;
    for (int k = 0; k < n_win; ++k) inwin |= (e >= wl[k] && e < wh[k]);
    const bool ok = a < A && b < B && isfinite(e) && inwin;
    const uint32_t C = (uint32_t)ec.n_bnd + 1u;
    const uint32_t G = (uint32_t)n_subsets * A_s * C;
    const uint32_t v = (uint32_t)(a % n_subsets) * A_s + a / n_subsets;
    keys[j] = ok ? (v * C + energy_class(ec, e)) * (uint32_t)B + (uint32_t)b : G * (uint32_t)B;
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

size_t sort_batch_scratch_bytes(int64_t n, int64_t G, int R) {
    const int64_t nblk = (n + kSortChunk - 1) / kSortChunk;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += bump_bytes(bytes); };
    add(4 * n); add(4 * n); add(4 * n); add(4 * n);    // keys/vals ping-pong (reused by bp_order)
    add(4 * 256 * (nblk > 0 ? nblk : 1));
    add(4 * n); add(2 * n); add(4 * n); add(2 * n);     // perm, bins, energies, realisations
    add(2 * n); add(2 * n); add(4 * n);                 // concatenated events
    add(4 * (G + 1)); add(4 * (G + 1)); add(4 * G); add(4 * G);
    add(8 * (R + 1));
    add(sizeof(Tile) * (size_t)(n / kETMin + G + 1));
    return b;
}

// Groups of the batched sort: (subset, angle within the subset, class), with
// A_s = ceil(A / n_subsets) angle slots per subset (empty past the last angle).
int sort_events_batch(lm_handle* h, const lm_events* evs, int R, int n_subsets,
                      SortedEvents* out, char*& arena, cudaStream_t st) {
    const ModelConst& m = h->mc;
    const int A = m.A, B = m.B, C = h->n_classes;
    const int A_s = (A + n_subsets - 1) / n_subsets;
    const int64_t V = (int64_t)n_subsets * A_s;
    const int64_t G = V * C;
    std::vector<int64_t> off(R + 1, 0);
    for (int r = 0; r < R; ++r) off[r + 1] = off[r] + evs[r].n;
    const int64_t n = off[R];
    std::vector<int> angle_of_group(G), lines_of_group(G);
    for (int64_t v = 0; v < V; ++v) {
        const int ai = (int)(v % A_s), s = (int)(v / A_s);
        const int a = ai * n_subsets + s;
        for (int c = 0; c < C; ++c) {
            angle_of_group[v * C + c] = a < A ? a : 0;
            lines_of_group[v * C + c] = h->class_lines[c];
        }
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
    out->group_start = bump<int>(arena, G + 1);
    out->tile_start = bump<int>(arena, G + 1);
    int* d_angle_of_group = bump<int>(arena, G);
    int* d_lines_of_group = bump<int>(arena, G);
    int64_t* d_off = bump<int64_t>(arena, R + 1);
    out->tiles = bump<Tile>(arena, n / kETMin + G + 1);
    out->tile_ev = h->tile_ev;
    out->n_groups = (int)G;
    out->n_classes = C;
    out->angle_of_group = d_angle_of_group;
    out->lines_of_group = d_lines_of_group;

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
    LMMEW_CUDA(cudaMemcpyAsync(d_angle_of_group, angle_of_group.data(), 4 * G,
                               cudaMemcpyHostToDevice, st));
    LMMEW_CUDA(cudaMemcpyAsync(d_lines_of_group, lines_of_group.data(), 4 * G,
                               cudaMemcpyHostToDevice, st));
    if (n > 0) {
        const Windows wn = windows_of(m);
        uint32_t *kin = out->tmp_keys0, *kout = out->tmp_keys1;
        uint32_t *vin = out->tmp_vals0, *vout = out->tmp_vals1;
        k_keys_batch<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            c_angle, c_bin, c_energy, n, A, B, n_subsets, A_s, m.n_win, wn.w01, wn.w23, wn.w45,
            wn.w67, h->ecls, kin, vin, h->d_status);
        ++h->launches;
        LMMEW_CUDA(cudaGetLastError());
        int rc = radix_sort_pairs(h, n, key_bits((uint64_t)G * (uint64_t)B), kin, kout, vin, vout,
                                  out->tmp_hist, st);
        if (rc != LMMEW_OK) return rc;
        k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kin, vin, c_energy, n, B, out->perm,
                                                             out->bin, out->energy);
        k_real_of<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out->perm, n, d_off, R, out->real);
        k_bounds<<<(unsigned)((G + 1 + 127) / 128), 128, 0, st>>>(kin, n, (int)G, B,
                                                                 out->group_start);
        h->launches += 3;
        LMMEW_CUDA(cudaGetLastError());
    } else {
        LMMEW_CUDA(cudaMemsetAsync(out->group_start, 0, sizeof(int) * (G + 1), st));
    }
    k_tile_scan<<<1, 1024, 0, st>>>(out->group_start, (int)G, out->tile_ev, out->tile_start);
    k_tiles<<<(unsigned)((G + 127) / 128), 128, 0, st>>>(out->group_start, out->tile_start,
                                                         d_angle_of_group, (int)G, out->tile_ev,
                                                         out->bin, d_lines_of_group, h->d_crange,
                                                         h->mc.B, h->mc.np, out->tiles);
    h->launches += 2;
    LMMEW_CUDA(cudaGetLastError());
    out->h_group_start.resize(G + 1);
    out->h_tile_start.resize(G + 1);
    int status = 0;
    LMMEW_CUDA(cudaMemcpyAsync(out->h_group_start.data(), out->group_start, 4 * (G + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(out->h_tile_start.data(), out->tile_start, 4 * (G + 1),
                               cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (status != 0) LMMEW_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    const int rc = status_error(status);
    if (rc != LMMEW_OK) return rc;
    out->n_valid = out->h_group_start[G];
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
    k_tile_scan<<<1, 1024, 0, st>>>(se->group_start, G, tile_ev, se->tile_start);
    k_tiles<<<(unsigned)((G + 127) / 128), 128, 0, st>>>(se->group_start, se->tile_start,
                                                         se->angle_of_group, G, tile_ev, se->bin,
                                                         se->lines_of_group, h->d_crange, h->mc.B,
                                                         h->mc.np, se->tiles);
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
