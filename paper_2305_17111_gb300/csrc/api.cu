// C ABI entry points (include/lmmew.h): argument checks, scratch management,
// work planning and the sequence of kernels of each call.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "lmmew_internal.cuh"

namespace lmmew {

namespace {
thread_local std::string g_err;
constexpr size_t kRowBudgetFloats = size_t(1) << 30;   // 4 GiB of row block per chunk
}  // namespace

int set_error(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_error(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LMMEW_ERR_OOM : LMMEW_ERR_CUDA;
}

namespace {

int ensure(lm_handle* h, Scratch& s, size_t bytes, cudaStream_t st) {
    if (s.bytes >= bytes) return LMMEW_OK;
    LMMEW_CUDA(cudaStreamSynchronize(st));
    if (s.ptr) {
        cudaFree(s.ptr);
        s.ptr = nullptr;
        s.bytes = 0;
    }
    const size_t want = bytes + bytes / 8;
    if (cudaMalloc(&s.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LMMEW_ERR_OOM, "cannot allocate " + std::to_string(want >> 20) +
                                            " MiB of scratch");
    }
    s.bytes = want;
    (void)h;
    return LMMEW_OK;
}

// Row-kernel autotuner.  It times, with CUDA events on the caller's stream,
// candidate launch shapes on a sample of the workload: whole angles of the
// first subset, taken until they hold kTuneEvents events.  After one
// warm-up launch it tries every events-per-tile size (32, 64 or 128 where
// the FP32 form has the small-tile kernels) x work-unit order at the
// occupancy limit of CTAs per SM, then the best of those with one CTA per SM
// fewer.  The sample runs without forward sums or stored rows.  The choice
// is kept per handle for each workload class: log2 of the call's mean
// events per angle, the scatter model, the precision and whether energy
// classes are on, so a call of a class tuned before needs no event counts on
// the host.  Every choice gives bit-identical results: a tile's size changes
// only which exact-zero terms it skips.
constexpr int64_t kTuneEvents = 16384;

uint64_t tune_key_for(const lm_handle* h, double mean_events_per_angle) {
    int bucket = 0;
    while (bucket < 40 && (double)(int64_t(2) << bucket) <= mean_events_per_angle) ++bucket;
    return 1ull | ((uint64_t)bucket << 8) | ((uint64_t)h->scatter_model << 4) |
           ((uint64_t)h->prec << 2) | ((uint64_t)(h->n_classes > 1) << 1);
}

// True if the class has a shape: the class in use keeps the current one (it
// may have been set by lm_set_tile_events), a class tuned before gets its
// stored shape back, the surrogate models take 128-event tiles (the network
// kernel dominates and has its own launch shape).
bool tune_known(lm_handle* h, uint64_t key) {
    if (h->tune_key == key) return true;
    const auto hit = h->tune_cache.find(key);
    if (hit != h->tune_cache.end()) {
        h->tile_ev = hit->second.tile_ev;
        h->unit_order = hit->second.unit_order;
        h->grid_per_sm = hit->second.grid_per_sm;
        h->tune_ms = hit->second.ms;
        h->tune_key = key;
        return true;
    }
    if (h->scatter_model == LMMEW_SCATTER_SURROGATE ||
        h->scatter_model == LMMEW_SCATTER_SURROGATE_COARSE) {
        h->tile_ev = kET;
        h->unit_order = 0;
        h->grid_per_sm = 0;
        h->tune_key = key;
        h->tune_ms = 0.f;
        return true;
    }
    return false;
}

// Times the candidates on the sorted events (host counts required) and
// stores the choice for the class; the events leave re-cut into tiles of the
// chosen size.
int autotune_run(lm_handle* h, SortedEvents& se, int first_ranks, uint64_t key, cudaStream_t st) {
    // whole angle ranks (each n_classes groups) of the first subset
    const int C = se.n_classes;
    int g1 = 0;
    int64_t ev = 0;
    for (int r = 0; r < first_ranks && ev < kTuneEvents; ++r) {
        ev += se.h_group_start[(r + 1) * C] - se.h_group_start[r * C];
        g1 = (r + 1) * C;
    }
    if (ev == 0) return recut_tiles(h, &se, h->tile_ev, st);
    const bool small_tiles = h->prec == 0 && h->mc.W <= 4;
    const int sizes[3] = {kET, 64, 32};
    const int n_sizes = small_tiles ? 3 : 1;
    cudaEvent_t ta = nullptr, tb = nullptr;
    LMMEW_CUDA(cudaEventCreate(&ta));
    const cudaError_t ce = cudaEventCreate(&tb);
    if (ce != cudaSuccess) {
        cudaEventDestroy(ta);
        return cuda_error(ce, "cudaEventCreate");
    }
    const int prof = h->prof_on;
    h->prof_on = 0;   // the trial launches are not part of any timed work
    int rc = LMMEW_OK;
    int reps = 1;
    // one trial: the sample in tiles of `size` events, unit order, CTAs per SM;
    // the shortest of `reps` launches (two when a launch is under 2 ms)
    auto trial = [&](int size, int order, int grid, float* ms_out) -> int {
        int r = recut_tiles(h, &se, size, st);
        if (r != LMMEW_OK) return r;
        RowLaunch L{se.tiles, se.h_tile_start[0], se.h_tile_start[g1], se.bin, se.energy,
                    nullptr, nullptr, 0, 0, nullptr, 0, ev};
        L.tile_ev = se.tile_ev;
        h->unit_order = order;
        h->grid_per_sm = grid;
        float tmin = 3.0e38f;
        for (int rep = 0; rep < reps; ++rep) {
            cudaError_t e = cudaEventRecord(ta, st);
            if (e == cudaSuccess) {
                r = launch_row(h, L, st);
                if (r != LMMEW_OK) return r;
                e = cudaEventRecord(tb, st);
            }
            if (e == cudaSuccess) e = cudaEventSynchronize(tb);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ta, tb);
            if (e != cudaSuccess) return cuda_error(e, "timing a trial row launch");
            tmin = std::min(tmin, ms);
        }
        *ms_out = tmin;
        return LMMEW_OK;
    };
    const int max_grid = h->row_blocks[h->prec];
    float best = 3.0e38f, warm = 0.f;
    int best_size = kET, best_order = 0, best_grid = max_grid;
    rc = trial(kET, 0, max_grid, &warm);          // warm-up; sets the repeat count
    if (rc == LMMEW_OK && warm < 2.0f) reps = 2;
    // tile size x unit order at the occupancy limit, then the best of those
    // with one CTA per SM fewer
    for (int si = 0; si < n_sizes && rc == LMMEW_OK; ++si) {
        for (int order = 0; order < 2 && rc == LMMEW_OK; ++order) {
            float ms = 0.f;
            rc = trial(sizes[si], order, max_grid, &ms);
            if (rc == LMMEW_OK && ms < best) {
                best = ms;
                best_size = sizes[si];
                best_order = order;
            }
        }
    }
    if (rc == LMMEW_OK && max_grid > 1) {
        float ms = 0.f;
        rc = trial(best_size, best_order, max_grid - 1, &ms);
        if (rc == LMMEW_OK && ms < best) {
            best = ms;
            best_grid = max_grid - 1;
        }
    }
    cudaEventDestroy(ta);
    cudaEventDestroy(tb);
    h->prof_on = prof;
    if (rc != LMMEW_OK) return rc;
    h->tile_ev = best_size;
    h->unit_order = best_order;
    h->grid_per_sm = best_grid;
    h->tune_key = key;
    h->tune_ms = best;
    h->tune_cache[key] = lm_handle::TuneChoice{best_size, best_order, best_grid, best};
    return recut_tiles(h, &se, best_size, st);
}

// The tuner for callers whose sort read the counts back (the batch and the
// planned paths): the class from the call's mean events per angle.
int autotune_row(lm_handle* h, SortedEvents& se, int first_ranks, cudaStream_t st) {
    const uint64_t key = tune_key_for(h, (double)se.n_total / h->mc.A);
    if (tune_known(h, key)) return recut_tiles(h, &se, h->tile_ev, st);
    return autotune_run(h, se, first_ranks, key, st);
}

struct Chunk {
    int t0, t1;         // tile range
    int64_t e0, e1;     // sorted event range
};

// Split the tiles of groups [g0, g1) into chunks of at most max_events events.
std::vector<Chunk> plan_chunks(const SortedEvents& se, int g0, int g1, int64_t max_events) {
    std::vector<Chunk> out;
    Chunk cur{-1, -1, 0, 0};
    for (int r = g0; r < g1; ++r) {
        for (int t = se.h_tile_start[r]; t < se.h_tile_start[r + 1]; ++t) {
            const int64_t b = se.h_group_start[r] + (int64_t)(t - se.h_tile_start[r]) * se.tile_ev;
            const int64_t e = std::min<int64_t>(b + se.tile_ev, se.h_group_start[r + 1]);
            if (cur.t0 >= 0 && (e - cur.e0) > max_events) {
                out.push_back(cur);
                cur.t0 = -1;
            }
            if (cur.t0 < 0) cur = Chunk{t, t, b, b};
            cur.t1 = t + 1;
            cur.e1 = e;
        }
    }
    if (cur.t0 >= 0) out.push_back(cur);
    return out;
}

int check_events(const lm_handle* h, const lm_events* ev) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    if (!ev) return set_error(LMMEW_ERR_INVALID_ARG, "events is NULL");
    if (ev->n < 0) return set_error(LMMEW_ERR_INVALID_ARG, "negative event count");
    if (ev->n >= (int64_t(1) << 31))
        return set_error(LMMEW_ERR_INVALID_ARG, "at most 2^31 - 1 events per call");
    if (ev->n > 0 && (!ev->angle || !ev->bin || !ev->energy_keV))
        return set_error(LMMEW_ERR_INVALID_ARG, "event arrays are NULL");
    return LMMEW_OK;
}

int row_stride_of(const lm_handle* h) { return (h->mc.nq + 3) & ~3; }

}  // namespace

int launch_row_profiled(lm_handle* h, const RowLaunch& L, cudaStream_t st) {
    if (!h->prof_on) return launch_row(h, L, st);
    if (h->prof_used + 2 > h->prof_ev.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            LMMEW_CUDA(cudaEventCreate(&e));
            h->prof_ev.push_back(e);
        }
    }
    cudaEvent_t e0 = h->prof_ev[h->prof_used], e1 = h->prof_ev[h->prof_used + 1];
    LMMEW_CUDA(cudaEventRecord(e0, st));
    const int rc = launch_row(h, L, st);
    if (rc != LMMEW_OK) return rc;
    LMMEW_CUDA(cudaEventRecord(e1, st));
    h->prof_used += 2;
    h->prof_launches += 1;
    h->prof_terms_dense += (double)L.n_events * (double)h->terms_per_event;
    h->prof_elems += (double)L.n_events * (double)h->mc.nq;
    return LMMEW_OK;
}

// The row launch L, whose tiles belong to ranks [r_lo, r_hi) of the sort
// (rank r_lo + i holds angle a_first + i a_step).  With the exact scatter
// model and streamed path tables, the ranks go in blocks of as many angles
// as the table buffer holds: each block's tables are built unless they are
// resident, and the launch is clipped on the device to the block's tiles.
int launch_row_ranks(lm_handle* h, const RowLaunch& L, const SortedEvents& se, int r_lo,
                     int r_hi, int a_first, int a_step, cudaStream_t st) {
    if (!h->tab_slots || h->scatter_model != LMMEW_SCATTER_EXACT || h->mc.np == 0)
        return launch_row_profiled(h, L, st);
    if (!L.range)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED, "streamed path tables need a planned row range");
    const int C = se.n_classes;
    for (int r0 = r_lo; r0 < r_hi; r0 += h->tab_slots) {
        const int r1 = std::min(r_hi, r0 + h->tab_slots);
        int rc = stream_tables(h, a_first + (r0 - r_lo) * a_step, a_step, r1 - r0, st);
        if (rc == LMMEW_OK) rc = launch_clip_range(h, L.range, se, r0 * C, r1 * C, h->d_clip, st);
        if (rc != LMMEW_OK) return rc;
        RowLaunch Lc = L;
        Lc.range = h->d_clip;
        if (r0 != r_lo) Lc.n_events = 0;
        rc = launch_row_profiled(h, Lc, st);
        if (rc != LMMEW_OK) return rc;
    }
    return LMMEW_OK;
}

ForwardPlan forward_plan(const lm_handle* h, int64_t n, int64_t cap_max) {
    ForwardPlan p;
    p.G = sort_groups(h, h->mc.A);
    const int te = h->tile_ev;
    p.n = n;
    // at most ceil(n / te) + G tiles: one row block of that many whole tiles
    // when it fits cap_max, else blocks of as many tiles as fit
    const int64_t tiles_max = (n + te - 1) / te + p.G;
    p.tpc = (int)std::max<int64_t>(1, std::min<int64_t>(tiles_max, cap_max / te));
    p.cap = (int64_t)p.tpc * te;
    p.blocks = (int)((tiles_max + p.tpc - 1) / p.tpc);
    return p;
}

size_t forward_region_bytes(const lm_handle* h, const ForwardPlan& p) {
    return sort_scratch_bytes(p.n, p.G) + bump_bytes(sizeof(float) * h->mc.nq) +
           bump_bytes(sizeof(float) * (size_t)h->mc.nqt * p.cap) +
           bump_bytes(sizeof(ChunkRange) * (size_t)p.blocks);
}

int forward_async(lm_handle* h, const lm_events* ev, const float* image, float* out_y,
                  const GroupArrays& ga, const ForwardPlan& p, char* arena, cudaStream_t st) {
    SortedEvents se;
    int rc = sort_events_async(h, ev, ga, p.G, &se, arena, st);
    if (rc != LMMEW_OK) return rc;
    float* lam_v = bump<float>(arena, h->mc.nq);
    float* ypart = bump<float>(arena, (size_t)h->mc.nqt * p.cap);
    ChunkRange* ranges = bump<ChunkRange>(arena, p.blocks);
    rc = launch_gather_image(h, image, lam_v, st);
    if (rc == LMMEW_OK) rc = launch_plan(h, se, 1, p.blocks, p.tpc, ranges, st);
    for (int k = 0; k < p.blocks && rc == LMMEW_OK; ++k) {
        RowLaunch L{se.tiles, 0, p.tpc, se.bin, se.energy, lam_v, nullptr, 0, 0, ypart, p.cap,
                    k == 0 ? p.n : 0};
        L.tile_ev = se.tile_ev;
        L.range = ranges + k;
        rc = launch_row_ranks(h, L, se, 0, h->mc.A, 0, 1, st);   // one subset: rank = angle
        if (rc == LMMEW_OK)
            rc = launch_forward_out_range(h, ypart, p.cap, p.cap, ranges + k, se.perm, out_y, st);
    }
    if (rc == LMMEW_OK) rc = launch_invalid_out(h, se.group_start + p.G, p.n, se.perm, out_y, st);
    return rc;
}

}  // namespace lmmew

using namespace lmmew;

extern "C" {

const char* lm_last_error(void) { return g_err.c_str(); }

int lm_create(const lm_geometry* g, const lm_attenuation* at, const lm_lines* ln,
              const lm_energy_model* em, const uint8_t* support, int n_subsets, lm_handle** out) {
    if (!out) return set_error(LMMEW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !at || !ln || !em) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    if (g->n < 1 || g->n > 4096) return set_error(LMMEW_ERR_INVALID_ARG, "n must be in 1..4096");
    if (!(g->pixel_cm > 0.f) || !isfinite(g->pixel_cm))
        return set_error(LMMEW_ERR_INVALID_ARG, "pixel_cm must be positive");
    if (g->n_angles < 1 || g->n_angles > 65535 || g->n_bins < 1 || g->n_bins > 65535)
        return set_error(LMMEW_ERR_INVALID_ARG, "n_angles and n_bins must be in 1..65535");
    if ((int64_t)g->n_angles * g->n_bins >= (int64_t(1) << 31))
        return set_error(LMMEW_ERR_INVALID_ARG, "n_angles * n_bins too large");
    if (n_subsets < 1 || n_subsets > g->n_angles)
        return set_error(LMMEW_ERR_INVALID_ARG, "n_subsets must be in 1..n_angles");
    if (!at->rho) return set_error(LMMEW_ERR_INVALID_ARG, "rho is NULL");
    if (at->n_knots < 1 || at->n_knots > LMMEW_MAX_KNOTS || !at->knot_keV || !at->mu_water_cm)
        return set_error(LMMEW_ERR_INVALID_ARG, "1..16 attenuation knots required");
    for (int i = 0; i + 1 < at->n_knots; ++i)
        if (!(at->knot_keV[i + 1] > at->knot_keV[i]))
            return set_error(LMMEW_ERR_INVALID_ARG, "knot energies must increase");
    if (at->scatter_n < 0 || (at->scatter_n > 0 && g->n % at->scatter_n != 0))
        return set_error(LMMEW_ERR_INVALID_ARG, "scatter_n must divide n (or be 0)");
    if (ln->n_lines < 1 || ln->n_lines > LMMEW_MAX_LINES || !ln->energy_keV || !ln->yield)
        return set_error(LMMEW_ERR_INVALID_ARG, "1..8 emission lines required");
    for (int w = 0; w < ln->n_lines; ++w)
        if (!(ln->energy_keV[w] > 0.f) || !(ln->yield[w] >= 0.f) || !isfinite(ln->yield[w]))
            return set_error(LMMEW_ERR_INVALID_ARG, "line energies must be > 0, yields >= 0");
    if (em->n_windows < 1 || em->n_windows > LMMEW_MAX_WINDOWS || !em->win_lo_keV || !em->win_hi_keV)
        return set_error(LMMEW_ERR_INVALID_ARG, "1..8 energy windows required");
    for (int k = 0; k < em->n_windows; ++k) {
        if (!(em->win_hi_keV[k] > em->win_lo_keV[k]))
            return set_error(LMMEW_ERR_INVALID_ARG, "each window needs lo < hi");
        for (int k2 = 0; k2 < k; ++k2)
            if (em->win_lo_keV[k] < em->win_hi_keV[k2] && em->win_lo_keV[k2] < em->win_hi_keV[k])
                return set_error(LMMEW_ERR_INVALID_ARG, "energy windows overlap");
    }
    if (!(em->fwhm_frac_ref > 0.f) || !(em->e_ref_keV > 0.f) || !isfinite(em->exponent))
        return set_error(LMMEW_ERR_INVALID_ARG, "energy resolution must be positive");
    const int n = g->n;
    for (int i = 0; i < n * n; ++i)
        if (!(at->rho[i] >= 0.f) || !isfinite(at->rho[i]))
            return set_error(LMMEW_ERR_INVALID_ARG, "rho must be finite and >= 0");

    lm_handle* h = new lm_handle();
    ModelConst& m = h->mc;
    std::memset(&m, 0, sizeof(m));
    m.n = n;
    m.h = g->pixel_cm;
    m.A = g->n_angles;
    m.B = g->n_bins;
    m.bin_w = g->bin_cm > 0.f ? (double)g->bin_cm : (double)n * g->pixel_cm / g->n_bins;
    m.r_det = g->r_det_cm > 0.f ? (double)g->r_det_cm : 0.5 * n * (double)g->pixel_cm;
    m.fwhm0 = g->coll_fwhm0_cm;
    m.slope = g->coll_fwhm_slope;
    m.T = g->scan_time > 0.f ? (double)g->scan_time : 1.0;
    m.S = at->scatter_n;
    m.f = m.S > 0 ? n / m.S : 1;
    m.cell_area = (m.f * m.h) * (m.f * m.h);
    m.W = ln->n_lines;
    for (int w = 0; w < m.W; ++w) {
        m.line_e[w] = ln->energy_keV[w];
        m.alpha[w] = ln->yield[w];
    }
    m.fwhm_frac = em->fwhm_frac_ref;
    m.e_ref = em->e_ref_keV;
    m.expo = em->exponent;
    m.n_win = em->n_windows;
    for (int k = 0; k < m.n_win; ++k) {
        m.win_lo[k] = em->win_lo_keV[k];
        m.win_hi[k] = em->win_hi_keV[k];
    }
    m.n_knots = at->n_knots;
    for (int i = 0; i < m.n_knots; ++i) {
        m.knot_e[i] = at->knot_keV[i];
        m.knot_mu[i] = at->mu_water_cm[i];
    }
    for (int i = 0; i < LMMEW_MAX_KNOTS; ++i)
        m.knot_slope[i] = i + 1 < m.n_knots
                              ? (m.knot_mu[i + 1] - m.knot_mu[i]) / (m.knot_e[i + 1] - m.knot_e[i])
                              : 0.0;
    h->n_subsets_default = n_subsets;
    int rc = build_tables(h, at->rho, support);
    if (rc == LMMEW_OK) build_energy_classes(h);
    if (rc == LMMEW_OK &&
        (cudaMalloc(&h->d_term_counter, sizeof(unsigned long long)) != cudaSuccess ||
         cudaMemset(h->d_term_counter, 0, sizeof(unsigned long long)) != cudaSuccess ||
         cudaMalloc(&h->d_work, sizeof(int)) != cudaSuccess))
        rc = set_error(LMMEW_ERR_OOM, "cannot allocate the term and work counters");
    if (rc == LMMEW_OK) rc = row_kernel_occupancy(h);
    if (rc != LMMEW_OK) {
        std::string keep = g_err;
        lm_destroy(h);
        g_err = keep;
        return rc;
    }
    // exponentials per event row: W per voxel (primary) + W per (voxel, scatter
    // point) path that exists (the emission voxel's own cell has none)
    {
        std::vector<int> q_pix(m.nq);
        cudaMemcpy(q_pix.data(), h->d_q_pix, sizeof(int) * m.nq, cudaMemcpyDeviceToHost);
        int64_t own = 0;
        if (m.S > 0) {
            std::vector<uint8_t> cell_has(m.S * m.S, 0);
            // a cell is a scatter point iff its mean density is positive
            for (int c = 0; c < m.S * m.S; ++c) {
                double sum = 0.0;
                const int mx = c % m.S, my = c / m.S;
                for (int iy = my * m.f; iy < (my + 1) * m.f; ++iy)
                    for (int ix = mx * m.f; ix < (mx + 1) * m.f; ++ix) sum += at->rho[iy * n + ix];
                cell_has[c] = sum > 0.0;
            }
            for (int pix : q_pix) own += cell_has[((pix / n) / m.f) * m.S + (pix % n) / m.f];
        }
        h->terms_per_event = (int64_t)m.W * ((int64_t)m.nq * (m.np + 1) - own);
    }
    *out = h;
    return LMMEW_OK;
}

int lm_destroy(lm_handle* h) {
    if (!h) return LMMEW_OK;
    cudaFree(h->d_q_pix);
    cudaFree(h->d_tab);
    cudaFree(h->d_cs);
    cudaFree(h->d_crange);
    cudaFree(h->d_g8);
    cudaFree(h->d_node_q);
    cudaFree(h->d_interp_node);
    cudaFree(h->d_interp_w);
    cudaFree(h->scratch_nodes.ptr);
    cudaFree(h->d_rho);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->d_tabh);
    cudaFree(h->d_tscale);
    cudaFree(h->d_cs_a);
    cudaFree(h->d_p_cell);
    cudaFree(h->d_p_rho);
    cudaFree(h->d_gqp);
    cudaFree(h->d_dqp);
    cudaFree(h->d_gp);
    cudaFree(h->d_on_det);
    cudaFree(h->d_inv);
    cudaFree(h->d_mu_line);
    cudaFree(h->d_clip);
    cudaFree(h->d_term_counter);
    cudaFree(h->d_work);
    cudaFree(h->d_cv);
    cudaFree(h->d_prim);
    cudaFree(h->d_sens_a);
    cudaFree(h->d_sens_a_prim);
    cudaFree(h->d_status);
    cudaFree(h->d_sens_sub);
    for (auto& kv : h->grp_cache) cudaFree(kv.second);
    cudaFree(h->scratch_sort.ptr);
    cudaFree(h->scratch_work.ptr);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    delete h;
    return LMMEW_OK;
}

int lm_model_info(const lm_handle* h, int64_t* out8) {
    if (!h || !out8) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    out8[0] = h->mc.nq;
    out8[1] = h->mc.np;
    out8[2] = h->mc.W;
    out8[3] = h->mc.A;
    out8[4] = h->mc.B;
    out8[5] = h->terms_per_event;
    out8[6] = (int64_t)h->tab_bytes;
    out8[7] = (int64_t)(h->setup_ms * 1000.0f);
    return LMMEW_OK;
}

int lm_sensitivity(lm_handle* h, int subset, double* out, lm_stream stream) {
    if (!h || !out) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    const int parts = h->n_subsets_default;
    if (subset < -1 || subset >= parts) return set_error(LMMEW_ERR_INVALID_ARG, "subset out of range");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = subset_sensitivity(h, parts, st);
    if (rc != LMMEW_OK) return rc;
    const double* src = h->d_sens_sub + (size_t)(subset < 0 ? parts : subset) * h->mc.nq;
    return launch_scatter_image_d(h, src, out, st);
}

// The planned forms of lm_forward / lm_backproject / lm_osem: the sort's
// counts are read back and the row blocks planned on the host.  The
// surrogate scatter models use them (their network kernel takes host tile
// ranges).
static int forward_planned(lm_handle* h, const lm_events* ev, const float* image, float* out_y,
                           lm_stream stream) {
    int rc = check_events(h, ev);
    if (rc != LMMEW_OK) return rc;
    if (ev->n > 0 && (!image || !out_y)) return set_error(LMMEW_ERR_INVALID_ARG, "NULL image/output");
    if (ev->n == 0) return LMMEW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const ModelConst& m = h->mc;
    rc = ensure(h, h->scratch_sort, sort_scratch_bytes(ev->n, sort_groups(h, m.A)), st);
    if (rc != LMMEW_OK) return rc;
    char* arena = (char*)h->scratch_sort.ptr;
    SortedEvents se;
    rc = sort_events(h, ev, 1, &se, arena, st);
    if (rc != LMMEW_OK) return rc;
    // the surrogate adds its scatter part to stored rows; the other models
    // need only the partial forward sums
    const bool keep_rows = h->scatter_model == LMMEW_SCATTER_SURROGATE ||
                           h->scatter_model == LMMEW_SCATTER_SURROGATE_COARSE;
    const int rs = row_stride_of(h);
    const int64_t max_ev =
        std::max<int64_t>(kET, (int64_t)(kRowBudgetFloats / (keep_rows ? rs : m.nqt)));
    std::vector<Chunk> chunks = plan_chunks(se, 0, se.n_groups, max_ev);
    int64_t biggest = 0;
    for (const Chunk& c : chunks) biggest = std::max(biggest, c.e1 - c.e0);
    rc = surrogate_prepare(h, biggest, st);
    if (rc != LMMEW_OK) return rc;
    rc = ensure(h, h->scratch_work,
                bump_bytes(sizeof(float) * m.nq) + bump_bytes(sizeof(float) * m.nqt * biggest) +
                    (keep_rows ? bump_bytes(sizeof(float) * rs * biggest) : 0),
                st);
    if (rc != LMMEW_OK) return rc;
    char* w = (char*)h->scratch_work.ptr;
    float* lam_v = bump<float>(w, m.nq);
    float* ypart = bump<float>(w, (size_t)m.nqt * std::max<int64_t>(biggest, 1));
    float* rows = keep_rows ? bump<float>(w, (size_t)rs * std::max<int64_t>(biggest, 1)) : nullptr;
    rc = launch_gather_image(h, image, lam_v, st);
    if (rc != LMMEW_OK) return rc;
    for (const Chunk& c : chunks) {
        RowLaunch L{se.tiles, c.t0, c.t1, se.bin, se.energy, lam_v, rows, c.e0, keep_rows ? rs : 0,
                    ypart, c.e1 - c.e0, c.e1 - c.e0};
        L.tile_ev = se.tile_ev;
        rc = launch_row_profiled(h, L, st);
        if (rc != LMMEW_OK) return rc;
        rc = launch_forward_out(h, ypart, c.e1 - c.e0, c.e0, c.e1 - c.e0, se.perm, out_y, st);
        if (rc != LMMEW_OK) return rc;
    }
    return LMMEW_OK;
}

static int backproject_planned(lm_handle* h, const lm_events* ev, const float* weight,
                               float* out_image, lm_stream stream) {
    int rc = check_events(h, ev);
    if (rc != LMMEW_OK) return rc;
    if (!out_image || (ev->n > 0 && !weight))
        return set_error(LMMEW_ERR_INVALID_ARG, "NULL weight/output");
    cudaStream_t st = (cudaStream_t)stream;
    const ModelConst& m = h->mc;
    if (ev->n == 0) {
        LMMEW_CUDA(cudaMemsetAsync(out_image, 0, sizeof(float) * m.n * m.n, st));
        return LMMEW_OK;
    }
    rc = ensure(h, h->scratch_sort, sort_scratch_bytes(ev->n, sort_groups(h, m.A)), st);
    if (rc != LMMEW_OK) return rc;
    char* arena = (char*)h->scratch_sort.ptr;
    SortedEvents se;
    rc = sort_events(h, ev, 1, &se, arena, st);
    if (rc != LMMEW_OK) return rc;
    const int rs = row_stride_of(h);
    const int64_t max_ev = std::max<int64_t>(kET, (int64_t)(kRowBudgetFloats / rs));
    std::vector<Chunk> chunks = plan_chunks(se, 0, se.n_groups, max_ev);
    int64_t biggest = 0, parts = 0;
    for (const Chunk& c : chunks) {
        biggest = std::max(biggest, c.e1 - c.e0);
        parts += bp_parts(c.e1 - c.e0);
    }
    rc = surrogate_prepare(h, biggest, st);
    if (rc != LMMEW_OK) return rc;
    rc = ensure(h, h->scratch_work,
                bump_bytes(sizeof(float) * rs * biggest) + bump_bytes(sizeof(float) * parts * m.nq) +
                    bump_bytes(sizeof(double) * m.nq),
                st);
    if (rc != LMMEW_OK) return rc;
    char* w = (char*)h->scratch_work.ptr;
    float* rows = bump<float>(w, (size_t)rs * biggest);
    float* bpart = bump<float>(w, (size_t)std::max<int64_t>(parts, 1) * m.nq);
    double* num = bump<double>(w, m.nq);
    int64_t row0 = 0;
    for (const Chunk& c : chunks) {
        RowLaunch L{se.tiles, c.t0, c.t1, se.bin, se.energy, nullptr, rows, c.e0, rs, nullptr, 0,
                    c.e1 - c.e0};
        L.tile_ev = se.tile_ev;
        rc = launch_row_profiled(h, L, st);
        if (rc != LMMEW_OK) return rc;
        rc = launch_bp_partial(h, rows, rs, nullptr, 0, c.e1 - c.e0, se.perm + c.e0, weight, bpart,
                               row0, nullptr, st);
        if (rc != LMMEW_OK) return rc;
        row0 += bp_parts(c.e1 - c.e0);
    }
    rc = launch_voxel_reduce(h, bpart, parts, num, st);
    if (rc != LMMEW_OK) return rc;
    return launch_num_to_image(h, num, out_image, st);
}

static int osem_planned(lm_handle* h, const lm_events* ev, int n_subsets, int n_iters,
                        int start_iter, int start_subset, float* image, double* loglik,
                        lm_stream stream) {
    int rc = check_events(h, ev);
    if (rc != LMMEW_OK) return rc;
    const ModelConst& m = h->mc;
    if (!image) return set_error(LMMEW_ERR_INVALID_ARG, "image is NULL");
    if (n_subsets < 1 || n_subsets > m.A)
        return set_error(LMMEW_ERR_INVALID_ARG, "n_subsets must be in 1..n_angles");
    if (n_iters < 0 || start_iter < 0 || start_iter > n_iters || start_subset < 0 ||
        start_subset >= n_subsets)
        return set_error(LMMEW_ERR_INVALID_ARG, "iteration range out of bounds");
    cudaStream_t st = (cudaStream_t)stream;
    rc = subset_sensitivity(h, n_subsets, st);
    if (rc != LMMEW_OK) return rc;
    rc = ensure(h, h->scratch_sort, sort_scratch_bytes(ev->n, sort_groups(h, m.A)), st);
    if (rc != LMMEW_OK) return rc;
    char* arena = (char*)h->scratch_sort.ptr;
    SortedEvents se;
    rc = sort_events(h, ev, n_subsets, &se, arena, st);
    if (rc != LMMEW_OK) return rc;
    rc = autotune_row(h, se, (m.A + n_subsets - 1) / n_subsets, st);
    if (rc != LMMEW_OK) return rc;

    // angle ranks of each subset and the chunks of its events
    const int rs = row_stride_of(h);
    const int64_t max_ev = std::max<int64_t>(kET, (int64_t)(kRowBudgetFloats / rs));
    std::vector<std::vector<Chunk>> plan(n_subsets);
    int64_t biggest = 0, parts_max = 0;
    {
        int r = 0;
        for (int s = 0; s < n_subsets; ++s) {
            const int cnt = (m.A - s + n_subsets - 1) / n_subsets;
            plan[s] = plan_chunks(se, r * se.n_classes, (r + cnt) * se.n_classes, max_ev);
            int64_t parts = 0;
            for (const Chunk& c : plan[s]) {
                biggest = std::max(biggest, c.e1 - c.e0);
                parts += bp_parts(c.e1 - c.e0);
            }
            parts_max = std::max(parts_max, parts);
            r += cnt;
        }
    }
    const size_t need = bump_bytes(sizeof(float) * m.nq) + bump_bytes(sizeof(float) * rs * biggest) +
                        bump_bytes(sizeof(float) * m.nqt * biggest) +
                        bump_bytes(sizeof(float) * std::max<int64_t>(parts_max, 1) * m.nq) +
                        bump_bytes(sizeof(double) * std::max<int64_t>(parts_max, 1)) +
                        bump_bytes(sizeof(double) * m.nq);
    rc = surrogate_prepare(h, biggest, st);
    if (rc != LMMEW_OK) return rc;
    rc = ensure(h, h->scratch_work, need, st);
    if (rc != LMMEW_OK) return rc;
    char* w = (char*)h->scratch_work.ptr;
    float* lam_v = bump<float>(w, m.nq);
    float* rows = bump<float>(w, (size_t)rs * std::max<int64_t>(biggest, 1));
    float* ypart = bump<float>(w, (size_t)m.nqt * std::max<int64_t>(biggest, 1));
    float* bpart = bump<float>(w, (size_t)std::max<int64_t>(parts_max, 1) * m.nq);
    double* llpart = bump<double>(w, std::max<int64_t>(parts_max, 1));
    double* num = bump<double>(w, m.nq);

    rc = launch_gather_image(h, image, lam_v, st);
    if (rc != LMMEW_OK) return rc;
    for (int it = start_iter; it < n_iters; ++it) {
        for (int s = (it == start_iter ? start_subset : 0); s < n_subsets; ++s) {
            int64_t row0 = 0;
            for (const Chunk& c : plan[s]) {
                const int64_t cnt = c.e1 - c.e0;
                RowLaunch L{se.tiles, c.t0, c.t1, se.bin, se.energy, lam_v, rows, c.e0, rs, ypart,
                            cnt, cnt};
                L.tile_ev = se.tile_ev;
                rc = launch_row_profiled(h, L, st);
                if (rc != LMMEW_OK) return rc;
                rc = launch_bp_partial(h, rows, rs, ypart, cnt, cnt, nullptr, nullptr, bpart, row0,
                                       loglik ? llpart : nullptr, st);
                if (rc != LMMEW_OK) return rc;
                row0 += bp_parts(cnt);
            }
            if (row0 > 0) {
                rc = launch_voxel_reduce(h, bpart, row0, num, st);
            } else {
                LMMEW_CUDA(cudaMemsetAsync(num, 0, sizeof(double) * m.nq, st));
            }
            if (rc != LMMEW_OK) return rc;
            rc = launch_update(h, lam_v, num, h->d_sens_sub + (size_t)s * m.nq, llpart, row0,
                               loglik ? loglik + (size_t)it * n_subsets + s : nullptr, st);
            if (rc != LMMEW_OK) return rc;
        }
    }
    return launch_scatter_image(h, lam_v, image, st);
}

static bool surrogate_model(const lm_handle* h) {
    return h->scatter_model == LMMEW_SCATTER_SURROGATE ||
           h->scatter_model == LMMEW_SCATTER_SURROGATE_COARSE;
}

int lm_forward(lm_handle* h, const lm_events* ev, const float* image, float* out_y,
               lm_stream stream) {
    int rc = check_events(h, ev);
    if (rc != LMMEW_OK) return rc;
    if (ev->n > 0 && (!image || !out_y)) return set_error(LMMEW_ERR_INVALID_ARG, "NULL image/output");
    if (ev->n == 0) return LMMEW_OK;
    if (surrogate_model(h)) return forward_planned(h, ev, image, out_y, stream);
    cudaStream_t st = (cudaStream_t)stream;
    GroupArrays ga;
    rc = group_arrays(h, 1, &ga);
    if (rc != LMMEW_OK) return rc;
    const ForwardPlan fp = forward_plan(h, ev->n, (int64_t)(kRowBudgetFloats / h->mc.nqt));
    rc = ensure(h, h->scratch_sort, forward_region_bytes(h, fp), st);
    if (rc != LMMEW_OK) return rc;
    return forward_async(h, ev, image, out_y, ga, fp, (char*)h->scratch_sort.ptr, st);
}

int lm_backproject(lm_handle* h, const lm_events* ev, const float* weight, float* out_image,
                   lm_stream stream) {
    int rc = check_events(h, ev);
    if (rc != LMMEW_OK) return rc;
    if (!out_image || (ev->n > 0 && !weight))
        return set_error(LMMEW_ERR_INVALID_ARG, "NULL weight/output");
    cudaStream_t st = (cudaStream_t)stream;
    const ModelConst& m = h->mc;
    if (ev->n == 0) {
        LMMEW_CUDA(cudaMemsetAsync(out_image, 0, sizeof(float) * m.n * m.n, st));
        return LMMEW_OK;
    }
    if (surrogate_model(h)) return backproject_planned(h, ev, weight, out_image, stream);
    GroupArrays ga;
    rc = group_arrays(h, 1, &ga);
    if (rc != LMMEW_OK) return rc;
    const int64_t n = ev->n;
    const int G = sort_groups(h, m.A), rs = row_stride_of(h);
    const ForwardPlan fp = forward_plan(h, n, (int64_t)(kRowBudgetFloats / rs));
    const int64_t ppc = bp_parts(fp.cap);
    rc = ensure(h, h->scratch_sort, sort_scratch_bytes(n, G), st);
    if (rc == LMMEW_OK)
        rc = ensure(h, h->scratch_work,
                    bump_bytes(sizeof(float) * (size_t)rs * fp.cap) +
                        bump_bytes(sizeof(float) * (size_t)fp.blocks * ppc * m.nq) +
                        bump_bytes(sizeof(double) * m.nq) +
                        bump_bytes(sizeof(ChunkRange) * (size_t)fp.blocks),
                    st);
    if (rc != LMMEW_OK) return rc;
    char* arena = (char*)h->scratch_sort.ptr;
    SortedEvents se;
    rc = sort_events_async(h, ev, ga, G, &se, arena, st);
    if (rc != LMMEW_OK) return rc;
    char* w = (char*)h->scratch_work.ptr;
    float* rows = bump<float>(w, (size_t)rs * fp.cap);
    float* bpart = bump<float>(w, (size_t)fp.blocks * ppc * m.nq);
    double* num = bump<double>(w, m.nq);
    ChunkRange* ranges = bump<ChunkRange>(w, fp.blocks);
    rc = launch_plan(h, se, 1, fp.blocks, fp.tpc, ranges, st);
    for (int k = 0; k < fp.blocks && rc == LMMEW_OK; ++k) {
        RowLaunch L{se.tiles, 0, fp.tpc, se.bin, se.energy, nullptr, rows, 0, rs, nullptr, 0,
                    k == 0 ? n : 0};
        L.tile_ev = se.tile_ev;
        L.range = ranges + k;
        rc = launch_row_ranks(h, L, se, 0, m.A, 0, 1, st);   // one subset: rank = angle
        if (rc == LMMEW_OK)
            rc = launch_bp_partial_range(h, rows, rs, nullptr, 0, fp.cap, ranges + k, se.perm,
                                         weight, bpart, (int64_t)k * ppc, nullptr, st);
    }
    if (rc == LMMEW_OK) rc = launch_voxel_reduce_ranges(h, bpart, ranges, fp.blocks, ppc, num, st);
    if (rc != LMMEW_OK) return rc;
    return launch_num_to_image(h, num, out_image, st);
}

int lm_osem(lm_handle* h, const lm_events* ev, int n_subsets, int n_iters, int start_iter,
            int start_subset, float* image, double* loglik, lm_stream stream) {
    int rc = check_events(h, ev);
    if (rc != LMMEW_OK) return rc;
    const ModelConst& m = h->mc;
    if (!image) return set_error(LMMEW_ERR_INVALID_ARG, "image is NULL");
    if (n_subsets < 1 || n_subsets > m.A)
        return set_error(LMMEW_ERR_INVALID_ARG, "n_subsets must be in 1..n_angles");
    if (n_iters < 0 || start_iter < 0 || start_iter > n_iters || start_subset < 0 ||
        start_subset >= n_subsets)
        return set_error(LMMEW_ERR_INVALID_ARG, "iteration range out of bounds");
    if (surrogate_model(h))
        return osem_planned(h, ev, n_subsets, n_iters, start_iter, start_subset, image, loglik,
                            stream);
    cudaStream_t st = (cudaStream_t)stream;
    rc = subset_sensitivity(h, n_subsets, st);
    if (rc != LMMEW_OK) return rc;
    GroupArrays ga;
    rc = group_arrays(h, n_subsets, &ga);
    if (rc != LMMEW_OK) return rc;
    const int64_t n = ev->n;
    const int G = sort_groups(h, m.A);
    rc = ensure(h, h->scratch_sort, sort_scratch_bytes(n, G), st);
    if (rc != LMMEW_OK) return rc;
    char* arena = (char*)h->scratch_sort.ptr;
    SortedEvents se;
    rc = sort_events_async(h, ev, ga, G, &se, arena, st);
    if (rc != LMMEW_OK) return rc;
    // launch shape: a class tuned before needs no counts; a new class is
    // tuned once (set-up: the counts are read back and trial launches timed)
    const int first_ranks = (m.A + n_subsets - 1) / n_subsets;
    const uint64_t key = tune_key_for(h, (double)n / m.A);
    // (the trial launches would read every angle of the first ranks: with
    // streamed tables the handle's tile size is kept as it is)
    const bool streamed = h->tab_slots && h->scatter_model == LMMEW_SCATTER_EXACT && m.np > 0;
    if (!streamed && !tune_known(h, key)) {
        rc = read_back_counts(h, &se, st);
        if (rc == LMMEW_OK) rc = autotune_run(h, se, first_ranks, key, st);
        if (rc != LMMEW_OK) return rc;
    }
    rc = recut_tiles_async(h, &se, h->tile_ev, st);
    if (rc != LMMEW_OK) return rc;

    // row blocks of whole tiles, sized from the event count alone: a subset
    // has at most ceil(n / tile_ev) + (its groups) tiles
    const int te = se.tile_ev, C = se.n_classes, rs = row_stride_of(h);
    const int64_t g_sub = (int64_t)first_ranks * C;
    const int64_t tiles_max = (n + te - 1) / te + g_sub;
    const int tpc = (int)std::max<int64_t>(
        1, std::min<int64_t>(tiles_max, (int64_t)(kRowBudgetFloats / rs) / te));
    const int64_t cap = (int64_t)tpc * te;
    const int blocks = (int)((tiles_max + tpc - 1) / tpc);
    const int64_t ppc = bp_parts(cap);
    rc = ensure(h, h->scratch_work,
                bump_bytes(sizeof(float) * m.nq) + bump_bytes(sizeof(float) * (size_t)rs * cap) +
                    bump_bytes(sizeof(float) * (size_t)m.nqt * cap) +
                    bump_bytes(sizeof(float) * (size_t)blocks * ppc * m.nq) +
                    bump_bytes(sizeof(double) * (size_t)blocks * ppc) +
                    bump_bytes(sizeof(double) * m.nq) +
                    bump_bytes(sizeof(ChunkRange) * (size_t)n_subsets * blocks),
                st);
    if (rc != LMMEW_OK) return rc;
    char* w = (char*)h->scratch_work.ptr;
    float* lam_v = bump<float>(w, m.nq);
    float* rows = bump<float>(w, (size_t)rs * cap);
    float* ypart = bump<float>(w, (size_t)m.nqt * cap);
    float* bpart = bump<float>(w, (size_t)blocks * ppc * m.nq);
    double* llpart = bump<double>(w, (size_t)blocks * ppc);
    double* num = bump<double>(w, m.nq);
    ChunkRange* ranges = bump<ChunkRange>(w, (size_t)n_subsets * blocks);
    rc = launch_gather_image(h, image, lam_v, st);
    if (rc == LMMEW_OK) rc = launch_plan(h, se, n_subsets, blocks, tpc, ranges, st);
    // the first rank of each subset (subsets ascending, angles ascending inside one)
    std::vector<int> r_first(n_subsets + 1, 0);
    for (int s = 0; s < n_subsets; ++s) r_first[s + 1] = r_first[s] + (m.A - s + n_subsets - 1) / n_subsets;
    for (int it = start_iter; it < n_iters && rc == LMMEW_OK; ++it) {
        for (int s = (it == start_iter ? start_subset : 0); s < n_subsets && rc == LMMEW_OK; ++s) {
            const ChunkRange* rg = ranges + (size_t)s * blocks;
            for (int k = 0; k < blocks && rc == LMMEW_OK; ++k) {
                RowLaunch L{se.tiles, 0, tpc, se.bin, se.energy, lam_v, rows, 0, rs, ypart, cap,
                            (s == 0 && k == 0) ? n : 0};
                L.tile_ev = te;
                L.range = rg + k;
                rc = launch_row_ranks(h, L, se, r_first[s], r_first[s + 1], s, n_subsets, st);
                if (rc == LMMEW_OK)
                    rc = launch_bp_partial_range(h, rows, rs, ypart, cap, cap, rg + k, nullptr,
                                                 nullptr, bpart, (int64_t)k * ppc,
                                                 loglik ? llpart : nullptr, st);
            }
            if (rc == LMMEW_OK) rc = launch_voxel_reduce_ranges(h, bpart, rg, blocks, ppc, num, st);
            if (rc == LMMEW_OK)
                rc = launch_update_ranges(h, lam_v, num, h->d_sens_sub + (size_t)s * m.nq, llpart,
                                          rg, blocks, ppc,
                                          loglik ? loglik + (size_t)it * n_subsets + s : nullptr,
                                          st);
        }
    }
    if (rc != LMMEW_OK) return rc;
    return launch_scatter_image(h, lam_v, image, st);
}

int lm_check(lm_handle* h, lm_stream stream) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    return take_status(h, (cudaStream_t)stream);
}

int lm_osem_batch(lm_handle* h, int n_real, const lm_events* events, int n_subsets, int n_iters,
                  float* images, double* loglik, lm_stream stream) {
    if (!h || !events || !images) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    const ModelConst& m = h->mc;
    if (n_real < 1 || n_real > 65535) return set_error(LMMEW_ERR_INVALID_ARG, "1..65535 realisations");
    if (n_subsets < 1 || n_subsets > m.A)
        return set_error(LMMEW_ERR_INVALID_ARG, "n_subsets must be in 1..n_angles");
    if (n_iters < 0) return set_error(LMMEW_ERR_INVALID_ARG, "negative iteration count");
    int64_t n_total = 0;
    for (int r = 0; r < n_real; ++r) {
        int rc = check_events(h, &events[r]);
        if (rc != LMMEW_OK) return rc;
        n_total += events[r].n;
    }
    if (n_total >= (int64_t(1) << 31))
        return set_error(LMMEW_ERR_INVALID_ARG, "at most 2^31 - 1 events per batch");
    if (h->tab_slots && h->scatter_model == LMMEW_SCATTER_EXACT && m.np > 0)
        return set_error(LMMEW_ERR_NOT_IMPLEMENTED,
                         "batched reconstruction needs every angle's path tables resident "
                         "(lm_set_table_streaming(h, 0)) or a surrogate or scatter-free model");
    const int R = n_real;
    const int A_s = (m.A + n_subsets - 1) / n_subsets;
    const int64_t V = (int64_t)n_subsets * A_s;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->graph_exec) {   // the previous batch's graph (its launch finished before this call's sync)
        LMMEW_CUDA(cudaStreamSynchronize(st));
        cudaGraphExecDestroy(h->graph_exec);
        cudaGraphDestroy(h->graph);
        h->graph_exec = nullptr;
        h->graph = nullptr;
    }
    int rc = subset_sensitivity(h, n_subsets, st);
    if (rc != LMMEW_OK) return rc;
    rc = ensure(h, h->scratch_sort, sort_batch_scratch_bytes(n_total, V * h->n_classes, R), st);
    if (rc != LMMEW_OK) return rc;
    char* arena = (char*)h->scratch_sort.ptr;
    SortedEvents se;
    rc = sort_events_batch(h, events, R, n_subsets, &se, arena, st);
    if (rc != LMMEW_OK) return rc;
    rc = autotune_row(h, se, A_s, st);
    if (rc != LMMEW_OK) return rc;

    // plan: per subset, row blocks of whole tiles (all realisations mixed)
    const int rs = row_stride_of(h);
    const int64_t max_ev = std::max<int64_t>(kET, (int64_t)(kRowBudgetFloats / rs));
    struct RowBlock { int t0, t1; int64_t e0, e1; int c0, c1; };
    std::vector<RowBlock> blocks;
    std::vector<int> blk_off(n_subsets + 1, 0);
    for (int s = 0; s < n_subsets; ++s) {
        blk_off[s] = (int)blocks.size();
        RowBlock cur{-1, -1, 0, 0, 0, 0};
        const int64_t C = se.n_classes;
        for (int64_t v = (int64_t)s * A_s * C; v < (int64_t)(s + 1) * A_s * C; ++v) {
            int64_t e = se.h_group_start[v];
            const int64_t e_end = se.h_group_start[v + 1];
            int t = se.h_tile_start[v];
            for (; e < e_end; ++t) {
                const int64_t cnt = std::min<int64_t>(se.tile_ev, e_end - e);
                if (cur.t0 >= 0 && cur.e1 - cur.e0 + cnt > max_ev) {
                    blocks.push_back(cur);
                    cur.t0 = -1;
                }
                if (cur.t0 < 0) cur = RowBlock{t, t, e, e, 0, 0};
                cur.t1 = t + 1;
                cur.e1 = e + cnt;
                e += cnt;
            }
        }
        if (cur.t0 >= 0) blocks.push_back(cur);
    }
    blk_off[n_subsets] = (int)blocks.size();
    const int n_blk = (int)blocks.size();
    const int64_t G = (int64_t)n_blk * R;
    if (G >= (int64_t(1) << 31))
        return set_error(LMMEW_ERR_INVALID_ARG, "realisations x row blocks too large for one batch");
    int64_t biggest = 1;
    for (const RowBlock& b : blocks) biggest = std::max(biggest, b.e1 - b.e0);
    rc = surrogate_prepare(h, biggest, st);   // before the graph capture
    if (rc != LMMEW_OK) return rc;
    // back-projection chunks: up to 128 events of one realisation in one block;
    // a subset's slots run realisation-major, so each realisation's partial
    // sums are one contiguous run of slots.  Chunks of a subset: at most its
    // events / 128 plus one per (block, realisation) run.
    size_t max_chunks = 1, parts_max = 1;
    for (int s = 0; s < n_subsets; ++s) {
        const int64_t ev_s = se.h_group_start[(size_t)(s + 1) * A_s * se.n_classes] -
                             se.h_group_start[(size_t)s * A_s * se.n_classes];
        const size_t c = (size_t)(ev_s / kBpChunkEvents) + (size_t)(blk_off[s + 1] - blk_off[s]) * R;
        max_chunks += c;
        parts_max = std::max(parts_max, c);
    }
    const size_t need = bump_bytes(sizeof(float) * (size_t)R * m.nq) +
                        bump_bytes(sizeof(float) * (size_t)rs * biggest) +
                        bump_bytes(sizeof(float) * (size_t)m.nqt * biggest) +
                        bump_bytes(sizeof(float) * parts_max * m.nq) +
                        bump_bytes(sizeof(double) * parts_max) +
                        bump_bytes(sizeof(double) * (size_t)R * m.nq) +
                        bump_bytes(sizeof(BpChunk) * max_chunks) +
                        bump_bytes(sizeof(int) * (size_t)n_subsets * (R + 1)) +
                        bump_bytes(sizeof(int64_t) * (size_t)(n_blk + 1)) +
                        bump_bytes(sizeof(int) * (size_t)(G + 1));
    rc = ensure(h, h->scratch_work, need, st);
    if (rc != LMMEW_OK) return rc;
    char* w = (char*)h->scratch_work.ptr;
    float* lam_v = bump<float>(w, (size_t)R * m.nq);
    float* rows = bump<float>(w, (size_t)rs * biggest);
    float* ypart = bump<float>(w, (size_t)m.nqt * biggest);
    float* bpart = bump<float>(w, parts_max * m.nq);
    double* llpart = bump<double>(w, parts_max);
    double* num = bump<double>(w, (size_t)R * m.nq);
    BpChunk* d_bp = bump<BpChunk>(w, max_chunks);
    int* d_part = bump<int>(w, (size_t)n_subsets * (R + 1));
    int64_t* d_blk_start = bump<int64_t>(w, (size_t)n_blk + 1);
    int* d_grp_start = bump<int>(w, (size_t)G + 1);
    std::vector<int64_t> blk_start(n_blk + 1, se.n_total);
    for (int b = 0; b < n_blk; ++b) blk_start[b] = blocks[b].e0;
    if (n_blk > 0)
        LMMEW_CUDA(cudaMemcpyAsync(d_blk_start, blk_start.data(), 8 * (size_t)(n_blk + 1),
                                   cudaMemcpyHostToDevice, st));
    std::vector<int> grp;   // grp[b * R + r]: first entry of (block b, realisation r)
    rc = bp_order_batch(h, &se, R, d_blk_start, n_blk, d_grp_start, grp, st);
    if (rc != LMMEW_OK) return rc;
    std::vector<BpChunk> bp;
    std::vector<int> part_start((size_t)n_subsets * (R + 1), 0);
    for (int s = 0; s < n_subsets; ++s) {
        // slot of each (realisation, block) run, realisation-major
        const int b0 = blk_off[s], b1 = blk_off[s + 1];
        std::vector<int> slot0((size_t)(b1 - b0) * R);
        int slot = 0;
        for (int r = 0; r < R; ++r) {
            part_start[(size_t)s * (R + 1) + r] = slot;
            for (int b = b0; b < b1; ++b) {
                const int64_t cnt = grp[(size_t)b * R + r + 1] - grp[(size_t)b * R + r];
                slot0[(size_t)(b - b0) * R + r] = slot;
                slot += (int)((cnt + kBpChunkEvents - 1) / kBpChunkEvents);
            }
        }
        part_start[(size_t)s * (R + 1) + R] = slot;
        // chunks in block order, each block's chunks one contiguous list
        for (int b = b0; b < b1; ++b) {
            blocks[b].c0 = (int)bp.size();
            for (int r = 0; r < R; ++r) {
                const int64_t g0 = grp[(size_t)b * R + r], g1 = grp[(size_t)b * R + r + 1];
                int sl = slot0[(size_t)(b - b0) * R + r];
                for (int64_t e = g0; e < g1; e += kBpChunkEvents, ++sl)
                    bp.push_back(BpChunk{e, (int)std::min<int64_t>(kBpChunkEvents, g1 - e), sl});
            }
            blocks[b].c1 = (int)bp.size();
        }
    }
    if (!bp.empty())
        LMMEW_CUDA(cudaMemcpyAsync(d_bp, bp.data(), sizeof(BpChunk) * bp.size(),
                                   cudaMemcpyHostToDevice, st));
    LMMEW_CUDA(cudaMemcpyAsync(d_part, part_start.data(), sizeof(int) * part_start.size(),
                               cudaMemcpyHostToDevice, st));
    rc = launch_images_batch(h, R, images, lam_v, true, st);
    if (rc != LMMEW_OK) return rc;

    if (n_iters == 0) return launch_images_batch(h, R, images, lam_v, false, st);

    // the whole reconstruction as one CUDA graph, replayed on the caller's stream
    if (!h->cap_stream) LMMEW_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = h->cap_stream;
    LMMEW_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < n_iters && rc == LMMEW_OK; ++it) {
        for (int s = 0; s < n_subsets && rc == LMMEW_OK; ++s) {
            for (int b = blk_off[s]; b < blk_off[s + 1]; ++b) {
                const RowBlock& c = blocks[b];
                RowLaunch L{se.tiles, c.t0, c.t1, se.bin, se.energy, lam_v, rows, c.e0, rs, ypart,
                            c.e1 - c.e0, c.e1 - c.e0, m.nq};
                L.tile_ev = se.tile_ev;
                L.ev_real = se.real;
                rc = launch_row(h, L, cs);
                if (rc != LMMEW_OK) break;
                rc = launch_bp_batch(h, rows, rs, ypart, c.e1 - c.e0, se.bp_idx, c.e0, d_bp + c.c0,
                                     c.c1 - c.c0, bpart, loglik ? llpart : nullptr, cs);
                if (rc != LMMEW_OK) break;
            }
            if (rc != LMMEW_OK) break;
            rc = launch_reduce_update_batch(
                h, R, bpart, d_part + (size_t)s * (R + 1), num, lam_v,
                h->d_sens_sub + (size_t)s * m.nq, llpart,
                loglik ? loglik + (size_t)it * n_subsets + s : nullptr, n_iters * n_subsets, cs);
        }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (rc != LMMEW_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ec != cudaSuccess) return cuda_error(ec, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_error(ei, "cudaGraphInstantiate");
    }
    h->graph = graph;
    h->graph_exec = exec;
    LMMEW_CUDA(cudaGraphLaunch(exec, st));
    return launch_images_batch(h, R, images, lam_v, false, st);
}

int lm_batch_tuning(const lm_handle* h, double* out5) {
    if (!h || !out5) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    out5[0] = h->unit_order;
    out5[1] = h->grid_per_sm;
    out5[2] = h->tune_key != 0 ? 1.0 : 0.0;
    out5[3] = h->tune_ms;
    out5[4] = h->tile_ev;
    return LMMEW_OK;
}

int lm_set_tile_events(lm_handle* h, int tile_events) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    if (tile_events != 32 && tile_events != 64 && tile_events != kET)
        return set_error(LMMEW_ERR_INVALID_ARG, "tile_events must be 32, 64 or 128");
    h->tile_ev = tile_events;
    return LMMEW_OK;
}

int lm_set_table_streaming(lm_handle* h, int max_angles) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    return set_table_streaming(h, max_angles);
}

int lm_table_streaming(const lm_handle* h, int* max_angles, int64_t* table_bytes) {
    if (!h || !max_angles || !table_bytes) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    *max_angles = h->tab_slots;
    *table_bytes = (int64_t)h->tab_bytes;
    return LMMEW_OK;
}

int lm_set_table_budget(int64_t bytes) {
    if (bytes < 0) return set_error(LMMEW_ERR_INVALID_ARG, "the table budget must be >= 0");
    g_table_budget = bytes;
    return LMMEW_OK;
}

int lm_set_energy_pruning(lm_handle* h, int enable) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    h->prune_lines = enable ? 1 : 0;
    build_energy_classes(h);
    return LMMEW_OK;
}

int lm_set_scatter_precision(lm_handle* h, int precision) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    return set_precision(h, precision);
}

int lm_profile_enable(lm_handle* h, int enable) {
    if (!h) return set_error(LMMEW_ERR_INVALID_ARG, "handle is NULL");
    h->prof_on = enable ? 1 : 0;
    return LMMEW_OK;
}

int lm_profile_read(lm_handle* h, double* out5) {
    if (!h || !out5) return set_error(LMMEW_ERR_INVALID_ARG, "NULL argument");
    double ms = 0.0;
    for (size_t i = 0; i + 1 < h->prof_used; i += 2) {
        LMMEW_CUDA(cudaEventSynchronize(h->prof_ev[i + 1]));
        float t = 0.f;
        LMMEW_CUDA(cudaEventElapsedTime(&t, h->prof_ev[i], h->prof_ev[i + 1]));
        ms += t;
    }
    unsigned long long evaluated = 0;
    if (h->d_term_counter) {
        LMMEW_CUDA(cudaMemcpy(&evaluated, h->d_term_counter, sizeof(evaluated),
                              cudaMemcpyDeviceToHost));
        LMMEW_CUDA(cudaMemset(h->d_term_counter, 0, sizeof(evaluated)));
    }
    out5[0] = ms;
    out5[1] = (double)h->prof_launches;
    out5[2] = (double)evaluated;
    out5[3] = h->prof_elems;
    out5[4] = (double)h->launches;
    h->launches = 0;
    h->prof_used = 0;
    h->prof_launches = 0;
    h->prof_terms_dense = 0.0;
    h->prof_elems = 0.0;
    return LMMEW_OK;
}

}  // extern "C"
