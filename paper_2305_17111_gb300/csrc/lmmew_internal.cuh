// Internal declarations shared by the translation units of liblmmew.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <map>
#include <vector>

#include "lmmew.h"

namespace lmmew {

// ---------------------------------------------------------------- tiling
constexpr int kQT = 32;     // voxels per q-tile of the row kernel
constexpr int kPC = 32;     // scatter points per pipeline stage
constexpr int kET = 128;    // largest tile: events per tile (kEPL per lane, 32 lanes)
constexpr int kEPL = kET / 32;
constexpr int kETMin = 32;  // smallest tile (one event per lane); tile arrays are sized for it
constexpr int kCPad = 36;   // floats per staged collimator row (32 + 4 pad)
constexpr int kRowThreads = 256;
constexpr float kNegHuge = -1.0e30f;   // log2 weight of an absent path
constexpr float kPosHuge = 1.0e30f;    // its negative (square-root form of the tables)
// Collimator probabilities of scatter points below this fraction of the
// largest point probability of the same (angle, bin) are stored as exactly 0,
// and the row kernel never visits a run of points that are all 0 for the
// tile's bins.  A dropped term is below 1e-7 of the (angle, bin)'s largest
// collimator factor times its own path weight; over every event of the small
// parity cases and 1 500 of the 64 x 64 workload (FP64 restatement on the
// oracle's path data, random images) the forward value moves by 1.0e-7
// relative at most, the size of the FP32 rounding of the sums.  Relative to
// the bin's own largest factor, the floor keeps the far-tail points of bins
// outside the object's shadow, where they carry the whole value.  Voxel
// (unscattered) probabilities keep every value.
constexpr float kCollimatorFloorRel = 1e-7f;

// Status bits written by kernels into the handle's device status word.
constexpr int kStatusOutOfRange = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusTables = 4;   // a row launch met an angle whose path tables were not resident

// ---------------------------------------------------------------- model
// Model constants passed by value to the setup kernels (FP64).
struct ModelConst {
    int n, A, B, S, W, n_win, n_knots;
    int nq, np, f;            // support voxels, scatter points, pixels per cell side
    int nqt, npc;             // q-tiles, p-chunks
    double h, bin_w, r_det, fwhm0, slope, T, cell_area;
    double fwhm_frac, e_ref, expo;
    double line_e[LMMEW_MAX_LINES], alpha[LMMEW_MAX_LINES], kn_norm[LMMEW_MAX_LINES];
    double win_lo[LMMEW_MAX_WINDOWS], win_hi[LMMEW_MAX_WINDOWS];
    double knot_e[LMMEW_MAX_KNOTS], knot_mu[LMMEW_MAX_KNOTS];
    double knot_slope[LMMEW_MAX_KNOTS];   // (mu[s+1] - mu[s]) / (e[s+1] - e[s])
};

// Per-line FP32 constants of the energy response used by the hot kernel.
struct LineConst {
    float e[LMMEW_MAX_LINES];      // line energy
    float nk[LMMEW_MAX_LINES];     // -log2(e) / (2 sigma_E(E)^2)
    float norm[LMMEW_MAX_LINES];   // 1 / (sqrt(2 pi) sigma_E(E))
};

// One tile of events: one angle and one energy class, up to tile_ev (<= kET)
// consecutive sorted events.
struct Tile {
    int a;          // detector angle
    int begin;      // first sorted event (index into the sorted arrays)
    int count;      // 1..tile_ev
    int b_lo_hi;    // (b_lo << 16) | b_hi: bin range of the tile's events
    int r;          // realisation (0 outside batched reconstruction)
    int lines;      // bit w set: line w's single scatter can reach the tile's energies
    // run [p_lo, p_hi) of the angle's point order with non-zero collimator
    // probability for some bin of the tile (p_lo >= p_hi: none)
    int p_lo, p_hi;
};

// Energy classes of the recorded energy.  A photon of line w that scatters
// once leaves with E' between the backscatter energy E_w / (1 + 2 E_w / m_e c^2)
// and E_w; the detector blurs E' by a Gaussian of sigma_E(E').  Line w's
// reach is [lo_w, hi_w] = the union of E' -+ kScatterReachSigmas sigma_E(E')
// over those E'.  The 2W reach ends, sorted, cut the energy axis into classes;
// inside one class every line's reach either covers the class or misses it,
// so the class fixes which lines' single-scatter terms the row kernel
// evaluates.  A term of a line out of reach has an energy factor below
// exp(-kScatterReachSigmas^2 / 2) = exp(-32) of its own path's peak.
constexpr float kScatterReachSigmas = 8.0f;
struct EnergyClasses {
    int n_bnd;                          // class boundaries (0: one class, every line)
    float bnd[2 * LMMEW_MAX_LINES];     // ascending; class = #{k : bnd[k] <= E_hat}
};

struct Scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Work of one row block (a chunk of whole tiles), written on the device by
// the planning kernel so that the host needs no event counts: tiles
// [x, y) and sorted events [z, w) (x = y: nothing to do).
typedef int4 ChunkRange;

}  // namespace lmmew

struct lm_handle {
    lmmew::ModelConst mc;
    lmmew::LineConst lc;
    int n_subsets_default;
    // geometry on the device
    int* d_q_pix = nullptr;        // [nq] pixel index of each support voxel
    float* d_tab = nullptr;        // [A][nqt][npc][3][W][kQT][kPC]  nlh, sr, m (square-root form)
    float* d_cs = nullptr;         // [A][npc][B][kCPad] collimator prob. of scatter points,
                                   // points in each angle's ascending-u order
    int2* d_crange = nullptr;      // [A][B] ordered points with non-zero probability: [first, last+1)
    float* d_cv = nullptr;         // [A][B][nq] collimator prob. of voxels
    float* d_prim = nullptr;       // [A][W][nq] alpha_w exp(-mu_w gamma_det)
    double* d_sens_a = nullptr;    // [A][nq] per-angle sensitivity (FP64)
    int* d_status = nullptr;       // device status word
    // energy classes of the sort and the lines each class evaluates
    lmmew::EnergyClasses ecls{};
    int n_classes = 1;
    int class_lines[2 * LMMEW_MAX_LINES + 1] = {};
    int prune_lines = 1;           // 0: every tile evaluates every line (lm_set_energy_pruning)
    // device copies of the sort's group arrays, one set per subset partition
    // (rank of each angle [A], angle and line mask of each group [G]) for the
    // energy classes grp_classes; emptied when the classes change
    int grp_classes = 0;
    std::map<int, int*> grp_cache;
    size_t tab_bytes = 0;
    // Streamed path tables: with tab_slots > 0, d_tab holds the tables of at
    // most tab_slots angles, a0 + i astep (i < tab_count), rebuilt by k_scatter
    // when a row launch needs other angles; 0: every angle resident
    int tab_slots = 0;
    int tab_a0 = 0, tab_astep = 1, tab_count = 0;
    // what k_scatter needs to rebuild tables, kept from the set-up
    double* d_cs_a = nullptr;      // [A][2] cos, sin of each detector direction
    int* d_p_cell = nullptr;       // [np] cell of each scatter point
    double* d_p_rho = nullptr;     // [np] its mean density
    double* d_gqp = nullptr;       // [nq][np] voxel-to-point line integrals of rho
    double* d_dqp = nullptr;       // [nq][np] voxel-to-point distances
    double* d_gp = nullptr;        // [A][np] point-to-detector line integrals
    double* d_on_det = nullptr;    // [A][np] collimator mass of each point on the detector
    int* d_inv = nullptr;          // [A][np] point of each slot of an angle's point order
    double* d_mu_line = nullptr;   // [W] mu_water at each line energy
    lmmew::ChunkRange* d_clip = nullptr;   // a row launch's tiles clipped to one angle block
    // cached subset sensitivities for the last partition asked for
    int sens_parts = 0;
    double* d_sens_sub = nullptr;  // [parts][nq]
    // growable scratch arena
    lmmew::Scratch scratch_sort;   // sorted events of the current call
    lmmew::Scratch scratch_work;   // row blocks and partial sums
    int sm_count = 0;
    int row_blocks_per_sm = 0;
    int row_blocks[3] = {0, 0, 0};   // resident row-kernel CTAs per SM, per precision
    // launch shape of the row kernel (set by the batch autotuner)
    int unit_order = 0;            // 0: tile-major units, 1: voxel-tile-major units
    int grid_per_sm = 0;           // persistent CTAs per SM (0: occupancy maximum)
    cudaStream_t cap_stream = nullptr;     // private stream for CUDA-graph capture
    cudaGraphExec_t graph_exec = nullptr;  // last batched reconstruction graph
    cudaGraph_t graph = nullptr;
    uint64_t tune_key = 0;         // workload class the current launch shape belongs to
    struct TuneChoice {
        int tile_ev, unit_order, grid_per_sm;
        float ms;
    };
    std::map<uint64_t, TuneChoice> tune_cache;   // every workload class tuned on this handle
    int tile_ev = lmmew::kET;      // events per tile of the row kernel: 32, 64 or 128 (tuned)
    float tune_ms = 0.f;           // the tuned row launch's time
    // scatter-term precision: 0 FP32, 1 FP16, 2 BF16 (reduced-precision form)
    int prec = 0;
    int tabh_prec = 0;
    float* d_tabh = nullptr;       // reduced-precision copy of d_tab
    float* d_tscale = nullptr;     // [A][nqt][npc] block scales 2^base
    // learned scatter surrogate
    float* d_g8 = nullptr;         // [A][nq][8] rho line integrals along theta_a + k pi/4 (cm)
    float* d_rho = nullptr;        // [n][n] relative density (surrogate inputs)
    double mu_line[LMMEW_MAX_LINES] = {};   // mu_water at each line energy
    const struct lm_surrogate* surrogate = nullptr;   // scatter model when set
    int scatter_model = 0;         // 0 exact, 1 surrogate, 2 none, 3 surrogate on the coarse grid
    // coarse-grid surrogate: network nodes and each voxel's interpolation
    int n_nodes = 0;
    int coarse_stride = 2;         // node spacing in pixels (lm_set_coarse_stride)
    int* d_node_q = nullptr;       // [n_nodes] support voxel of each node
    int4* d_interp_node = nullptr; // [nq] up to 4 nodes of each voxel (-1: none)
    float4* d_interp_w = nullptr;  // [nq] their weights (sum 1)
    lmmew::Scratch scratch_nodes;  // [block events][n_nodes] network outputs
    double* d_sens_a_prim = nullptr;   // [A][nq] unscattered part of the sensitivity
    int sens_prim_only = 0;
    float setup_ms = 0.f;
    int64_t terms_per_event = 0;   // exponentials per event row (primary + scatter)
    // optional timing of the row kernel (CUDA events around each launch)
    int prof_on = 0;
    std::vector<cudaEvent_t> prof_ev;   // pairs
    size_t prof_used = 0;
    double prof_ms = 0.0;
    int64_t prof_launches = 0;
    double prof_terms_dense = 0.0;   // terms of the rows without the exact-zero skip
    double prof_elems = 0.0;
    int64_t launches = 0;          // kernels this library launched (all kinds)
    unsigned long long* d_term_counter = nullptr;   // exponentials evaluated while timing
    int* d_work = nullptr;         // row kernel's next-unit counter, zeroed before each launch
};

namespace lmmew {

// Error reporting (thread-local message).
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);
#define LMMEW_CUDA(call)                                              \
    do {                                                              \
        cudaError_t e__ = (call);                                     \
        if (e__ != cudaSuccess) return ::lmmew::cuda_error(e__, #call); \
    } while (0)

// setup.cu
int build_tables(lm_handle* h, const float* rho_host, const uint8_t* support_host);
// setup.cu: the path tables of angles a0 + i astep (i < count) into the
// streamed table buffer (nothing to do if they are resident), and the switch
// between streamed (max_angles > 0) and resident (0) tables
int stream_tables(lm_handle* h, int a0, int astep, int count, cudaStream_t st);
int set_table_streaming(lm_handle* h, int max_angles);
// setup.cu: tables larger than this are streamed by lm_create (0: no limit
// beyond the device's free memory)
extern int64_t g_table_budget;
// events.cu: the energy classes of the handle's lines and energy model
void build_energy_classes(lm_handle* h);
int subset_sensitivity(lm_handle* h, int n_subsets, cudaStream_t st);

// events.cu: validation + stable sort by (subset rank of angle, energy class,
// bin).  A group is one (angle rank, energy class): n_classes consecutive
// groups per angle rank.
struct SortedEvents {
    uint16_t* bin = nullptr;     // [n] sorted bins
    float* energy = nullptr;     // [n] sorted energies
    uint32_t* perm = nullptr;    // [n] caller index of each sorted event
    int* group_start = nullptr;  // [G+1] device: first sorted event of each group
    Tile* tiles = nullptr;       // [max_tiles]
    int* tile_start = nullptr;   // [G+1] first tile of each group
    int64_t n_valid = 0;
    int tile_ev = kET;           // events per tile the tiles were cut with
    int n_groups = 0;            // groups G the tiles are cut in
    int n_classes = 1;           // groups per angle rank
    const int* angle_of_group = nullptr;   // device [n_groups]: angle of each group
    const int* lines_of_group = nullptr;   // device [n_groups]: line mask of each group
    // batched sort only
    uint16_t* real = nullptr;    // [n] realisation of each sorted event
    uint32_t* bp_idx = nullptr;  // [n] back-projection order (bp_order_batch)
    uint32_t *tmp_keys0 = nullptr, *tmp_keys1 = nullptr, *tmp_vals0 = nullptr,
             *tmp_vals1 = nullptr, *tmp_hist = nullptr;
    int64_t n_total = 0;
    // host copies
    std::vector<int> h_group_start;  // [G+1]
    std::vector<int> h_tile_start;   // [G+1]
};
// Groups of a sort over A angle ranks (A * n_classes) and the line mask of
// each class.
int sort_groups(const lm_handle* h, int A);
size_t sort_scratch_bytes(int64_t n, int G);
int sort_events(lm_handle* h, const lm_events* ev, int n_subsets, SortedEvents* out,
                char*& arena, cudaStream_t st);

// events.cu: the sort without any host read-back: every size the later
// kernels need stays on the device (group_start[G] = valid events,
// tile_start[G] = tiles).  The group arrays come from the handle's cache
// (group_arrays) or, for callers that may not allocate, from ga.
struct GroupArrays {
    const int* rank_of_angle;    // [A]
    const int* angle_of_group;   // [G]
    const int* lines_of_group;   // [G]
};
int group_arrays(lm_handle* h, int n_subsets, GroupArrays* out);   // cached per partition
int sort_events_async(lm_handle* h, const lm_events* ev, const GroupArrays& ga, int G,
                      SortedEvents* out, char*& arena, cudaStream_t st);
// Group arrays of one subset (angles in natural order) built on the device
// into a caller-provided region (no allocation, no copy from the host).
GroupArrays group_arrays_into(lm_handle* h, char*& arena, cudaStream_t st);
// Tiles re-cut on the device only (no read-back).
int recut_tiles_async(lm_handle* h, SortedEvents* se, int tile_ev, cudaStream_t st);
// Read back the group and tile starts of an async sort (synchronises).
int read_back_counts(lm_handle* h, SortedEvents* se, cudaStream_t st);
// Synchronises the stream, then returns (and clears) the error the device
// status word holds: LMMEW_ERR_OUT_OF_RANGE, LMMEW_ERR_TIMEOUT or LMMEW_OK.
int take_status(lm_handle* h, cudaStream_t st);
// api.cu: the forward projection without host read-back, shared by
// lm_forward and lm_forward_noalloc.  One set of all groups, row blocks of
// tpc tiles (cap events), `blocks` of them: enough for any n events.
struct ForwardPlan {
    int G;
    int64_t n, cap;
    int tpc, blocks;
};
ForwardPlan forward_plan(const lm_handle* h, int64_t n, int64_t cap_max);
size_t forward_region_bytes(const lm_handle* h, const ForwardPlan& p);
int forward_async(lm_handle* h, const lm_events* ev, const float* image, float* out_y,
                  const GroupArrays& ga, const ForwardPlan& p, char* arena, cudaStream_t st);
// Row blocks of n_sets consecutive rank ranges (the subsets of a partition
// into n_subsets, or all ranks for n_subsets = 1): set s, block k covers
// tiles [T0 + k tpc, T0 + (k + 1) tpc) of the set's tiles [T0, T1).
int launch_plan(lm_handle* h, const SortedEvents& se, int n_subsets, int blocks_per_set,
                int tiles_per_block, ChunkRange* ranges, cudaStream_t st);
// events.cu: a row block's range clipped on the device to the tiles of groups
// [g0, g1) (one angle block of streamed path tables); row base and events
// stay the block's
int launch_clip_range(lm_handle* h, const ChunkRange* in, const SortedEvents& se, int g0, int g1,
                      ChunkRange* out, cudaStream_t st);

size_t sort_batch_scratch_bytes(int64_t n, int64_t G, int R);
int sort_events_batch(lm_handle* h, const lm_events* evs, int R, int n_subsets,
                      SortedEvents* out, char*& arena, cudaStream_t st);
int bp_order_batch(lm_handle* h, SortedEvents* se, int R, const int64_t* blk_start, int n_blk,
                   int* grp_start, std::vector<int>& h_grp_start, cudaStream_t st);
// Re-cut the sorted groups into tiles of tile_ev events (h_tile_start updated).
int recut_tiles(lm_handle* h, SortedEvents* se, int tile_ev, cudaStream_t st);

// row.cu: fused system-matrix row kernel
struct RowLaunch {
    const Tile* tiles;
    int tile_begin, tile_end;
    const uint16_t* ev_bin;
    const float* ev_e;
    const float* lam_v;     // [nq] image on the voxel list (may be null: no forward sums)
    float* rows;            // null: do not store rows
    int64_t row_base;       // sorted index of row 0
    int row_stride;
    float* ypart;           // [nqt][ypart_stride], indexed by sorted event - row_base
    int64_t ypart_stride;
    int64_t n_events;       // events covered by the tile range (for accounting)
    int lam_stride = 0;     // batched: image of realisation r at lam_v + r * lam_stride
    int tile_ev = kET;      // events per tile the tiles were cut with (32, 64 or 128)
    const uint16_t* ev_real = nullptr;   // batched: realisation of each sorted event
    int skip_scatter = 0;   // unscattered terms only (the surrogate adds the rest)
    const ChunkRange* range = nullptr;   // if set: tiles and row_base read on the device
};
int launch_row(lm_handle* h, const RowLaunch& L, cudaStream_t st);
int set_precision(lm_handle* h, int prec);
// mlp.cu: the surrogate's rows (adds the learned scatter part to rows k_row
// wrote without scatter, then the partial forward sums)
int launch_surrogate_rows(lm_handle* h, const RowLaunch& L, cudaStream_t st);
// mlp.cu: nodes of the coarse-grid surrogate and each voxel's interpolation
// (built once per handle), and the node-output scratch for a row block of
// up to max_events events (called by the planners before any capture)
int build_coarse_nodes(lm_handle* h);
int surrogate_prepare(lm_handle* h, int64_t max_events, cudaStream_t st);
size_t row_smem_bytes(const lm_handle* h);
int row_kernel_occupancy(lm_handle* h);

// em.cu
int launch_forward_out(lm_handle* h, const float* ypart, int64_t ypart_stride, int64_t begin,
                       int64_t count, const uint32_t* perm, float* out_y, cudaStream_t st);
int launch_bp_partial(lm_handle* h, const float* rows, int row_stride, const float* ypart,
                      int64_t ypart_stride, int64_t count, const uint32_t* perm,
                      const float* weight, float* bpart, int64_t bpart_row0, double* llpart,
                      cudaStream_t st);
int64_t bp_parts(int64_t count);
int launch_voxel_reduce(lm_handle* h, const float* bpart, int64_t n_parts, double* num,
                        cudaStream_t st);
int launch_update(lm_handle* h, float* lam_v, const double* num, const double* sens,
                  const double* llpart, int64_t n_ll, double* loglik_out, cudaStream_t st);
// The same steps with the sizes on the device: row block k of a set holds
// ranges[k].w - ranges[k].z events, its ypart / rows indexed from
// ranges[k].z, its back-projection partials at slots [k * ppc, ...).
int launch_forward_out_range(lm_handle* h, const float* ypart, int64_t ypart_stride,
                             int64_t capacity, const ChunkRange* range, const uint32_t* perm,
                             float* out_y, cudaStream_t st);
int launch_invalid_out(lm_handle* h, const int* n_valid, int64_t n, const uint32_t* perm,
                       float* out_y, cudaStream_t st);
int launch_bp_partial_range(lm_handle* h, const float* rows, int row_stride, const float* ypart,
                            int64_t ypart_stride, int64_t capacity, const ChunkRange* range,
                            const uint32_t* perm, const float* weight, float* bpart,
                            int64_t slot0, double* llpart, cudaStream_t st);
int launch_voxel_reduce_ranges(lm_handle* h, const float* bpart, const ChunkRange* ranges,
                               int n_blocks, int64_t ppc, double* num, cudaStream_t st);
int launch_update_ranges(lm_handle* h, float* lam_v, const double* num, const double* sens,
                         const double* llpart, const ChunkRange* ranges, int n_blocks,
                         int64_t ppc, double* loglik_out, cudaStream_t st);
constexpr int kBpChunkEvents = 128;   // events per back-projection partial sum
struct BpChunk {
    int64_t begin;   // first entry of the back-projection order
    int count;       // 1..128 events, all of one realisation
    int slot;        // partial-sum slot of the sub-iteration
};
int launch_bp_batch(lm_handle* h, const float* rows, int row_stride, const float* ypart,
                    int64_t ypart_stride, const uint32_t* bp_idx, int64_t row_base,
                    const BpChunk* chunks, int n_chunks, float* bpart, double* llpart,
                    cudaStream_t st);
int launch_reduce_update_batch(lm_handle* h, int R, const float* bpart, const int* part_start,
                               double* num, float* lam_v, const double* sens,
                               const double* llpart, double* loglik, int ll_stride,
                               cudaStream_t st);
int launch_images_batch(lm_handle* h, int R, float* images, float* lam_v, bool to_voxels,
                        cudaStream_t st);
int launch_gather_image(lm_handle* h, const float* image, float* lam_v, cudaStream_t st);
int launch_scatter_image(lm_handle* h, const float* lam_v, float* image, cudaStream_t st);
int launch_scatter_image_d(lm_handle* h, const double* v, double* image, cudaStream_t st);
int launch_num_to_image(lm_handle* h, const double* num, float* image, cudaStream_t st);

// Inputs of the learned scatter surrogate for one (event, voxel q, line w).
// Geometry in cm in the frame of detector angle a: depth t = x cos + y sin,
// detector coordinate u = -x sin + y cos.  The recorded energy fixes, through
// Compton's relation, the scattering angle phi a single scatter needs to
// bring E_w down to e_hat: 1 - cos(phi) = kappa = m_e c^2 (1/e_hat - 1/E_w).
// The scatter point p* on the bin's projection line (u = u_b) seen from q at
// that angle to the detector direction dominates S_w; its position,
// distance and density are inputs, together with the optical depths
// mu_w(E_w) x rho-integral from q to the image edge along theta_a + k pi/4.
//   0-1 x, y      2-3 cos, sin of theta_a   4 u_b   5 e_hat   6-8 line one-hot
//   9-16 optical depths   17 u_b - u_q   18 t_q   19 kappa   20 e_hat / E_w
//   21 |u_b - u_q|   22-23 p*   24 |p* - q|   25 cos(phi)   26 h / (|p* - q| + h)
//   27 [kappa < 0]   28 rho(p*)   29-31 zero
constexpr int kSurrogateIn = 32;
constexpr float kSurrogateEps = 1e-8f;   // target = ln(S + eps)
// The surrogate is evaluated only for recorded energies within this many
// energy-resolution sigmas of the energies single scatter of the line can
// have (backscatter energy to E_w): outside, the exact term is below
// exp(-32) of its largest value and the surrogate's part is 0.
constexpr float kSurrogateReachSigmas = kScatterReachSigmas;
constexpr float kElectronRestKeV = 510.99895f;
// Division in the network's input features: the fast approximate form on the
// device (about 2 ulp; the inputs are rounded to BF16 afterwards), IEEE on the
// host.
__host__ __device__ __forceinline__ float feature_div(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
// The 32 inputs of one (event, voxel, line); g8 holds the 8 rho line
// integrals of the voxel at this angle.  Every kernel builds them here, so
// they all compute the same values.
__host__ __device__ __forceinline__ void surrogate_features(float xq, float yq, float ca, float sa,
                                                            float ub, float e_hat, int w,
                                                            float e_line, float mu_w,
                                                            const float* g8, const float* rho,
                                                            int n, float h, float* f) {
    f[0] = xq * 0.05f;
    f[1] = yq * 0.05f;
    f[2] = ca;
    f[3] = sa;
    f[4] = ub * 0.05f;
    f[5] = (e_hat - 150.f) * 0.01f;
    f[6] = w == 0 ? 1.f : 0.f;
    f[7] = w == 1 ? 1.f : 0.f;
    f[8] = w == 2 ? 1.f : 0.f;
    for (int k = 0; k < 8; ++k) f[9 + k] = mu_w * g8[k] * 0.25f;
    // detector coordinate and depth of the voxel, the Compton kappa of the
    // recorded energy, and the scatter point p* on the bin's projection line
    const float uq = -xq * sa + yq * ca, tq = xq * ca + yq * sa;
    const float du = ub - uq;
    const float kappa = kElectronRestKeV * (feature_div(1.f, e_hat) - feature_div(1.f, e_line));
    const float c = fminf(fmaxf(1.f - kappa, -1.f), 1.f);
    const float s = fmaxf(sqrtf(fmaxf(1.f - c * c, 0.f)), 0.05f);
    const float lim = n * h;
    const float dt = fminf(fmaxf(feature_div(fabsf(du) * c, s), -lim), lim);
    const float tp = tq + dt;
    const float xp = tp * ca - ub * sa, yp = tp * sa + ub * ca;
    f[17] = du * 0.2f;
    f[18] = tq * 0.05f;
    f[19] = fminf(fmaxf(kappa, -2.f), 4.f) * 0.5f;
    f[20] = feature_div(e_hat, e_line);
    f[21] = fabsf(du) * 0.2f;
    f[22] = xp * 0.05f;
    f[23] = yp * 0.05f;
    const float r = sqrtf(dt * dt + du * du);
    f[24] = r * 0.05f;
    f[25] = c;
    f[26] = feature_div(h, r + h);
    f[27] = kappa < 0.f ? 1.f : 0.f;
    const float gx = floorf(feature_div(xp, h) + 0.5f * n), gy = floorf(feature_div(yp, h) + 0.5f * n);
    f[28] = (gx >= 0.f && gx < (float)n && gy >= 0.f && gy < (float)n) ? rho[(int)gy * n + (int)gx]
                                                                      : 0.f;
    f[29] = f[30] = f[31] = 0.f;
}

#ifdef __CUDACC__
// Shared-memory addresses, the global timer and mbarriers (every wait on an
// mbarrier is bounded in time), and the bulk asynchronous copy engine.
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per pipeline wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for a barrier phase with a time limit; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer();
    while (!mbar_try_wait(bar, parity))
        if (global_timer() - t0 > kWaitLimitNs) return false;
    return true;
}

// Packed pairs of FP32 values (Blackwell's f32x2 arithmetic): one instruction,
// two IEEE round-to-nearest results.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
#endif

// Bump allocation from a scratch arena (256-byte aligned).
template <class T>
inline T* bump(char*& arena, size_t count) {
    uintptr_t p = reinterpret_cast<uintptr_t>(arena);
    p = (p + 255) & ~uintptr_t(255);
    T* out = reinterpret_cast<T*>(p);
    arena = reinterpret_cast<char*>(p + sizeof(T) * count);
    return out;
}
inline size_t bump_bytes(size_t bytes) { return ((bytes + 255) / 256) * 256 + 256; }

}  // namespace lmmew
