/*
 * lmmew.h -- C ABI of the GB300 (sm_103a) list-mode multi-energy-window
 * (LM-MEW) OSEM library for 2-D SPECT of isotopes with several emission peaks
 * (Rahman et al., arXiv 2305.17111).
 *
 * The problem (paper Sec. "Problem formulation"): a voxelised activity lambda
 * (Q voxels), W emission lines E_0^w with yields alpha_w, and J list-mode
 * events, each with a detector angle, a detected position (here a detector
 * bin) and a recorded energy.  The library evaluates, on the GPU, the
 * path-based model of Sec. "Likelihood of list-mode data using path-based
 * formalism" -- for every event and voxel the system-matrix element
 *
 *   a_j[q] = sum_w alpha_w sum_{P in P_q} pr(A_j | P, E_0^w) s(P, E_0^w)
 *
 * over the unscattered path and the single-scatter paths through a grid of
 * scatter points (Eq. s_p with n = 0, 1) -- and runs the LM-OSEM update of
 * Eq. (os-lm-mlem) with (z_bar_update_os).  The model's readings where the
 * paper is silent are:
 *   - pr(A|P,E) = collimator bin probability (Gaussian, FWHM = fwhm0 +
 *     slope * depth, integrated over the bin) x energy-resolution Gaussian
 *     density (FWHM/E = frac (E/E_ref)^exponent) at the recorded energy;
 *   - scatter subpaths: scatter_n x scatter_n cells, density = cell mean,
 *     quadrature weight A_p / (2 pi d), the emission voxel's own cell skipped,
 *     Klein-Nishina normalised to the image plane, scatter probability per cm
 *     = mu;
 *   - sensitivity = the row integrated over the detector and the windows;
 *   - subsets interleave angles: subset(a) = a mod n_subsets;
 *   - mu(r, E) = rho(r) mu_water(E), mu_water linear between knots.
 *
 * Conventions (all entry points):
 *   - return 0 (LMMEW_OK) or a negative LMMEW_ERR_* code; lm_last_error()
 *     gives a message for the calling thread;
 *   - geometry, maps and spectra are HOST pointers, copied by lm_create;
 *   - events, images and outputs are DEVICE pointers owned by the caller; the
 *     library never frees or permutes them (it sorts a private copy);
 *   - work is queued on the caller's CUDA stream (a cudaStream_t; 0 = the
 *     legacy default stream).  lm_forward, lm_backproject and lm_osem with
 *     the exact or the scatter-free model, and lm_forward_noalloc, queue
 *     their kernels and return without waiting for the stream: events are
 *     validated on the device and the work is sized from the event count
 *     alone.  Errors found on the device (an event out of range, a pipeline
 *     wait that ran out of time) set the handle's status word, which
 *     lm_check reports (it synchronises the stream).  Set-up steps
 *     synchronise: the first call of a subset partition (sensitivities,
 *     group tables), scratch that has to grow, and lm_osem's first call of a
 *     workload class (the launch-shape tuner, see lm_batch_tuning).
 *     lm_osem_batch and the surrogate scatter models read the event counts
 *     back once per call;
 *   - a handle serves one stream at a time;
 *   - there is no CPU fallback: every step runs in this library's kernels.
 *
 * Images are n*n arrays in raster order [iy*n + ix]; pixel (ix, iy) has its
 * centre at ((ix + 0.5 - n/2) h, (iy + 0.5 - n/2) h) cm.  Detector angle a is
 * theta_a = 2 pi a / n_angles; the detector normal is (cos, sin), the
 * detector coordinate u = -x sin + y cos, and bin b covers
 * u in [-n_bins w/2 + b w, -n_bins w/2 + (b+1) w).
 */
#ifndef LMMEW_H
#define LMMEW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LMMEW_OK 0
#define LMMEW_ERR_INVALID_ARG -1     /* bad sizes, pointers or physics parameters */
#define LMMEW_ERR_OUT_OF_RANGE -2    /* an event's angle, bin or energy is outside the model */
#define LMMEW_ERR_CUDA -3            /* a CUDA call failed (message has the CUDA error) */
#define LMMEW_ERR_OOM -4             /* device allocation failed */
#define LMMEW_ERR_TIMEOUT -5         /* a kernel's bounded pipeline wait ran out */
#define LMMEW_ERR_NOT_IMPLEMENTED -6

#define LMMEW_MAX_LINES 8
#define LMMEW_MAX_WINDOWS 8
#define LMMEW_MAX_KNOTS 16

/* Opaque handle: owns the device tables of one scanner + object model. */
typedef struct lm_handle lm_handle;

/* A cudaStream_t, declared without including the CUDA headers. */
struct CUstream_st;
typedef struct CUstream_st* lm_stream;

/* Scanner and grid (paper Sec. "SPECT simulation"). */
typedef struct {
    int32_t n;               /* image is n x n pixels, n >= 1 */
    float pixel_cm;          /* pixel size h, cm */
    int32_t n_angles;        /* detector angles over 360 degrees, 1..65535 */
    int32_t n_bins;          /* detector bins, 1..65535 */
    float bin_cm;            /* bin width; <= 0 means n * pixel_cm / n_bins */
    float r_det_cm;          /* detector face distance from the centre; <= 0 means n * pixel_cm / 2 */
    float coll_fwhm0_cm;     /* collimator FWHM at the detector face, cm */
    float coll_fwhm_slope;   /* FWHM growth per cm of depth */
    float scan_time;         /* T; <= 0 means 1 */
} lm_geometry;

/* Attenuation (paper Sec. "Synthetic phantom model": water with varying
 * density, mu linear in energy between knots). */
typedef struct {
    const float* rho;          /* host, n*n relative density (water = 1), >= 0 */
    int32_t n_knots;           /* 1..16 */
    const float* knot_keV;     /* host, increasing */
    const float* mu_water_cm;  /* host, water attenuation at the knots, 1/cm */
    int32_t scatter_n;         /* scatter grid scatter_n^2 cells; must divide n; 0 = no scatter */
} lm_attenuation;

/* Emission lines E_0^w and yields alpha_w (paper Sec. "Problem formulation"). */
typedef struct {
    int32_t n_lines;           /* 1..8 */
    const float* energy_keV;   /* host */
    const float* yield;        /* host, >= 0 */
} lm_lines;

/* Detector energy response and acceptance windows. */
typedef struct {
    float fwhm_frac_ref;       /* FWHM / E at e_ref_keV (paper: 0.10 at 140 keV) */
    float e_ref_keV;
    float exponent;            /* FWHM / E ~ (E / e_ref)^exponent (paper: -0.5) */
    int32_t n_windows;         /* 1..8, non-overlapping [lo, hi) */
    const float* win_lo_keV;   /* host */
    const float* win_hi_keV;   /* host */
} lm_energy_model;

/* List-mode events (paper Sec. "Problem formulation": angle, detected
 * position, recorded energy).  DEVICE pointers, n entries each. */
typedef struct {
    const uint16_t* angle;     /* 0 .. n_angles-1 */
    const uint16_t* bin;       /* 0 .. n_bins-1 */
    const float* energy_keV;   /* inside one of the windows */
    int64_t n;                 /* >= 0 */
} lm_events;

/* Build the model: copies the host inputs, builds on the GPU the path
 * integrals of Eq. (radpath) (exact line integrals through the density map),
 * the path sensitivities of Eq. (s_p) for every voxel, scatter point, angle
 * and line, the collimator tables and the per-angle sensitivity image (FP64).
 * support: host n*n mask of the voxels that form the model (the LM-OSEM
 * support, paper App. "GPU implementation": voxels with non-zero initial
 * activity); NULL means rho > 0.  n_subsets (>= 1) is the default subset
 * partition used by lm_sensitivity.  Work runs on the legacy default stream
 * and is complete when the call returns.  On success *out owns all device
 * memory of the model; free it with lm_destroy.
 * The single-scatter path tables take 12 bytes per (angle, line, support
 * voxel, scatter point), padded to blocks of 32 voxels x 32 points: 1.6 GB
 * for 60 angles x 3 lines x 864 x 864, 14 GB for 120 x 3 x 3464 x 900.  A
 * model whose tables (with the set-up's line integrals) do not fit 90 % of
 * the device's free memory, or the table budget of lm_set_table_budget, is
 * created with streamed tables (see lm_set_table_streaming); one whose
 * set-up and the tables of a single angle do not fit is refused with
 * LMMEW_ERR_OOM and a message giving the sizes, before anything is
 * allocated for them.
 * Errors: INVALID_ARG (sizes, NULL pointers, scatter_n not dividing n,
 * non-positive collimator or energy blur anywhere in the model, overlapping
 * windows), OOM, CUDA. */
int lm_create(const lm_geometry* geometry, const lm_attenuation* attenuation,
              const lm_lines* lines, const lm_energy_model* energy,
              const uint8_t* support, int n_subsets, lm_handle** out);

/* Sensitivity image of Eq. (os-lm-mlem)'s denominator,
 *   sens_s[q] = T sum_{a in s} sum_w alpha_w sum_{P in P_q} s(P, E_0^w)
 *               x Prob(response on the detector and inside a window),
 * accumulated in FP64.  subset in [0, n_subsets) of the handle's default
 * partition, or -1 for all angles.  out: DEVICE double[n*n], zero outside
 * the support.  Errors: INVALID_ARG, CUDA. */
int lm_sensitivity(lm_handle* h, int subset, double* out, lm_stream stream);

/* Forward projection y_j = sum_q a_j[q] image[q] (the denominator of
 * Eq. z_bar_update_os), FP32 with hierarchical sums.  image: DEVICE
 * float[n*n] (pixels outside the support are ignored); out_y: DEVICE
 * float[events->n], in the caller's event order; an event out of range gets
 * NaN and sets the status word (reported by lm_check).
 * Errors (returned): INVALID_ARG, OOM, CUDA; (by lm_check) OUT_OF_RANGE,
 * TIMEOUT. */
int lm_forward(lm_handle* h, const lm_events* events, const float* image, float* out_y,
               lm_stream stream);

/* Forward projection that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * while they run -- a process whose device memory is already reserved by
 * another allocator (a framework's caching allocator, a fixed budget), or a
 * steady-state loop in which the allocation and the device synchronisation
 * that cudaMalloc/cudaFree imply are not allowed.  It computes exactly what
 * lm_forward computes (same kernels, same order, bit-identical results), with
 * all of its scratch in one 16 MiB array in the library's static device
 * memory, which every GPU that loads the library holds until the process
 * exits.  The call rejects, with LMMEW_ERR_INVALID_ARG and a message, event
 * counts whose scratch would exceed 16 MiB (about 31 + 4*ceil(nq/32) bytes
 * per event, nq = support voxels: some 160 000 events for a 32x32 model of
 * 484 voxels, 34 000 for a 128x128 model of 3 464); use lm_forward for
 * those.  Its first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current: make that
 * first call before any stream capture.  The address is kept for the rest of
 * the process, so the library must not be used across a cudaDeviceReset.
 * Every call shares the one array and
 * it keeps the last call's contents (each call writes every word it reads
 * before reading it): calls that overlap on the GPU -- two streams, two host
 * threads, or a call queued before an earlier one finished on another
 * stream -- race, so serialise them.  Like lm_forward it queues its work
 * without waiting for the stream; events out of range get NaN and are
 * reported by lm_check.  Arguments as lm_forward; the caller still provides
 * events, image and output.  It runs the exact and the scatter-free models;
 * the surrogate models keep a row block of the whole event list, so with
 * them it returns LMMEW_ERR_NOT_IMPLEMENTED before queueing anything (use
 * lm_forward). */
int lm_forward_noalloc(lm_handle* h, const lm_events* events, const float* image, float* out_y,
                       lm_stream stream);

/* Back projection out[q] = sum_j weight_j a_j[q].  weight: DEVICE
 * float[events->n] in the caller's order; out_image: DEVICE float[n*n],
 * zero outside the support; events out of range contribute nothing.
 * Errors: as lm_forward. */
int lm_backproject(lm_handle* h, const lm_events* events, const float* weight,
                   float* out_image, lm_stream stream);

/* LM-OSEM (Eq. os-lm-mlem with z_bar_update_os; Algorithm 1):
 *   for it in [start_iter, n_iters), s in [start_subset (first iteration
 *   only), n_subsets):
 *     y_j = sum_q a_j[q] lambda_q for the events of subset s,
 *     lambda_q <- lambda_q (sum_{j in s, y_j > 0} a_j[q] / y_j) / sens_s[q]
 *     (0 where sens_s[q] = 0).
 * image: DEVICE float[n*n], lambda^0 in, lambda out; pixels outside the
 * support are set to 0.  loglik: NULL or DEVICE double[n_iters*n_subsets];
 * entry it*n_subsets + s receives sum_{j in s, y_j > 0} log y_j -
 * sum_q lambda_q sens_s[q] at the image entering that sub-iteration
 * (Eq. lll_med without J log T - log J!).  Resuming with the image returned
 * by an earlier call and the next (start_iter, start_subset) reproduces an
 * uninterrupted run bit for bit.  The row kernel's launch shape is chosen by
 * the autotuner described at lm_batch_tuning before the first sub-iteration.
 * Errors: as lm_forward. */
int lm_osem(lm_handle* h, const lm_events* events, int n_subsets, int n_iters,
            int start_iter, int start_subset, float* image, double* loglik,
            lm_stream stream);

/* Waits for the stream, then reports (and clears) what the handle's earlier
 * calls found on the device: LMMEW_ERR_OUT_OF_RANGE (an event's angle or bin
 * outside the model, or its energy outside every window: the paper's events
 * lie on the detector and in the windows, Sec. "Problem formulation"),
 * LMMEW_ERR_TIMEOUT (a kernel's bounded pipeline wait ran out), or LMMEW_OK.
 * Errors: INVALID_ARG, CUDA. */
int lm_check(lm_handle* h, lm_stream stream);

/* Arithmetic of the single-scatter sum (the reduced-precision form).
 * LMMEW_PREC_FP32 (default): every term in FP32.  LMMEW_PREC_FP16 /
 * LMMEW_PREC_BF16: d = E_hat - E' stays FP32, the Gaussian exponent
 * (relative to the largest log2 path weight of each 32-voxel x 32-point block)
 * and ex2 run on packed FP16 / BF16 pairs, the per-line sum in that type,
 * everything is accumulated in FP32; unscattered terms, the sensitivity (FP64)
 * and the log-likelihood (FP64) are unchanged.  Applies to the handle's later
 * lm_forward / lm_backproject / lm_osem calls.  The first switch to a reduced
 * precision builds its tables (8 KiB per line per block, synchronously).
 * Errors: INVALID_ARG, NOT_IMPLEMENTED (more than 4 lines), OOM, CUDA. */
#define LMMEW_PREC_FP32 0
#define LMMEW_PREC_FP16 1
#define LMMEW_PREC_BF16 2
int lm_set_scatter_precision(lm_handle* h, int precision);

/* Batched LM-OSEM over n_real independent realisations (noise realisations
 * of the same object: same handle, own events, own image).  Each
 * sub-iteration runs as one persistent row-kernel launch over the events of
 * every realisation (plus per-realisation back projection, FP64 log-likelihood
 * and update), and the whole n_iters x n_subsets sequence is captured once as
 * a CUDA graph and replayed on the caller's stream.  Before the capture the
 * autotuner described at lm_batch_tuning chooses the row kernel's launch
 * shape.
 * events: HOST array of n_real lm_events (device pointers inside); images:
 * DEVICE float[n_real][n*n], lambda^0 in, lambda out; loglik: NULL or DEVICE
 * double[n_real][n_iters*n_subsets].  Every realisation's result equals
 * lm_osem's on its own events bit for bit while each subset's events (all
 * realisations together) fit one row block; beyond that the back
 * projection's event chunks break at row-block edges and results agree to
 * FP32 rounding.  Errors: as lm_osem. */
int lm_osem_batch(lm_handle* h, int n_real, const lm_events* events, int n_subsets, int n_iters,
                  float* images, double* loglik, lm_stream stream);

/* The row-kernel launch shape chosen by the last autotune.  lm_osem and
 * lm_osem_batch time, before their first sub-iteration, launch shapes on a
 * sample of their events (whole angles of the first subset, about 16 384
 * events): every events-per-tile size (32, 64 or 128 for the FP32 form with
 * at most 4 lines, else 128) x work-unit order at the occupancy limit of
 * CTAs per SM, then the best of those with one CTA per SM fewer.  The fastest
 * shape is stored on the handle for the workload class (log2 of the sample's
 * mean events per angle, the scatter model and the precision): each class is
 * timed once per handle, and a call of a class met before takes its stored
 * shape.  Every shape gives bit-identical results.  lm_forward and
 * lm_backproject use the last chosen shape.  out5[0] = work-unit order
 * (0 tile-major, 1 voxel-tile-major), out5[1] = CTAs per SM (0: the
 * occupancy limit), out5[2] = 1 if tuned, out5[3] = the chosen shape's time
 * on the sample (ms), out5[4] = events per tile.  Not part of the paper's
 * method.  Errors: INVALID_ARG. */
int lm_batch_tuning(const lm_handle* h, double* out5);

/* Sets the events per row-kernel tile (32, 64 or 128) for the following
 * calls, until an autotune replaces it; lm_osem and lm_osem_batch keep it
 * while their workload class stays the one last tuned.  Results do not
 * depend on it.  Not part of the paper's method.  Errors: INVALID_ARG. */
int lm_set_tile_events(lm_handle* h, int tile_events);

/* Streamed single-scatter path tables.  The tables the row kernel reads hold
 * the per-path quantities of Eq. (s_p) with n = 1 for every (angle, line,
 * voxel, scatter point): 12 bytes x A x W x Q x P (1.6 GB for 64^2 with a
 * 64^2 scatter grid, 14 GB for 128^2).  The paper computes them per detector
 * angle inside the angle's kernel (Algorithm 1); here they are tabulated
 * once, which costs memory that grows as A W Q P.  With max_angles > 0 the
 * handle keeps the tables of at most max_angles angles: each row launch of
 * lm_forward, lm_backproject and lm_osem covers its angles in blocks of that
 * many, rebuilding a block's tables on the device (the set-up's own kernel,
 * so the values are the same bits) unless they are the resident ones.
 * Results are bit-identical to resident tables.  Each rebuilt angle costs
 * about 0.6 of its share of lm_create's set-up (the sensitivity sums are
 * not repeated): at 64^2 with a 64^2 scatter grid about 15 ms per OSEM
 * iteration, which then takes 33-41 ms instead of 18.
 * max_angles = 0 (or >= n_angles) makes every angle resident again.
 * lm_create streams by itself when all angles' tables do not fit 90 % of the
 * free device memory or the process's table budget (lm_set_table_budget),
 * with as many angles as fit half the free memory (or the budget).
 * Streamed tables serve the exact scatter model of lm_forward,
 * lm_forward_noalloc, lm_backproject and lm_osem; lm_osem keeps the
 * handle's tile size instead of autotuning; the reduced-precision form
 * (lm_set_scatter_precision), lm_osem_batch with the exact model and
 * lm_surrogate_sample return NOT_IMPLEMENTED until the tables are resident
 * again.  The call synchronises the device.  Not part of the paper's
 * method.  Errors: INVALID_ARG (max_angles < 0), NOT_IMPLEMENTED (reduced
 * precision selected), OOM (the new buffer does not fit: the old one is
 * kept). */
int lm_set_table_streaming(lm_handle* h, int max_angles);

/* The table mode: *max_angles = angles the streamed buffer holds (0: every
 * angle resident), *table_bytes = device bytes of the table buffer.  Errors:
 * INVALID_ARG. */
int lm_table_streaming(const lm_handle* h, int* max_angles, int64_t* table_bytes);

/* Process-wide limit in bytes on the path tables lm_create keeps resident;
 * a model whose tables exceed it is created with streamed tables (see
 * lm_set_table_streaming).  0 (the default): only the device's free memory
 * limits them.  Applies to later lm_create calls of every thread.  Not part
 * of the paper's method.  Errors: INVALID_ARG (bytes < 0). */
int lm_set_table_budget(int64_t bytes);

/* Energy-window pruning of the single-scatter terms (on by default).  A
 * photon of line w scattered once leaves with E' between its backscatter
 * energy E_w / (1 + 2 E_w / m_e c^2) and E_w (Compton's relation, paper
 * Sec. "Likelihood of list-mode data using path-based formalism"), and the
 * detector blurs E' by the energy-resolution Gaussian sigma_E(E').  With
 * pruning on, the events of every call are sorted by (angle, energy class,
 * bin); a class is a range of recorded energies in which each line's reach
 * [min (E' - 8 sigma_E(E')), max (E' + 8 sigma_E(E'))] is either wholly in
 * or out, and the row kernel evaluates the single-scatter terms of the lines
 * in reach only.  A skipped term's energy factor is below exp(-32) of its
 * path's peak, so forward projections move by far less than FP32 rounding.
 * enable = 0 evaluates every line for every event (one class).  Applies to
 * the handle's later calls.  Not part of the paper's method.  Errors:
 * INVALID_ARG. */
int lm_set_energy_pruning(lm_handle* h, int enable);

/* ---------------------------------------------------------------------
 * Learned surrogate of the single-scatter term (not in the paper: the
 * paper evaluates Eq. s_p with n = 1 exactly; this replaces that sum by a
 * small network, trained on samples of the exact sum).
 *
 * The network maps 32 inputs of one (event, voxel, line w) -- voxel x, y,
 * detector direction cos/sin, bin centre, recorded energy, line one-hot (up
 * to 3 lines) and the optical depth mu_w(E_w) x (rho line integral from the
 * voxel to the image edge along theta_a + k pi/4, k = 0..7) -- through three
 * 128-wide GELU (tanh form) layers to ln(S_w + 1e-8), S_w the single-scatter
 * part of the system-matrix element for that line.  Weights BF16 for the
 * tensor-core kernels, FP32 masters, Adam.  Parameter vector (FP32):
 * W1[128][32], b1[128], W2[128][128], b2, W3[128][128], b3, w4[128], b4. */
typedef struct lm_surrogate lm_surrogate;

/* Number of FP32 parameters (37 377). */
int lm_surrogate_param_count(void);

/* New network with Xavier-uniform weights drawn from a SplitMix64 stream of
 * `seed`.  Errors: INVALID_ARG, OOM, CUDA. */
int lm_surrogate_create(uint64_t seed, lm_surrogate** out);
int lm_surrogate_destroy(lm_surrogate* s);

/* Copy the FP32 parameters to / from HOST memory (param_count floats). */
int lm_surrogate_get_params(const lm_surrogate* s, float* host_out);
int lm_surrogate_set_params(lm_surrogate* s, const float* host_in);

/* Network outputs for n input rows.  x: DEVICE float[n][32] (rounded to
 * BF16 inside); out: DEVICE float[n].  Asynchronous on the stream. */
int lm_surrogate_forward(lm_surrogate* s, const float* x, int64_t n, float* out, lm_stream stream);

/* Gradient of the weighted mean squared error
 *   L = (1/n) sum_i v_i (net(x_i) - target_i)^2
 * with respect to the parameters.  x: DEVICE float[n][32], target: DEVICE
 * float[n], weight: DEVICE float[n] or NULL (all v_i = 1), grad_out: DEVICE
 * float[param_count]; loss_out: NULL or HOST.  Synchronises the stream. */
int lm_surrogate_gradient(lm_surrogate* s, const float* x, const float* target,
                          const float* weight, int64_t n, float* grad_out, double* loss_out,
                          lm_stream stream);

/* Adam training (beta 0.9 / 0.999, eps 1e-8, bias-corrected) for `steps`
 * minibatches of `batch` rows drawn with replacement from the n DEVICE
 * samples: row i of the minibatch of step k (counted over the surrogate's
 * life) is SplitMix64(seed ^ SplitMix64(k * 0x100000001b3 + i)) mod n, with
 * SplitMix64(z) the generator's output for state z.  Sample weights
 * v_i = exp(weight_power (t_i - max_j t_j)), normalised to mean 1 over the n
 * samples (weight_power 0: unweighted), so that with targets ln(S + eps)
 * the loss counts each sample by (S + eps)^weight_power.  loss_history:
 * NULL or HOST double[steps] (each minibatch's loss before its update; this
 * synchronises every step).  Synchronises the stream.
 * Errors: INVALID_ARG (n <= 0, n >= 2^32, batch not in 1..2^20, lr <= 0,
 * weight_power not in [0, 64]), OOM, CUDA. */
int lm_surrogate_train(lm_surrogate* s, const float* x, const float* target, int64_t n, int steps,
                       int batch, float lr, float weight_power, uint64_t seed,
                       double* loss_history, lm_stream stream);

/* n training samples from a model: events drawn uniformly from `events`
 * (device), voxels uniformly from the support, lines uniformly; x_out:
 * DEVICE float[n][32] inputs, target_out: DEVICE float[n] = ln(S_w + 1e-8)
 * with S_w the exact single-scatter sum of the model's tables (FP32 terms,
 * FP64 sum).  SplitMix64 of `seed`.  Errors: INVALID_ARG, NOT_IMPLEMENTED
 * (more than 3 lines), CUDA. */
int lm_surrogate_sample(lm_handle* h, const lm_events* events, int64_t n, uint64_t seed,
                        float* x_out, float* target_out, lm_stream stream);

/* Scatter model of the handle's later lm_forward / lm_osem calls:
 * LMMEW_SCATTER_EXACT (default, s ignored), LMMEW_SCATTER_SURROGATE (the
 * network s, evaluated for every (event, voxel, line); s must outlive its
 * use), LMMEW_SCATTER_NONE (unscattered paths only: the method without a
 * scatter model), LMMEW_SCATTER_SURROGATE_COARSE (the network s evaluated on
 * a half-resolution grid of emission positions and interpolated: see below).
 * The coarse form evaluates the network at the support voxels whose pixel
 * coordinates are both multiples of the node stride s (2 by default, see
 * lm_set_coarse_stride), and at any support voxel none of whose four
 * surrounding nodes is in the support, and gives every other voxel the
 * bilinear interpolation of its surrounding nodes that lie in the support,
 * the weights renormalised to sum to 1.  About 1/s^2 of the network
 * evaluations; the single-scatter part is smooth in the emission position,
 * and at 0.6 cm pixels the interpolation moves forward projections by about
 * 0.4 % on average with s = 2, 0.9 % with s = 3.  Not part of the paper's
 * method.
 * Errors: INVALID_ARG, NOT_IMPLEMENTED (surrogate with more than 3 lines),
 * OOM, CUDA. */
#define LMMEW_SCATTER_EXACT 0
#define LMMEW_SCATTER_SURROGATE 1
#define LMMEW_SCATTER_NONE 2
#define LMMEW_SCATTER_SURROGATE_COARSE 3
int lm_set_scatter_model(lm_handle* h, int model, const lm_surrogate* s);

/* Node stride s (2, 3 or 4 pixels) of the coarse-grid surrogate for the
 * handle's later calls (default 2); the node tables are rebuilt.  Not part
 * of the paper's method.  Errors: INVALID_ARG, OOM, CUDA. */
int lm_set_coarse_stride(lm_handle* h, int stride);

/* Free every device buffer of the handle (NULL is ignored). */
int lm_destroy(lm_handle* h);

/* Message describing the calling thread's last error ("" if none). */
const char* lm_last_error(void);

/* Row-kernel timing, for throughput accounting (an instrument of this
 * library, not part of the paper's method).  While enabled, CUDA events are
 * recorded on the caller's stream around every launch of the fused
 * system-matrix row kernel.  lm_profile_read synchronises those events and
 * writes out5[0] = total row-kernel time in ms, out5[1] = row-kernel
 * launches, out5[2] = exponentials those launches evaluated for real
 * (event, voxel) pairs -- one per path term whose collimator factor is not
 * an exact zero -- counted on the device, out5[3] = system-matrix elements
 * (events x support voxels),
 * out5[4] = kernels of every kind this handle launched (counted whether or
 * not timing is enabled); then it resets the counters.
 * Errors: INVALID_ARG, CUDA. */
int lm_profile_enable(lm_handle* h, int enable);
int lm_profile_read(lm_handle* h, double* out5);

/* Model sizes, for work accounting: out8[0] = voxels in the support,
 * out8[1] = scatter points with rho > 0, out8[2] = emission lines,
 * out8[3] = angles, out8[4] = bins, out8[5] = exponentials per event row,
 * out8[6] = bytes of device tables, out8[7] = set-up time in microseconds. */
int lm_model_info(const lm_handle* h, int64_t* out8);

/* Exponential throughput of the current GPU (an instrument of this library,
 * not part of the paper's method): times kernels of independent dependent
 * chains of ex2.approx.ftz.f32, ex2.approx.f16x2 and ex2.approx.ftz.bf16x2
 * on every SM and writes out4[0..2] = exponential results per clock per SM
 * for each (two results per packed instruction), out4[3] = the SM clock in
 * MHz the rates refer to (the device's maximum).  Synchronises the stream;
 * allocates and frees 1 MiB of device memory.  Errors: INVALID_ARG, CUDA. */
int lm_probe_ex2_rate(lm_stream stream, double* out4);

/* Self-test of the bounded waits of the pipelined kernels (an instrument of
 * this library): launches one warp that waits, through the same bounded wait
 * the row and tensor-core kernels use, on an mbarrier nothing arrives on.
 * The wait gives up after its limit (2 s), the kernel sets the timeout status
 * and returns; nothing stays in flight and the context remains usable.
 * Writes the time waited (ms) to *waited_ms and returns LMMEW_ERR_TIMEOUT (the
 * expected outcome); any other code means the wait did not behave.
 * Synchronises the device. */
int lm_selftest_wait_timeout(double* waited_ms);

#ifdef __cplusplus
}
#endif
#endif /* LMMEW_H */
