/*
 * lmosem: list-mode OS-LM-MLEM attenuation and scatter compensation for 2-D
 * SPECT on one GB300 (sm_103a).
 *
 * Method: Rahman, Laforest, Jha, "A list-mode OSEM-based attenuation and
 * scatter compensation method for SPECT", ISBI 2020 (arXiv:2002.12471).
 *
 * C ABI.  Plain pointers and sizes only.  Conventions:
 *  - Pointers named d_* are CUDA device memory owned by the caller; h_* are
 *    host memory owned by the caller.  The context copies what it keeps and
 *    owns every buffer it allocates (freed by lmosem_destroy).
 *  - All device work is enqueued on the stream given to lmosem_create.  A
 *    call returns once its work is enqueued, except where it must read a
 *    result back (noted per function); those calls synchronise the stream.
 *  - Every function returns a status code; none throws or aborts.  After an
 *    error lmosem_last_error(ctx) holds a one-line message.  A context is not
 *    thread-safe.
 *  - The image is a vector over the emission support: d_f[q] is the activity
 *    of pixel support[q] (see lmosem_support).  Support and scatter pixels are
 *    listed in increasing row-major pixel index (pixel n = iy * nx + ix).
 *
 * Geometry (the model's frozen reading of the scanner, paper Section 3):
 *  pixel (ix, iy) has centre ((ix + 1/2 - nx/2) D, (iy + 1/2 - ny/2) D);
 *  detector angle a has theta_a = angle0 + 2 pi a / n_angles, photons reach
 *  it travelling along omega_a = (cos, sin) theta_a; the event position is
 *  u = p . (-sin theta_a, cos theta_a), continuous, |u| <= n_bins bin_mm / 2;
 *  depth d = R - p . omega_a sets the collimator response
 *  FWHM_u = coll_fwhm0 + coll_fwhm_slope d.  Energy resolution is
 *  FWHM_E(E) = fwhm_frac_e0 sqrt(E0 E); events outside [e_lo, e_hi] are not
 *  acquired.
 */
#ifndef LMOSEM_H
#define LMOSEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LMOSEM_OK = 0,
    LMOSEM_EINVAL = 1,   /* an argument is out of range; nothing was enqueued      */
    LMOSEM_ENOMEM = 2,   /* a device allocation failed                              */
    LMOSEM_ECUDA = 3,    /* a CUDA call failed (message holds the CUDA error)       */
    LMOSEM_ETIMEOUT = 4, /* a bounded device wait ran out                           */
    LMOSEM_ENUMERIC = 5, /* a non-finite value appeared in the image                */
    LMOSEM_ESTATE = 6,   /* called out of order (e.g. iterate before build_model)   */
    LMOSEM_ENOTIMPL = 7  /* the requested form is not built                         */
} lmosem_status;

typedef struct lmosem_ctx lmosem_ctx; /* opaque; owns all device buffers */

/* Object: the mu-map at the photopeak energy (a CT-derived attenuation map;
 * paper Section 1) and the emission support (paper Section 2.2: the cost scales
 * with the number of non-zero voxels N_nz). */
typedef struct {
    int32_t nx, ny;          /* grid size, 1..2048 each                           */
    double pixel_mm;         /* pixel pitch D > 0                                 */
    const double* h_mu_per_mm; /* host, ny*nx row-major, finite, >= 0             */
    const uint8_t* h_support;  /* host, ny*nx, nonzero = emission pixel;
                                  NULL selects {mu > 0}                            */
} lmosem_object;

typedef struct {
    int32_t n_angles;        /* >= 1                                              */
    double angle0_rad;
    int32_t n_bins;          /* detector extent n_bins * bin_mm                   */
    double bin_mm;
    double radius_mm;        /* > distance of every support/scatter pixel centre  */
    double coll_fwhm0_mm;    /* > 0                                               */
    double coll_fwhm_slope;  /* >= 0                                              */
} lmosem_geometry;

typedef struct {
    double e0_kev;           /* photopeak (159 keV for I-123)                      */
    double fwhm_frac_e0;     /* energy FWHM at E0 / E0, > 0                        */
    double e_lo_kev, e_hi_kev; /* acquisition window, e_lo < e_hi                  */
} lmosem_energy;

typedef struct {
    /* Scatter paths (n, m) whose position kernel is evaluated farther than
     * k_sigma collimator sigmas from the event are left out of p_jn.
     * 0 selects the default 6 (entries change by < 3e-7 of the row maximum). */
    float k_sigma;
    /* Upper bound (bytes) of the per-angle scatter-weight tables kept on the
     * device while a model is built; 0 selects 4 GiB. */
    int64_t table_budget_bytes;
    /* Kernel timing for benchmarks.  1: bracket every kernel launch with
     * CUDA events on the context stream so that lmosem_profile_read can
     * report device time per kernel class (OSEM iterations are then launched
     * one kernel at a time).  2: the same, except that OSEM iterations keep
     * their CUDA-graph replay on non-default streams and are not timed. */
    int32_t profile;
    /* Clock-cycle budget of every bounded device wait (the mbarrier waits of
     * the TMA-ring OSEM pass, the tensor-core surrogate and the batch
     * scheduler's work queue; the path sum and the other passes wait only at
     * CTA barriers); 0 selects 2e9 (about one second).
     * A wait that runs out abandons its kernel and the call returns
     * LMOSEM_ETIMEOUT; the context stays usable.  Tests set a tiny budget
     * (here or with lmosem_set_wait_budget) to exercise that path. */
    int64_t wait_budget_cycles;
    /* Streaming-pass implementation (tuning knobs; 0 = automatic, which is
     * 1): 1 = rows double-buffered in registers, 2 = rows staged in a
     * shared-memory ring by bulk (TMA) copies, ring_rows rows per stage
     * (1..8) and ring_stages stages (2..8), 3 = each thread's row vectors
     * staged in its own slots of a shared-memory ring by cp.async (several
     * row groups in flight, the arithmetic of 1), 4 = every sub-iteration of
     * the call in one persistent cooperative launch: the ring of 3, a
     * bounded grid barrier, the update of each CTA's slice of the support,
     * a second barrier, and the copies of the next subset's rows in flight
     * across both barriers. */
    int32_t pass_variant;
    int32_t ring_rows;
    int32_t ring_stages;
    /* Scatter-surrogate inference: 0 = automatic (2), 1 = the chain of
     * separate tcgen05 products that training uses (activations through
     * HBM), 2 = fused tcgen05 kernel (one persistent CTA per SM, activations
     * kept on chip, TMEM accumulators). */
    int32_t surrogate_kernel;
    /* Register pass (pass_variant 1): row groups fetched into L2 ahead of
     * their register loads by bulk prefetches, this many groups ahead;
     * -1 = none, 0 = automatic (rows wide enough to be processed one at a
     * time: about 48 KB ahead per CTA; none otherwise), 1..16. */
    int32_t prefetch_groups;
    /* Energy cut of the scatter terms: a term U_jm W_a(n, m) phi(E_j; E', sigma_E)
     * of the sum of paper Eq. 2 is left out when the event energy E_j lies
     * farther than e_sigma energy sigmas sigma_E(E') from the Compton energy
     * E'_a(n', m) of every support pixel n' of the 128-pixel column tile
     * that holds n.  Every term left out is below 2^(-e_sigma^2 log2(e) / 2)
     * of its value at E_j = E' (1.5e-8 at 6).  0 selects the default 6;
     * a negative value keeps every term (the exact sum); EINVAL above 20. */
    float e_sigma;
} lmosem_options;

/* Kernel classes reported by lmosem_profile_read. */
typedef enum {
    LMOSEM_K_TABLES = 0,   /* attenuation line integrals and per-angle parameters */
    LMOSEM_K_SORT = 1,     /* event check and (subset, angle, class, position) sort */
    LMOSEM_K_WTABLE = 2,   /* per-angle scatter weight tables                     */
    LMOSEM_K_PATHSUM = 3,  /* per-event path-sum model build                      */
    LMOSEM_K_QUANTIZE = 4, /* row scaling to FP16/BF16                            */
    LMOSEM_K_SENS = 5,     /* subset sensitivities                                */
    LMOSEM_K_PASS = 6,     /* streaming OSEM pass (forward, back-projection, LL)  */
    LMOSEM_K_UPDATE = 7,   /* per-subset reduction and multiplicative update      */
    LMOSEM_K_OTHER = 8,
    LMOSEM_K_SURROGATE = 9, /* scatter surrogate: features, loss, Adam, combine */
    LMOSEM_K_MLP = 10,      /* scatter surrogate: the MLP products (tensor cores) */
    LMOSEM_K_COUNT = 11
} lmosem_kernel_class;

typedef enum {
    LMOSEM_MODEL_FP32 = 0,          /* p_jn cached as FP32                           */
    LMOSEM_MODEL_FP16_SCALED = 1,   /* p_jn = c_j h_jn, h FP16 with max_n h = 2^15   */
    LMOSEM_MODEL_BF16_SCALED = 2,   /* p_jn = c_j h_jn, h BF16 with max_n h = 1      */
    LMOSEM_MODEL_SURROGATE_FP32 = 3 /* FP32; scatter part from the loaded surrogate  */
} lmosem_model_fmt;

/* Scatter surrogate parameters: one FP32 blob of LMOSEM_SURROGATE_PARAMS
 * values, in this order: W1 (256 x 8, row-major, out x in), b1 (256), W2, b2,
 * W3, b3 (256 x 256, 256), W4, b4, W5 (1 x 256), b5 (1), the 28 coefficients
 * c of a quadratic baseline, mu, sigma.  The network (ReLU after every hidden
 * layer) maps eight inputs x, the event and the pixel in the detector frame
 * of the event's angle theta (omega = (cos theta, sin theta), t = (-sin theta,
 * cos theta), p the pixel centre, u_a(p) = p.t, mu the map at E0):
 *   (u - u_a(p)) / 50 mm, p.omega / 100 mm, u_a(p) / 100 mm,
 *   (theta - pi) / pi, (E - 137.5 keV) / 37.5 keV,
 *   (integral of mu from the pixel centre to the grid edge along omega - 1.5) / 1.5,
 *   (integral of mu along the event's line {s omega + u t} from s = p.omega
 *    on, towards the detector - 1.5) / 1.5,
 *   (integral of mu along that whole line - 1.5) / 1.5,
 * to y with
 *   log p^scat_jn = c . phi(x) + mu + sigma y   (natural log),
 * phi(x) = (1, x_1 .. x_6, x_i x_k for i <= k <= 6) in that order.  The two
 * line integrals are interpolated bilinearly in u and s from exact integrals
 * at nodes half a pixel apart.  A blob with zero coefficients is the network
 * alone. */
#define LMOSEM_SURROGATE_PARAMS 199967

/* Create a context: validate the problem, copy the mu-map and support to the
 * device and build the attenuation tables (integrals of mu along omega_a from
 * every pixel centre to the grid edge, and between every support and scatter
 * pixel centre; Siddon's ray parametrisation).  Synchronises the stream.
 * opts may be NULL.  stream is a cudaStream_t (NULL = legacy default stream).
 * EINVAL: any field out of the ranges above, empty support, radius too small. */
lmosem_status lmosem_create(const lmosem_object* obj, const lmosem_geometry* geom,
                            const lmosem_energy* energy, const lmosem_options* opts,
                            void* stream, lmosem_ctx** out);

void lmosem_destroy(lmosem_ctx* ctx);

const char* lmosem_last_error(const lmosem_ctx* ctx);
const char* lmosem_status_string(lmosem_status st);

/* Number of emission-support pixels N_nz and of scatter pixels {mu > 0}. */
int32_t lmosem_n_support(const lmosem_ctx* ctx);
int32_t lmosem_n_scatter(const lmosem_ctx* ctx);

/* Copy the support pixel indices (N_nz int32, increasing) to host memory. */
lmosem_status lmosem_support(const lmosem_ctx* ctx, int32_t* h_out);

/* Subset sensitivities s^i_q (denominator of paper Eq. 7, without T): the
 * probability that a photon emitted in support pixel q is acquired at an
 * angle of subset i, summed over the primary path and every first-order
 * in-plane scatter path.  Subset i holds the angles a with a mod n_subsets
 * == i.  Terms in FP32, accumulation in FP64.  Kept in the context; also
 * copied to d_sens (n_subsets x N_nz FP64, row-major) when d_sens != NULL.
 * EINVAL: n_subsets not in [1, n_angles]. */
lmosem_status lmosem_sensitivity(lmosem_ctx* ctx, int32_t n_subsets, double* d_sens);

/* Build and cache the list-mode system model for J events (paper Eq. 2 with
 * Eq. 4: p_jq = sum over paths P from pixel q of pr(A_j|P) s_eff(P), the
 * primary path plus every first-order in-plane Compton path (q, m) with
 * attenuation, Klein-Nishina weight, energy blur and collimator response).
 * Events are three device arrays of length n_events (angle index, position
 * in mm, energy in keV).  The context sorts them by (subset, angle, energy
 * class, u), the class splitting at E0 (1 - fwhm_frac_e0 / 2), and keeps
 * the sorted copy; the caller's arrays are not modified and may be
 * freed on return.  Synchronises the stream (input check).
 * EINVAL: n_events < 1 or >= 2^31, n_subsets not in [1, n_angles], an angle
 * outside [0, n_angles), |u| > extent/2, E outside [e_lo, e_hi], NaN.
 * ENOMEM: the model does not fit.  Any earlier model is released first. */
lmosem_status lmosem_build_model(lmosem_ctx* ctx, const int32_t* d_angle, const float* d_u_mm,
                                 const float* d_e_kev, int64_t n_events, int32_t n_subsets,
                                 lmosem_model_fmt fmt);

/* Binned form (the paper's binning experiment, Section 4): the data are
 * photon counts per (angle, detector position bin, energy bin) instead of a
 * list of events.  Position bins are the detector's n_bins bins of bin_mm;
 * energy bin k is [h_e_edges[k], h_e_edges[k + 1]].  A row of the model is a
 * bin with a positive count, and its model is the event model integrated
 * over the bin: p_iq = the probability that an emission in pixel q is
 * detected at the bin's angle with position and energy inside the bin (each
 * Gaussian density of lmosem_build_model replaced by its mass on the bin).
 * lmosem_init_image, lmosem_iterate and lmosem_loglik then weight every row
 * by its count (a bin holding n_i photons acts as n_i identical events), and
 * lmosem_model_rows takes the ordinals of the positive bins in dense
 * (angle, position bin, energy bin) order.  FP32 model only.
 * d_counts: device float32 [n_angles][n_bins][n_ebins], finite, >= 0.
 * h_e_edges: host, n_ebins + 1 increasing energies; the first must equal the
 * window's e_lo and the last its e_hi (relative 1e-9), so that the bins tile
 * the window the sensitivity integrates over.  Synchronises the stream.
 * EINVAL: n_ebins not in 1..8, bad edges, a negative or non-finite count, no
 * positive count, n_subsets not in [1, n_angles].  ENOTIMPL: fmt other than
 * FP32.  Any earlier model is released first. */
lmosem_status lmosem_build_model_binned(lmosem_ctx* ctx, const float* d_counts, int32_t n_ebins,
                                        const double* h_e_edges, int32_t n_subsets,
                                        lmosem_model_fmt fmt);

/* Batching form: one model for n_real independent list-mode data sets (noise
 * realisations; the paper repeats its study over multiple noise realisations,
 * Section 3) of the same object and scanner.  The events of realisation r are
 * d_*[h_event_offsets[r] .. h_event_offsets[r+1]) (host offsets, n_real + 1,
 * from 0, not decreasing; realisations may differ in size and may be empty).
 * The model is FP32 (ENOTIMPL for the scaled formats).  Afterwards use the
 * *_batch calls; the single-data-set calls return ESTATE.  Synchronises.
 * EINVAL: as lmosem_build_model, or n_real outside 1..1536, bad offsets. */
lmosem_status lmosem_build_model_batch(lmosem_ctx* ctx, const int32_t* d_angle, const float* d_u_mm,
                                       const float* d_e_kev, const int64_t* h_event_offsets,
                                       int32_t n_real, int32_t n_subsets, lmosem_model_fmt fmt);

/* Starting images of a batched model: d_f[r * N_nz + q] = J_r / (T sum s). */
lmosem_status lmosem_init_image_batch(lmosem_ctx* ctx, double acq_time, float* d_f);

/* n_iters OS-LM-MLEM iterations (paper Eqs. 7-9) of every realisation, all in
 * one persistent kernel launch (replayed as a CUDA graph on a non-default
 * stream).  d_f: n_real x N_nz FP32 images, updated in place.  The rows of a
 * (realisation, subset) are split into chunks of the tile size set by
 * lmosem_set_batch_tiles / lmosem_autotune_batch (default 512 rows, 2 CTAs
 * per SM).  Synchronises.  ETIMEOUT: a bounded wait of the persistent kernel
 * ran out (images then partly updated). */
lmosem_status lmosem_iterate_batch(lmosem_ctx* ctx, int32_t n_iters, double acq_time, float* d_f);

/* Autotuner of the batched iterations: times one iteration of every
 * (chunk rows in {128..2048}, CTAs per SM in {1..4}) candidate on a scratch
 * copy of d_f (not modified), keeps the fastest for this context and writes
 * it to h_choice[0..1] (may be NULL).  Synchronises. */
lmosem_status lmosem_autotune_batch(lmosem_ctx* ctx, double acq_time, const float* d_f,
                                    int32_t* h_choice);

/* Set the batched tiles directly (e.g. a choice cached from an earlier
 * autotuning): chunk_rows in [8, 2^20], ctas_per_sm in [1, 16]. */
lmosem_status lmosem_set_batch_tiles(lmosem_ctx* ctx, int32_t chunk_rows, int32_t ctas_per_sm);

/* Support initialiser (paper Sec. 2.2, last paragraph: the cost grows with
 * the non-zero voxels, so the object's boundary is first estimated from a
 * crude OSEM reconstruction of the binned data).  Bins the events into the
 * sinogram (angle x position bin, every energy of the window), reconstructs
 * it over the whole grid with a crude projector (collimator response
 * integrated over each bin; no attenuation, scatter or energy) by n_iters
 * iterations of OSEM with n_subsets angle subsets (a mod n_subsets), and
 * writes h_support[n] = 1 for the pixels within `dilate` pixels (square
 * neighbourhood) of one with f_n >= threshold * max f, else 0 (host,
 * nx * ny bytes, row-major; pass it to lmosem_create of the reconstruction).
 * d_image (device, nx * ny FP32, may be NULL) receives the crude image.  The
 * context's own support is not used.  Synchronises.  EINVAL for events out
 * of range (as lmosem_build_model) or arguments outside 1 <= n_subsets <=
 * n_angles, 1 <= n_iters <= 1000, 0 < threshold <= 1, 0 <= dilate <= 8. */
lmosem_status lmosem_binned_support(lmosem_ctx* ctx, const int32_t* d_angle, const float* d_u_mm,
                                    const float* d_e_kev, int64_t n_events, int32_t n_subsets, int32_t n_iters,
                                    double threshold, int32_t dilate, uint8_t* h_support, float* d_image);

/* Scatter surrogate (the learned form of the first-order scatter sum of paper
 * Eq. 2; the paper itself evaluates that sum exactly).
 *
 * Training samples: builds the exact model of the given events with the
 * primary path left out (replacing any cached model, which is released
 * afterwards) and writes, for every (event k, support pixel q) at row
 * k * N_nz + q: the eight scaled inputs (d_features, 8 floats per row) and the
 * natural log of the exact scatter entry (d_log_scatter; entries below 1e-30
 * are clamped).  d_rel_log (may be NULL) receives each entry's log minus the
 * largest log of its event's row (<= 0), which lmosem_surrogate_train can use
 * to draw training pairs in proportion to their share of their row: the EM
 * update weighs every event alike, and most pairs of a row carry little of
 * it.  Synchronises.  EINVAL as lmosem_build_model. */
lmosem_status lmosem_surrogate_samples(lmosem_ctx* ctx, const int32_t* d_angle, const float* d_u_mm,
                                       const float* d_e_kev, int64_t n_events, float* d_features,
                                       float* d_log_scatter, float* d_rel_log);

typedef struct {
    int32_t steps;     /* Adam steps (>= 1)                                        */
    int32_t batch;     /* rows per minibatch, multiple of 64, 64..65536            */
    float lr;          /* learning rate (the last 20% of the steps use lr / 10)    */
    uint64_t seed;     /* minibatch sampling (rows drawn with replacement)         */
    float target_floor; /* > 0: targets below (largest target - target_floor) are
                         * raised to that level, so that the fit is spent on the
                         * entries that carry the model (log units); with
                         * d_rel_log the largest target of the same event's row
                         * (every event then keeps its row's shape); 0: none     */
    int32_t residual_fit; /* 1: fit the quadratic baseline to the (floored) targets
                           * by least squares first and train the network on the
                           * residual; 0: zero baseline                           */
    float magnitude_power; /* alpha > 0 with d_rel_log: minibatch rows drawn with
                            * probability proportional to exp(alpha rel_log), i.e.
                            * (entry / largest entry of its row)^alpha; 0: uniform */
} lmosem_train_opts;

/* Train the surrogate on n samples (features n x 8, targets n = log scatter,
 * d_rel_log n or NULL: see lmosem_surrogate_samples and magnitude_power)
 * with the library's tensor-core forward and backward kernels and Adam (FP32
 * parameters and moments, BF16 products, FP32 accumulation).  d_weights holds
 * the initial parameters on entry (the baseline coefficients are refitted or
 * zeroed, and mu and sigma recomputed from the (floored) targets minus the
 * baseline) and the trained ones on return.  h_loss_curve (steps doubles, may
 * be NULL) receives the minibatch loss of every step.  Synchronises. */
lmosem_status lmosem_surrogate_train(lmosem_ctx* ctx, const float* d_features, const float* d_targets,
                                     const float* d_rel_log, int64_t n, const lmosem_train_opts* opts,
                                     float* d_weights, double* h_loss_curve);

/* Gradient of the mean squared error of the network output against the
 * standardised targets ((t - mu) / sigma with the blob's mu, sigma) over all
 * n rows (n <= 65536), in the blob layout (mu, sigma entries zero), and the
 * loss in *h_loss.  Synchronises. */
lmosem_status lmosem_surrogate_grad(lmosem_ctx* ctx, const float* d_weights, const float* d_features,
                                    const float* d_targets, int64_t n, float* d_grad, double* h_loss);

/* Network output y for n rows of scaled inputs (log p^scat = mu + sigma y).
 * Synchronises. */
lmosem_status lmosem_surrogate_infer(lmosem_ctx* ctx, const float* d_weights, const float* d_features,
                                     int64_t n, float* d_out);

/* Copy trained parameters into the context for LMOSEM_MODEL_SURROGATE_FP32
 * model builds. */
lmosem_status lmosem_surrogate_load(lmosem_ctx* ctx, const float* d_weights);

/* The exact path sum as the judge and the fallback of the surrogate form.
 * The surrogate replaces the first-order scatter sum of paper Eq. 2 (with
 * Eq. 4; Section 2.2), so every LMOSEM_MODEL_SURROGATE_FP32 build is checked
 * against that sum: n_check_rows sorted rows, evenly spaced over the model
 * (row (k + 1/2) J / K of K, so every subset and angle group is sampled),
 * are rebuilt with the exact path sum and compared with the surrogate's
 * rows.  When the relative L2 error over those rows exceeds tol (taken after
 * the energy gate of lmosem_set_surrogate_gate, when it is on), the build
 * replaces the whole model with the exact path sum.  tol = 0: measure only,
 * never rebuild.  Defaults: tol 1e-2, 512 rows (0 selects 512).  Applies to
 * the builds that follow.  EINVAL: tol negative or not finite, n_check_rows
 * not in [0, 65536]. */
lmosem_status lmosem_set_surrogate_check(lmosem_ctx* ctx, double tol, int32_t n_check_rows);

/* Result of the check of the current model (see lmosem_set_surrogate_check):
 * *h_rel_err = relative L2 error of the sampled surrogate rows against the
 * exact ones, *h_row_max = the largest per-row relative L2 error, *h_exact =
 * 1 when the check rebuilt the model with the exact path sum (the model then
 * holds exact FP32 rows), 0 when it holds the surrogate's rows.  Any pointer
 * may be NULL.  ESTATE: the current model was not built in the surrogate
 * form. */
lmosem_status lmosem_surrogate_check(const lmosem_ctx* ctx, double* h_rel_err, double* h_row_max,
                                     int32_t* h_exact);

/* Energy gate of the surrogate form: the exact path sum as a per-energy
 * fallback.  The surrogate replaces the first-order scatter sum of paper Eq. 2
 * (Section 2.2); its error is largest for events well below the photopeak,
 * whose rows are almost all scatter, and the EM update (Eq. 8) weighs every
 * event's row alike.  With row_tol > 0 (and the check of
 * lmosem_set_surrogate_check on), the network builds the check's sampled
 * rows first and the check groups them in energy bins of bin_kev from the
 * window's lower edge; the highest bin whose mean per-row relative L2 error
 * exceeds row_tol marks the cut.  Every model row whose event energy lies
 * below the top of that bin is then built by the exact path sum (bitwise the
 * exact build's row), the others by the network, and the check's error is
 * taken with the former exact.  The exact rows pass through device scratch of
 * at most 8 GiB at a time (ENOMEM from the build when that does not fit).  row_tol = 0: off
 * (the default).  bin_kev = 0 selects 5 keV.  Applies to the builds that
 * follow.  EINVAL: a negative or non-finite argument. */
lmosem_status lmosem_set_surrogate_gate(lmosem_ctx* ctx, double row_tol, double bin_kev);

/* Result of the energy gate of the current surrogate-form model:
 * *h_e_cut_kev = the energy below which rows are exact (the window's lower
 * edge when none are; its upper edge when all are), *h_frac_exact = the
 * fraction of the model's rows that hold the exact path sum (1 after a whole
 * rebuild by the check).  Any pointer may be NULL.  ESTATE: the current model
 * was not built in the surrogate form. */
lmosem_status lmosem_surrogate_gate(const lmosem_ctx* ctx, double* h_e_cut_kev, double* h_frac_exact);

/* Uniform starting image on the support, T sum_q s_q f_q = J (FP32, N_nz);
 * J is the number of events, or the sum of the counts of a binned model.
 * ESTATE: no model or sensitivity. */
lmosem_status lmosem_init_image(lmosem_ctx* ctx, double acq_time, float* d_f);

/* n_iters global OS-LM-MLEM iterations (paper Eqs. 7-9): for every subset i
 * in index order, y_j = sum_q p_jq f_q over the subset's events, then
 * f_q <- f_q sum_j p_jq / y_j / (T s^i_q) (events with y_j = 0 add nothing;
 * f_q = 0 where s^i_q = 0).  d_f (N_nz FP32) is updated in place.  When
 * d_loglik != NULL, d_loglik[t] (FP64, device) receives the log-likelihood
 * of paper Eq. 3 (without log J!) of the image after iteration t; this costs
 * one extra read of the model per iteration.
 * ESTATE: no model, or the sensitivity was computed for another subset count. */
lmosem_status lmosem_iterate(lmosem_ctx* ctx, int32_t n_iters, double acq_time, float* d_f,
                             double* d_loglik);

/* The expected count of every subset for the image d_f: d_out[i] =
 * T sum_q s^i_q f_q (FP64, fixed-order reduction), n_subsets values.  Right
 * after the sub-iteration of subset i this equals the number of its events
 * (or the sum of its counts) with y_j > 0: the count conservation of the EM
 * update (paper Eq. 7), a cheap check of a reconstruction.
 * ESTATE: no sensitivity for the model's subset count. */
lmosem_status lmosem_subset_totals(lmosem_ctx* ctx, double acq_time, const float* d_f, double* d_out);

/* Log-likelihood of paper Eq. 3 (without log J!) of the image d_f:
 * sum_j log(T y_j) - T sum_q s_q f_q, FP64 reduction, into d_out[0]. */
lmosem_status lmosem_loglik(lmosem_ctx* ctx, double acq_time, const float* d_f, double* d_out);

/* One whole reconstruction from host buffers, the end-to-end call of the
 * library: copies the n_events events (host arrays as for lmosem_build_model;
 * pinned memory makes the copies asynchronous, pageable memory also works) to
 * the device on the context stream, computes the subset sensitivities, builds
 * and caches the model in format fmt, starts from the uniform image, runs
 * n_iters OS-LM-MLEM iterations (paper Eqs. 7-9) and copies the image
 * (N_nz FP32) to h_f and, when h_loglik != NULL, the log-likelihood of paper
 * Eq. 3 (without log J!) of that image to h_loglik[0].  The model and the
 * sensitivity stay in the context; the device copies of the events and the
 * image are released.  Synchronises.  Errors as lmosem_sensitivity,
 * lmosem_build_model, lmosem_iterate and lmosem_loglik; h_f is written only
 * on success. */
lmosem_status lmosem_reconstruct(lmosem_ctx* ctx, const int32_t* h_angle, const float* h_u_mm,
                                 const float* h_e_kev, int64_t n_events, int32_t n_subsets,
                                 lmosem_model_fmt fmt, int32_t n_iters, double acq_time, float* h_f,
                                 double* h_loglik);

/* Copy model rows back as FP32 (dequantised for the scaled forms):
 * d_out[k * N_nz + q] = p_{j_k, q} for the caller's original event indices
 * j_k = d_event_ids[k] (device int64, each in [0, J)).  For tests and tools. */
lmosem_status lmosem_model_rows(lmosem_ctx* ctx, const int64_t* d_event_ids, int64_t n,
                                float* d_out);

/* Bytes of the cached model (rows x padded columns x element size + scales). */
int64_t lmosem_model_bytes(const lmosem_ctx* ctx);

/* Number of kernel launches this context has enqueued so far. */
int64_t lmosem_launch_count(const lmosem_ctx* ctx);

/* Path terms that the path-sum kernels formed in their last row build on
 * this context (paper Eq. 2 with Eq. 4: one term per (event, support pixel)
 * for the primary path and one per (event, support pixel, scatter pixel)
 * whose term the position cut (k_sigma) and the energy cut (e_sigma) keep).
 * After lmosem_build_model or lmosem_build_model_batch with an FP32, FP16
 * or BF16 format that is the whole model.  A surrogate build runs the path
 * sum on the rows its exact judge and energy gate recompute, one set of
 * rows at a time, and the count covers the last such set.  Padding columns
 * are not counted.  Synchronises the context stream.  EINVAL: the path sum
 * has not run on this context. */
lmosem_status lmosem_model_terms(lmosem_ctx* ctx, int64_t* h_terms);

/* Change the clock-cycle budget of the bounded device waits (see
 * lmosem_options.wait_budget_cycles; 0 restores 2e9) for the calls that
 * follow, e.g. to let a test build the model and then make one pass time
 * out.  EINVAL: negative budget. */
lmosem_status lmosem_set_wait_budget(lmosem_ctx* ctx, int64_t cycles);

/* Measured throughput of the exponential unit (ex2.approx.ftz.f32 per
 * second on the current device): grid = SMs x ctas_per_sm CTAs of `threads`
 * threads, each running 8 independent chains of `iters` steps (one ex2 and
 * one FP32 add per step), timed with CUDA events after one warm-up launch on
 * `stream`.  The paper has no counterpart; the path sum of Eq. 2 costs one
 * ex2 per term, so this rate bounds it.  Synchronises.  EINVAL: ctas_per_sm
 * not in 1..32, threads not a multiple of 32 in 32..1024, iters not in
 * 1..2^32, NULL output.  ECUDA: a launch or the timing failed. */
lmosem_status lmosem_measure_ex2_rate(void* stream, int32_t ctas_per_sm, int32_t threads, int64_t iters,
                                      double* h_per_second);

/* Device time (ms) and launch count per kernel class since the last read,
 * from the CUDA events of a context created with opts->profile != 0.
 * h_ms and h_launches hold LMOSEM_K_COUNT entries.  Synchronises the stream.
 * ESTATE: profiling is off. */
lmosem_status lmosem_profile_read(lmosem_ctx* ctx, double* h_ms, int64_t* h_launches);

/* One OS-LM-MLEM sub-iteration that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc or cudaFree, for example an application whose own
 * allocator owns all device memory, or a processing loop that must not make
 * calls that can synchronise the whole device.  It needs no context: the
 * caller passes the model rows of one subset and the image, and the per-CTA
 * partial back-projections use a 4 MiB array of static device memory that
 * the library reserves on every GPU that loads it, until the process exits.
 *
 *   d_rows     device, n_rows x ld FP32 model rows p_jq of the subset's
 *              events (row-major, 16-byte aligned, ld a multiple of 4 and at
 *              most 8192); columns n_support..ld-1 are read and multiplied by
 *              zero, so they must hold finite values (zeros recommended)
 *   d_f        device, n_support FP32 image, updated in place:
 *              f_q <- f_q sum_j p_jq / y_j / (T s_q), y_j = sum_q p_jq f_q;
 *              rows with y_j = 0 add nothing; f_q = 0 where s_q = 0
 *   d_sens_i   device, n_support FP64 subset sensitivities s_q (without T)
 *   acq_time   T > 0
 *   stream     cudaStream_t the work is enqueued on (NULL: legacy stream)
 *
 * EINVAL: null pointers, n_rows < 1, n_support < 1 or above 8192 (the
 * widest row the register pass holds: 256 threads x 8 vectors of 4 floats;
 * the static array then holds 128 per-CTA partials), ld out of range or
 * misaligned rows.  ECUDA: a CUDA error from earlier work was still pending
 * when the call began (nothing runs and the error is left for the caller to
 * read), or the set-up or one of this call's launches failed.
 * The first call on each device, with that device current, looks up the
 * address of the static array (cudaGetSymbolAddress), caches it and loads
 * every kernel the entry point can launch, so later calls load nothing; make
 * that first call before any stream capture.  The cached address belongs to
 * the device's primary context: after cudaDeviceReset on that device this
 * entry point must not be called again in the same process.  All calls share
 * the array and each call overwrites what it needs, so calls whose work
 * overlaps on the GPU (different streams or threads) race and must be
 * serialised by the caller. */
lmosem_status lmosem_osem_subiter_noalloc(const float* d_rows, int64_t n_rows, int32_t n_support,
                                          int64_t ld, float* d_f, const double* d_sens_i,
                                          double acq_time, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LMOSEM_H */
