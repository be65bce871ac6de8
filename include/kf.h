/*
 * kf.h -- C interface of the GB300 Kalman-filter track fit and build step.
 *
 * The operations follow arXiv:1705.02876 (Cerati et al., "Parallelized
 * Kalman-Filter-Based Reconstruction of Particle Tracks on Many-Core
 * Processors and GPUs"):
 *   - Section 2.1: the track state is 6 global parameters (x, y, z, px, py,
 *     pz) with a 6x6 covariance, a hit is a 3-D point with a 3x3 covariance;
 *   - Section 2: the Kalman filter folds multiple-scattering estimates into
 *     the trajectory; fitting applies the filter over a known hit set
 *     without branching; building explores several candidates per seed;
 *   - Section 4.1: matrices are stored matrix-major (element (i,j) of all
 *     tracks contiguous) so that consecutive threads read consecutive words;
 *   - Section 4.2: one GPU thread per track for fitting; one event does not
 *     fill the GPU, so several events are processed together;
 *   - Sections 3 and 4.3: building keeps the best N candidates per seed,
 *     ranked by number of hits and chi2 ("clone engine"), hits partitioned
 *     into spatial bins.
 *
 * Conventions shared by every call:
 *   - Layout is structure-of-arrays, track index fastest: an array written
 *     [a][b][T] holds element (a, b) of track t at ((a * B) + b) * T + t.
 *   - A symmetric matrix is packed as its lower triangle, row by row:
 *     (0,0), (1,0), (1,1), (2,0), (2,1), (2,2), ...  (21 floats for 6x6,
 *     6 floats for 3x3).
 *   - Units: cm, GeV, tesla.  Charge is +1 or -1.
 *   - Every array pointer is device memory owned by the caller unless its
 *     comment says "host".  Pointers must be aligned to their element size.
 *     The library never frees, reallocates or retains caller memory after a
 *     call's work has completed on the stream.
 *   - Calls enqueue work on the caller's stream and return without
 *     synchronising; results are valid once that stream reaches them.
 *   - Return value: KF_OK (0) or a negative KF_ERR_* code; kf_last_error()
 *     describes the last failure on that context.  Per-track problems never
 *     fail a call: they set bits in out_flags.
 *   - A context may be used by one host thread at a time, and the work of
 *     its calls must not overlap on the GPU (one stream per context, or
 *     synchronise between streams): calls share the context's scratch.
 */
#ifndef KF_H
#define KF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kf_context kf_context;
typedef struct CUstream_st *kf_stream; /* a cudaStream_t; NULL is the legacy default stream */

/* status codes */
#define KF_OK 0
#define KF_ERR_ARG (-1)         /* null / misaligned pointer, bad size or option */
#define KF_ERR_CUDA (-2)        /* a CUDA runtime or driver call failed */
#define KF_ERR_TIMEOUT (-3)     /* a bounded device-side wait expired */
#define KF_ERR_NOMEM (-4)       /* the context could not grow its scratch */
#define KF_ERR_UNSUPPORTED (-5) /* no sm_103a device, or a feature off on this device */
#define KF_ERR_TOO_LARGE (-6)   /* a size exceeds what kf_fit_tracks_noalloc's fixed scratch serves */

/* per-track flags in out_flags */
#define KF_FLAG_UNREACHABLE 1u       /* a layer's cylinder is not reached: fit stops there */
#define KF_FLAG_LEFT_BARREL 2u       /* the crossing lies beyond |z| = z_half: fit stops */
#define KF_FLAG_INVERSION_FAILED 4u  /* S = H C H^T + V not positive definite: update skipped */
#define KF_FLAG_NAN_INPUT 8u         /* non-finite seed or used hit: outputs are the seed */
#define KF_FLAG_FP64_PATH 16u        /* at least one update used extended precision: a float-float
                                        gain or the FP64 update */
#define KF_FLAG_PSD_REPAIRED 32u     /* the FP64 path clamped the covariance */

#define KF_MAX_LAYERS 32

/* precision_mode */
#define KF_PRECISION_FP32 0   /* every step in FP32 */
#define KF_PRECISION_ROUTED 1 /* FP32, with ill-conditioned updates redone in FP64 */

/* launch_mode */
#define KF_LAUNCH_AUTO 0      /* one persistent launch over all events, graph-captured */
#define KF_LAUNCH_PER_EVENT 1 /* one plain launch per event (needs event_offsets) */
#define KF_LAUNCH_FLAT 2      /* one plain launch over all tracks */

/*
 * Detector: n_layers concentric cylinders of radius r[l] (strictly
 * increasing, > 0) and length 2 z_half, each x_over_x0[l] radiation lengths
 * thick at normal incidence, in a uniform field bz_tesla along z
 * (Section 3.2: equally spaced fixed-length cylinders).  Host memory.
 */
typedef struct {
    int n_layers;            /* 1 .. KF_MAX_LAYERS */
    const float *r;          /* host, [n_layers] */
    const float *x_over_x0;  /* host, [n_layers], >= 0 */
    float z_half;
    float bz_tesla;
} kf_geometry;

typedef struct {
    /* precision routing (fit and build) */
    int precision_mode;      /* KF_PRECISION_* */
    float cond_max;          /* an update whose S has a correlation matrix R (S scaled to unit
                                diagonal) with det R < 27 / (4 cond_max) runs in FP64, so
                                every FP32 update has cond_2(R) <= cond_max */
    float pt_lo, pt_hi;      /* tracks with pT outside [pt_lo, pt_hi] GeV update in FP64 */
    float gain_max;          /* > 0: an update with C_ii > gain_max V_ii (i = x, y, z) forms
                                its gain (S^-1 and K) in float-float; 0 = off */
    /* launch shape (fit) */
    int launch_mode;         /* KF_LAUNCH_* */
    int tracks_per_block;    /* 0 = autotuned, else 32, 64, 128 or 256 */
    int reg_cap;             /* registers per thread of the persistent fit: 0 = autotuned,
                                -1 = uncapped, 168, 128, 96 or 80 */
    int hit_prefetch;        /* layers of hits the persistent fit loads ahead of their
                                update: 0 = autotuned, 1 = the next layer into registers,
                                2 or 4 = through a ring in shared memory (cp.async) */
    /* building */
    int max_cands;           /* N candidates kept per seed, 1 (best hit) .. 8 */
    float chi2_cut;          /* hits with a larger chi2 increment are incompatible */
    float window_nsigma;     /* search window half-width in sigmas */
    float hit_sigma_rphi;    /* nominal hit resolution used for the window, cm */
    float hit_sigma_z;
    float window_max_dphi;   /* cap of the window's phi half-width, rad */
    float window_max_dz;     /* cap of its z half-width, cm */
    int n_phi_bins;          /* hit bins per layer, in phi ... (0 = autotuned) */
    int n_z_bins;            /* ... and in z (0 = autotuned); at most 16,384 bins */
    int use_proposal;        /* 1: the learned proposal keeps the top-k in-window hits */
    int topk;
    int build_variant;       /* learned build: -1 autotuned, 0 one proposal pass, 1 speculative */
} kf_options;

/* Fill *opt with the defaults: routed precision (cond_max 1e4, pT in
 * [0.25, 200], gain_max 0), automatic launch, N = 6, chi2 cut 30, 3-sigma window
 * capped at 0.05 rad and 5 cm, 0.01/0.1 cm nominal resolution, autotuned hit
 * bins, proposal off, top-k 4, the learned build's form autotuned. */
void kf_options_default(kf_options *opt);

/* Create a context on CUDA device `device` (requires compute capability
 * 10.3).  The context owns scratch memory, the autotuner's choices, captured
 * CUDA graphs and the proposal network's weights. */
int kf_context_create(kf_context **ctx, int device);
void kf_context_destroy(kf_context *ctx);

/* Text of the last error on ctx (never NULL; "" after success). */
const char *kf_last_error(const kf_context *ctx);

/*
 * Kalman-filter fit of n_tracks tracks (Sections 2 and 4.2).
 *
 * For each track, starting from its seed, for each layer l in order:
 *   1. propagate the state along the helix of the uniform field to its first
 *      forward crossing of cylinder l; if there is none, set
 *      KF_FLAG_UNREACHABLE and stop; if |z| > z_half there, set
 *      KF_FLAG_LEFT_BARREL and stop (the state stays at the previous layer);
 *   2. transport the covariance, C' = J C J^T, with J the Jacobian of the
 *      crossing state with respect to the previous state;
 *   3. add multiple-scattering noise on the momentum block,
 *      Q = theta0^2 (|p|^2 I3 - p p^T), theta0 the Highland width for
 *      x_over_x0[l] / |cos(incidence)| radiation lengths and beta = 1;
 *   4. if bit l of hit_mask is set, update with the hit: S = C_xx + V,
 *      K = C[:, 0:3] S^-1, x += K (m - x_xyz), C -= K C[0:3, :],
 *      chi2 += (m - x_xyz)^T S^-1 (m - x_xyz).
 *
 * Inputs (device, caller-owned, read only):
 *   seed_state [6][T], seed_cov [21][T] packed, charge [T] (int8, +1/-1),
 *   hit_pos [L][3][T], hit_cov [L][6][T] packed, hit_mask [T]
 *   (bit l set = a hit on layer l; values of absent hits are not read).
 * event_offsets: host, [n_events + 1], event e holds tracks
 *   event_offsets[e] .. event_offsets[e+1]-1; may be NULL (one event).  Only
 *   KF_LAUNCH_PER_EVENT launches by event; the other modes pack all events
 *   into one launch.
 * Outputs (device, caller-owned, written): out_state [6][T], out_cov [21][T]
 *   packed, out_chi2 [T], out_ndof [T] = 3 n_hits - 6, out_flags [T].
 * n_tracks may be 0 (nothing is launched).  Inputs and outputs must not
 * overlap.  opt may be NULL (defaults).
 */
int kf_fit_tracks(kf_context *ctx, const kf_geometry *geom, int64_t n_tracks,
                  const int64_t *event_offsets, int n_events,
                  const float *seed_state, const float *seed_cov, const int8_t *charge,
                  const float *hit_pos, const float *hit_cov, const uint32_t *hit_mask,
                  float *out_state, float *out_cov, float *out_chi2, int16_t *out_ndof,
                  uint32_t *out_flags, const kf_options *opt, kf_stream stream);

/*
 * kf_fit_tracks from and to host memory (the paper's events live on the host;
 * Section 4.2 streams several events to the GPU concurrently, and Section 4.3
 * finds host-device transfers about half of the GPU build's wall time).
 *
 * chunk_tracks = 0 and every array page-locked memory the device can address
 * (cudaMallocHost, cudaHostAlloc, cudaHostRegister): one persistent fit
 * launch reads the inputs and writes the outputs where they are, over the
 * host link; nothing is staged.  Otherwise the batch is cut into chunks of
 * chunk_tracks tracks (0: 262,144); each chunk is copied in, fitted (the
 * persistent fit, all of the chunk's events in one launch) and copied out on
 * one of three internal streams, so the transfers of one chunk overlap the
 * fit of another.
 *
 * Arrays: the layouts of kf_fit_tracks, all in host memory owned by the
 * caller; pageable memory takes the chunked path through the driver's
 * staging, slower.  The call returns when every output is in host memory.
 * Device staging (about 3 x 591 B x chunk_tracks at 10 layers) is kept by the
 * context and grown on demand (KF_ERR_NOMEM).  opt->launch_mode is ignored;
 * the shape is opt->tracks_per_block / opt->reg_cap / opt->hit_prefetch when
 * set, else 64 tracks per block, 128 registers and the register prefetch (no
 * tuning runs).
 */
int kf_fit_tracks_host(kf_context *ctx, const kf_geometry *geom, int64_t n_tracks, const float *seed_state,
                       const float *seed_cov, const int8_t *charge, const float *hit_pos, const float *hit_cov,
                       const uint32_t *hit_mask, float *out_state, float *out_cov, float *out_chi2,
                       int16_t *out_ndof, uint32_t *out_flags, int64_t chunk_tracks, const kf_options *opt);

/*
 * Combinatorial track building, the clone engine (Sections 3, 3.1 and 4.3):
 * starting from each seed, layer by layer, every candidate is propagated to
 * the layer (same steps as kf_fit_tracks: helix, transport, scattering) and
 * yields one child per compatible hit plus one child without a hit; the
 * children of a seed are ranked by number of hits (more first), then chi2
 * (less first), then candidate index, then hit index within the layer (the
 * hole first), and the best max_cands survive, each updated with its hit.
 * max_cands = 1 is the best-hit approach (Section 3).  A hit is compatible
 * if it lies within the window
 *   |dphi| <= window_nsigma sqrt(sigma_rphi,pred^2 + hit_sigma_rphi^2) / r,
 *   |dz|   <= window_nsigma sqrt(sigma_z,pred^2 + hit_sigma_z^2)
 * around the predicted crossing, the half-widths capped at window_max_dphi and
 * window_max_dz (a prediction that has lost its precision, as near a
 * tangential crossing, does not search the whole layer), and its chi2
 * increment is at most chi2_cut.  A candidate that cannot reach a layer, or crosses it beyond |z| = z_half,
 * stops and yields only its hole child from then on (its flags record why).
 * Hits are first sorted into n_phi_bins x n_z_bins bins per (event, layer)
 * in context scratch (Section 3: hits partitioned spatially).  Where opt
 * leaves the bin grid 0 an autotuner chooses it: the first call of a workload
 * class (layers, N, mode, the seed and hit counts' sizes in powers of two)
 * times five grids of up to 16,384 bins on the caller's buffers and keeps the
 * fastest (kf_build_tuned_shape reports it); with the learned proposal it
 * also chooses between one proposal pass and a speculative plain pass whose
 * flagged seeds alone are rebuilt with the proposal (opt->build_variant
 * fixes that choice: 0 the single pass, 1 the speculative form).  The results
 * depend on neither choice.
 *
 * geom: the layers to build over (host).
 * hit_offsets: host, [n_events][L + 1]; the hits of event e on layer l are
 *   hit_offsets[e][l] .. hit_offsets[e][l+1]-1 of hit_pos [3][n_hits] and
 *   hit_cov [6][n_hits] (device); events stored back to back, each holding
 *   fewer than 2^27 hits; n_hits < 2^31.
 * Seeds (device): seed_event [S] (int32; a seed of an event outside
 *   0..n_events-1 builds nothing), seed_state [6][S], seed_cov [21][S]
 *   packed, seed_charge [S], all at a radius inside the first layer.
 * Outputs (device), slot j of seed s = rank j after the last layer:
 *   out_hit_idx [S][N][L] (index into hit_pos, -1 = no hit on that layer),
 *   out_chi2 [S][N], out_nhits [S][N] (-1 for an empty slot),
 *   out_state [6][S*N], out_cov [21][S*N] packed, out_flags [S][N];
 *   N = opt->max_cands (1..8).
 * Scratch: 16 bytes per hit plus 4 (n_phi_bins n_z_bins + 1) bytes per
 * (event, layer) (16,384 bins when tuned), kept by the context and grown on
 * demand (KF_ERR_NOMEM).
 * The call copies hit_offsets to the device and waits for that copy.
 */
int kf_build_tracks(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
                    const float *hit_pos, const float *hit_cov, int64_t n_hits, int64_t n_seeds,
                    const int32_t *seed_event, const float *seed_state, const float *seed_cov,
                    const int8_t *seed_charge, int32_t *out_hit_idx, float *out_chi2, int16_t *out_nhits,
                    float *out_state, float *out_cov, uint32_t *out_flags, const kf_options *opt,
                    kf_stream stream);

/*
 * kf_build_tracks from and to host memory.  The paper's GPU build spent about
 * half of its wall time moving events between host and device (Section 4.3)
 * and fed the device from several CPU threads at once (Section 4.2).  Here the
 * events are cut into batches of events_per_batch events (0: 16), and a
 * pipeline of three streams overlaps the upload of one batch's hits and
 * seeds, the build of the previous one and the download of the outputs of the
 * one before that, through three rings of device buffers kept by the context.
 *
 * Arguments: those of kf_build_tracks, with every array in host memory owned
 * by the caller (page-locked memory -- cudaMallocHost, cudaHostAlloc,
 * cudaHostRegister -- lets the copies run asynchronously; pageable memory
 * works through the driver's staging, without the overlap).  Seeds must be
 * grouped by event: seed_event non-decreasing, every value in 0..n_events-1.
 * out_hit_idx holds indices into the caller's hit_pos, as kf_build_tracks
 * writes them.  The outputs equal kf_build_tracks' for the same inputs and
 * options (the build does not depend on how the events are batched).  The
 * call returns when every output is in host memory.  Device memory: three
 * batches' inputs and outputs plus the binning scratch of one batch, kept by
 * the context and grown on demand (KF_ERR_NOMEM).
 */
int kf_build_tracks_host(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
                         const float *hit_pos, const float *hit_cov, int64_t n_hits, int64_t n_seeds,
                         const int32_t *seed_event, const float *seed_state, const float *seed_cov,
                         const int8_t *seed_charge, int32_t *out_hit_idx, float *out_chi2, int16_t *out_nhits,
                         float *out_state, float *out_cov, uint32_t *out_flags, int events_per_batch,
                         const kf_options *opt);

/*
 * The shape the build autotuner picked for builds of n_layers layers, N =
 * max_cands, mode (0 plain, 1 logged, 2 learned proposal), n_seeds seeds and
 * n_hits hits (their size classes, powers of two), with the bin grid left to
 * the tuner (opt->n_phi_bins = opt->n_z_bins = 0): the grid, and for the
 * learned proposal whether it runs speculatively (*speculative = 1: a plain
 * pass flags the seeds one of whose windows held more than topk hits and the
 * proposal pass rebuilds those only; the others' builds are the same either
 * way).  speculative may be NULL.  KF_ERR_ARG if no such build has run on ctx.
 */
int kf_build_tuned_shape(kf_context *ctx, int n_layers, int max_cands, int mode, int64_t n_seeds, int64_t n_hits,
                         int *n_phi_bins, int *n_z_bins, int *speculative);

/*
 * kf_build_tracks that also records the training set of the learned proposal
 * (kf_proposal_*): one row for every (candidate, hit) pair whose hit lies in
 * the candidate's window, in the order the GPU meets them.  The build itself
 * is the plain one (opt->use_proposal must be 0) and its outputs are those of
 * kf_build_tracks.  The paper has no counterpart: the rows are the labelled
 * examples the plain build gives for free.
 *
 * log_features [log_capacity][12]: the pair's proposal inputs (see below).
 * log_labels [log_capacity]: 1 if the pair became one of the surviving
 *   candidates at that layer, else 0.
 * log_ref [log_capacity][4] (int32): seed, candidate slot at the start of
 *   the layer, build layer, hit index into hit_pos.
 * log_count (device, one uint64): set to the number of pairs met, which may
 *   exceed log_capacity; rows beyond the capacity are not written.
 * All device memory owned by the caller.  Rows appear in no fixed order
 * (atomic claims), so two calls give the same rows in different orders.
 */
int kf_build_tracks_logged(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
                           const float *hit_pos, const float *hit_cov, int64_t n_hits, int64_t n_seeds,
                           const int32_t *seed_event, const float *seed_state, const float *seed_cov,
                           const int8_t *seed_charge, int32_t *out_hit_idx, float *out_chi2, int16_t *out_nhits,
                           float *out_state, float *out_cov, uint32_t *out_flags, const kf_options *opt,
                           float *log_features, float *log_labels, int32_t *log_ref, int64_t log_capacity,
                           uint64_t *log_count, kf_stream stream);

/*
 * The learned hit proposal.  The paper has no learned component: this network
 * is the ranking the build step can use for a candidate's in-window hits
 * (kf_options.use_proposal), so that only the best top-k of them get the full
 * Kalman chi2.  It is a perceptron 12 -> 64 -> 64 -> 1 with ReLU activations
 * whose logit scores a (candidate, hit) pair.
 *
 * In kf_build_tracks with use_proposal = 1 (weights loaded by
 * kf_proposal_load, else KF_ERR_ARG) a candidate whose window holds more
 * than topk (1..8) hits scores all of them and computes the chi2 of only the
 * topk best by logit (ties to the lower hit index within the layer); the chi2
 * cut, ranking and update are unchanged.  A window of topk hits or fewer is
 * searched exhaustively, as without the proposal.
 *
 * weights: KF_PROPOSAL_PARAMS float32 values, in this order: W1 [12][64]
 *   (input-major), b1 [64], W2 [64][64], b2 [64], W3 [64], b3.
 * features: float32 [n][12], one row per pair: the residual of the hit in the
 *   layer's local frame (radial, tangential, z) divided by the square roots
 *   of the matching diagonal entries of S = H C H^T + V; log10 of the six
 *   diagonal entries of the predicted covariance C; q / pT; the layer's index
 *   among the build layers divided by their number; the candidate's holes so
 *   far.  labels: float32 [n], 1 = the plain build kept the pair, 0 = not.
 * All arrays are device memory owned by the caller.
 */
#define KF_PROPOSAL_PARAMS 5057

/* Mean binary cross-entropy on the logits over the n pairs and its gradient
 * with respect to the weights (grad [KF_PROPOSAL_PARAMS], device), in FP32;
 * *loss (host, may be NULL) receives the loss and makes the call wait. */
int kf_proposal_gradient(kf_context *ctx, const float *weights, const float *features, const float *labels,
                         int64_t n, float *grad, float *loss, kf_stream stream);

/* Train the weights in place (FP32 master weights) with Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8) on mini-batches of `batch` pairs, `epochs` passes
 * over the data, each in a fixed pseudo-random order.  epoch_loss (host, may
 * be NULL) receives the mean loss of each epoch and makes the call wait. */
int kf_proposal_train(kf_context *ctx, float *weights, const float *features, const float *labels, int64_t n,
                      int epochs, int batch, float learning_rate, float *epoch_loss, kf_stream stream);

/* Load weights into the context for inference: copied, with W1, W2 and W3
 * rounded to BF16 (the network's inference weights) and the biases kept in
 * FP32. */
int kf_proposal_load(kf_context *ctx, const float *weights, kf_stream stream);

/* kf_proposal_load with the weights given as bytes: weights (device) holds the
 * 5,057 FP32 parameters in the order above, bytes must be 20,228
 * (KF_ERR_ARG otherwise); enqueued on the legacy default stream. */
int kf_load_proposal(kf_context *ctx, const void *weights, size_t bytes);

/* Logits [n] of the loaded network for the pairs' features [n][12] (device),
 * on the tensor cores: the network's BF16 weights, each activation carried as
 * a pair of BF16 numbers (hi, and the rounding of what hi leaves over), FP32
 * accumulation; the result is the FP32 evaluation of the BF16-weight network
 * to about 2^-16 of each activation.  Uses the engine chosen by measurement
 * (KF_SCORE_AUTO of kf_proposal_score_with). */
int kf_proposal_score(kf_context *ctx, const float *features, int64_t n, float *logits, kf_stream stream);

/* kf_proposal_score with the tensor-core instruction family named:
 *   KF_SCORE_MMA_SYNC: warp-level mma.sync.m16n8k16, each warp scoring 32 rows
 *     with the weights in shared memory and the accumulators in registers;
 *   KF_SCORE_TCGEN05: tcgen05.mma, each CTA scoring 128-row tiles with the
 *     weights staged once in shared memory and both layers' accumulators in
 *     tensor memory.  Its waits for the tensor cores are bounded: a wait that
 *     expires leaves that CTA's remaining rows unwritten and sets the flag
 *     kf_proposal_status reports;
 *   KF_SCORE_AUTO: the one kf_proposal_score uses.
 * Both give the same logits within FP32 rounding. */
#define KF_SCORE_AUTO 0
#define KF_SCORE_MMA_SYNC 1
#define KF_SCORE_TCGEN05 2
int kf_proposal_score_with(kf_context *ctx, const float *features, int64_t n, float *logits, int engine,
                           kf_stream stream);

/* *expired = 1 if a bounded device-side wait of the scoring has expired on
 * this context since it was created, else 0.  Synchronises with the device. */
int kf_proposal_status(kf_context *ctx, int *expired);

/*
 * Seeding from hits (the paper seeds from the true hits of each simulated
 * track and leaves realistic seeding for later, Section 2): triplets of hits
 * on the three seed layers of every event that a track from the beam line
 * above pt_min could have made, and the seed fit's inputs built from them.
 *
 * A triplet (h0, h1, h2) of one event, with the hits' own radii r_i, azimuths
 * phi_i and z_i, is a seed when |phi_1 - phi_0| <= w01 and |phi_2 - phi_1| <=
 * w12 (w_ab = asin(R_b / 2 R_min) - asin(R_a / 2 R_min) + d0_max (1/R_a +
 * 1/R_b), R_a the layers' radii, R_min = pt_min / (0.0029979 |Bz|)); the line
 * through (r_0, z_0), (r_1, z_1) meets r = 0 within z0_max and predicts z at
 * r_2 within dz_max; and the circle through the three (x, y) points has pT >=
 * pt_min and passes within d0_max of the beam line.  Its charge follows the
 * turning sense (positive charges turn clockwise in Bz > 0); a triplet with
 * pT above pt_both_charges, straighter than three hits resolve, is seeded
 * with both charges.
 */
typedef struct {
    float pt_min;           /* GeV */
    float d0_max;           /* cm, distance of the circle to the beam line */
    float z0_max;           /* cm, |z| where the (r, z) line meets the beam line */
    float dz_max;           /* cm, |z_2 - the line's prediction| */
    float pt_both_charges;  /* GeV */
    float pt_unresolved;    /* GeV, the seed fit's starting pT of a two-charge triplet */
    float p_sigma_resolved;    /* momentum sigma of the seed fit's start, relative */
    float p_sigma_unresolved;  /* the same for a two-charge triplet */
    int n_phi_bins, n_z_bins;  /* bins of the seed layers' hits */
} kf_seeding;

/* Defaults: pt_min 0.3, d0_max 0.15, z0_max 4, dz_max 0.8, pt_both_charges 2,
 * pt_unresolved 6, p_sigma_resolved 0.3, p_sigma_unresolved 1, 256 x 64 bins. */
void kf_seeding_default(kf_seeding *opt);

/*
 * Find the triplets.  geom: the three seed layers (host).  hit_offsets: host
 * [n_events][4]; event e's hits of seed layer l are hit_offsets[e][l] ..
 * hit_offsets[e][l+1]-1 of hit_pos [3][n_hits] (device), events back to back,
 * n_hits < 2^31.  *n_seeds (host) receives the number of seeds (a triplet
 * seeded with both charges counts twice); the call waits for the search.
 * The seeds stay in the context until the next search, in no fixed order.
 */
int kf_seed_triplets(kf_context *ctx, const kf_geometry *geom, int n_events, const int64_t *hit_offsets,
                     const float *hit_pos, int64_t n_hits, const kf_seeding *opt, int64_t *n_seeds,
                     kf_stream stream);

/*
 * The first n (<= *n_seeds of the last search) seeds as the seed fit's inputs,
 * in kf_fit_tracks' layouts with T = n (device, caller-owned): out_state
 * [6][n] (1 cm before the first hit along the circle's tangent, pT from the
 * circle, or pt_unresolved for a two-charge triplet, whose curvature the hits
 * do not measure, pz from the first chord's slope), out_cov [21][n]
 * (diagonal: sigma 10% of each position component and p_sigma_resolved, or
 * p_sigma_unresolved for a two-charge triplet, of each momentum component,
 * floors 1e-4 cm, 1e-3 GeV),
 * out_charge [n], out_hit_pos [3][3][n], out_hit_cov [3][6][n] (the three
 * hits, from hit_pos [3][H] / hit_cov [6][H] of the search), out_mask [n] (= 7);
 * out_event [n] and out_hits [3][n] (indices into hit_pos) identify each
 * seed.
 */
int kf_seed_fetch(kf_context *ctx, const kf_geometry *geom, const float *hit_pos, const float *hit_cov,
                  const kf_seeding *opt, int64_t n, int32_t *out_event, int32_t *out_hits, float *out_state,
                  float *out_cov, int8_t *out_charge, float *out_hit_pos, float *out_hit_cov, uint32_t *out_mask,
                  kf_stream stream);

/*
 * The fit followed by the Kalman smoother: at every layer the estimate that
 * uses all of the track's hits (Section 2 names a final fit with a smoother,
 * after building, as the step giving each track's best parameters).  The
 * forward pass is kf_fit_tracks' per-track fit (routed precision as set in
 * opt); the backward pass is the Rauch-Tung-Striebel recursion in each layer's
 * local coordinates (t, z, px, py, pz), where the covariances are positive
 * definite, with Cp^-1 from a Cholesky factorisation scaled to unit diagonal.
 *
 * Inputs: the layouts of kf_fit_tracks (device, caller-owned).
 * Outputs (device, caller-owned): out_state [L][6][T] and out_cov [L][21][T]
 *   packed, the smoothed estimate after every layer the fit reached, NaN on
 *   the other layers and on every layer of a track with a non-finite input;
 *   out_reached [T] (int16) the number of layers reached (0 for such a
 *   track); out_flags [T] as kf_fit_tracks (INVERSION_FAILED also when a
 *   predicted covariance could not be factorised, the layer then keeping its
 *   filtered estimate).
 * No scratch: the backward pass recomputes each layer's prediction from the
 * filtered estimate the forward pass left in the outputs.  One thread per
 * track, one launch; opt->launch_mode and the shape are ignored.
 */
int kf_smooth_tracks(kf_context *ctx, const kf_geometry *geom, int64_t n_tracks, const float *seed_state,
                     const float *seed_cov, const int8_t *charge, const float *hit_pos, const float *hit_cov,
                     const uint32_t *hit_mask, float *out_state, float *out_cov, int16_t *out_reached,
                     uint32_t *out_flags, const kf_options *opt, kf_stream stream);

/*
 * Batched covariance transport C <- J C J^T for n general (dense) 6x6
 * Jacobians: the batched small-matrix product the paper measures on the GPU
 * (Section 4.1, 6x6 products in a Matriplex-style layout against batched
 * cuBLAS).  One thread per matrix, J and C in registers; no structure of J is
 * assumed (the fit's own transport exploits it).
 *
 * J: device float [36][n], J[i][j] of matrix t at (6 i + j) n + t.
 * C: device float [21][n], packed lower triangle, read and overwritten.
 * n may be 0.  KF_ERR_ARG on a NULL or misaligned pointer.
 */
int kf_transport_batch(kf_context *ctx, int64_t n, const float *J, float *C, kf_stream stream);

/*
 * Launch shape the autotuner picked for the persistent fit of n_layers layers
 * and a batch of n_tracks' size class (powers of two), once a KF_LAUNCH_AUTO
 * fit of that class has run on ctx.  Writes tracks per block, the register
 * cap per thread (-1: uncapped) and the hit prefetch depth (kf_options).
 * KF_ERR_ARG if that class has not been tuned.
 */
int kf_fit_tuned_shape(kf_context *ctx, int n_layers, int64_t n_tracks, int *tracks_per_block,
                       int *reg_cap, int *hit_prefetch);

/*
 * The fit for callers that cannot allocate device memory.  The paper has no
 * counterpart to this entry point.
 *
 * kf_fit_tracks needs a kf_context, and kf_context_create calls cudaMalloc.
 * Callers that work inside a device-memory pool they do not own, loops that
 * must not touch the allocator after start-up, or hosts that forbid
 * allocation while their own work is in flight can call this instead.  It
 * runs the same persistent fit kernel (same steps, inputs, outputs and flags
 * as kf_fit_tracks, all events in one launch) and allocates nothing: the
 * kernel's only scratch, the 4-byte counter from which its warps claim
 * 32-track units, is a fixed array in the library's device memory that every
 * GPU loading the library holds until the process exits.
 *
 *   - Runs on the current CUDA device.  The first call on a device looks up
 *     that array's device address once (cudaGetSymbolAddress); make that
 *     first call before any stream capture.
 *   - Each call clears the counter on `stream` before its launch.  All calls
 *     on a device share the counter, so calls whose work overlaps on the GPU
 *     (different streams, not ordered) race and give wrong results: order
 *     them on one stream or synchronise.
 *   - n_tracks must be at most KF_NOALLOC_MAX_TRACKS (2^36, the limit of
 *     kf_fit_tracks too); larger batches return KF_ERR_TOO_LARGE, and so does
 *     a launch that would hold more than 16,384 resident warps (the 32-bit
 *     counter must not wrap while every warp makes its last claim; a GB300
 *     holds at most 152 x 64 = 9,728).
 *   - No tuning runs.  The shape is opt->tracks_per_block, opt->reg_cap and
 *     opt->hit_prefetch where set, else 64 tracks per block, no register cap
 *     and the register prefetch (depth 1).  Only the (block, cap, depth)
 *     combinations the autotuner of kf_fit_tracks chooses from are compiled
 *     in: blocks 32/64/128/256 with cap none/168/128/96/80 at depth 1 (cap
 *     168 only below 256 threads, cap 96 only below 256), and at depths 2
 *     and 4 the caps 128 (all blocks) and 96 (below 256); another combination
 *     returns KF_ERR_ARG.  opt->launch_mode is ignored.  There is no context,
 *     so failures are reported by the return code only: KF_ERR_ARG (a bad
 *     argument or an uncompiled shape), KF_ERR_TOO_LARGE, KF_ERR_CUDA (a CUDA
 *     call failed, including the shape's shared-memory opt-in or occupancy
 *     query).
 */
#define KF_NOALLOC_MAX_TRACKS (68719476736LL)
int kf_fit_tracks_noalloc(const kf_geometry *geom, int64_t n_tracks, const float *seed_state,
                          const float *seed_cov, const int8_t *charge, const float *hit_pos,
                          const float *hit_cov, const uint32_t *hit_mask, float *out_state,
                          float *out_cov, float *out_chi2, int16_t *out_ndof, uint32_t *out_flags,
                          const kf_options *opt, kf_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* KF_H */
