/*
 * scstat.h -- C ABI of the GB300 (sm_103a) library that evaluates the
 * semi-coherent search statistic Upsilon_N of Bandopadhyay & Moore,
 * "A GPU-accelerated semi-coherent hierarchical search for stellar-mass
 * binary inspiral signals in LISA", arXiv:2408.13170.
 *
 * What one evaluation computes, for every particle theta_p
 * (Sec. II.A Eq. inner_prod, Sec. II.B Eq. semi-coherent_O and Upsilon_N):
 *
 *   z_{p,n}  = sum_{k in segment n} sum_{alpha in {A,E} (or {A,E,T})}
 *                  4 df d_alpha(f_k) conj(h_alpha(theta_p, f_k)) / S_alpha(f_k)
 *   hh_{p,n} = sum_{k in segment n} sum_alpha 4 df |h_alpha|^2 / S_alpha
 *   x_{p,n}  = max_phi Re{z e^{-i phi}} = |z_{p,n}|
 *   Upsilon_N(p) = sum_n x_{p,n}^2 / hh_{p,n}      (terms with hh = 0 add 0)
 *
 * with h_alpha the (2,2)-mode frequency-domain inspiral (TaylorF2 to 3.5PN
 * with the leading eccentric term) times the LISA TDI A/E (and, on a stream loaded with
 * scs_set_data_aet, T) transfer function at t = t(f) (Sec. IV).
 *
 * Conventions shared by all calls
 *  - Every function returns 0 (SCS_OK) or a negative SCS_E* code; the text
 *    of the last error of a context is returned by scs_last_error().
 *  - Pointers may be host or device memory; the library detects which with
 *    cudaPointerGetAttributes.  Host arrays are copied and the call returns
 *    after the result has been copied back (synchronous); when every array
 *    of a call is device memory the call is asynchronous on the given stream.
 *  - A context is bound to one device and is not thread-safe.
 *  - Particle layout: params is row-major P x 8:
 *      {Mc [Msun, detector frame], q = m1/m2 >= 1, f0 [Hz, GW frequency at
 *       t = 0, the start of the observation], lambda, beta [ecliptic
 *       longitude/latitude, rad], iota [inclination, rad], psi
 *       [polarisation, rad], e0 [orbital eccentricity at f0, 0 <= e0 <= 0.3]}.
 *  - Waveform (Sec. IV, TaylorF2Ecc): the non-spinning TaylorF2 phase to
 *    3.5PN plus the leading-order eccentric term
 *    -(2355/1462) e0^2 (f/f0)^{-19/9} times the Newtonian term; amplitude
 *    f^{-7/6}.
 *  - Non-physical particles (Mc <= 0, q < 1, f0 <= 0, a non-finite entry,
 *    e0 < 0 or e0 > 0.3, or f0 already past the last stable orbit
 *    v = 6^{-1/2}) get stat = -inf; a particle whose support misses the data
 *    band gets 0.
 *  - Support of a particle: grid bins k with f_k >= f0, t(f_k) <= T_obs and
 *    v(f_k) <= 6^{-1/2}.
 */
#ifndef SCSTAT_H
#define SCSTAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCS_OK 0
#define SCS_EINVAL (-1)       /* bad argument (size, pointer, value) */
#define SCS_ENOMEM (-2)       /* device allocation failed */
#define SCS_ECUDA (-3)        /* a CUDA runtime call or kernel failed */
#define SCS_ENODATA (-4)      /* stream has no data or no segments yet */
#define SCS_ETIMEOUT (-5)     /* a bounded device-side wait gave up (reserved:
                                 no kernel of this library waits) */
#define SCS_EUNSUPPORTED (-6) /* valid request the library does not do */

/* evaluation paths */
#define SCS_FP64 0   /* every bin in FP64, double-double phase */
#define SCS_MIXED 1  /* FP64 anchors + FP32 split-phase bins, Kahan sums */
#define SCS_SPLINE 2 /* comparison path built like the paper's GPU design (Sec. IV):
                        phase and amplitude x transfer functions exact on a sparse
                        node grid, cubic splines onto the FFT grid (FP64 phase
                        spline, FP32 products, Kahan sums); see scs_set_spline */

/* segmentations */
#define SCS_EQUAL_WIDTH 0 /* n-th edge floor(n K / N) over the whole grid */
#define SCS_EQUAL_SNR2 1  /* equal squared SNR per segment, per particle */

typedef struct scs_ctx scs_ctx; /* opaque, owned by the library */

/* Create a context on CUDA device `device` using evaluation path `path`
 * (SCS_FP64 or SCS_MIXED).  *out receives the context (NULL on failure).
 * SCS_SPLINE is accepted too.
 * Errors: SCS_EINVAL (bad device/path/out), SCS_ECUDA, SCS_ENOMEM. */
int scs_create(scs_ctx **out, int device, int path);

/* Wait for the work queued on the context's stream, then release every
 * device buffer of the context and the context itself (no counterpart in
 * the paper).  NULL is ignored; no error is returned. */
void scs_destroy(scs_ctx *ctx);

/* NUL-terminated text of the last error on this context (owned by the
 * context, valid until the next call on it; "null context" for NULL).
 * Never fails. */
const char *scs_last_error(const scs_ctx *ctx);

/* Switch the evaluation path of later calls (SCS_FP64, SCS_MIXED or
 * SCS_SPLINE; the swarm calls refuse SCS_SPLINE with SCS_EUNSUPPORTED).
 * Errors: SCS_EINVAL (unknown path). */
int scs_set_path(scs_ctx *ctx, int path);

/* Node grid of the SCS_SPLINE path.  Sec. IV evaluates the waveform and the
 * response on a grid about 1000 times coarser than the FFT grid and
 * spline-interpolates them onto it; here each particle's nodes are
 * k_lo, k_lo + S, ..., k_hi with S the largest power of two
 * <= 2^max_log2_spacing (default 10: 1024 bins) for which twice the cubic
 * spline's phase error bound (5/384) S^4 max|d^4 Phi/dk^4| stays below 1e-6
 * turns, the phase tolerance of the mixed path's anchors.  The splines are
 * not-a-knot cubic splines of the unwrapped total phase Phi (turns, FP64
 * coefficients) and of the real and imaginary parts of G_A, G_E (and G_T),
 * G = A(f) R(f) (FP32 coefficients).  An evaluation on this path
 * synchronises with the host once (to size the node scratch) and allocates.
 *   max_log2_spacing  3 .. 14.
 * Errors: SCS_EINVAL. */
int scs_set_spline(scs_ctx *ctx, int max_log2_spacing);

/* ---- Test-only: model switch ----
 * Replaces, for every later call on the context (evaluation on both paths,
 * edges, supports, templates, injection, swarm iterations), the waveform and
 * the response by test models that have closed forms:
 *   SCS_MODEL_TF2           the search model (default): TaylorF2 to 3.5PN
 *                           with the leading eccentric term, amplitude
 *                           f^{-7/6} (Sec. IV);
 *   SCS_MODEL_NEWTONIAN     the same with the leading (Newtonian) phase term
 *                           only: a power-law chirp (e0 must be 0);
 *   SCS_MODEL_LINEAR_CHIRP  App. A's constant-amplitude linear chirp
 *                           f(t) = f0 + fdot t: phase (f - f0)^2 / (2 fdot)
 *                           - 1/8 turns, t(f) = (f - f0)/fdot, amplitude 1,
 *                           params[0] read as fdot [Hz/s] > 0, q ignored, no
 *                           last-stable-orbit cut, e0 must be 0;
 *   SCS_RESPONSE_TDI        the rigid-adiabatic TDI A, E (and T) response
 *                           (default);
 *   SCS_RESPONSE_IDENTITY   h_A = h, h_E = h_T = 0, no Doppler modulation.
 * Errors: SCS_EINVAL (unknown model). */
#define SCS_MODEL_TF2 0
#define SCS_MODEL_NEWTONIAN 1
#define SCS_MODEL_LINEAR_CHIRP 2
#define SCS_RESPONSE_TDI 0
#define SCS_RESPONSE_IDENTITY 1
int scs_debug_set_model(scs_ctx *ctx, int waveform, int response);

/* Load one data stream (Sec. II.A: data d_alpha on the FFT grid with
 * one-sided PSD S_alpha; Sec. IV: grid f_k = f_first + k df, k = 0..K-1,
 * df = 1/T_obs).
 *   stream_id  0 <= stream_id < 1024, slot to (re)fill.
 *   A, E       K complex values each, interleaved (re, im), FP64.
 *   S_A, S_E   K one-sided PSD values each (> 0, finite); S_E may be NULL
 *              (then S_E = S_A).
 *   f_first, df, K, T_obs   grid; requires K >= 1, df > 0, f_first > 0 and
 *              |df T_obs - 1| <= 1e-12.
 * The library copies and pre-whitens the data (d~ = 4 df d / S,
 * w = 4 df / S) in FP64 and FP32; the caller keeps ownership of its
 * buffers and may free them on return.  Any segmentation previously set on
 * the stream is kept if N <= K.
 * Errors: SCS_EINVAL (sizes, non-positive or non-finite PSD), SCS_ENOMEM,
 * SCS_ECUDA. */
int scs_set_data(scs_ctx *ctx, int stream_id, const double *A, const double *E,
                 const double *S_A, const double *S_E, double f_first,
                 double df, int64_t K, double T_obs);

/* As scs_set_data, with the third TDI channel T = (X + Y + Z)/sqrt3 and its
 * PSD S_T (the search uses all three channels, Sec. I; T's response, like
 * A's and E's, from the rigid-adiabatic model of Sec. IV).  Every later
 * evaluation, edge, log-likelihood and injection on the stream then sums
 * over A, E and T: z_n gains w_T d_T conj(h_T), [h|h]_n gains w_T |h_T|^2,
 * <d|d> gains w_T |d_T|^2.  scs_set_data on the slot drops the channel.
 *   T    K complex values, interleaved (re, im), FP64 (host or device).
 *   S_T  K one-sided PSD values (> 0, finite).
 * Errors: as scs_set_data; SCS_EINVAL also for a null T or S_T. */
int scs_set_data_aet(scs_ctx *ctx, int stream_id, const double *A, const double *E,
                     const double *T, const double *S_A, const double *S_E,
                     const double *S_T, double f_first, double df, int64_t K,
                     double T_obs);

/* Choose the segmentation of a stream (Sec. II.B): N segments, 1 <= N <= K,
 * mode SCS_EQUAL_WIDTH (edges floor(n K/N) shared by all particles) or
 * SCS_EQUAL_SNR2 (per particle: the cumulative template power
 * sum_alpha w |h_alpha|^2, evaluated exactly on the anchor bins
 * k_lo, k_lo + 1024, ..., k_hi and integrated by the trapezoid rule, is cut
 * at n/N of its total by linear inverse interpolation; bin k belongs to
 * segment n iff kappa_n <= k < kappa_{n+1}).
 * Errors: SCS_EINVAL, SCS_ENODATA (no data on the stream). */
int scs_set_segments(scs_ctx *ctx, int stream_id, int N, int mode);

/* Evaluate Upsilon_N for P particles on one stream (Sec. II.B).
 *   params   P x 8 doubles (layout above), host or device.
 *   P        number of particles, 1 <= P <= 2^24.
 *   stat     P doubles: Upsilon_N per particle.
 *   seg_x    NULL, or P x N doubles: x_{p,n} = |z_{p,n}| (row-major).
 *   seg_hh   NULL, or P x N doubles: hh_{p,n} = [h|h]_n.
 *   cuda_stream  cudaStream_t to run on (NULL: the context's stream).
 * A call holds at most 2^31 - 1 (particle, work chunk) pairs: P times the
 * stream's ceil(K / tile) chunks (scs_set_tile); a larger call is rejected
 * with SCS_EINVAL and must be split.
 * Errors: SCS_EINVAL, SCS_ENODATA, SCS_ENOMEM, SCS_ECUDA, SCS_ETIMEOUT. */
int scs_eval_stat(scs_ctx *ctx, int stream_id, const double *params,
                  int64_t P, double *stat, double *seg_x, double *seg_hh,
                  void *cuda_stream);

/* Semi-coherent log-likelihood (Sec. II.B) of P templates a_p h(theta_p):
 *   log L_N = -<d|d>/2 - a^2 <h|h>/2 + a O_N,  O_N = sum_n x_n,
 *   <h|h> = sum_n [h|h]_n,
 * on the stream's segmentation, where h(theta) is this library's template
 * (Sec. IV form f^{-7/6} T_alpha e^{-i Psi}, the normalisation of
 * scs_waveform) and a_p = amp[p] carries the physical amplitude (NULL: 1).
 *   loglike P doubles (-inf for non-physical particles); overlap (O_N) and
 *   hh (<h|h>) P doubles each of the unit templates, may be NULL.  Any array
 *   host or device.  Uses the evaluation of scs_eval_stat with per-segment
 *   outputs (P x N doubles of scratch).
 * Errors: as scs_eval_stat. */
int scs_eval_loglike(scs_ctx *ctx, int stream_id, const double *params, int64_t P,
                     const double *amp, double *loglike, double *overlap, double *hh,
                     void *cuda_stream);

/* Several data streams in one evaluation (one persistent launch): item i
 * evaluates particles P_offsets[i] .. P_offsets[i+1]-1 of params on stream
 * stream_ids[i] with that stream's grid, data and segmentation (streams may
 * differ in length, band, N and mode).  Used to batch independent swarms or
 * search tiles (Sec. IV: tiles searched independently).
 *   stream_ids  n_items ints; P_offsets  n_items + 1 int64, P_offsets[0] = 0,
 *               non-decreasing, P = P_offsets[n_items] in [1, 2^24].
 *   params      P x 8 doubles; stat  P doubles (host or device).
 * Per-particle results are identical to scs_eval_stat on the same stream.
 * The (particle, work chunk) pairs of all items together are limited as in
 * scs_eval_stat.
 * Errors: SCS_EINVAL, SCS_ENODATA, SCS_ENOMEM, SCS_ECUDA. */
int scs_batch_eval(scs_ctx *ctx, const int *stream_ids, const int64_t *P_offsets,
                   int n_items, const double *params, double *stat, void *cuda_stream);

/* ---- Device-side particle swarm (Sec. III.A; multi-swarm, Sec. III.B) ----
 * One swarm state per context.  Swarm s owns particles swarm_offsets[s] ..
 * swarm_offsets[s+1]-1 and searches data stream stream_ids[s] with that
 * stream's segmentation.  An iteration evaluates Upsilon_N of every particle
 * of every swarm in one batched launch (as scs_batch_eval), then on the device:
 *   personal best  Psi_p <- theta_p where Upsilon(theta_p) > best_p (strict);
 *   swarm best     Xi_s <- the best personal best of the swarm if it beats
 *                  the swarm's record (strict; lowest particle index on ties);
 *   velocity       u = Omega v + Phi_P r_P (Psi_p - theta) + Phi_G r_G (Xi_s - theta)
 *                  per dimension (Eq. PSO_velocity_rule), evaluated as
 *                  ((Omega v) + ((Phi_P r_P) (Psi - theta))) + ((Phi_G r_G) (Xi - theta))
 *                  with every operation rounded once (no contraction);
 *   clamp          v = u if |u| >= eps, else eps with the sign of u, sign(0)
 *                  = +1 (Eq. PSO_min_velocity);
 *   move           theta <- theta + v; lambda (dimension 3) and psi (6) wrap
 *                  into [lo, hi); the others reflect at a bound that was
 *                  crossed (2 bound - theta, velocity negated) and are then
 *                  clipped to [lo, hi].  Dimension 7 (e0) is searched (and
 *                  reflects) when prior_hi[7] > prior_lo[7]; with
 *                  prior_hi[7] == prior_lo[7] it stays at prior_lo[7] and
 *                  draws no random numbers.
 * r_P, r_G: outputs 0 and 1 of Philox4x32-10 (Salmon et al., SC'11) with key
 * (seed mod 2^32, seed >> 32) and counter (particle, iteration, dimension, 0),
 * mapped to (x + 1/2) 2^-32.  The iteration counter lives on the device.
 * Initial state: theta = lo + u0 (hi - lo), v = (u1 - 1/2) 0.2 (hi - lo) with
 * (u0, u1) from counter (particle, 2^32 - 1, dimension, 1); best values -inf.
 * Particles whose statistic is -inf (non-physical) never become bests. */

/* Create (or replace) the swarm state and initialise it on the device.
 *   n_swarms       1 .. 1024.
 *   stream_ids     n_swarms data streams, each with data and segmentation set.
 *   swarm_offsets  n_swarms + 1 int64, [0] = 0, strictly increasing, total P <= 2^24.
 *   prior_lo/hi    8 doubles each; hi > lo in dimensions 0..6 (host memory).
 *   seed           Philox key.
 * Hyper-parameters default to the N = 100 row of Table III for every swarm.
 * Synchronous.  Errors: SCS_EINVAL, SCS_ENODATA, SCS_ENOMEM, SCS_ECUDA. */
int scs_pso_create(scs_ctx *ctx, int n_swarms, const int *stream_ids,
                   const int64_t *swarm_offsets, const double *prior_lo,
                   const double *prior_hi, uint64_t seed, void *cuda_stream);

/* Set Omega, Phi_P, Phi_G (Eq. PSO_velocity_rule) and eps[8] (minimum
 * speeds, Eq. PSO_min_velocity; parameter order of params, >= 0) of one
 * swarm, or of every swarm if swarm = -1 (Table III gives them per segment
 * count).  Waits for the work on cuda_stream first.
 * Errors: SCS_EINVAL (swarm out of range, non-finite coefficient, eps < 0),
 * SCS_ENODATA (no swarm), SCS_EUNSUPPORTED (spline path). */
int scs_pso_set_hyper(scs_ctx *ctx, int swarm, double Omega, double PhiP, double PhiG,
                      const double *eps, void *cuda_stream);

/* Run iters (0 .. 100000) iterations, asynchronously on cuda_stream (NULL:
 * the context's stream).  use_graph = 1 captures iters whole iterations into
 * one CUDA graph on the first call (and again when iters, the path or a
 * swarm's stream data or segmentation changed) and launches it; use_graph = 0
 * launches the same kernels directly.  Both give identical states.  The
 * swarm evaluates with its own scratch, separate from the other calls.
 * Errors: SCS_EINVAL, SCS_ENODATA, SCS_ENOMEM, SCS_ECUDA. */
int scs_pso_run(scs_ctx *ctx, int iters, int use_graph, void *cuda_stream);

/* Copy the state out (each pointer may be NULL to skip; host or device):
 * pos, vel, best_pos P x 8; best_val P; swarm_pos S x 8; swarm_val S;
 * stat P (statistic of the positions evaluated last, i.e. before the last
 * move); iteration = iterations run since create.  Synchronous.
 * Errors: SCS_ENODATA (no swarm), SCS_EUNSUPPORTED (spline path), SCS_ECUDA. */
int scs_pso_get(scs_ctx *ctx, double *pos, double *vel, double *best_pos, double *best_val,
                double *swarm_pos, double *swarm_val, double *stat, int64_t *iteration,
                void *cuda_stream);

/* Overwrite parts of the state (NULL pointers keep that part; host or
 * device) and set the iteration counter (0 .. 2^32 - 1).  Synchronous.
 * Errors: SCS_EINVAL (iteration out of range), SCS_ENODATA (no swarm),
 * SCS_EUNSUPPORTED (spline path), SCS_ECUDA. */
int scs_pso_set(scs_ctx *ctx, const double *pos, const double *vel, const double *best_pos,
                const double *best_val, const double *swarm_pos, const double *swarm_val,
                int64_t iteration, void *cuda_stream);

/* Checkpoint of the whole swarm (layout, seed, prior box, hyper-parameters,
 * state, iteration) into a caller-owned buffer: with buf = NULL, *len
 * receives the size; otherwise *len is the buffer's size on input and the
 * bytes written on output.  scs_pso_load recreates the swarm from such a
 * buffer (the referenced streams must exist in this context); the run then
 * continues bit for bit as it would have without the checkpoint.
 * A checkpoint whose sizes, swarm coefficients (finite, eps >= 0) or
 * convergence rule (delta >= 0, window >= 1) fail the checks of the setters
 * is refused before the current swarm is touched.
 * Errors: SCS_EINVAL (small buffer, not a checkpoint or a corrupt one), as
 * create. */
int scs_pso_save(scs_ctx *ctx, void *buf, size_t *len, void *cuda_stream);
int scs_pso_load(scs_ctx *ctx, const void *buf, size_t len, void *cuda_stream);

/* Work tile of a stream: its bins are cut into chunks of 2^log2_chunk
 * (11 .. 14, default 12 = 4096 bins); a work item is one chunk x up to 32
 * particles.  The tile sets where FP32 block sums are handed to the FP64
 * merge: results for different tiles agree to FP32 rounding (~1e-8
 * relative); one tile always gives the same bits.
 * Errors: SCS_EINVAL, SCS_ENODATA. */
int scs_set_tile(scs_ctx *ctx, int stream_id, int log2_chunk);

/* Autotuner: times full evaluations of the given particles (P x 8, host or
 * device; the stream's data and segmentation must be set) with every tile
 * log2_chunk = 11 .. 14 on cuda_stream, each started with a cold L2 (a
 * 192 MB buffer is written before it), keeps the fastest (the smallest tile
 * within 2% of the fastest) for the stream and
 * returns it in *log2_chunk (may be NULL); ms (may be NULL) receives the
 * four best-of-three times.  Synchronous; allocates.
 * Errors: as scs_eval_stat. */
int scs_autotune(scs_ctx *ctx, int stream_id, const double *params, int64_t P,
                 int *log2_chunk, double *ms, void *cuda_stream);

/* ---- The hierarchical multi-swarm search on the device (Sec. III.B, App. B) ----
 * Convergence rule: a swarm has converged when its best value has not grown by
 * more than delta over the last `window` evaluations (the paper: 2 over 50,
 * the default).  The record is kept on the device by every iteration.
 * Errors: SCS_EINVAL (delta negative or not finite, window < 1), SCS_ENODATA
 * (no swarm), SCS_EUNSUPPORTED (spline path). */
int scs_pso_set_convergence(scs_ctx *ctx, double delta, int window);

/* converged[S] (may be NULL): 1 for each converged swarm; *iteration (may be
 * NULL): iterations run.  Returns 1 when every swarm has converged, 0 when
 * not, a negative SCS_E* code on error.  Synchronous on cuda_stream. */
int scs_pso_status(scs_ctx *ctx, int *converged, int64_t *iteration, void *cuda_stream);

/* Forget the personal and swarm bests and the convergence records (positions
 * and velocities are kept): for a new objective, e.g. the next rung of the
 * segment ladder (App. B).  Synchronous.
 * Errors: SCS_ENODATA (no swarm), SCS_EUNSUPPORTED (spline path), SCS_ECUDA. */
int scs_pso_reset_bests(scs_ctx *ctx, void *cuda_stream);

/* The current swarm layout (it changes with scs_pso_regroup, Sec. III.B):
 * *n_swarms, stream_ids[S] and swarm_offsets[S + 1] (host; each may be
 * NULL to skip it).
 * Errors: SCS_ENODATA (no swarm), SCS_EUNSUPPORTED (spline path). */
int scs_pso_layout(scs_ctx *ctx, int *n_swarms, int *stream_ids, int64_t *swarm_offsets);

/* k-means of P positions (P x 8, host or device) in the prior box: features
 * M_c, q, f0, beta, iota normalised to the box and lambda, psi on circles of
 * circumference one; centroid 0 is particle 0, centroid j the particle
 * farthest from centroids 0 .. j-1 (lowest index among equals); then `iters`
 * Lloyd steps (nearest centroid, lowest index among equals; an empty cluster
 * keeps its centroid).  labels[P] (host) receive the cluster of each
 * particle, centroids (host, may be NULL) k x 9 features.  1 <= k <= P.
 * The clustering step of the multi-swarm search (Sec. III.B); usable alone.
 * Errors: SCS_EINVAL (sizes, k, iters outside 0 .. 1000), SCS_ENOMEM,
 * SCS_ECUDA. */
int scs_kmeans(scs_ctx *ctx, const double *pos, int64_t P, const double *prior_lo,
               const double *prior_hi, int k, int iters, int *labels, double *centroids,
               void *cuda_stream);

/* Re-cluster the swarms (Sec. III.B): for each data stream, k-means with
 * n_clusters centroids (seeded with that stream's swarm bests, then as
 * scs_kmeans) over all particles of its swarms; every non-empty cluster
 * becomes a swarm (particles renumbered: stream by stream, cluster by
 * cluster, in their previous order), so swarms can merge, split or appear;
 * the total number of particles is kept.  Bests are forgotten; each new
 * swarm takes the hyper-parameters of its stream's first old swarm.
 * Synchronous.
 * Errors: SCS_EINVAL (n_clusters outside 1 .. 1024, iters outside
 * 0 .. 1000), SCS_ENODATA (no swarm), SCS_ENOMEM, SCS_ECUDA. */
int scs_pso_regroup(scs_ctx *ctx, int n_clusters, int iters, void *cuda_stream);

/* The hierarchical search (Sec. III.B): for each rung r of the ladder
 * (n_rungs segment counts, e.g. {100, 50, 10, 1}): every swarm stream gets
 * N = ladder[r] equal-SNR^2 segments, every swarm the hyper-parameter row
 * hyper_rows[r] (Omega, Phi_P, Phi_G, eps[8]), the bests are reset, and
 * iterations run in CUDA graphs of chunk_iters until all swarms have
 * converged or max_iters have run (iters_out[r], may be NULL); between rungs
 * the swarms are re-clustered into n_clusters per stream (0: not).
 * Errors: SCS_EINVAL (ladder, rows or counts out of range), SCS_ENODATA,
 * SCS_ENOMEM, SCS_ECUDA. */
int scs_pso_search(scs_ctx *ctx, const int *ladder, int n_rungs, const double *hyper_rows,
                   int n_clusters, int chunk_iters, int max_iters, int64_t *iters_out,
                   void *cuda_stream);

/* Template h_A, h_E (Sec. IV: h_alpha = T_alpha(theta, f) A(f) e^{-i Psi(f)},
 * A(f) = f^{-7/6}) of one particle on the stream's grid, FP64, complex
 * interleaved, zero outside the support.
 *   theta  8 doubles; hA, hE  2K doubles each (host or device).
 * Errors: SCS_EINVAL (also for a non-physical theta), SCS_ENODATA,
 * SCS_ECUDA. */
int scs_waveform(scs_ctx *ctx, int stream_id, const double *theta, double *hA,
                 double *hE, void *cuda_stream);

/* As scs_waveform, and h_T of the third channel (T = (X + Y + Z)/sqrt3) in
 * hT (2K doubles, host or device), on any stream's grid.
 * Errors: as scs_waveform. */
int scs_waveform_aet(scs_ctx *ctx, int stream_id, const double *theta, double *hA,
                     double *hE, double *hT, void *cuda_stream);

/* Add an injection to the loaded data of a stream: d += snr h/sqrt(<h|h>)
 * with h the template of theta (Sec. IV: injected signals scaled to a target
 * SNR), over A, E and, on a stream loaded with scs_set_data_aet, T.
 * *hh_out (may be NULL) receives <h|h> of the un-normalised template.
 * Synchronous.
 * Errors: SCS_EINVAL, SCS_ENODATA, SCS_ECUDA. */
int scs_inject(scs_ctx *ctx, int stream_id, const double *theta, double snr,
               double *hh_out);

/* Support and anchor stride of P particles (diagnostics): k_lo[P], k_hi[P]
 * (the bins with f >= f0, t(f) <= T_obs and v <= 6^{-1/2}, Sec. IV;
 * k_hi < k_lo: empty; both -1: non-physical) and the mixed path's
 * strides (may be NULL): bits 0-7 log2 of the phase-anchor stride B, bits
 * 8-15 log2 of the response sub-span Br.  Host or device pointers.
 * Errors: SCS_EINVAL, SCS_ENODATA, SCS_ENOMEM, SCS_ECUDA. */
int scs_support(scs_ctx *ctx, int stream_id, const double *params, int64_t P,
                int64_t *k_lo, int64_t *k_hi, int32_t *log2_stride,
                void *cuda_stream);

/* Segment edges of P particles under the stream's segmentation (Sec. II.B:
 * equal width, or equal squared SNR per segment): e[P x (N+1)] with segment
 * n = [e_n, e_{n+1}) in grid bins (int64, host or device).
 * Errors: SCS_EINVAL, SCS_ENODATA, SCS_ENOMEM, SCS_ECUDA. */
int scs_segment_edges(scs_ctx *ctx, int stream_id, const double *params,
                      int64_t P, int64_t *edges, void *cuda_stream);

/* Stage timing of scs_eval_stat (CUDA events recorded on the call's
 * stream while enabled; adds no synchronisation to the call itself).
 * scs_last_timings blocks until the last profiled call has finished and
 * writes ms[4]: particle set-up and work list, segment edges, main
 * evaluation kernel, cross-chunk fix-up.
 * Errors: SCS_EINVAL, SCS_ENODATA (nothing profiled yet), SCS_ECUDA. */
int scs_set_profiling(scs_ctx *ctx, int enable);
int scs_last_timings(scs_ctx *ctx, double *ms);

/* Counters of the last profiled scs_eval_stat / scs_batch_eval (profiling
 * enabled; blocks until that call has finished): out[0] = particles
 * evaluated, out[1] = particles whose equal-SNR^2 edges were recomputed from
 * FP64 anchor powers because an edge lay within the double-float guard band
 * of a bin boundary (-1 if the call computed no equal-SNR^2 edges); entries
 * from 2 on are 0.  n >= 1 entries are written.
 * Errors: SCS_EINVAL, SCS_ENODATA (nothing profiled yet), SCS_ECUDA. */
int scs_last_counters(scs_ctx *ctx, int64_t *out, int n);

/* Index checks of the debug build.  A library compiled with -DSCS_DEBUG
 * (the package's build.build(debug=True): _build/libscstat_debug.so; the
 * Python binding loads it when the environment has SCS_DEBUG=1) tests the
 * indices of the evaluation kernels' accesses -- data and weight loads,
 * work-list slots, (particle, chunk) records, edge tables, the grid table and
 * the equal-SNR^2 anchor slots -- against the sizes of their arrays; a
 * failing test skips its access (so a bad index is reported instead of
 * reading or writing out of bounds) and the first failure is kept.  This call
 * waits for the device, then reads and clears that record:
 *   check  0 if no test failed, else which: 1 data or weight load, 2 work-list
 *          slot, 3 record, 4 edge table, 5 grid table, 6 anchor slots;
 *   index  the failing index, clamped to [0, 2^48 - 1] (-1 if none).
 * Returns SCS_OK in a debug build; otherwise SCS_EUNSUPPORTED with check = 0
 * (the normal build has no tests).  Errors: SCS_EINVAL (null argument),
 * SCS_ECUDA. */
int scs_debug_error(scs_ctx *ctx, int *check, long long *index);

/* scs_eval_stat without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc at evaluation time -- services whose device memory is entirely
 * owned by another allocator (a memory pool sized at start-up leaves
 * nothing for a library to take), and loops that must not pay an
 * allocation's latency or its implicit device synchronisation.
 *   Same evaluation as scs_eval_stat (path and segmentation of the context
 *   and stream), without per-segment outputs.  params (P x 8) and stat (P)
 *   must be device memory.  Asynchronous on cuda_stream (NULL: the
 *   context's stream).
 *   Scratch: a fixed 64 MiB device array inside the library, held by every
 *   GPU that loads it until the process exits; no cudaMalloc, cudaFree or
 *   allocating library routine is called.  Calls whose scratch would exceed
 *   it are rejected with SCS_EINVAL and a message giving the bytes needed
 *   (roughly 20 + 75 C bytes per particle, C = ceil(K/4096) chunks, plus
 *   4 (N+1) + 16 (K/1024 + 2) bytes per particle for equal-SNR^2 segments).
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress, a synchronous runtime call); later calls on that
 *   device reuse it.
 *   The stream table of the call is handed to the device as a kernel
 *   argument, so no host buffer is read after the call returns.
 *   Every call shares the array and it keeps the previous call's contents:
 *   calls that overlap on the GPU (different streams, or different contexts
 *   on one device) race and must be serialised by the caller.
 * The stream's data (scs_set_data or scs_set_data_aet) and segmentation must already be set.
 * Errors: SCS_EINVAL (sizes, host pointers), SCS_ENODATA, SCS_ECUDA,
 * SCS_EUNSUPPORTED (device index >= 64). */
int scs_eval_stat_noalloc(scs_ctx *ctx, int stream_id, const double *params,
                          int64_t P, double *stat, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SCSTAT_H */
