/*
 * ec3r.h - C ABI of the B300 (sm_103a) hot path of EC3R-SLAM submap fusion.
 *
 * The paper (EC3R-SLAM, arXiv 2510.02080) builds local submaps with a
 * feed-forward model, registers every new submap against connected submaps
 * through the keyframes they share with a weighted Umeyama Sim(3) solve
 * (Sec. III-C, "Sim3 Point Cloud Registration", Eq. (sim3)), adds the
 * results as relative Sim(3) constraints to a submap pose graph
 * (Sec. III-E), and places every submap point in global coordinates
 * (Sec. III-C, "Point Correction").  This library does those three steps on
 * the GPU, batched, plus the reverse-mode derivative of the registration.
 *
 * Conventions shared by every call
 *  - All pointers named d_* are device pointers (cudaMalloc'd or equivalent,
 *    on the context's device); h_* are host pointers.  The caller owns every
 *    buffer it passes; the library never frees or keeps them past the call.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL means the legacy default stream).  A returned EC3R_OK means the
 *    arguments were valid and the work was enqueued; per-pair and device-side
 *    conditions (degenerate pairs, non-positive pivots, capacity overflow,
 *    timeouts) are reported in device status words and by
 *    ec3r_sync_status().
 *  - The context owns its workspace.  A call that needs more workspace than
 *    the context holds grows it (cudaMalloc) before enqueueing; such a call
 *    must not be made while `stream` is being captured into a CUDA graph
 *    (it returns EC3R_ERR_CAPTURE instead).
 *  - One context per host thread / stream at a time; contexts are
 *    independent.
 *  - Similarities act as x -> s R x + t; R is row-major.
 */
#ifndef EC3R_H
#define EC3R_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EC3R_OK = 0,
  EC3R_ERR_INVALID_ARG = 1, /* bad pointer, size or option; nothing enqueued */
  EC3R_ERR_CUDA = 2,        /* a CUDA runtime call failed; see ec3r_last_error */
  EC3R_ERR_OOM = 3,         /* workspace allocation failed */
  EC3R_ERR_CAPACITY = 4,    /* fuse_points: output capacity exceeded */
  EC3R_ERR_NOT_SPD = 5,     /* pose graph: non-positive pivot in Cholesky */
  EC3R_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
  EC3R_ERR_DEGENERATE = 7,  /* at least one registration pair was degenerate */
  EC3R_ERR_CAPTURE = 8      /* workspace growth requested during stream capture */
} ec3r_status;

/* Per-pair status bits written by ec3r_align_submaps (0 = solved). */
#define EC3R_PAIR_FEW_POINTS 1u  /* fewer than 3 valid correspondences */
#define EC3R_PAIR_ZERO_WEIGHT 2u /* total weight <= 0 or not finite */
#define EC3R_PAIR_RANK 4u        /* source variance <= 0 or sigma2 <= 1e-4 sigma1 */
#define EC3R_PAIR_NONFINITE 8u   /* non-finite moments or result */
#define EC3R_PAIR_BAD_INPUT 16u  /* link offsets or frame indices out of range */

typedef struct {
  double s;     /* scale, > 0 */
  double R[9];  /* rotation, row-major */
  double t[3];  /* translation */
} ec3r_sim3;

typedef struct ec3r_ctx ec3r_ctx;

/* Create a context on CUDA device `device`.  Allocates its status words. */
ec3r_status ec3r_create(ec3r_ctx** out, int device);
/* Destroy a context and free its workspace (synchronises the device). */
void ec3r_destroy(ec3r_ctx* ctx);
/* Human-readable text of the last error of this context (never NULL). */
const char* ec3r_last_error(const ec3r_ctx* ctx);
const char* ec3r_status_string(ec3r_status st);
/* Library version, e.g. "ec3r 0.1 sm_103a". */
const char* ec3r_version(void);

/*
 * Wait for `stream`, then read and clear the context's device status words.
 * Returns EC3R_ERR_CAPACITY, EC3R_ERR_NOT_SPD, EC3R_ERR_TIMEOUT or
 * EC3R_ERR_INVALID_ARG (an index argument was out of range) if one of those
 * was raised by work enqueued since the last call, EC3R_ERR_CUDA if the
 * stream reports an error, else EC3R_OK.  Degenerate registration pairs are
 * reported in the per-pair status array, not here.
 */
ec3r_status ec3r_sync_status(ec3r_ctx* ctx, void* stream);

/*
 * Bounded waits.  A kernel that waits on work of other CTAs or on its own
 * asynchronous copies (the persistent registration's per-pair solves, the
 * tensor-core similarity's mbarriers) gives up after a limit, raises
 * EC3R_ERR_TIMEOUT at ec3r_sync_status and returns; the context stays usable.
 * ec3r_set_wait_limit sets that limit in seconds (0: the default of two
 * seconds; at most 3600) for later calls of this context.
 *
 * ec3r_inject makes such a wait run out on purpose, for tests of that path
 * (no fault, trap or unbounded wait is involved): EC3R_INJECT_LOOPS_NO_COPY -
 * the similarity kernel's producer starts no copy, so its MMA thread's first
 * wait gives up; EC3R_INJECT_ALIGN_NO_EPOCH - the registration's solves publish
 * no epoch, so the next sweep's waits give up.  0 turns injection off.  Both
 * calls drop the context's cached graphs.  EC3R_ERR_INVALID_ARG for a bad
 * value.
 */
#define EC3R_INJECT_LOOPS_NO_COPY 1u
#define EC3R_INJECT_ALIGN_NO_EPOCH 2u
ec3r_status ec3r_set_wait_limit(ec3r_ctx* ctx, double seconds);
ec3r_status ec3r_inject(ec3r_ctx* ctx, unsigned what);

/*
 * Tracing.  With profiling on, calls launch their kernels directly (no cached
 * graph) and bracket every kernel launch with a CUDA event pair recorded on
 * the launching stream.  ec3r_profile_read waits for those events, returns
 * per kernel name the summed duration (ms) and the launch count, in first-
 * launch order, and clears the record.  `names` receives up to `max_kernels`
 * NUL-terminated names of `name_len` bytes each; *n_kernels the number of
 * distinct kernels recorded (which may exceed max_kernels).
 */
ec3r_status ec3r_profile(ec3r_ctx* ctx, int enable);
ec3r_status ec3r_profile_read(ec3r_ctx* ctx, int max_kernels, char* names, int name_len,
                              double* total_ms, int64_t* launches, int* n_kernels);

/* ------------------------------------------------------------------------ */
/* Registration: batched Huber-IRLS weighted Umeyama (Sec. III-C, Eq. (sim3))*/
/* ------------------------------------------------------------------------ */

typedef enum { EC3R_PREC_FP32C = 0, EC3R_PREC_FP64 = 1 } ec3r_precision;
typedef enum { EC3R_WEIGHT_PRODUCT = 0, EC3R_WEIGHT_SRC = 1 } ec3r_weight_rule;

typedef struct {
  float huber_delta; /* Huber threshold on |s R p + t - q| (target units), > 0 */
  int iters;         /* number of weighted Umeyama solves, 1..64 */
  float conf_min;    /* valid iff c_p > conf_min and c_q > conf_min */
  int weight_rule;   /* ec3r_weight_rule: w = c_p c_q or w = c_p */
  int precision;     /* ec3r_precision: FP32 blocked/pairwise moments or FP64 */
  int want_cost;     /* 1: also write the final weighted residual (one more sweep) */
} ec3r_align_opts;

/* Fills `o` with the defaults: delta 0.02, 10 iterations, conf_min 0,
 * product weights, FP32 moments, no cost. */
void ec3r_align_opts_default(ec3r_align_opts* o);

/*
 * Register `n_pairs` submap pairs in one batched call (Sec. III-C, Eq. (sim3)
 * and the weighted Umeyama solution it names, wrapped in Huber IRLS).
 *
 * Frames.  d_xyz is a bank of `n_frames` pointmaps, float32 [n_frames][hw][3]
 * (x, y, z interleaved per pixel, as the feed-forward model writes them), and
 * d_conf their confidences, float32 [n_frames][hw].  Both are read only.
 *
 * Pairs.  Pair k owns links d_link_off[k] .. d_link_off[k+1]-1 (int32
 * [n_pairs+1], device, non-decreasing, d_link_off[0] = 0 and
 * d_link_off[n_pairs] = n_links).  Link l says that pixel i of frame
 * d_src[l] (a point p_i of the current submap) and pixel i of frame
 * d_tgt[l] (its counterpart q_i in the other submap) are the same keyframe
 * pixel: the correspondences of Sec. III-C.  Frame indices must lie in
 * [0, n_frames).  Offsets that do not form such an array (out of range,
 * decreasing anywhere, wrong first or last value) mark every pair of the call
 * EC3R_PAIR_BAD_INPUT; a link with an out-of-range frame marks its pair.
 * Nothing out of range is read, and either case raises EC3R_ERR_INVALID_ARG at
 * ec3r_sync_status.  A pair with no link is degenerate (EC3R_PAIR_FEW_POINTS).
 *
 * Weights.  Correspondence i is valid when p_i, q_i, c_p, c_q are finite and
 * c_p > cmin and c_q > cmin, where cmin = d_pair_conf_min[k] if that
 * pointer is non-NULL (float32 [n_pairs]) else opts->conf_min.  Its base
 * weight is w_i = c_p c_q (or c_p).  Normalising the weights does not change
 * the solution, so none is applied.
 *
 * Iteration.  Solve 1 uses w; solve k >= 2 uses w_i h_i with
 * h_i = min(1, delta / r_i), r_i = |s R p_i + t - q_i| under solve k-1.
 *
 * Output.  d_out[k] (device) receives the last solve, mapping p to q;
 * d_pair_status[k] (int32, device) the EC3R_PAIR_* bits (0 = solved; a
 * degenerate pair gets the identity).  d_pair_cost (nullable, float64
 * [n_pairs]) receives sum omega r(S)^2 / sum omega with the last weights
 * when opts->want_cost is set.  With FP32 moments the last sweep and solve
 * then run in a second kernel that also forms the cost's sums, so the results
 * with and without want_cost differ at FP32 rounding level, as between sweep
 * variants.
 *
 * Launches.  A set-up kernel, then, with FP32 moments, two persistent
 * launches that run every sweep and solve: the first sweep, which also stores
 * each correspondence's weight (NaN where it is invalid), then the later
 * sweeps, which read that weight in place of both confidences (28 instead of
 * 32 bytes per correspondence) and start as the first launch's CTAs retire.
 * Tiles of pixels are handed out iteration by iteration to resident CTAs, the
 * CTA that completes a pair's tiles of an iteration solves that pair, and a
 * pair's next sweep waits only for its own solve (a bounded wait: one that
 * runs out raises EC3R_ERR_TIMEOUT at ec3r_sync_status).  With want_cost the
 * last sweep is one more launch that starts as the persistent CTAs retire and
 * also accumulates the sums from which the cost under the last solve follows
 * exactly (no extra pass over the correspondences).  With FP64 accumulation,
 * `iters` x (sweep, solve) grids and, with want_cost, a cost sweep.
 * Replayed from a CUDA graph cached per argument set when `stream` is not
 * itself being captured.
 *
 * Variants.  The FP32 path has variants (pixels per tile x CTAs per SM of the
 * persistent launch, and one grid per sweep and per solve instead:
 * ec3r_align_variant_info).  The tile size groups the FP32 sums, so results
 * of different variants differ at FP32 rounding level; each variant is
 * deterministic.  Unless one is forced (ec3r_align_set_variant), the first
 * call of each problem-size bucket (the power of two of the link pixels and
 * of the pair count) on 16-byte aligned pointmaps with hw a multiple of 4
 * times every variant on its own inputs - three runs each after a warm-up,
 * synchronising with `stream` - and the fastest serves the bucket from then
 * on; such a first call must not be made while `stream` is captured (a
 * captured first call uses variant 0 untimed).  Other pointmaps use one fixed
 * configuration.
 *
 * Workspace: 4 bytes per link pixel (the stored weights, which
 * ec3r_align_submaps_backward also reads), 300 bytes per 4096 link pixels,
 * 4 bytes per link, and per pair
 * 444 bytes plus 448 bytes per iteration (the checkpoints that
 * ec3r_align_submaps_backward reuses).
 */
ec3r_status ec3r_align_submaps(ec3r_ctx* ctx, const float* d_xyz, const float* d_conf,
                               int64_t n_frames, int64_t hw, int n_pairs, int64_t n_links,
                               const int32_t* d_link_off, const int32_t* d_src,
                               const int32_t* d_tgt, const float* d_pair_conf_min,
                               const ec3r_align_opts* opts, ec3r_sim3* d_out,
                               int32_t* d_pair_status, double* d_pair_cost, void* stream);

/*
 * Reverse-mode derivative of ec3r_align_submaps (the paper has no gradient;
 * this differentiates the registration above, for training on top of it).
 *
 * Same inputs and options as the forward call (FP32 moments only).  Given
 * d_grad_S (float64 [n_pairs][13], device: dL/ds, dL/dR row-major, dL/dt of
 * each pair's output) and d_grad_cost (float64 [n_pairs], device, nullable:
 * dL/dcost of the weighted residual that want_cost reports), it writes the
 * gradient with respect to every input point and confidence of the frame
 * bank: d_grad_xyz (float32 [n_frames][hw][3]) and d_grad_conf (float32
 * [n_frames][hw]); frames used by several links receive the sum, accumulated
 * in link order (deterministic).  Invalid correspondences and degenerate pairs
 * get zero.
 *
 * Checkpoints.  Every ec3r_align_submaps call keeps, in its context, the
 * estimate and the moments of every solve, each pair's final status and its
 * cost, and issues a new token (ec3r_align_token).  With fwd_token = 0 the
 * backward call first runs the forward pass itself (into context-owned
 * outputs, with want_cost = 1 exactly when d_grad_cost is given) and uses its
 * checkpoints: always correct.  With fwd_token = the
 * token of the last ec3r_align_submaps call on this context, the backward
 * call reuses that call's checkpoints instead; that call must have had the
 * same inputs (pointers and sizes) and options, and want_cost = 1 if
 * d_grad_cost is given, else EC3R_ERR_INVALID_ARG (nothing enqueued).  By
 * passing a token the caller asserts that the frames, confidences, links and
 * thresholds have not been modified since that call (the library cannot see
 * an in-place rewrite); that call's output buffers are never read, so they
 * may have been freed or reused.
 * It then differentiates all `iters` solves, unrolled (the Huber weights of
 * solve k depend on solve k-1): one reduction sweep per Huber iteration
 * (iters - 1 of them; the sums of the cost term come from the forward's last
 * sweep) and one final sweep that writes the per-point gradients.  The rotation is
 * differentiated in its polar form, with 1/(d_i + d_j) factors.  The Huber
 * weight has a kink at r = delta; there the one-sided derivative of the
 * branch taken by the FP32 forward is used.
 *
 * Errors: EC3R_ERR_INVALID_ARG (nothing enqueued) for a NULL context, opts,
 * d_grad_xyz or d_grad_conf, a NULL d_grad_S with n_pairs > 0, n_pairs < 0,
 * opts->precision other
 * than EC3R_PREC_FP32C, or a fwd_token that does not qualify (above);
 * n_pairs = 0 only zeroes d_grad_xyz and d_grad_conf.  The forward call's own checks apply when it is
 * run with fwd_token = 0.
 * Workspace (context-owned, beyond the forward's): 96 bytes per tile of 8192
 * pixels, 32 bytes per link pixel (per-link gradients, summed into frames
 * that several links share), 348 bytes per pair plus 136 bytes per pair and
 * iteration, and 4 bytes per frame.
 */
ec3r_status ec3r_align_submaps_backward(ec3r_ctx* ctx, const float* d_xyz, const float* d_conf,
                                        int64_t n_frames, int64_t hw, int n_pairs,
                                        int64_t n_links, const int32_t* d_link_off,
                                        const int32_t* d_src, const int32_t* d_tgt,
                                        const float* d_pair_conf_min, const ec3r_align_opts* opts,
                                        uint64_t fwd_token, const double* d_grad_S,
                                        const double* d_grad_cost, float* d_grad_xyz,
                                        float* d_grad_conf, void* stream);

/*
 * Sweep variants of ec3r_align_submaps (FP32 moments): their count, and for
 * variant v its tile size (pixels), CTAs per SM and whether it is the
 * persistent launch (1) or one grid per sweep and per solve (0)
 * (EC3R_ERR_INVALID_ARG for v out of range).  ec3r_align_set_variant forces
 * variant v for every later call on the context, or, with v = -1 (the
 * default), lets each size bucket use the variant its first call timed
 * fastest.  ec3r_align_last_variant gives the variant of the last call (-1: a
 * mode without variants) and, if ms is not NULL (float
 * [ec3r_align_variant_count()]), every variant's median time in ms from the
 * timing of that call's bucket (-1 where none was measured).
 */
/*
 * Share of the SMs that the backward call's reduction sweeps take (the
 * HBM-bound part of ec3r_align_submaps_backward).  With ctas_per_sm = 0 (the
 * default) each sweep launches one CTA per tile of 8192 link pixels, as many
 * resident per SM as fit (four): the fastest sweep when nothing else runs.
 * With 1..4 each sweep launches ctas_per_sm CTAs per SM that stride over the
 * tiles, which leaves room on every SM for latency-bound work that the caller
 * runs beside the backward call on another stream (for instance the pose
 * graph).  The gradients are bit-identical for every value (each tile's
 * partial sums have a fixed slot).  Later calls of this context use the
 * value; a change drops the context's cached graphs.  EC3R_ERR_INVALID_ARG for
 * a NULL context or a value outside 0..4.
 */
ec3r_status ec3r_align_backward_set_ctas_per_sm(ec3r_ctx* ctx, int ctas_per_sm);

int ec3r_align_variant_count(void);
ec3r_status ec3r_align_variant_info(int v, int* tile_pixels, int* ctas_per_sm,
                                    int* persistent);
ec3r_status ec3r_align_set_variant(ec3r_ctx* ctx, int v);
ec3r_status ec3r_align_last_variant(const ec3r_ctx* ctx, int* variant, float* ms);

/*
 * Token of the last successful ec3r_align_submaps call on this context (a new
 * nonzero value per call; 0 if there is none, or if the last call failed),
 * for ec3r_align_submaps_backward.  NULL context: 0.
 */
uint64_t ec3r_align_token(const ec3r_ctx* ctx);

/*
 * Registration without allocation.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory at all, such
 * as code running inside a memory arena it does not own, real-time loops
 * where an allocation's implicit synchronisation and unbounded latency are
 * not allowed, or hosts whose allocator belongs to another framework.
 *
 * It computes exactly what ec3r_align_submaps computes, with the same
 * arguments (minus the context) and the same kernels, but its scratch lives
 * in one fixed device array inside the library (about 2.8 MB, held on every
 * GPU that loads the library until the process exits).  It calls no
 * cudaMalloc or cudaFree and needs no context.  Limits, checked before any
 * work is enqueued (EC3R_ERR_INVALID_ARG when exceeded):
 *   n_pairs <= EC3R_NOALLOC_MAX_PAIRS, n_links <= EC3R_NOALLOC_MAX_LINKS,
 *   n_links * ceil(hw / 8192) <= EC3R_NOALLOC_MAX_TILES.
 * It runs on the current CUDA device.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (each call resets what must start fresh): calls whose
 * work overlaps on the GPU - on different streams, or from different
 * threads - race and corrupt each other; serialise them.  Out-of-range
 * offsets or frames are reported only in d_pair_status (EC3R_PAIR_BAD_INPUT).
 */
#define EC3R_NOALLOC_MAX_PAIRS 1024
#define EC3R_NOALLOC_MAX_LINKS 4096
#define EC3R_NOALLOC_MAX_TILES 16384
ec3r_status ec3r_align_submaps_noalloc(const float* d_xyz, const float* d_conf,
                                       int64_t n_frames, int64_t hw, int n_pairs,
                                       int64_t n_links, const int32_t* d_link_off,
                                       const int32_t* d_src, const int32_t* d_tgt,
                                       const float* d_pair_conf_min,
                                       const ec3r_align_opts* opts, ec3r_sim3* d_out,
                                       int32_t* d_pair_status, double* d_pair_cost,
                                       void* stream);

/* ------------------------------------------------------------------------ */
/* Registration straight from depth maps and cameras (Sec. III-C: a submap   */
/* is the inverse projection of the predicted depths through the predicted   */
/* cameras, one point per keyframe pixel)                                    */
/* ------------------------------------------------------------------------ */

/* A frame's pinhole camera and its pose in its submap. */
typedef struct {
  float fx, fy, cx, cy; /* focal lengths and principal point, pixels */
  float R[9];           /* camera -> submap rotation, row-major */
  float t[3];           /* camera -> submap translation */
} ec3r_camera;          /* 64 bytes */

/*
 * The registration of ec3r_align_submaps applied to the pointmaps
 *   X(v, u) = R (d(v, u) * ((u - cx) / fx, (v - cy) / fy, 1)) + t
 * of every frame (pixel row v, column u; u, v integers; d the depth along the
 * optical axis), without forming them: each link is swept in its two cameras'
 * frames and reads 4-byte depths (16 bytes per correspondence with the
 * confidences instead of 32).  A pixel whose depth is not finite or not > 0
 * is invalid (like a non-finite point).
 *
 * d_depth and d_conf: float32 [n_frames][H][W], device.  d_cams: ec3r_camera
 * [n_frames], device.  Pairs, links, pair thresholds, options, outputs,
 * statuses and the cost are as for ec3r_align_submaps (the output Sim(3) maps
 * src-submap coordinates to tgt-submap coordinates), except that only FP32
 * moments are offered (opts->precision must be EC3R_PREC_FP32C) and the call
 * keeps no checkpoints for ec3r_align_submaps_backward.  H * W < 2^31.
 * Workspace is context-owned; first calls (and calls with larger problems)
 * allocate and must not be captured.
 */
ec3r_status ec3r_align_submaps_depth(ec3r_ctx* ctx, const float* d_depth, const float* d_conf,
                                     const ec3r_camera* d_cams, int64_t n_frames, int H, int W,
                                     int n_pairs, int64_t n_links, const int32_t* d_link_off,
                                     const int32_t* d_src, const int32_t* d_tgt,
                                     const float* d_pair_conf_min, const ec3r_align_opts* opts,
                                     ec3r_sim3* d_out, int32_t* d_pair_status,
                                     double* d_pair_cost, void* stream);

/* ------------------------------------------------------------------------ */
/* Pose graph: Sim(3) submap poses refined by Gauss-Newton (Sec. III-E)     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int iters;          /* Gauss-Newton iterations, 0..1000 */
  int fixed_node;     /* node held constant (gauge), 0 <= fixed_node < n_nodes */
  double lm_lambda;   /* >= 0; the normal matrix is H + lm_lambda I (0: Gauss-Newton) */
  int init_by_chaining; /* 1: first set every node by chaining relative transforms */
  int lm_adaptive;    /* 1: Levenberg-Marquardt with adaptive damping from lm_lambda > 0 */
} ec3r_pg_opts;

/* Fills `o` with the defaults: 10 iterations, node 0 fixed, lambda 0, chaining on,
 * fixed damping. */
void ec3r_pg_opts_default(ec3r_pg_opts* o);

/*
 * Refine submap poses d_nodes (ec3r_sim3 [n_nodes], device, in/out: submap ->
 * world) against the relative transforms of `n_edges` edges, minimising
 * chi^2 = sum_e e_e^T Omega_e e_e with e = log_Sim3(T_ij^-1 T_i^-1 T_j)
 * (Sec. III-E), so an edge (i, j) is satisfied when T_j = T_i T_ij.
 *
 * Structure.  h_i, h_j (int32 [n_edges], HOST) give each edge's endpoints,
 * in [0, n_nodes) and distinct.  The structure is analysed on the host once
 * (nested-dissection or minimum-degree ordering, whichever is estimated
 * cheaper; block fill of the Cholesky factor) and cached
 * in the context; a call with a new structure allocates and must not be made
 * during stream capture (EC3R_ERR_CAPTURE).  The first pose-graph call of a
 * context also uploads a constant table.  A structure whose factor ends in a
 * dense block of more than 3200 nodes is rejected (EC3R_ERR_INVALID_ARG).
 *
 * Data.  d_Tij (ec3r_sim3 [n_edges], device) are the measured T_ij; d_info
 * (float64 [n_edges][49], row-major symmetric Omega, device) or NULL for the
 * identity.  The tangent order is (rho, phi, sigma): translation, rotation
 * vector, log-scale; T <- T Exp(delta) is the update.
 *
 * Chaining.  With init_by_chaining, every node except the fixed one is first
 * set by composing relative transforms along a spanning tree made of the
 * edges, in input order, that join two unconnected parts of the graph, walked
 * from the fixed node (T_j = T_i T_ij along an edge, T_i = T_j T_ij^-1
 * against it); nodes not connected to the fixed node become the identity.
 *
 * Iteration.  `iters` Gauss-Newton steps on all nodes but the fixed one, each
 * solving (H + lambda I) delta = -g by an FP64 block Cholesky factorisation.
 * d_chi2 (float64 [iters+1], device, nullable) receives chi^2 before each
 * step and after the last.  A non-positive pivot skips that step's update and
 * raises EC3R_ERR_NOT_SPD at ec3r_sync_status.
 *
 * With lm_adaptive = 1 the iterations are Levenberg-Marquardt (the paper's
 * choice): lambda starts at lm_lambda (0 < lm_lambda <= 1e10); a step is kept
 * when its factorisation succeeds and chi^2 decreases, and lambda is divided by
 * 10 (not below 1e-10); otherwise the poses are restored and lambda is
 * multiplied by 10 (not above 1e10).  A rejected step is not an error.
 */
ec3r_status ec3r_pose_graph_correct(ec3r_ctx* ctx, int n_nodes, ec3r_sim3* d_nodes, int n_edges,
                                    const int32_t* h_i, const int32_t* h_j,
                                    const ec3r_sim3* d_Tij, const double* d_info,
                                    const ec3r_pg_opts* opts, double* d_chi2, void* stream);

/* ------------------------------------------------------------------------ */
/* Fusion: confidence-filtered transform of submap points into the global   */
/* map (Sec. III-C "Point Correction": global coordinates of all points)    */
/* ------------------------------------------------------------------------ */

/*
 * Append every point of `n_submaps` submaps whose confidence is strictly
 * greater than `conf_threshold` (NaN is dropped) to a global point buffer,
 * transformed by its submap's pose.
 *
 * d_xyz float32 [n_submaps][pts_per_submap][3] and d_conf float32
 * [n_submaps][pts_per_submap] hold the submaps (pts_per_submap = frames*H*W;
 * flat point g = m*pts_per_submap + i in submap-major order).  d_poses[m]
 * (ec3r_sim3, device) maps submap m to the world; the point is computed in
 * float32 from the float32-rounded pose (s R rounded once, then FMA).
 *
 * Kept points are written in ascending g at positions *d_cursor,
 * *d_cursor + 1, ...: d_out_xyz float32 [capacity][3] and d_out_idx int64
 * [capacity] (= index_base + g).  *d_cursor (int64, device, in/out) is
 * advanced by the number of kept points, so successive calls stream into one
 * buffer.  Positions at or beyond `capacity` are not written; the cursor
 * still advances and ec3r_sync_status then returns EC3R_ERR_CAPACITY.
 * Workspace: 1036 bytes per 8192 points (tile counts, offsets, keep mask).
 */
ec3r_status ec3r_fuse_points(ec3r_ctx* ctx, int n_submaps, int64_t pts_per_submap,
                             const float* d_xyz, const float* d_conf, const ec3r_sim3* d_poses,
                             float conf_threshold, int64_t index_base, float* d_out_xyz,
                             int64_t* d_out_idx, int64_t capacity, int64_t* d_cursor,
                             void* stream);

/*
 * The same fusion in two calls, for callers that know the confidences before
 * the poses (the count needs no pose, so it can run while the poses are
 * still being corrected).
 *
 * ec3r_fuse_count writes, for every tile of 8192 consecutive points of every
 * submap (tile t = m * ceil(pts_per_submap / 8192) + i / 8192 for point i of
 * submap m), its number of kept points to d_tile_counts[t] (int32
 * [n_tiles], device, caller-owned) and its keep mask to d_keep_mask (uint32
 * [n_tiles * 256], device, caller-owned: bit j % 32 of word t * 256 + j / 32
 * says whether point j of tile t is kept; bits past a tile's last point are
 * 0).  ec3r_fuse_points_counted then scans the counts and scatters the points
 * the mask keeps, without reading the confidences, and produces exactly the
 * output of ec3r_fuse_points with the same d_conf and conf_threshold (the
 * other arguments as there).  The counts and the mask are not checked.
 */
ec3r_status ec3r_fuse_count(ec3r_ctx* ctx, int n_submaps, int64_t pts_per_submap,
                            const float* d_conf, float conf_threshold, int32_t* d_tile_counts,
                            uint32_t* d_keep_mask, void* stream);
ec3r_status ec3r_fuse_points_counted(ec3r_ctx* ctx, int n_submaps, int64_t pts_per_submap,
                                     const float* d_xyz, const int32_t* d_tile_counts,
                                     const uint32_t* d_keep_mask, const ec3r_sim3* d_poses,
                                     int64_t index_base, float* d_out_xyz, int64_t* d_out_idx,
                                     int64_t capacity, int64_t* d_cursor, void* stream);

/*
 * ec3r_fuse_points on the pointmaps of depth frames (Sec. III-C: submaps are
 * the inverse projection of the predicted depths through the predicted
 * cameras), without forming them.  Frame f of submap m is d_depth / d_conf
 * float32 [n_submaps*frames][H][W] entry m*frames + f with camera
 * d_cams[m*frames + f] (ec3r_camera, device; pixel and camera conventions of
 * ec3r_align_submaps_depth).  A pixel has a point when its frame's camera is
 * finite with nonzero focal lengths and its depth is finite and > 0; it is kept
 * when, in addition, its confidence is strictly greater than conf_threshold.
 * The kept point is s_m R_m (R_f x + t_f) + t_m with x the camera-frame point,
 * evaluated in float32 from the composite pose rounded once to float32.
 * Outputs, flat indices (g = index_base + (m*frames + f)*H*W + v*W + u),
 * cursor and capacity behave exactly as in ec3r_fuse_points.  H * W < 2^31.
 * Reads 8 bytes per pixel twice (count and scatter) instead of 4 + 16.
 */
ec3r_status ec3r_fuse_points_depth(ec3r_ctx* ctx, int n_submaps, int frames, int H, int W,
                                   const float* d_depth, const float* d_conf,
                                   const ec3r_camera* d_cams, const ec3r_sim3* d_poses,
                                   float conf_threshold, int64_t index_base, float* d_out_xyz,
                                   int64_t* d_out_idx, int64_t capacity, int64_t* d_cursor,
                                   void* stream);

/* ------------------------------------------------------------------------ */
/* Point correction (Sec. III-C "Point Correction"): sparse-map points that  */
/* correspond to submap pixels take those pixels' global coordinates         */
/* ------------------------------------------------------------------------ */

/*
 * For every sparse-map point i (d_points float32 [n_points][3], device,
 * in/out) with a reference d_refs[i] = g (int64, device: the flat submap point
 * g = m*pts_per_submap + k of ec3r_fuse_points, or -1 for none), replace the
 * point by T_m(X_g) when the submap point is valid: its confidence is
 * strictly greater than conf_threshold and its coordinates are finite; the
 * point is computed exactly as ec3r_fuse_points computes the fused point of
 * g (float32 from the float32-rounded pose, same FMA order).  Other points are
 * left unchanged.  d_xyz / d_conf / d_poses as for ec3r_fuse_points.
 * d_n_corrected (int64, device, nullable) is incremented by the number of
 * corrected points.  A reference < -1 or >= n_submaps*pts_per_submap leaves
 * its point unchanged and makes ec3r_sync_status return EC3R_ERR_INVALID_ARG.
 * No workspace; one launch.
 */
ec3r_status ec3r_correct_points(ec3r_ctx* ctx, int64_t n_points, float* d_points,
                                const int64_t* d_refs, int n_submaps, int64_t pts_per_submap,
                                const float* d_xyz, const float* d_conf,
                                const ec3r_sim3* d_poses, float conf_threshold,
                                int64_t* d_n_corrected, void* stream);

/* ------------------------------------------------------------------------ */
/* Global loop retrieval (Sec. III-D "Loop Retrieval and Verification")     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int stride;       /* similarities between every stride-th keyframe (the paper's N) */
  int radius;       /* neighbourhood half-width around a similar pair, keyframes */
  int gap;          /* minimum keyframe distance j - i of a loop */
  float tau_global; /* coarse threshold (paper: 0.93) */
  float tau_local;  /* neighbourhood threshold (paper: 0.96) */
} ec3r_loop_opts;

typedef struct {
  int a, b;         /* coarse pair: sampled keyframes a*stride < b*stride */
  int i, j;         /* best keyframe pair of its neighbourhood, i < j */
  float s_coarse;   /* cosine of a and b from the BF16 tensor-core contraction */
  float s;          /* cosine of i and j in FP32 */
} ec3r_loop;        /* 24 bytes */

/*
 * Loop candidates among n keyframe embeddings d_emb (float32 [n][d], device;
 * d a positive multiple of 64).  Similarity is the cosine of two embeddings.
 * Every stride-th keyframe is normalised in FP32 and rounded to BF16; their
 * similarity matrix S = A A^T (upper triangle) is a tensor-core contraction
 * with FP32 accumulation; a coarse pair (a, b), a < b, qualifies when
 * (b - a) * stride >= gap and S_ab > tau_global.  For each, the keyframes
 * within `radius` of a*stride and of b*stride (with j - i >= gap) are compared
 * by FP32 cosines; the best pair (largest cosine; ties: smallest i, then j)
 * is a loop candidate when its cosine is > tau_local.
 *
 * d_loops (ec3r_loop [capacity], device) receives the candidates in no
 * particular order; d_counts (int64 [2], device) receives the number of coarse
 * pairs and of candidates (counting those past a buffer: ec3r_sync_status then
 * returns EC3R_ERR_CAPACITY; the coarse buffer is context-owned and holds at
 * least 2^20 pairs).  d_sim (float32 [m][m], m = ceil(n / stride), device,
 * nullable) receives the upper triangle of S (diagonal included; the lower
 * triangle is not written).  Workspace is context-owned; not graph-captured.
 * A bounded wait that runs out raises EC3R_ERR_TIMEOUT at ec3r_sync_status.
 */
ec3r_status ec3r_loop_candidates(ec3r_ctx* ctx, const float* d_emb, int n, int d,
                                 const ec3r_loop_opts* opts, ec3r_loop* d_loops,
                                 int64_t capacity, int64_t* d_counts, float* d_sim,
                                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* EC3R_H */
