/*
 * gsvr.h -- C ABI of libgsvr.so: the analytic-PSF slice forward model over
 * anisotropic 3D Gaussians, its adjoint and the Adam step, on one B300 GPU.
 *
 * Method (paper "Fast and Explicit: Slice-to-Volume Reconstruction via 3D
 * Gaussian Primitives with Analytic PSF Modeling"):
 *  - Sec. 2.1, Eq. 1 / Eq. 3: a slice pixel u of slice i is the volume
 *    convolved with the slice-oriented PSF, read at x = T_i(u) = R_i u + t_i.
 *  - Sec. 2.2: the volume is a sum of N Gaussians, 11 parameters each
 *    (mean mu, log-space scales ls, quaternion q = (w,x,y,z), amplitude c),
 *    Sigma_j = R(q) diag(exp(2 ls)) R(q)^T.
 *  - Sec. 2.3, Eq. 4: Sigma_obs = Sigma_j + R_i Sigma_PSF R_i^T, Sigma_PSF
 *    diagonal in slice coordinates; Eq. 5 (numerator): the pixel receives
 *    c_j f exp(-1/2 v^T Sigma_obs^-1 v), v = x - mu_j, with
 *    f = sqrt(det Sigma_j / det Sigma_obs) (the exact convolution of a
 *    unit-mass PSF; GSVR_NORM_EXACT) or f = 1 (GSVR_NORM_LITERAL).
 *  - Sec. 2.4: per slice a rigid motion (axis-angle r, translation tau) that
 *    moves the slice and rotates its PSF: R_i = Rod(r) R0_i,
 *    t_i = Rod(r) c0_i + tau, (R0_i, c0_i) the slice's nominal frame.
 *  - Loss: L = sum_p w_p (I_hat_p - I_p)^2, w_p = 1 / |sampled pixels|.
 *  - Optimisation Details (appendix): Adam, per-group learning rates
 *    (mu, s: 2.5e-2; q, c: 1e-2; rotation 2.5e-3; translation 1e-1).
 *
 * Conventions shared by every call:
 *  - Units: millimetres and radians.  float32 data unless stated.
 *  - Every call is asynchronous on the context's CUDA stream unless it says
 *    it synchronises; pointers passed in are only read during the call (data
 *    is copied), so the caller may reuse them when the call returns (host
 *    pointers) or after the stream reaches the call (device pointers).
 *  - `mem` arguments say where a pointer lives: GSVR_MEM_HOST (pageable or
 *    pinned host memory) or GSVR_MEM_DEVICE (memory of the context's device).
 *  - Every call returns a gsvr_status.  Argument errors return immediately
 *    with GSVR_ERR_INVALID_ARG and change nothing.  Errors found on the device
 *    (capacity overflow in fixed-capacity mode, non-finite values, a wait
 *    that ran out) are latched in a device status word and returned by
 *    gsvr_sync_status().  gsvr_last_error() describes the last failure.
 *  - A context is not thread-safe; distinct contexts are independent.
 *
 * Parameter vector theta (component-major structure of arrays), N Gaussians,
 * M slices (slices ordered stack by stack, slice index k within a stack):
 *   [0,N) mu_x [N,2N) mu_y [2N,3N) mu_z [3N,6N) ls_0..2 [6N,10N) q_w,q_x,q_y,q_z
 *   [10N,11N) c   then 6 floats per slice i at 11N + 6i: r_0..2, tau_0..2.
 * Pixels: global index = (first pixel of slice i) + row * W + col, slices in
 * the order above; pixel (row, col) sits at slice-local
 * u = ((col - (W-1)/2) dx, (row - (H-1)/2) dy, 0).
 */
#ifndef GSVR_H
#define GSVR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSVR_ABI_VERSION 1

typedef struct gsvr_ctx gsvr_ctx; /* opaque; owns all of its device buffers */

typedef enum gsvr_status {
    GSVR_OK = 0,
    GSVR_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or value */
    GSVR_ERR_CUDA = 2,        /* a CUDA runtime call failed (see gsvr_last_error) */
    GSVR_ERR_CAPACITY = 3,    /* fixed-capacity buffers overflowed; results of that call are invalid */
    GSVR_ERR_NONFINITE = 4,   /* a parameter, observation or the loss is not finite */
    GSVR_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    GSVR_ERR_STATE = 6,       /* call out of order (e.g. backward before forward) */
    GSVR_ERR_NOMEM = 7        /* device allocation failed */
} gsvr_status;

enum { GSVR_MEM_HOST = 0, GSVR_MEM_DEVICE = 1 };
enum { GSVR_NORM_EXACT = 0, GSVR_NORM_LITERAL = 1 };

/* One stack of parallel, contiguous slices (no gap), Sec. 2.1 / Sec. 3.2.
 * Slice k (0-based) of n is centred at origin + (k - (n-1)/2) * thickness * n_hat,
 * n_hat = third column of R.  Sigma_PSF = diag((fwhm / 2.355)^2) in slice axes. */
typedef struct gsvr_stack_desc {
    int32_t n_slices, H, W, reserved;
    float dx, dy, thickness;  /* pixel spacing along slice x (columns), y (rows); slice thickness */
    float R[9];               /* row-major 3x3; columns = slice x, slice y, slice normal in world */
    float origin[3];          /* world position of the stack centre */
    float fwhm[3];            /* PSF full width at half maximum along slice x, y, normal */
} gsvr_stack_desc;

typedef struct gsvr_config {
    float cutoff_rel;       /* drop a (pixel, Gaussian) pair when exp(-1/2 v^T Sigma_obs^-1 v) < cutoff_rel;
                               0 -> 1e-7 (truncated mass below 1e-7 of the amplitude) */
    int32_t tile_h, tile_w; /* pixel tile shape used for binning; 0 -> 16 x 16; each in [4, 32] */
    int32_t norm_mode;      /* GSVR_NORM_EXACT (default) or GSVR_NORM_LITERAL */
    int32_t fixed_capacity; /* 0: the library grows its buffers as needed (reads two counts back
                               per forward, synchronising the stream); 1: buffers keep the
                               capacities below, nothing synchronises, overflow -> GSVR_ERR_CAPACITY */
    int32_t timing;         /* 1: record CUDA events around each stage (see gsvr_get_kernel_times) */
    int64_t cap_records;    /* initial / fixed capacity of (slice, Gaussian) records; 0 -> auto */
    int64_t cap_keys;       /* initial / fixed capacity of (tile, record) keys; 0 -> auto */
    uint64_t seed;          /* seed of the device pixel sampler */
} gsvr_config;

typedef struct gsvr_adam_cfg {
    float lr_mu, lr_ls, lr_q, lr_c, lr_rot, lr_trans; /* per-group learning rates */
    float beta1, beta2, eps;                          /* 0 -> 0.9, 0.999, 1e-8 */
    int32_t step_every;                               /* StepLR (App. A.1): rates x gamma every step_every
                                                         steps; 0 = constant rates */
    float gamma;                                      /* StepLR factor; 0 -> 1 */
} gsvr_adam_cfg;

/* Device views of context-owned buffers (valid until the next gsvr_set_* call that
 * resizes them, or gsvr_destroy).  The caller may read and write them on the
 * context's stream. */
typedef struct gsvr_views {
    float *theta;    /* 11N + 6M parameter vector */
    float *grad;     /* dL/dtheta, same layout (written by gsvr_backward) */
    float *adam_m;   /* Adam first moments, same layout */
    float *adam_v;   /* Adam second moments, same layout */
    float *pred;     /* I_hat per global pixel; only the sampled pixels are written */
    float *rbar;     /* dL/dI_hat per global pixel; only the sampled pixels are written */
    double *loss;    /* scalar loss of the last forward */
    int64_t n_gauss, n_slices, n_pixels, n_params;
} gsvr_views;

/* Counters of the last forward (synchronises the stream). */
typedef struct gsvr_stats {
    int64_t n_sampled;       /* pixels in the current sample */
    int64_t n_records;       /* (slice, Gaussian) candidates of the slab test (each one record; those
                                failing the exact Mahalanobis cut carry no keys) */
    int64_t n_keys;          /* (tile, record) keys sorted */
    int64_t pairs_evaluated; /* (pixel, Gaussian) pairs the evaluation kernels visit, each pass */
    int64_t n_tiles;         /* pixel tiles in all slices */
    int64_t tile_px_max;     /* pixels per tile (tile_h * tile_w) */
    int64_t cap_records, cap_keys;
} gsvr_stats;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `cfg` may be NULL for
 * defaults.  *out receives the context.  Synchronous. */
gsvr_status gsvr_create(gsvr_ctx **out, int device, void *cuda_stream, const gsvr_config *cfg);

/* Release every buffer of the context (synchronises its stream first). */
gsvr_status gsvr_destroy(gsvr_ctx *ctx);

/* Acquisition geometry (Sec. 2.1, Sec. 3.2): n_stacks stack descriptions in host
 * memory.  Defines M (slices) and the pixel count; invalidates observations,
 * poses and the sample.  Synchronous. */
gsvr_status gsvr_set_stacks(gsvr_ctx *ctx, int32_t n_stacks, const gsvr_stack_desc *stacks);

/* Observed slice intensities I (float32, one per global pixel) and the pixel
 * mask (uint8, nonzero = usable), both `mem`.  mask may be NULL (all usable).
 * Requires gsvr_set_stacks.  Makes the sample "every masked pixel". */
gsvr_status gsvr_set_observations(gsvr_ctx *ctx, const float *I, const uint8_t *mask, int32_t mem);

/* The N Gaussians (Sec. 2.2): theta_g = the first 11N entries of the
 * parameter vector, `mem`.  Resets the Adam moments of the Gaussians. */
gsvr_status gsvr_set_gaussians(gsvr_ctx *ctx, int64_t N, const float *theta_g, int32_t mem);

/* The M slice motions (Sec. 2.4): pose[6i + 0..2] = axis-angle r,
 * pose[6i + 3..5] = translation tau, `mem`.  Resets the pose Adam moments. */
gsvr_status gsvr_set_poses(gsvr_ctx *ctx, const float *pose, int32_t mem);

/* Mark slices whose pose the optimiser must not move (gauge fixing: a joint
 * rigid motion of volume and slices leaves L unchanged).  frozen: M bytes,
 * host memory; NULL clears. */
gsvr_status gsvr_set_frozen(gsvr_ctx *ctx, const uint8_t *frozen);

/* Sample = the listed global pixels (int32, `mem`, any order; duplicates count
 * once; unmasked pixels are dropped).  n < 0: every masked pixel.
 * w_p = 1 / (number of distinct usable pixels listed).  Indices are checked on
 * the device (host and device lists alike): an index outside [0, pixels) is
 * skipped and makes the next gsvr_sync_status return GSVR_ERR_INVALID_ARG. */
gsvr_status gsvr_set_pixel_sample(gsvr_ctx *ctx, const int32_t *idx, int64_t n, int32_t mem);

/* Sample n masked pixels uniformly without replacement on the device: the
 * first n values of a keyed random permutation of the masked pixels (SplitMix64
 * round keys from (seed, step), a 4-round multiply/xor-shift bijection on
 * ceil(log2(#masked)) bits, cycle walking).  n must not exceed #masked. */
gsvr_status gsvr_sample_pixels(gsvr_ctx *ctx, int64_t n, uint64_t step);

/* Forward pass (Eq. 4, Eq. 5 numerator with the normalisation of norm_mode,
 * MSE loss) over the current sample: per-Gaussian and per-slice preprocessing,
 * Mahalanobis cut of every (slice, Gaussian) pair at cutoff_rel, (tile, record)
 * key emission and radix sort, fused tile evaluation.  Writes pred, rbar and
 * loss (see gsvr_views).  In growing mode this synchronises twice to size
 * buffers. */
gsvr_status gsvr_forward(gsvr_ctx *ctx);

/* Adjoint of the last forward: dL/dtheta for every Gaussian parameter and
 * every slice pose, recomputing each pair from the sorted tile lists (nothing
 * per pair is stored by the forward).  Requires a forward since the last
 * change of parameters, sample or observations.  dL/dI_hat is read from the
 * rbar buffer (gsvr_views) at the sampled pixels: the forward writes the
 * loss's values there, and a caller may overwrite them (for example with the
 * gradient of a downstream loss of the predictions) before this call. */
gsvr_status gsvr_backward(gsvr_ctx *ctx);

/* One Adam step (bias-corrected, no weight decay) on theta with the last
 * gradient; `step` is the 1-based step count used for bias correction and the
 * StepLR schedule. */
gsvr_status gsvr_adam_step(gsvr_ctx *ctx, const gsvr_adam_cfg *cfg, int64_t step);

/* ---- Batched form: several independent reconstructions in one context ----
 * Subjects: stack_subject[s] is the subject of stack s (subjects 0..n-1, each a
 * contiguous run of stacks in order); gauss_count[k] Gaussians belong to subject
 * k, in order (subject 0's first, each parameter component-major over all N as
 * above).  A Gaussian is evaluated only against its own subject's slices, pixel
 * weights are 1 / (the subject's sampled pixels) and losses are kept per
 * subject; one set of launches serves all subjects (the evaluation kernels are
 * persistent over the work items of every subject).  Host tables; call after
 * gsvr_set_gaussians and gsvr_set_observations; n = 1 restores one subject. */
gsvr_status gsvr_set_subjects(gsvr_ctx *ctx, int32_t n, const int32_t *stack_subject, const int64_t *gauss_count);

/* Device sampler per subject: n_per_subject masked pixels of every subject
 * (all of them where a subject has fewer), uniformly without replacement;
 * subject k uses the keyed permutation of gsvr_sample_pixels with seed
 * seed + k * 0x9E3779B97F4A7C15. */
gsvr_status gsvr_sample_pixels_subjects(gsvr_ctx *ctx, int64_t n_per_subject, uint64_t step);

/* Per-subject MSE losses of the last forward into host `out` (n >= number of
 * subjects).  Synchronises. */
gsvr_status gsvr_get_subject_losses(gsvr_ctx *ctx, double *out, int32_t n);

/* Retire subjects from (active[k] = 0) or return them to (1) the batched
 * sampler (gsvr_sample_pixels_subjects and captured iterations): a retired
 * subject draws no pixels, so it adds no work and receives zero gradient, and
 * its Adam moments (Gaussians and slice poses) are zeroed when it is retired,
 * so Adam leaves its parameters unchanged (with the scale regulariser on, its
 * Gaussians still follow the regulariser's gradient).  Its loss reads 0.  A
 * subject returned to the sample restarts Adam from zero moments.  active:
 * host array of n_subj flags, NULL = every subject active; at least one must
 * stay active.  Drops a captured CUDA graph (the sample size changes: capture
 * again).  Synchronises.  Errors: GSVR_ERR_STATE (before the Gaussians and
 * observations, during graph capture), GSVR_ERR_INVALID_ARG (no active
 * subject). */
gsvr_status gsvr_set_subject_active(gsvr_ctx *ctx, const uint8_t *active);

/* Grow the record / key capacities to at least the given counts (never
 * shrinks; contents are regenerated by the next forward).  In fixed-capacity
 * mode this is how a caller makes room after a GSVR_ERR_CAPACITY or before the
 * counts reach the capacity (gsvr_get_stats reports both).  A captured graph
 * is dropped when a buffer moves.  Synchronises. */
gsvr_status gsvr_reserve(gsvr_ctx *ctx, int64_t cap_records, int64_t cap_keys);

/* ---- CUDA graph of one optimisation iteration ----
 * gsvr_graph_capture records, on the context's (non-default) stream: the
 * per-subject device sampler (n_per_subject < 0: keep the current sample),
 * forward, backward, Adam with `cfg`, and the advance of a device iteration
 * counter that the sampler's step and Adam's bias correction / schedule read
 * (so every replay is the next iteration).  Requires fixed_capacity = 1 and a
 * prior successful forward at these capacities.  gsvr_graph_launch replays it
 * `iterations` times (asynchronous); gsvr_set_step sets the counter (the next
 * iteration uses step and Adam step step + 1).  Capacity overflow during replay
 * is reported by gsvr_sync_status. */
gsvr_status gsvr_graph_capture(gsvr_ctx *ctx, int64_t n_per_subject, const gsvr_adam_cfg *cfg);
gsvr_status gsvr_graph_launch(gsvr_ctx *ctx, int32_t iterations);
gsvr_status gsvr_set_step(gsvr_ctx *ctx, int64_t step);

/* ---- Launch shape and autotuner ----
 * How the tile stage cuts the work; it does not change what is computed (the
 * Mahalanobis cut and the records are exact per pixel; only the rounding order
 * of the per-pixel sums follows the tiles).  The paper fixes no launch shape
 * (its Sec. 2.5 kernels process fixed batches of points); these are the
 * B300 kernels' knobs.
 *   tile_h, tile_w      pixel tile (each in [4, 32]; 0 -> 16), with
 *                       tile_h * ceil(tile_w / px) <= 256 for the forward's px
 *   fwd_px_per_thread   forward pixels per thread along a tile row: 1, 2, 4, 8 or 16
 *                       (0 -> 8 when tile_w > 16, 16 when 12 < tile_w <= 16,
 *                       4 when tile_w == 12, else 2); the launch is refused when
 *                       the forward's groups x tile pixels exceed its shared
 *                       buffer (max(128 x fwd_px_per_thread, 1024) floats)
 *   fwd_blocks_per_sm,
 *   bwd_blocks_per_sm   CTAs per SM of the persistent evaluation kernels
 *                       (0 -> as many as fit; larger requests are clamped;
                       -1 -> one CTA per work item, scheduled by the hardware)
 *   queue_order         0: work items in tile order; 1: longest items first
 *                       (one extra 9-bit radix sort of the items per forward)
 *   ms                  written by gsvr_autotune: measured ms per iteration,
 *                       -1 for a shape that was invalid or overflowed a fixed
 *                       capacity */
typedef struct gsvr_tiling {
    int32_t tile_h, tile_w;
    int32_t fwd_px_per_thread;
    int32_t fwd_blocks_per_sm, bwd_blocks_per_sm;
    int32_t queue_order;
    float ms;
} gsvr_tiling;

/* Apply a launch shape.  A new tile shape rebuilds every tile-ordered table
 * (pixel tiles, masked-pixel order, subject ranges) from the stored stack
 * descriptions, observations and mask; parameters, Adam moments, subjects and
 * frozen slices are kept; the pixel sample becomes every masked pixel and a
 * captured graph is dropped.  Synchronises.  GSVR_ERR_INVALID_ARG for a shape
 * outside the limits above (the context is then unchanged). */
gsvr_status gsvr_set_tiling(gsvr_ctx *ctx, const gsvr_tiling *t);

/* Objective (Sec. 2.5, "Loss Function").  loss_kind 0: the MSE data term
 * sum_p w_p (I_hat - I)^2 (default); 1: the paper's L1 data term
 * sum_p w_p |I_hat - I| (subgradient sign(0) = 0).  lambda_reg > 0 adds the
 * scale regulariser lambda_reg sum_j sum_k (exp(ls_jk) - s_target)^2 (scales
 * in mm; the paper's s_target = 1.6 mm, lambda_reg = 2.5e-3) to the loss and
 * its gradient to the log-scales; in the batched form it enters the total
 * loss only, not the per-subject losses.  Applies to both forward models.
 * GSVR_ERR_INVALID_ARG for another loss_kind, lambda_reg < 0 or not finite,
 * s_target <= 0 or not finite.  Synchronises the stream. */
gsvr_status gsvr_set_objective(gsvr_ctx *ctx, int32_t loss_kind, float lambda_reg, float s_target);

/* Content-adaptive initialisation of the means (Sec. 2.5, "Content-Adaptive
 * Initialization"): n means drawn from P_init proportional to
 * (1 - lambda_init) |grad I_i(u)| + lambda_init over the masked pixels of the
 * observations, each placed at its pixel's world position T_i(u) under
 * `pose` (host, M x 6 (r, tau) per slice; NULL = no motion), jittered
 * uniformly within the pixel's voxel (dx x dy x slice thickness).
 * Deterministic: |grad I| by central differences (one-sided at the border) in
 * float32 with every operation rounded alone, integer weights
 * floor(1024 ((1 - lambda) |grad I| + lambda)), an int64 cumulative sum T,
 * draw k = the first pixel whose cumulative weight exceeds
 * floor(SplitMix64(seed, k) T / 2^64), jitter uniforms = 24-bit fractions of
 * SplitMix64(seed, 2^40 + 3 k + a).
 * mu: device [3][n] (x row, y row, z row, as the parameter vector's means);
 * pix: device [n] (the drawn global pixels) or NULL; *total_weight (host, may be
 * NULL) = T.  Synchronises.  GSVR_ERR_STATE before stacks and observations;
 * GSVR_ERR_INVALID_ARG for n < 0 or > 2^30, lambda_init outside [0, 1], a
 * non-finite pose, or T = 0 (no masked pixel carries weight). */
gsvr_status gsvr_init_means(gsvr_ctx *ctx, const float *pose, int64_t n, float lambda_init, uint64_t seed, float *mu,
                            int32_t *pix, int64_t *total_weight);

/* Per-slice outlier terms (Sec. 2.4): a learnable intensity scale sigma_i
 * (Eq. 5's factor: every prediction of slice i is sigma_i times the model) and
 * an aleatoric weight omega_i, read as the pixel loss
 * w_p (l(I_hat - I) / omega_i + log omega_i) with l the data term of
 * gsvr_set_objective.  Both are held as logarithms (log sigma_i, log omega_i),
 * 2 M floats, zero (sigma = omega = 1) when switched on.  The forward also
 * writes their gradients (they need no backward pass); gsvr_adam_step steps
 * them with lr_log_sigma / lr_log_omega on the same schedule as the other
 * groups; a frozen slice (gsvr_set_frozen) keeps its sigma (the intensity
 * gauge: sigma_i and the amplitudes trade off).  enable = 0 switches them
 * off (predictions and loss as without them).  gsvr_set_stacks switches them
 * off.  Both forward models.  GSVR_ERR_STATE before gsvr_set_stacks;
 * GSVR_ERR_INVALID_ARG for negative or non-finite rates.  Synchronises. */
gsvr_status gsvr_set_slice_weights(gsvr_ctx *ctx, int32_t enable, float lr_log_sigma, float lr_log_omega);
/* Device views of the per-slice terms (log sigma_i for i < M, then log
 * omega_i) and of their gradients; the caller may write the parameters
 * between calls.  GSVR_ERR_STATE when they are off. */
gsvr_status gsvr_slice_weight_views(gsvr_ctx *ctx, float **params, float **grads, int32_t *M);

/* Normalised top-K forward model (Sec. 2.2, Eq. 2; Eq. 5 with sigma_i = 1;
 * Sec. 2.5 "Sparse Computation (Top-K)").  With K >= 1 every later forward
 * predicts a sampled pixel as
 *     I_hat = sum_{j in S} c_j E_j / (sum_{j in S} E_j + delta),
 *     E_j = exp(-1/2 v^T Sigma_obs,ij^-1 v), v = T_i(u) - mu_j,
 *     Sigma_obs,ij = Sigma_j + R_i Sigma_PSF R_i^T (Eq. 4, no normalisation factor),
 * S = the K Gaussians whose means are nearest the pixel's world position in
 * Euclidean distance (ties to the smaller index), found exactly by a shell
 * search of a uniform grid over the means (about 16 means per cell, at most
 * 2^16 cells).  The grid is rebuilt every `refresh_every` forwards (1 = every
 * forward: exact neighbours; larger values select the neighbours by the means
 * as of the last build, as the paper's periodically refreshed index does,
 * while the ratio itself uses the current means).
 * The loss is the one gsvr_set_objective selects; gsvr_backward gives the
 * exact gradient for the neighbour sets of the last forward (the selection
 * is piecewise constant).
 * K = 0 restores the plain sum of gsvr_forward.  One subject only
 * (GSVR_ERR_STATE otherwise, at gsvr_forward).
 * Arguments: 0 <= K <= 128; delta > 0 and finite; refresh_every >= 1; else
 * GSVR_ERR_INVALID_ARG.  Synchronises the stream; sizes the buffers when
 * Gaussians are set (GSVR_ERR_NOMEM on failure). */
gsvr_status gsvr_set_topk(gsvr_ctx *ctx, int32_t K, float delta, int32_t refresh_every);

/* Neighbour sets of the last top-K forward (synchronises): *n_out = number of
 * sampled pixels; with host buffers pix [cap], nbr [cap][K], cnt [cap] (all
 * non-NULL, cap >= *n_out) also the sampled global pixels in evaluation order,
 * their neighbours (Gaussian indices, in no particular order) and neighbour
 * counts (K, or N when N < K).  Passing all three NULL only queries *n_out.
 * GSVR_ERR_STATE without a current top-K forward. */
gsvr_status gsvr_get_topk_neighbors(gsvr_ctx *ctx, int32_t *pix, int32_t *nbr, int32_t *cnt, int64_t cap,
                                    int64_t *n_out);
gsvr_status gsvr_get_tiling(gsvr_ctx *ctx, gsvr_tiling *out);

/* The built-in candidate shapes: writes min(cap, total) of them to out and the
 * total count to *n (out may be NULL when cap = 0). */
gsvr_status gsvr_tune_space_default(gsvr_tiling *out, int32_t cap, int32_t *n);

/* Time each candidate (`iterations` timed iterations of device sample of
 * n_per_subject pixels per subject -- 0 keeps every masked pixel -- forward and
 * backward, after one untimed iteration; CUDA events on the context's stream),
 * write cand[c].ms, apply the fastest and return its index in *best (may be
 * NULL).  Parameters are not updated.  Afterwards the context's pixel sample is
 * unspecified: draw one before the next forward.  Synchronises. */
gsvr_status gsvr_autotune(gsvr_ctx *ctx, gsvr_tiling *cand, int32_t n_cand, int64_t n_per_subject,
                          int32_t iterations, int32_t *best);

/* End to end from host buffers: copy theta (11N + 6M floats, host) and the
 * pixel sample (n int32 global indices, host; n < 0 = every masked pixel) to
 * the device, run forward and backward, copy dL/dtheta (host, 11N + 6M floats)
 * and the loss (host double) back.  Synchronises.  grad_out or loss_out may be
 * NULL. */
gsvr_status gsvr_step_host(gsvr_ctx *ctx, const float *theta, const int32_t *idx, int64_t n, float *grad_out,
                           double *loss_out);

/* Copy the current sample (global pixel indices, in the library's tile order)
 * to host memory `out` of `cap` int32 entries; *n_out receives the sample size
 * (entries beyond cap are not written).  Synchronises. */
gsvr_status gsvr_get_sample(gsvr_ctx *ctx, int32_t *out, int64_t cap, int64_t *n_out);

gsvr_status gsvr_get_views(gsvr_ctx *ctx, gsvr_views *out);
gsvr_status gsvr_get_stats(gsvr_ctx *ctx, gsvr_stats *out);

/* Stages timed when gsvr_config.timing = 1. */
enum {
    GSVR_STAGE_SAMPLE = 0,   /* device pixel sampler and tile ranges */
    GSVR_STAGE_PREP = 1,     /* Gaussian covariances and slice frames */
    GSVR_STAGE_BIN = 2,      /* Mahalanobis cut, records, keys, radix sort, tile ranges, gather */
    GSVR_STAGE_FWD_EVAL = 3, /* forward tile evaluation kernel */
    GSVR_STAGE_BWD_EVAL = 4, /* backward tile evaluation kernel */
    GSVR_STAGE_GRAD = 5,     /* per-Gaussian and per-slice gradient epilogue */
    GSVR_STAGE_ADAM = 6,     /* fused Adam */
    GSVR_N_STAGES = 8
};

typedef struct gsvr_kernel_times {
    double ms[GSVR_N_STAGES];     /* device time per stage since gsvr_timing_reset (CUDA events
                                     on the context stream) */
    int64_t calls[GSVR_N_STAGES]; /* executions of each stage */
    int64_t pairs_evaluated;      /* pixel x record pairs the forward visited since the reset */
    int64_t kernel_launches;      /* kernels this library launched since the reset (all contexts) */
    int64_t bwd_pairs_evaluated;  /* pixel x record pairs the backward evaluated since the reset
                                     (each record over its in-cut box inside the tile) */
} gsvr_kernel_times;

/* Clear the stage timers and counters. */
gsvr_status gsvr_timing_reset(gsvr_ctx *ctx);

/* Read the stage timers (synchronises). */
gsvr_status gsvr_get_kernel_times(gsvr_ctx *ctx, gsvr_kernel_times *out);

/* Diagnostic pass over the current forward's tile lists (synchronises):
 * *useful = (pixel, Gaussian) pairs with exp(-1/2 v^T Sigma_obs^-1 v) >= cutoff_rel,
 * *evaluated = pairs the evaluation kernels visit.  Requires a current forward. */
gsvr_status gsvr_count_pairs(gsvr_ctx *ctx, int64_t *useful, int64_t *evaluated);

/* Synchronise the stream; return and clear the device status word
 * (GSVR_OK, GSVR_ERR_CAPACITY, GSVR_ERR_NONFINITE or GSVR_ERR_TIMEOUT). */
gsvr_status gsvr_sync_status(gsvr_ctx *ctx);

/* Text of the last error of this context (static storage owned by ctx);
 * ctx NULL gives the last error of gsvr_create. */
const char *gsvr_last_error(gsvr_ctx *ctx);

/* Measurement helper (not part of the method): float32 FFMA and MUFU ex2.approx
 * throughput of the whole device in instructions per second (best of three
 * launches of independent dependency chains filling every SM) and the SM count;
 * the roofline denominators of the ALU-bound tile kernels.  Synchronous;
 * allocates a 1 KB buffer. */
gsvr_status gsvr_alu_peaks(int device, double *ffma_per_s, double *ex2_per_s, double *sm_count);

/* Measurement helper (not part of the method): float64 DFMA throughput of the
 * whole device in instructions per second, measured the same way; the roofline
 * denominator of the float64 metric passes of gsvr_volume_metrics.
 * Synchronous; allocates a 1 KB buffer. */
gsvr_status gsvr_fp64_peak(int device, double *dfma_per_s);

/* Measurement helper (not part of the method): packed two-wide float32 FMA
 * (PTX fma.rn.f32x2) throughput of the whole device in instructions per
 * second (each instruction two FMAs), measured the same way; with the FFMA
 * rate it fixes the roofline of tile kernels that use packed arithmetic.
 * Synchronous; allocates a 1 KB buffer. */
gsvr_status gsvr_ffma2_peak(int device, double *ffma2_per_s);

/* Coarse-to-fine densification: split, clone and prune of the Gaussians.  The
 * paper names progressive densification (after 3D Gaussian Splatting, Kerbl
 * et al. 2023) as future work ("Limitations and Future Work": start with few
 * large Gaussians, split adaptively) without giving a rule; this is the rule:
 *  - statistic: per Gaussian the sums of ||dL/dmu_j|| and of dL/dmu_j over the
 *    backward passes since the last densification (gsvr_densify_accumulate
 *    after each gsvr_backward) and the number of those passes;
 *  - decision (float32): prune when |c_j| < prune_amplitude; else, when the
 *    mean norm (sum / passes; 0 with no pass) exceeds grad_threshold, split if
 *    the largest log-scale exceeds log_scale_threshold, clone otherwise; else
 *    keep;
 *  - split: two children at mu_j +- d a (a = the principal axis, the
 *    rotation's column of the largest log-scale, first on ties;
 *    d = s sqrt(1 - 1/phi^2), s that scale), principal scale s / phi: the pair
 *    has the parent's mean and covariance;
 *  - clone: two copies at mu_j +- delta u (u = direction of the summed mean
 *    gradient, the principal axis if it is zero; delta = clone_offset x the
 *    smallest scale);
 *  - amplitudes: mass_preserving = 1 (the plain sum) gives c phi / 2 (split) or
 *    c / 2 (clone), keeping the summed mass; 0 (the normalised top-K model,
 *    where c is a colour) keeps c;
 *  - layout: Gaussians in index order, a kept one once (with its Adam
 *    moments), a split or cloned one as its two children (+ first; moments 0),
 *    a pruned one not at all; slice poses and their moments unchanged. */
typedef struct gsvr_densify_cfg {
    float grad_threshold;      /* split or clone above this mean ||dL/dmu_j|| */
    float log_scale_threshold; /* split (not clone) above this largest log-scale */
    float prune_amplitude;     /* remove when |c_j| is below it (0: never), >= 0 */
    float split_factor;        /* phi > 1 (3D Gaussian Splatting uses 1.6) */
    float clone_offset;        /* kappa >= 0 */
    int32_t mass_preserving;   /* 1 or 0, see above */
    int64_t max_gaussians;     /* refuse above this count (0: 2^26) */
} gsvr_densify_cfg;

/* Add ||dL/dmu_j|| and dL/dmu_j of the gradient buffer (the last
 * gsvr_backward) to the statistics and count one pass.  The statistics restart
 * (zero) after gsvr_set_gaussians and gsvr_densify.  Asynchronous; graph
 * capturable once sized (one call outside capture sizes them). */
gsvr_status gsvr_densify_accumulate(gsvr_ctx *ctx);

/* Read (set = 0) or write (set = 1) the statistics: acc = host float[4 N]
 * (per Gaussian: sum of norms, sum of the three gradient components), count =
 * passes.  Synchronises.  GSVR_ERR_INVALID_ARG for NULL pointers (acc may be
 * NULL when N = 0) or a negative count. */
gsvr_status gsvr_densify_stats(gsvr_ctx *ctx, float *acc, int32_t *count, int32_t set);

/* Apply the rule above to the context's Gaussians: the parameter vector and
 * Adam moments are rebuilt for the new count N' (views from gsvr_get_views
 * change), the gradient is zeroed, capacities follow N', a captured CUDA graph
 * is dropped, and the statistics restart.  counts (host int64[4], may be NULL)
 * = {N', split, cloned, pruned}.  Synchronises.  Errors: GSVR_ERR_INVALID_ARG
 * (bad configuration), GSVR_ERR_STATE (no Gaussians, a batched context, during
 * graph capture), GSVR_ERR_CAPACITY (N' > max_gaussians; nothing changed). */
gsvr_status gsvr_densify(gsvr_ctx *ctx, const gsvr_densify_cfg *cfg, int64_t *counts);

/* Image-quality metrics of a reconstructed volume X against its ground truth
 * Y on the same grid: the evaluation of Sec. 3 (Table 1 reports PSNR, SSIM and
 * NCC; the paper does not state their parameters, the readings are these).
 *   PSNR = 10 log10(L^2 / MSE) over the masked voxels, L = data_range.
 *   NCC  = the Pearson correlation of X and Y over the masked voxels.
 *   SSIM = Wang et al. (2004) with K1 = 0.01, K2 = 0.03 and the Gaussian window
 *          of standard deviation 1.5 voxels and radius 5, in 3D the product
 *          window of 11 x 11 x 11 voxels; near the grid border the window keeps
 *          its in-grid voxels and is renormalised over them; local moments are
 *          weighted population moments over every grid voxel of the window
 *          (masked or not); the SSIM map is averaged over the masked voxels.
 * Arguments:
 *   device       CUDA device (made current for the call; the previous one is
 *                restored).
 *   cuda_stream  cudaStream_t to issue the work on (NULL = legacy default).
 *   D, H, W      grid size; X, Y are float32 device arrays of D*H*W voxels,
 *                row-major with x fastest (index (z*H + y)*W + x).
 *   mask         uint8 device array of D*H*W voxels (non-zero = counted), or
 *                NULL for every voxel.
 *   data_range   L > 0.
 *   out          host double[3]: PSNR (dB; +inf when X = Y on the mask), mean
 *                SSIM, NCC (NaN when X or Y is constant on the mask).
 *   ssim_map     optional float64 device array of D*H*W voxels receiving the
 *                SSIM map at every voxel (masked or not); NULL = not written.
 *   msg, msg_len optional buffer for an error text.
 * Scratch of 80 bytes per voxel is kept per device between calls (grown with
 * cudaMalloc when a larger grid comes, held until the process exits); calls
 * are serialised on it.  Synchronises the stream.
 * Errors: GSVR_ERR_INVALID_ARG (no such device, a size <= 0 or above 2^30 per
 * axis, a NULL volume or out, data_range not finite and positive, a mask that
 * selects no voxel: out then holds NaN), GSVR_ERR_NOMEM (scratch), GSVR_ERR_CUDA. */
gsvr_status gsvr_volume_metrics(int device, void *cuda_stream, int64_t D, int64_t H, int64_t W, const float *X,
                                const float *Y, const uint8_t *mask, double data_range, double *out,
                                double *ssim_map, char *msg, int32_t msg_len);

/* Pixel weight of the loss (Sec. 2.5 takes the loss over the sampled points;
 * here w_p = 1 / |sample|, its mean).  n_total > 0 sets w_p = 1 / n_total for
 * every sampled pixel (every subject) instead of 1 / (this context's sample
 * size), so that contexts holding disjoint parts of one reconstruction's
 * slices (one per rank of a data-parallel split) each compute their exact
 * share of the global loss and gradient: summing the contexts' losses and
 * Gaussian gradients gives the global ones.  n_total = 0 restores the
 * default.  Drops a captured graph.
 * Errors: GSVR_ERR_INVALID_ARG (n_total < 0 or > 2^40), GSVR_ERR_STATE
 * (during graph capture). */
gsvr_status gsvr_set_sample_total(gsvr_ctx *ctx, int64_t n_total);

/* Test hook for failure detection (no counterpart in the paper).  Every
 * device-side wait of the library is bounded (1 s) and, when it runs out,
 * latches a status bit that gsvr_sync_status reports as GSVR_ERR_TIMEOUT while
 * the context stays usable.  To exercise that path without a fault, the next
 * n_forwards calls of gsvr_forward make every block of the tile evaluation
 * wait, for its first work item with records, on a shared-memory barrier that
 * nothing ever completes, bounded by limit_ns (1 us .. 1 s); the wait runs
 * out, the block stops taking work and still waits, with the normal bound,
 * for the copies it started.  That forward's results are invalid (GSVR_ERR_TIMEOUT at the next
 * gsvr_sync_status); the forwards after it are normal.
 * Errors: GSVR_ERR_INVALID_ARG (bad counts or limit), GSVR_ERR_STATE (during
 * graph capture). */
gsvr_status gsvr_test_wait_timeout(gsvr_ctx *ctx, int32_t n_forwards, int64_t limit_ns);

/* ---- checkpoint / resume.
 * The optimisation state of the reconstruction: the Gaussian parameters
 * (Sec. 2.2: mean, log-scales, quaternion, amplitude), the slice poses
 * (Sec. 2.4), the Adam moments and the position in the step schedule (App. A.1:
 * Adam with StepLR over hundreds of epochs, long enough that a run may need to
 * stop and resume).  A checkpoint is one versioned binary file (host byte
 * order): magic "GSVRCKPT", version 1, then tagged sections -- configuration
 * (cutoff, normalisation, sampler seed, launch shape), stack descriptions,
 * parameters with Adam m and v (11N + 6M float32 each), the device step
 * counter (gsvr_set_step; drives the device sampler and the StepLR / bias
 * correction of graph-replayed steps), frozen slices, objective, per-slice
 * weights with their Adam state, top-K settings, subject tables and active
 * flags, densification statistics -- and a 64-bit FNV-1a hash of all of it.
 * Observations and masks are inputs, not state: they are not stored. */
typedef struct gsvr_checkpoint_header {
    int32_t version, n_stacks, n_slices, reserved;
    int64_t n_pixels, n_gaussians, step;
} gsvr_checkpoint_header;

/* Writes the context's state to `path` (host file; written under path + ".tmp"
 * and renamed over `path`).  Synchronises the stream.
 * Errors: GSVR_ERR_STATE (no Gaussians yet, or during graph capture),
 * GSVR_ERR_INVALID_ARG (NULL path, the file cannot be written), GSVR_ERR_CUDA. */
gsvr_status gsvr_save(gsvr_ctx *ctx, const char *path);

/* Restores a state written by gsvr_save into a context that already holds the
 * same stacks (compared byte for byte) and its observations
 * (gsvr_set_stacks, gsvr_set_observations): Gaussians (N may differ from the
 * context's), poses, Adam moments, step counter, launch shape, sampler seed,
 * cutoff and normalisation, frozen slices, objective, slice weights, top-K
 * settings, subjects and densification statistics.  After it, the same pixel
 * sample gives bitwise the forward, the Gaussian gradient and the Adam step of
 * the Gaussians the saved context would have given (the slice-pose gradients
 * are float atomics in a thread-timing order: equal to rounding, on any run).  Drops a captured graph (capture again); the top-K
 * neighbour grid is rebuilt at the next forward.  The file is checked before
 * anything changes.
 * Errors: GSVR_ERR_INVALID_ARG (NULL path, unreadable file, bad magic,
 * unsupported version, hash mismatch, malformed section), GSVR_ERR_STATE
 * (stacks or observations not set, stacks differ, during graph capture),
 * GSVR_ERR_NOMEM, GSVR_ERR_CUDA.  A failure after the checks leaves the
 * context partly restored. */
gsvr_status gsvr_load(gsvr_ctx *ctx, const char *path);

/* Reads and checks a checkpoint file without a context or GPU: framing, magic,
 * version, hash and the sizes of the required sections; fills *out.
 * Errors: GSVR_ERR_INVALID_ARG (with the reason in msg when msg_len > 0). */
gsvr_status gsvr_checkpoint_info(const char *path, gsvr_checkpoint_header *out, char *msg, int32_t msg_len);

/* Forward pass without any device allocation (this entry point has no
 * counterpart in the paper; it exists for callers that cannot call cudaMalloc:
 * code running inside a host framework or plug-in whose device memory is owned
 * by someone else, or under a budget or in a region where allocating is not
 * allowed).  It needs no context and allocates nothing: every intermediate
 * buffer lives in one file-scope device array of 32 MiB that each GPU loading
 * this library holds until the process exits.  It runs the same kernels as
 * gsvr_forward with 16 x 16 pixel tiles and fixed capacities.
 *   device      CUDA device to run on (made current for the call).
 *   cuda_stream cudaStream_t to issue the work on (NULL = legacy default stream).
 *   stacks      n_stacks descriptions (host), as for gsvr_set_stacks.
 *   theta       11N + 6M float32 parameters (device), the layout above.
 *   I           observed intensity per global pixel (device float32).
 *   idx, n_idx  sampled global pixel indices (device int32, duplicates count
 *               once, at most 2^30 entries; an index outside [0, P) returns
 *               GSVR_ERR_INVALID_ARG); n_idx = -1 samples every pixel (idx may
 *               be NULL).
 *   cutoff_rel, norm_mode  as in gsvr_config (0 -> 1e-7).
 *   pred        per global pixel (device float32); only sampled pixels written.
 *   loss        the MSE loss (device double).
 *   msg, msg_len optional host buffer receiving an error description.
 * Limits: every pixel costs 29 bytes of the array (tile maps, sample lists,
 * residual, mask), so at most 1,157,049 pixels fit, fewer once the tiles
 * (about 1 KiB each) and Gaussians (40 bytes each) take their share; the rest
 * holds records at about 212 bytes each (a record, its candidate, tile box
 * and room for 4 keys with their sort buffers).  A problem whose pixel, tile
 * and Gaussian arrays leave no room for records is rejected with
 * GSVR_ERR_INVALID_ARG before any work; one whose (slice, Gaussian) records or
 * keys found on the device overflow that room returns GSVR_ERR_CAPACITY
 * (writes past the room are skipped; pred and loss are then incomplete).
 * Every call looks up the array's device address (cudaGetSymbolAddress);
 * the first call on a device also loads the library's device code there and
 * should come before any stream capture on that device.  Every call shares the array and leaves its contents behind (each
 * call clears what must start at zero), so calls that overlap on the GPU --
 * on different streams or threads -- race and must not be issued.  The call
 * synchronises `cuda_stream` before it returns (to report device status). */
gsvr_status gsvr_forward_noalloc(int device, void *cuda_stream, int32_t n_stacks, const gsvr_stack_desc *stacks,
                                 int64_t N, const float *theta, const float *I, const int32_t *idx, int64_t n_idx,
                                 float cutoff_rel, int32_t norm_mode, float *pred, double *loss, char *msg,
                                 int32_t msg_len);

/* ABI version (GSVR_ABI_VERSION of the built library). */
int32_t gsvr_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSVR_H */
