/*
 * gsvr_cnn.h -- C ABI of the slice-pose regression network in libgsvr.so.
 *
 * What it is for: the reconstruction's slice poses (Sec. 2.4: per slice a
 * rigid motion, axis-angle r and translation tau, composed with the slice's
 * nominal frame) start from a learned estimate instead of zero.  The paper
 * evaluates its method on residual motion of the size a learned
 * pre-alignment leaves (Sec. 3.2, "Data"); this network is that learned
 * step: it reads one slice image and regresses its 6-DoF motion, trained on
 * slices that the forward model of gsvr.h renders from synthetic Gaussian
 * volumes under random rigid motion.
 *
 * Network (fixed architecture):
 *   input  x: one 128 x 128 slice image (float32, row-major), rounded to
 *          bfloat16 on the device
 *   6 conv layers 3x3, stride 2, zero padding 1, channels
 *          1 -> 32 -> 64 -> 128 -> 256 -> 256 -> 512 (128^2 -> 2^2 positions),
 *          each + bias + ReLU; activations NHWC bfloat16, products on the
 *          tensor cores (bfloat16 operands, float32 accumulation)
 *   the final 2 x 2 x 512 map flattened position-major -> 2048 features
 *          (float32; the positions keep where the anatomy sits in the slice)
 *   concatenated with aux (25 floats per slice: the stack's nominal rotation
 *          R0 row-major (9) and a 16-d sinusoidal embedding of the slice's
 *          offset along the stack normal; the caller builds it)
 *   fc1 2073 -> 256 + ReLU, fc2 256 -> 6 (float32)
 *   output (r_0..2 in rad, tau_0..2 / 10 mm)
 *   loss   mean over the batch and the 6 outputs of (output - target)^2
 * Parameters: one float32 vector (master copy), in this order per layer l:
 *   conv_l weights [Co][3][3][Ci], conv_l bias [Co]  (l = 1..6),
 *   fc1 weights [256][2073], fc1 bias [256], fc2 weights [6][256], fc2 bias [6]
 *   (2,690,566 floats); the conv weights are rounded to bfloat16 at the start
 *   of every forward.
 *
 * Conventions: as in gsvr.h (device pointers are memory of the network's
 * device; calls are asynchronous on its stream unless stated; argument errors
 * return GSVR_ERR_INVALID_ARG and change nothing).  bfloat16 tensors are passed
 * as uint16_t bit patterns.
 */
#ifndef GSVR_CNN_H
#define GSVR_CNN_H

#include <stdint.h>

#include "gsvr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsvr_cnn gsvr_cnn; /* opaque; owns its parameters, Adam state and activations */

#define GSVR_CNN_IMAGE 128
#define GSVR_CNN_AUX 25
#define GSVR_CNN_OUT 6

/* Create a network on `device` / `stream` (NULL = legacy default stream) for
 * batches of at most max_batch slices (1..4096).  Parameters are initialised
 * from `seed`: conv and fc weights normal with variance 2 / fan_in, biases 0.
 * Adam moments start at 0. */
gsvr_status gsvr_cnn_create(gsvr_cnn **out, int32_t device, void *stream, int32_t max_batch, uint64_t seed);
gsvr_status gsvr_cnn_destroy(gsvr_cnn *net);
const char *gsvr_cnn_last_error(gsvr_cnn *net);

/* Synchronise and return-and-clear the network's device status word:
 * GSVR_ERR_TIMEOUT when a tensor-memory GEMM of an earlier call gave up a
 * bounded wait (its output was left unwritten), else GSVR_OK.  net NULL
 * synchronises the device and reads the word of the layer primitives. */
gsvr_status gsvr_cnn_sync_status(gsvr_cnn *net);

/* Device pointers to the float32 parameter and gradient vectors (layout above)
 * and their length.  The caller may read or overwrite the parameters between
 * calls (e.g. to load a checkpoint). */
gsvr_status gsvr_cnn_views(gsvr_cnn *net, float **params, float **grads, int64_t *n_params);

/* Forward pass of B slices: x device [B][128][128], aux device [B][25] ->
 * out device [B][6]. */
gsvr_status gsvr_cnn_forward(gsvr_cnn *net, const float *x, const float *aux, int32_t B, float *out);

/* Forward, loss against target (device [B][6]) and backward: the gradient of
 * the loss with respect to every parameter is written to the gradient vector
 * (overwritten).  loss (device, may be NULL) receives the loss as float64. */
gsvr_status gsvr_cnn_loss_backward(gsvr_cnn *net, const float *x, const float *aux, const float *target, int32_t B,
                                   double *loss);

/* One Adam step on every parameter from the gradient vector (bias-corrected
 * with step t >= 1; beta1/beta2/eps of 0 select 0.9 / 0.999 / 1e-8). */
gsvr_status gsvr_cnn_adam_step(gsvr_cnn *net, float lr, float beta1, float beta2, float eps, int64_t t);

/* ---- layer primitives (one conv layer 3x3 / stride 2 / pad 1, NHWC) ----
 * Shapes: x [B][H][W][Ci], w [Co][3][3][Ci], y / gy [B][OH][OW][Co] with
 * OH = (H + 1) / 2, OW = (W + 1) / 2.  Ci and Co must be multiples of 8 (the
 * tensor-core path moves 8 channels at a time; the forward and the weight
 * gradient also take Ci = 1 with Co = 32, the first layer); all pointers
 * device memory, 16-byte aligned.
 *
 * Layers with at least 64 output columns (Co for the forward, 4 Ci for the
 * input gradient) run as tcgen05.mma GEMMs with tensor-memory accumulators,
 * their operands fetched by tensor-map copies when the reduction channels (Ci
 * forward, Co input gradient) are a multiple of 64 and a 128-row tile is
 * whole output rows or whole images (OW and OH OW powers of two, OW <= 128),
 * else by per-thread 16-byte copies; a bounded wait that runs out there is
 * reported by gsvr_cnn_sync_status(NULL).
 *
 * gsvr_cnn_conv_forward: y = bf16(max(conv(x, w) + bias, 0)) when relu, else
 *   without the max; y32 (may be NULL) receives the float32 values before the
 *   bfloat16 rounding.
 * gsvr_cnn_conv_dgrad: dx = conv^T(gy, w) (the input gradient), times
 *   (mask > 0) elementwise when mask (shape of x) is given; dx (bfloat16)
 *   and dx32 (float32, may be NULL).  One GEMM in sub-pixel form: each output
 *   position feeds its 2 x 2 input pixels through the taps that reach them.
 * gsvr_cnn_conv_wgrad: dw [Co][3][3][Ci] += sum over positions of gy x-patch,
 *   db [Co] += sum of gy (float32, accumulated: zero them first; dw 16-byte
 *   aligned).  With Ci a multiple of 64 and the output grid tiled as above
 *   (64-position steps) it runs on tcgen05.mma with both operands MN-major,
 *   the position range split over CTAs that add their tiles atomically (the
 *   summation order, and so the last bits, vary from run to run). */
gsvr_status gsvr_cnn_conv_forward(void *stream, const uint16_t *x, int32_t B, int32_t H, int32_t W, int32_t Ci,
                                  const uint16_t *w, const float *bias, int32_t Co, int32_t relu, uint16_t *y,
                                  float *y32);
gsvr_status gsvr_cnn_conv_dgrad(void *stream, const uint16_t *gy, int32_t B, int32_t H, int32_t W, int32_t Ci,
                                const uint16_t *w, int32_t Co, const uint16_t *mask, uint16_t *dx, float *dx32);
gsvr_status gsvr_cnn_conv_wgrad(void *stream, const uint16_t *gy, const uint16_t *x, int32_t B, int32_t H, int32_t W,
                                int32_t Ci, int32_t Co, float *dw, float *db);

/* Dense GEMM C[M][N] = sum_k A[m][k] B[n][k] (bfloat16 row-major A [M][K] and
 * B [N][K], K a multiple of 8; C float32 row-major; all three 16-byte aligned) on the
 * tensor cores.  tensor_memory selects the kernel:
 *   1  tcgen05.mma, accumulators in tensor memory, operand tiles fetched by
 *      tensor-map copies (cp.async.bulk.tensor, 128-byte swizzle)
 *   2  tcgen05.mma with operand tiles gathered by 16-byte cp.async per thread
 *      (the path of convolution shapes that tensor-map tiles do not cover)
 *   0  mma.sync (register accumulators)
 * For 1 and 2 a bounded wait that runs out sets bit 4 of the device word
 * `status` and leaves C unwritten. */
gsvr_status gsvr_cnn_gemm(void *stream, const uint16_t *A, const uint16_t *B, int32_t M, int32_t N, int32_t K, float *C,
                          int32_t tensor_memory, unsigned *status);

#ifdef __cplusplus
}
#endif

#endif /* GSVR_CNN_H */
