/* cnn_oracle.c -- FP64 reference of the learned pose-initialisation network.
 *
 * TEST INFRASTRUCTURE ONLY (built into liboracle.so with gsvr_oracle.c; only
 * the tests, the smoke check and the benchmark's CPU baseline load it).  It
 * shares no code with the CUDA path.
 *
 * The network regresses a slice's 6-DoF motion (the pose p_i = (r_i, tau_i)
 * of Sec. 2.4, the per-slice rigid transform of Eq. 1) from the slice image,
 * standing in for the learned pre-alignment that produces the residual motion
 * model of Sec. 3.2 ("Data").  Every operation is written as its plain
 * definition with float64 accumulation:
 *
 *   conv 3x3, stride 2, zero padding 1, NHWC activations, weights [Co][3][3][Ci]:
 *     y[b][oh][ow][co] = bias[co] + sum_{kh,kw,ci} w[co][kh][kw][ci] x[b][2oh-1+kh][2ow-1+kw][ci]
 *   its input gradient (scatter of every product) and weight / bias gradients
 *   (sum over every output position).
 */
#include <stdint.h>
#include <string.h>

#include <omp.h>

/* y = conv(x, w) + bias, then max(., 0) when relu.  absy (may be NULL) gets
 * sum |bias| + sum |w x| per output (the rounding scale of the sum). */
void oracle_conv_fwd(int64_t B, int64_t H, int64_t W, int64_t Ci, int64_t Co, const double *x, const double *w,
                     const double *bias, int relu, double *y, double *absy) {
    const int64_t OH = (H + 1) / 2, OW = (W + 1) / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t b = 0; b < B; ++b)
        for (int64_t oh = 0; oh < OH; ++oh)
            for (int64_t ow = 0; ow < OW; ++ow)
                for (int64_t co = 0; co < Co; ++co) {
                    double s = bias ? bias[co] : 0.0;
                    double a = bias ? (bias[co] < 0 ? -bias[co] : bias[co]) : 0.0;
                    for (int64_t kh = 0; kh < 3; ++kh) {
                        const int64_t ih = 2 * oh - 1 + kh;
                        if (ih < 0 || ih >= H) continue;
                        for (int64_t kw = 0; kw < 3; ++kw) {
                            const int64_t iw = 2 * ow - 1 + kw;
                            if (iw < 0 || iw >= W) continue;
                            for (int64_t ci = 0; ci < Ci; ++ci) {
                                const double p = w[((co * 3 + kh) * 3 + kw) * Ci + ci] * x[((b * H + ih) * W + iw) * Ci + ci];
                                s += p;
                                a += p < 0 ? -p : p;
                            }
                        }
                    }
                    const int64_t o = ((b * OH + oh) * OW + ow) * Co + co;
                    y[o] = (relu && s < 0.0) ? 0.0 : s;
                    if (absy) absy[o] = a;
                }
}

/* dx[b][ih][iw][ci] = sum over the outputs that read x[b][ih][iw][ci] of
 * gy * w (the adjoint of oracle_conv_fwd without bias / relu). */
void oracle_conv_dgrad(int64_t B, int64_t H, int64_t W, int64_t Ci, int64_t Co, const double *gy, const double *w,
                       double *dx, double *absdx) {
    const int64_t OH = (H + 1) / 2, OW = (W + 1) / 2;
    memset(dx, 0, sizeof(double) * B * H * W * Ci);
    if (absdx) memset(absdx, 0, sizeof(double) * B * H * W * Ci);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < B; ++b)
        for (int64_t oh = 0; oh < OH; ++oh)
            for (int64_t ow = 0; ow < OW; ++ow)
                for (int64_t co = 0; co < Co; ++co) {
                    const double g = gy[((b * OH + oh) * OW + ow) * Co + co];
                    for (int64_t kh = 0; kh < 3; ++kh) {
                        const int64_t ih = 2 * oh - 1 + kh;
                        if (ih < 0 || ih >= H) continue;
                        for (int64_t kw = 0; kw < 3; ++kw) {
                            const int64_t iw = 2 * ow - 1 + kw;
                            if (iw < 0 || iw >= W) continue;
                            for (int64_t ci = 0; ci < Ci; ++ci) {
                                const double p = g * w[((co * 3 + kh) * 3 + kw) * Ci + ci];
                                dx[((b * H + ih) * W + iw) * Ci + ci] += p;
                                if (absdx) absdx[((b * H + ih) * W + iw) * Ci + ci] += p < 0 ? -p : p;
                            }
                        }
                    }
                }
}

/* dw[co][kh][kw][ci] = sum_{b,oh,ow} gy[b][oh][ow][co] x[b][2oh-1+kh][2ow-1+kw][ci],
 * db[co] = sum_{b,oh,ow} gy[b][oh][ow][co] (overwritten). */
void oracle_conv_wgrad(int64_t B, int64_t H, int64_t W, int64_t Ci, int64_t Co, const double *gy, const double *x,
                       double *dw, double *db, double *absdw) {
    const int64_t OH = (H + 1) / 2, OW = (W + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t co = 0; co < Co; ++co) {
        double sb = 0.0;
        for (int64_t t = 0; t < 9 * Ci; ++t) {
            dw[co * 9 * Ci + t] = 0.0;
            if (absdw) absdw[co * 9 * Ci + t] = 0.0;
        }
        for (int64_t b = 0; b < B; ++b)
            for (int64_t oh = 0; oh < OH; ++oh)
                for (int64_t ow = 0; ow < OW; ++ow) {
                    const double g = gy[((b * OH + oh) * OW + ow) * Co + co];
                    sb += g;
                    for (int64_t kh = 0; kh < 3; ++kh) {
                        const int64_t ih = 2 * oh - 1 + kh;
                        if (ih < 0 || ih >= H) continue;
                        for (int64_t kw = 0; kw < 3; ++kw) {
                            const int64_t iw = 2 * ow - 1 + kw;
                            if (iw < 0 || iw >= W) continue;
                            for (int64_t ci = 0; ci < Ci; ++ci) {
                                const double p = g * x[((b * H + ih) * W + iw) * Ci + ci];
                                dw[((co * 3 + kh) * 3 + kw) * Ci + ci] += p;
                                if (absdw) absdw[((co * 3 + kh) * 3 + kw) * Ci + ci] += p < 0 ? -p : p;
                            }
                        }
                    }
                }
        db[co] = sb;
    }
}
