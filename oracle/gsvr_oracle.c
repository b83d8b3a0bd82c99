/*
 * gsvr_oracle.c -- FP64 brute-force CPU oracle for the analytic-PSF slice
 * forward model over anisotropic 3D Gaussians, its gradient, the Adam step
 * and the pixel sampler.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py load this library.  It shares no
 * code, header, table or helper with the CUDA path, and the product path never
 * calls it.
 *
 * What it computes (paper sections / equations):
 *  - Gaussian primitive (Sec. 2.2, Eq. 2 numerator): mean mu, covariance
 *    Sigma = R S S^T R^T with S = diag(exp(ls)) (log-space scales, Nomenclature
 *    table) and R from the normalised quaternion q = (w, x, y, z); amplitude c.
 *  - Acquisition (Eq. 1, Eq. 3): pixel u of slice i sits at x = R_i u + t_i
 *    (u = (u_x, u_y, 0) in slice millimetres), and its value is the volume
 *    convolved with the slice PSF N(0, R_i Sigma_PSF R_i^T) evaluated at x.
 *  - Closed form (Eq. 4, Eq. 5 numerator): for each Gaussian,
 *    Sigma_obs = Sigma_j + R_i Sigma_PSF R_i^T and the pixel receives
 *    c_j * f * exp(-1/2 v^T Sigma_obs^-1 v), v = x - mu_j, where f is the
 *    exact-convolution normalisation sqrt(det Sigma_j / det Sigma_obs)
 *    (norm_mode 0) or 1 (norm_mode 1, the literal substitution of Eq. 5).
 *    EVERY (pixel, Gaussian) pair is summed; nothing is culled.
 *  - Motion (Sec. 2.4): per slice a 6-DoF motion (r, tau), r axis-angle.  The
 *    slice frame is R_i = Rod(r) R0_i, t_i = Rod(r) c0_i + tau.
 *  - Loss: L = sum_p w_p (I_hat_p - I_p)^2 (mean squared error, w_p = 1/|sample|).
 *  - Gradient of L with respect to mu, ls, q, c and (r, tau), written out in
 *    the 3D form (derivative of the expressions above, pair by pair).
 *  - Adam (the optimiser of the Optimization Details appendix, decoupled
 *    weight decay 0), per parameter group learning rate.
 *
 * Parameter vector layout (component-major SoA), N Gaussians, M slices:
 *   [0,N) mu_x  [N,2N) mu_y  [2N,3N) mu_z  [3N..6N) ls_0..2
 *   [6N..10N) q_w q_x q_y q_z   [10N,11N) c   [11N + 6i + k] pose of slice i
 *   (k = 0..2 axis-angle r, 3..5 translation tau).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n_slices, H, W, pad_;
    double dx, dy, thickness;
    double R[9];      /* row-major; columns are the slice x, y and normal axes in world */
    double origin[3]; /* world position of the stack centre */
    double fwhm[3];   /* PSF full width at half maximum along slice x, y, normal */
} or_stack;

typedef struct {
    double R0[9], c0[3]; /* nominal frame of the slice */
    double var[3];       /* diagonal of Sigma_PSF in slice coordinates */
    double dx, dy;
    int32_t H, W;
    int64_t pix_base;    /* first global pixel index of this slice */
} or_slice;

/* ---------------------------------------------------------------- 3x3 utils */
static void mat_mul(const double *A, const double *B, double *C) {
    double T[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
            T[3 * r + c] = s;
        }
    memcpy(C, T, sizeof T);
}
static void mat_mul_bt(const double *A, const double *B, double *C) { /* A B^T */
    double T[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * c + k];
            T[3 * r + c] = s;
        }
    memcpy(C, T, sizeof T);
}
static void mat_mul_at(const double *A, const double *B, double *C) { /* A^T B */
    double T[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * k + r] * B[3 * k + c];
            T[3 * r + c] = s;
        }
    memcpy(C, T, sizeof T);
}
static void mat_vec(const double *A, const double *v, double *o) {
    double t[3];
    for (int r = 0; r < 3; ++r) t[r] = A[3 * r] * v[0] + A[3 * r + 1] * v[1] + A[3 * r + 2] * v[2];
    memcpy(o, t, sizeof t);
}
static double det3(const double *A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}
/* inverse by the adjugate; returns the determinant */
static double inv3(const double *A, double *Ai) {
    double d = det3(A);
    double id = 1.0 / d;
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) * id;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) * id;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) * id;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return d;
}
static void skew(const double *v, double *K) {
    K[0] = 0.0;   K[1] = -v[2]; K[2] = v[1];
    K[3] = v[2];  K[4] = 0.0;   K[5] = -v[0];
    K[6] = -v[1]; K[7] = v[0];  K[8] = 0.0;
}

/* --------------------------------------------------------------- rotations */
/* Rotation matrix of the unit quaternion q/|q|, q = (w, x, y, z). */
void oracle_quat_to_rot(const double *q_in, double *R) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Rodrigues: exp of the skew matrix of the axis-angle vector r,
 * R = I + A K + B K^2 with A = sin(th)/th, B = (1 - cos th)/th^2. */
static void rod_coeffs(double th, double *A, double *B, double *dA, double *dB) {
    /* dA = A'(th)/th, dB = B'(th)/th (so that d/dr_k of A is dA * r_k) */
    if (th < 1e-3) {
        double t2 = th * th;
        *A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        *B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        *dA = -1.0 / 3.0 + t2 / 30.0 - t2 * t2 / 840.0;
        *dB = -1.0 / 12.0 + t2 / 180.0 - t2 * t2 / 6720.0;
    } else {
        double s = sin(th), c = cos(th);
        *A = s / th;
        *B = (1.0 - c) / (th * th);
        *dA = (th * c - s) / (th * th * th);
        *dB = (th * s - 2.0 * (1.0 - c)) / (th * th * th * th);
    }
}
void oracle_rodrigues(const double *r, double *R) {
    double th = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double A, B, dA, dB, K[9], K2[9];
    rod_coeffs(th, &A, &B, &dA, &dB);
    skew(r, K);
    mat_mul(K, K, K2);
    for (int e = 0; e < 9; ++e) R[e] = (e % 4 == 0 ? 1.0 : 0.0) + A * K[e] + B * K2[e];
}
/* dR/dr_k by the product rule on R = I + A(th) K + B(th) K^2. */
static void rodrigues_jac(const double *r, double J[3][9]) {
    double th = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double A, B, dA, dB, K[9], K2[9];
    rod_coeffs(th, &A, &B, &dA, &dB);
    skew(r, K);
    mat_mul(K, K, K2);
    for (int k = 0; k < 3; ++k) {
        double ek[3] = {0, 0, 0}, E[9], EK[9], KE[9];
        ek[k] = 1.0;
        skew(ek, E);
        mat_mul(E, K, EK);
        mat_mul(K, E, KE);
        for (int e = 0; e < 9; ++e)
            J[k][e] = dA * r[k] * K[e] + A * E[e] + dB * r[k] * K2[e] + B * (EK[e] + KE[e]);
    }
}

/* ------------------------------------------------------------ slice frames */
/* Stacks -> slices.  Slice k of a stack of n slices is centred at
 * origin + (k - (n-1)/2) * thickness * normal (contiguous slices, no gap);
 * its nominal rotation is the stack rotation; Sigma_PSF = diag((fwhm/2.355)^2).
 * Returns the number of slices; fills out (may be NULL to count). */
int64_t oracle_build_slices(int n_stacks, const or_stack *st, or_slice *out, int64_t *n_pixels) {
    int64_t m = 0, pix = 0;
    for (int s = 0; s < n_stacks; ++s) {
        for (int k = 0; k < st[s].n_slices; ++k) {
            if (out) {
                or_slice *o = &out[m];
                memcpy(o->R0, st[s].R, sizeof o->R0);
                double off = ((double)k - 0.5 * (st[s].n_slices - 1)) * st[s].thickness;
                for (int a = 0; a < 3; ++a) o->c0[a] = st[s].origin[a] + off * st[s].R[3 * a + 2];
                for (int a = 0; a < 3; ++a) {
                    double sg = st[s].fwhm[a] / 2.355;
                    o->var[a] = sg * sg;
                }
                o->dx = st[s].dx;
                o->dy = st[s].dy;
                o->H = st[s].H;
                o->W = st[s].W;
                o->pix_base = pix;
            }
            pix += (int64_t)st[s].H * st[s].W;
            ++m;
        }
    }
    if (n_pixels) *n_pixels = pix;
    return m;
}

typedef struct {
    double R[9], t[3];  /* world-from-slice rotation and slice centre */
    double Spsf[9];     /* R Sigma_PSF R^T */
    double rod[9];      /* Rod(r) */
} or_frame;

static void slice_frame(const or_slice *s, const double *pose, or_frame *f) {
    oracle_rodrigues(pose, f->rod);
    mat_mul(f->rod, s->R0, f->R);
    mat_vec(f->rod, s->c0, f->t);
    for (int a = 0; a < 3; ++a) f->t[a] += pose[3 + a];
    double D[9] = {s->var[0], 0, 0, 0, s->var[1], 0, 0, 0, s->var[2]}, T[9];
    mat_mul(f->R, D, T);
    mat_mul_bt(T, f->R, f->Spsf);
}

/* Exported for the geometry pins: world frame (R_i, t_i) of every slice. */
int oracle_slice_frames(int n_stacks, const or_stack *st, const double *pose, double *R_out, double *t_out) {
    int64_t npx;
    int64_t M = oracle_build_slices(n_stacks, st, NULL, &npx);
    or_slice *sl = (or_slice *)malloc(sizeof(or_slice) * (size_t)(M ? M : 1));
    oracle_build_slices(n_stacks, st, sl, &npx);
    for (int64_t i = 0; i < M; ++i) {
        or_frame f;
        slice_frame(&sl[i], pose + 6 * i, &f);
        memcpy(R_out + 9 * i, f.R, sizeof f.R);
        memcpy(t_out + 3 * i, f.t, sizeof f.t);
    }
    free(sl);
    return (int)M;
}

/* Decode a global pixel index into (slice, row, col) and its slice-local mm
 * coordinate u = ((col - (W-1)/2) dx, (row - (H-1)/2) dy, 0). */
static int64_t find_slice(const or_slice *sl, int64_t M, int64_t p) {
    int64_t lo = 0, hi = M - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (sl[mid].pix_base <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}
static void pixel_local(const or_slice *s, int64_t p, double *u) {
    int64_t loc = p - s->pix_base;
    int64_t row = loc / s->W, col = loc % s->W;
    u[0] = ((double)col - 0.5 * (s->W - 1)) * s->dx;
    u[1] = ((double)row - 0.5 * (s->H - 1)) * s->dy;
    u[2] = 0.0;
}

/* ---------------------------------------------------------------- Gaussians */
typedef struct {
    double mu[3], Rj[9], s2[3], Sig[9], det, c, qn[4], qnorm;
} or_gauss;

static void gauss_setup(int64_t N, const double *th, int64_t j, or_gauss *g) {
    for (int a = 0; a < 3; ++a) g->mu[a] = th[a * N + j];
    double q[4];
    for (int a = 0; a < 4; ++a) q[a] = th[(6 + a) * N + j];
    g->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a) g->qn[a] = q[a] / g->qnorm;
    oracle_quat_to_rot(q, g->Rj);
    double lsum = 0.0;
    for (int a = 0; a < 3; ++a) {
        double ls = th[(3 + a) * N + j];
        g->s2[a] = exp(2.0 * ls);
        lsum += ls;
    }
    double D[9] = {g->s2[0], 0, 0, 0, g->s2[1], 0, 0, 0, g->s2[2]}, T[9];
    mat_mul(g->Rj, D, T);
    mat_mul_bt(T, g->Rj, g->Sig);
    g->det = exp(2.0 * lsum);
    g->c = th[10 * N + j];
}

/* Gaussian covariance for the pins: Sigma (9 per Gaussian, row-major). */
void oracle_gauss_cov(int64_t N, const double *theta, double *Sig_out) {
    for (int64_t j = 0; j < N; ++j) {
        or_gauss g;
        gauss_setup(N, theta, j, &g);
        memcpy(Sig_out + 9 * j, g.Sig, sizeof g.Sig);
    }
}

/* One pair: value g = f * exp(-1/2 v^T P v) and the pieces the gradient needs. */
typedef struct {
    double P[9], v[3], Pv[3], e, f, g;
} or_pair;

static void eval_pair(const or_gauss *gj, const or_frame *fr, const double *x, int norm_mode, or_pair *pr) {
    double So[9];
    for (int e = 0; e < 9; ++e) So[e] = gj->Sig[e] + fr->Spsf[e];
    double dso = inv3(So, pr->P);
    for (int a = 0; a < 3; ++a) pr->v[a] = x[a] - gj->mu[a];
    mat_vec(pr->P, pr->v, pr->Pv);
    double d2 = pr->v[0] * pr->Pv[0] + pr->v[1] * pr->Pv[1] + pr->v[2] * pr->Pv[2];
    pr->e = exp(-0.5 * d2);
    pr->f = norm_mode == 0 ? sqrt(gj->det / dso) : 1.0;
    pr->g = pr->f * pr->e;
}

typedef struct {
    int64_t M, npx;
    or_slice *sl;
    or_frame *fr;
    or_gauss *g;
} or_model;

static int model_setup(int n_stacks, const or_stack *st, int64_t N, const double *theta, or_model *m) {
    m->M = oracle_build_slices(n_stacks, st, NULL, &m->npx);
    m->sl = (or_slice *)malloc(sizeof(or_slice) * (size_t)(m->M ? m->M : 1));
    m->fr = (or_frame *)malloc(sizeof(or_frame) * (size_t)(m->M ? m->M : 1));
    m->g = (or_gauss *)malloc(sizeof(or_gauss) * (size_t)(N ? N : 1));
    if (!m->sl || !m->fr || !m->g) return -1;
    oracle_build_slices(n_stacks, st, m->sl, &m->npx);
    for (int64_t i = 0; i < m->M; ++i) slice_frame(&m->sl[i], theta + 11 * N + 6 * i, &m->fr[i]);
    for (int64_t j = 0; j < N; ++j) gauss_setup(N, theta, j, &m->g[j]);
    return 0;
}
static void model_free(or_model *m) {
    free(m->sl);
    free(m->fr);
    free(m->g);
}

static void pixel_world(const or_model *m, int64_t p, int64_t *slice, double *u, double *x) {
    int64_t i = find_slice(m->sl, m->M, p);
    pixel_local(&m->sl[i], p, u);
    mat_vec(m->fr[i].R, u, x);
    for (int a = 0; a < 3; ++a) x[a] += m->fr[i].t[a];
    *slice = i;
}

/* Data loss of one residual r = pred - I: MSE w r^2 (loss_kind 0) or the
 * paper's L1 w |r| (loss_kind 1, Sec. 2.5 "Loss Function"), and its derivative
 * in r (the L1 subgradient takes sign(0) = 0). */
static double data_loss(int loss_kind, double w, double r) { return loss_kind ? w * fabs(r) : w * r * r; }
static double data_dloss(int loss_kind, double w, double r) {
    return loss_kind ? w * (double)((r > 0.0) - (r < 0.0)) : 2.0 * w * r;
}

/* Per-slice outlier terms (Sec. 2.4): slw = NULL, or 2 M values: log sigma_i
 * (intensity scale: the prediction is sigma_i times the model) then
 * log omega_i (aleatoric weight: a pixel of slice i costs
 * w (loss(r) / omega_i + log omega_i)).  pixel_terms gives, for a model value s
 * of slice i, the prediction, the loss and dL/ds; the per-slice derivatives
 * in log sigma_i and log omega_i are added to gsl (when not NULL). */
static void pixel_terms(const double *slw, int64_t M, int64_t i, int loss_kind, double w, double s, double I,
                        double *pred, double *L, double *dLds, double *gsl) {
    const double sig = slw ? exp(slw[i]) : 1.0, lw = slw ? slw[M + i] : 0.0, iw = exp(-lw);
    const double r = sig * s - I;
    const double l = data_loss(loss_kind, w, r), dl = data_dloss(loss_kind, w, r);
    *pred = sig * s;
    *L = l * iw + (slw ? w * lw : 0.0);
    *dLds = sig * dl * iw;
    if (gsl) {
        gsl[i] += dl * iw * sig * s;
        gsl[M + i] += w - l * iw;
    }
}

/* Sum of x[0..n) in index order with Neumaier's compensation: the result does
 * not depend on the thread schedule that produced the terms, and its error is
 * about one rounding of the total (a plain running sum would add a rounding
 * of the running total per term, which central differences of the loss
 * amplify by 1 / (2 h)). */
static double sum_in_order(const double *x, int64_t n) {
    double s = 0.0, c = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double t = s + x[k];
        c += fabs(s) >= fabs(x[k]) ? (s - t) + x[k] : (x[k] - t) + s;
        s = t;
    }
    return s + c;
}

/* Forward: pred[p] = sum over ALL Gaussians (times sigma_i); loss = sum_p of the
 * pixel losses. */
int oracle_forward(int n_stacks, const or_stack *st, int64_t N, const double *theta, int64_t P,
                   const int64_t *pix, const double *I_obs, double w_pix, int norm_mode, int loss_kind,
                   const double *slw, double *pred, double *loss) {
    or_model m;
    if (model_setup(n_stacks, st, N, theta, &m)) return -1;
    /* per-pixel loss terms, summed afterwards in pixel order (the sum is then
     * the same whatever the thread schedule) */
    double *lt = (double *)calloc((size_t)(P ? P : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t p = 0; p < P; ++p) {
        int64_t i;
        double u[3], x[3];
        pixel_world(&m, pix[p], &i, u, x);
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            or_pair pr;
            eval_pair(&m.g[j], &m.fr[i], x, norm_mode, &pr);
            s += m.g[j].c * pr.g;
        }
        double lp = 0.0, dl;
        pixel_terms(slw, m.M, i, loss_kind, w_pix, s, I_obs ? I_obs[p] : 0.0, &pred[p], &lp, &dl, NULL);
        lt[p] = I_obs ? lp : 0.0;
    }
    const double L = sum_in_order(lt, P);
    free(lt);
    if (loss) *loss = L;
    model_free(&m);
    return 0;
}

/* Number of (listed pixel, Gaussian) pairs with exp(-1/2 v^T Sigma_obs^-1 v) >= cutoff
 * (the pairs a per-pair truncation at `cutoff` keeps; Eq. 4 / Eq. 5 exponent). */
int64_t oracle_count_pairs(int n_stacks, const or_stack *st, int64_t N, const double *theta, int64_t P,
                           const int64_t *pix, double cutoff) {
    or_model m;
    if (model_setup(n_stacks, st, N, theta, &m)) return -1;
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : total)
    for (int64_t p = 0; p < P; ++p) {
        int64_t i;
        double u[3], x[3];
        pixel_world(&m, pix[p], &i, u, x);
        for (int64_t j = 0; j < N; ++j) {
            or_pair pr;
            eval_pair(&m.g[j], &m.fr[i], x, 0, &pr);
            total += pr.e >= cutoff ? 1 : 0;
        }
    }
    model_free(&m);
    return total;
}

/* Chain of a symmetric covariance gradient G (dL = tr(G dSigma)) through
 * Sigma = R diag(s^2) R^T, s = exp(ls), R = R(q/|q|): d ls (3) and d q (4). */
static void cov_chain(const or_gauss *g, const double *G, double *dls, double *dq) {
    double RtG[9], RtGR[9];
    mat_mul_at(g->Rj, G, RtG);
    mat_mul(RtG, g->Rj, RtGR);
    for (int k = 0; k < 3; ++k) dls[k] = 2.0 * g->s2[k] * RtGR[4 * k];
    /* dL/dR = 2 G R D */
    double D[9] = {g->s2[0], 0, 0, 0, g->s2[1], 0, 0, 0, g->s2[2]}, GR[9], GRD[9];
    mat_mul(G, g->Rj, GR);
    mat_mul(GR, D, GRD);
    for (int e = 0; e < 9; ++e) GRD[e] *= 2.0;
    double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
    /* partial derivatives of R(w,x,y,z) (unit-quaternion formula) */
    const double dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const double dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const double dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const double dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    double gq[4] = {0, 0, 0, 0};
    for (int e = 0; e < 9; ++e) {
        gq[0] += GRD[e] * dRw[e];
        gq[1] += GRD[e] * dRx[e];
        gq[2] += GRD[e] * dRy[e];
        gq[3] += GRD[e] * dRz[e];
    }
    /* through the normalisation q_hat = q / |q| */
    double dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    dq[0] = (gq[0] - w * dot) / g->qnorm;
    dq[1] = (gq[1] - x * dot) / g->qnorm;
    dq[2] = (gq[2] - y * dot) / g->qnorm;
    dq[3] = (gq[3] - z * dot) / g->qnorm;
}

/* The same chain with every product and sum taken in absolute value: the
 * componentwise scale of the float rounding of a computation that accumulates
 * the covariance gradient and projects it once (|dls_k|, |dq_c| bounds). */
static void cov_chain_abs(const or_gauss *g, const double *Gabs, double *dls, double *dq) {
    double R[9], D[9] = {g->s2[0], 0, 0, 0, g->s2[1], 0, 0, 0, g->s2[2]};
    for (int e = 0; e < 9; ++e) R[e] = fabs(g->Rj[e]);
    double RtG[9], RtGR[9];
    mat_mul_at(R, Gabs, RtG);
    mat_mul(RtG, R, RtGR);
    for (int k = 0; k < 3; ++k) dls[k] = 2.0 * g->s2[k] * RtGR[4 * k];
    double GR[9], GRD[9];
    mat_mul(Gabs, R, GR);
    mat_mul(GR, D, GRD);
    double w = fabs(g->qn[0]), x = fabs(g->qn[1]), y = fabs(g->qn[2]), z = fabs(g->qn[3]);
    const double dRw[9] = {0, 2 * z, 2 * y, 2 * z, 0, 2 * x, 2 * y, 2 * x, 0};
    const double dRx[9] = {0, 2 * y, 2 * z, 2 * y, 4 * x, 2 * w, 2 * z, 2 * w, 4 * x};
    const double dRy[9] = {4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, 2 * w, 2 * z, 4 * y};
    const double dRz[9] = {4 * z, 2 * w, 2 * x, 2 * w, 4 * z, 2 * y, 2 * x, 2 * y, 0};
    double gq[4] = {0, 0, 0, 0};
    for (int e = 0; e < 9; ++e) {
        gq[0] += 2.0 * GRD[e] * dRw[e];
        gq[1] += 2.0 * GRD[e] * dRx[e];
        gq[2] += 2.0 * GRD[e] * dRy[e];
        gq[3] += 2.0 * GRD[e] * dRz[e];
    }
    double n1 = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
    dq[0] = (gq[0] + w * n1) / g->qnorm;
    dq[1] = (gq[1] + x * n1) / g->qnorm;
    dq[2] = (gq[2] + y * n1) / g->qnorm;
    dq[3] = (gq[3] + z * n1) / g->qnorm;
}

/* Absolute-value version of pose_chain (componentwise rounding scale). */
static void pose_chain_abs(const or_slice *s, const double *pose, const double *GRabs, const double *Gtabs,
                           double *out6) {
    double J[3][9], G[9], R0[9], c0[3];
    rodrigues_jac(pose, J);
    for (int e = 0; e < 9; ++e) R0[e] = fabs(s->R0[e]);
    for (int a = 0; a < 3; ++a) c0[a] = fabs(s->c0[a]);
    mat_mul_bt(GRabs, R0, G);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[3 * a + b] += Gtabs[a] * c0[b];
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (int e = 0; e < 9; ++e) acc += G[e] * fabs(J[k][e]);
        out6[k] = acc;
    }
    for (int a = 0; a < 3; ++a) out6[3 + a] = Gtabs[a];
}

/* Chain of the slice-frame gradients (dL/dR_i, dL/dt_i) through
 * R_i = Rod(r) R0, t_i = Rod(r) c0 + tau: d r (3), d tau (3). */
static void pose_chain(const or_slice *s, const double *pose, const double *GR, const double *Gt, double *out6) {
    double J[3][9], G[9];
    rodrigues_jac(pose, J);
    /* dL/dRod = GR R0^T + Gt c0^T */
    mat_mul_bt(GR, s->R0, G);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[3 * a + b] += Gt[a] * s->c0[b];
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (int e = 0; e < 9; ++e) acc += G[e] * J[k][e];
        out6[k] = acc;
    }
    for (int a = 0; a < 3; ++a) out6[3 + a] = Gt[a];
}

/*
 * Forward + backward.  grad (11N + 6M) receives dL/dtheta.  absgrad, when not
 * NULL, receives for every entry the sum over pairs of |that pair's
 * contribution| (a condition-aware scale for comparing float32 sums).
 * When cutoff > 0 and trunc_pred / trunc_grad are not NULL they receive the
 * same sums restricted to the pairs with exp(-1/2 v^T Sigma_obs^-1 v) < cutoff,
 * i.e. the most a per-pair truncation at `cutoff` can change each output.
 * Only Gaussians with sel[j] != 0 get gradients (sel NULL = all); pose
 * gradients always include every pair of the selected Gaussians.
 */
int oracle_forward_backward(int n_stacks, const or_stack *st, int64_t N, const double *theta, int64_t P,
                            const int64_t *pix, const double *I_obs, double w_pix, int norm_mode, int loss_kind,
                            const double *slw, double *slw_grad, const uint8_t *sel, double *pred, double *loss,
                            double *grad, double *absgrad, double cutoff, double *trunc_pred, double *trunc_grad) {
    const int want_trunc = cutoff > 0.0 && trunc_grad != NULL && absgrad != NULL;
    or_model m;
    if (model_setup(n_stacks, st, N, theta, &m)) return -1;
    const int64_t M = m.M;
    double *rbar = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *px = (double *)malloc(sizeof(double) * 3 * (size_t)(P ? P : 1));
    double *pu = (double *)malloc(sizeof(double) * 3 * (size_t)(P ? P : 1));
    int64_t *psl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P ? P : 1));
    double *pmod = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *lt = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));  /* per-pixel loss terms */
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t p = 0; p < P; ++p) {
        int64_t i;
        pixel_world(&m, pix[p], &i, &pu[3 * p], &px[3 * p]);
        psl[p] = i;
        double s = 0.0, tr = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            or_pair pr;
            eval_pair(&m.g[j], &m.fr[i], &px[3 * p], norm_mode, &pr);
            s += m.g[j].c * pr.g;
            if (pr.e < cutoff) tr += fabs(m.g[j].c * pr.g);
        }
        double pr_, lp;
        pixel_terms(slw, M, i, loss_kind, w_pix, s, I_obs[p], &pr_, &lp, &rbar[p], NULL);
        if (pred) pred[p] = pr_;
        if (trunc_pred) trunc_pred[p] = tr;
        pmod[p] = s;
        lt[p] = lp;
    }
    const double L = sum_in_order(lt, P);
    free(lt);
    if (loss) *loss = L;
    if (slw_grad) {  /* per-slice sums in pixel order */
        memset(slw_grad, 0, sizeof(double) * (size_t)(2 * M));
        for (int64_t p = 0; p < P; ++p) {
            double a, b, c;
            pixel_terms(slw, M, psl[p], loss_kind, w_pix, pmod[p], I_obs[p], &a, &b, &c, slw_grad);
        }
    }
    memset(grad, 0, sizeof(double) * (size_t)(11 * N + 6 * M));
    if (absgrad) memset(absgrad, 0, sizeof(double) * (size_t)(11 * N + 6 * M));
    if (want_trunc) memset(trunc_grad, 0, sizeof(double) * (size_t)(11 * N + 6 * M));

    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    /* per-thread slice accumulators: dL/dR_i (9), dL/dt_i (3), |.| of the pose entries (6),
     * |.| of the truncated pairs' pose entries (6) */
    double *pacc = (double *)calloc((size_t)nthreads * (size_t)(M ? M : 1) * 24, sizeof(double));

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = pacc + (size_t)tid * (size_t)(M ? M : 1) * 24;
#pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < N; ++j) {
            if (sel && !sel[j]) continue;
            const or_gauss *gj = &m.g[j];
            double gmu[3] = {0, 0, 0}, GS[9] = {0}, gc = 0.0, glogdet = 0.0;
            double amu[3] = {0, 0, 0}, als[3] = {0, 0, 0}, aq[4] = {0, 0, 0, 0}, ac = 0.0;
            double tmu[3] = {0, 0, 0}, tls[3] = {0, 0, 0}, tq[4] = {0, 0, 0, 0}, tc = 0.0;
            for (int64_t p = 0; p < P; ++p) {
                int64_t i = psl[p];
                or_pair pr;
                eval_pair(gj, &m.fr[i], &px[3 * p], norm_mode, &pr);
                double a = rbar[p] * gj->c * pr.g;
                double dc = rbar[p] * pr.g;
                gc += dc;
                /* d/dSigma_obs of exp(-1/2 v^T P v) is 1/2 P v v^T P; the exact
                 * normalisation adds d/dSigma_obs of -1/2 log det Sigma_obs = -1/2 P. */
                const double pk = norm_mode == 0 ? 1.0 : 0.0;
                double Go[9];
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c)
                        Go[3 * r + c] = 0.5 * a * (pr.Pv[r] * pr.Pv[c] - pk * pr.P[3 * r + c]);
                for (int e = 0; e < 9; ++e) GS[e] += Go[e];
                for (int k = 0; k < 3; ++k) gmu[k] += a * pr.Pv[k];
                if (norm_mode == 0) glogdet += 0.5 * a; /* d(1/2 log det Sigma_j) */
                /* slice-frame contributions: x = R u + t, Sigma_obs contains R Sigma_PSF R^T */
                double dx[3] = {-a * pr.Pv[0], -a * pr.Pv[1], -a * pr.Pv[2]};
                double GR[9], D[9] = {0}, RD[9], GoRD[9];
                D[0] = m.sl[i].var[0]; D[4] = m.sl[i].var[1]; D[8] = m.sl[i].var[2];
                mat_mul(m.fr[i].R, D, RD);
                mat_mul(Go, RD, GoRD);
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c)
                        GR[3 * r + c] = dx[r] * pu[3 * p + c] + 2.0 * GoRD[3 * r + c];
                double *acc = my + 24 * i;
                const int cut = pr.e < cutoff;
                for (int e = 0; e < 9; ++e) acc[e] += GR[e];
                for (int k = 0; k < 3; ++k) acc[9 + k] += dx[k];
                if (absgrad) {
                    /* componentwise scales: |.| of every product and sum of the chain */
                    double d6[6], dls[3], dq[4], Ga[9], GRa[9], dxa[3], RDa[9], GoRDa[9];
                    for (int e = 0; e < 9; ++e) {
                        Ga[e] = fabs(Go[e]);
                        RDa[e] = fabs(RD[e]);
                    }
                    for (int k = 0; k < 3; ++k) dxa[k] = fabs(dx[k]);
                    mat_mul(Ga, RDa, GoRDa);
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c)
                            GRa[3 * r + c] = dxa[r] * fabs(pu[3 * p + c]) + 2.0 * GoRDa[3 * r + c];
                    pose_chain_abs(&m.sl[i], theta + 11 * N + 6 * i, GRa, dxa, d6);
                    for (int k = 0; k < 6; ++k) acc[12 + k] += fabs(d6[k]);
                    cov_chain_abs(gj, Ga, dls, dq);
                    for (int k = 0; k < 3; ++k) {
                        double v = dls[k] + (norm_mode == 0 ? fabs(a) : 0.0);
                        als[k] += v;
                        amu[k] += fabs(a * pr.Pv[k]);
                        if (cut) {
                            tls[k] += fabs(v);
                            tmu[k] += fabs(a * pr.Pv[k]);
                        }
                    }
                    for (int k = 0; k < 4; ++k) {
                        aq[k] += fabs(dq[k]);
                        if (cut) tq[k] += fabs(dq[k]);
                    }
                    ac += fabs(dc);
                    if (cut) {
                        tc += fabs(dc);
                        for (int k = 0; k < 6; ++k) acc[18 + k] += fabs(d6[k]);
                    }
                }
            }
            double dls[3], dq[4];
            cov_chain(gj, GS, dls, dq);
            for (int k = 0; k < 3; ++k) {
                grad[k * N + j] = gmu[k];
                grad[(3 + k) * N + j] = dls[k] + 2.0 * glogdet; /* log det Sigma_j = 2 sum ls */
            }
            for (int k = 0; k < 4; ++k) grad[(6 + k) * N + j] = dq[k];
            grad[10 * N + j] = gc;
            if (absgrad) {
                for (int k = 0; k < 3; ++k) {
                    absgrad[k * N + j] = amu[k];
                    absgrad[(3 + k) * N + j] = als[k];
                }
                for (int k = 0; k < 4; ++k) absgrad[(6 + k) * N + j] = aq[k];
                absgrad[10 * N + j] = ac;
            }
            if (want_trunc) {
                for (int k = 0; k < 3; ++k) {
                    trunc_grad[k * N + j] = tmu[k];
                    trunc_grad[(3 + k) * N + j] = tls[k];
                }
                for (int k = 0; k < 4; ++k) trunc_grad[(6 + k) * N + j] = tq[k];
                trunc_grad[10 * N + j] = tc;
            }
        }
    }
    for (int64_t i = 0; i < M; ++i) {
        double GR[9] = {0}, Gt[3] = {0}, ab[6] = {0}, tb[6] = {0};
        for (int t = 0; t < nthreads; ++t) {
            const double *acc = pacc + ((size_t)t * (size_t)M + (size_t)i) * 24;
            for (int e = 0; e < 9; ++e) GR[e] += acc[e];
            for (int k = 0; k < 3; ++k) Gt[k] += acc[9 + k];
            for (int k = 0; k < 6; ++k) ab[k] += acc[12 + k];
            for (int k = 0; k < 6; ++k) tb[k] += acc[18 + k];
        }
        double d6[6];
        pose_chain(&m.sl[i], theta + 11 * N + 6 * i, GR, Gt, d6);
        for (int k = 0; k < 6; ++k) {
            grad[11 * N + 6 * i + k] = d6[k];
            if (absgrad) absgrad[11 * N + 6 * i + k] = ab[k];
            if (want_trunc) trunc_grad[11 * N + 6 * i + k] = tb[k];
        }
    }
    free(pacc);
    free(rbar);
    free(pmod);
    free(px);
    free(pu);
    free(psl);
    model_free(&m);
    return 0;
}

/*
 * Adam (Kingma & Ba), bias-corrected, decoupled weight decay 0, one step t >= 1,
 * in place on theta, m, v.  Learning rate per group: lr[0] mu, lr[1] ls,
 * lr[2] q, lr[3] c, lr[4] pose rotation r, lr[5] pose translation tau.
 * Slices with frozen[i] != 0 keep their pose (and its moments) unchanged.
 */
void oracle_adam(int64_t N, int64_t M, double *theta, const double *grad, double *m, double *v,
                 const double *lr, double beta1, double beta2, double eps, int64_t t, const uint8_t *frozen) {
    int64_t n = 11 * N + 6 * M;
    double bc1 = 1.0 - pow(beta1, (double)t), bc2 = 1.0 - pow(beta2, (double)t);
    for (int64_t e = 0; e < n; ++e) {
        double rate;
        if (e < 3 * N) rate = lr[0];
        else if (e < 6 * N) rate = lr[1];
        else if (e < 10 * N) rate = lr[2];
        else if (e < 11 * N) rate = lr[3];
        else {
            int64_t i = (e - 11 * N) / 6, k = (e - 11 * N) % 6;
            if (frozen && frozen[i]) continue;
            rate = k < 3 ? lr[4] : lr[5];
        }
        m[e] = beta1 * m[e] + (1.0 - beta1) * grad[e];
        v[e] = beta2 * v[e] + (1.0 - beta2) * grad[e] * grad[e];
        double mh = m[e] / bc1, vh = v[e] / bc2;
        theta[e] -= rate * mh / (sqrt(vh) + eps);
    }
}

/*
 * Pixel sampler: n_s of n mask pixels, uniformly without replacement, as the
 * first n_s values of a keyed random permutation of [0, n).
 *  - SplitMix64 (Steele, Lea & Flood 2014), used as a counter-based generator:
 *    out(seed, ctr) = mix(seed + (ctr + 1) * 0x9E3779B97F4A7C15).
 *  - A bijection f on k-bit integers (2^k >= n) made of 4 rounds of
 *    x ^= key_r; x *= odd_r; x ^= x >> h (all mod 2^k, each step invertible),
 *    with round keys out(seed, 4 * step + r).
 *  - Cycle walking: y = f(x) until y < n (a permutation of [0, n)).
 */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t ctr) {
    uint64_t z = seed + (ctr + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

int oracle_sample_positions(int64_t n, int64_t n_s, uint64_t seed, uint64_t step, int64_t *out) {
    if (n_s > n || n <= 0) return -1;
    int k = 1;
    while ((1LL << k) < n) ++k;
    uint64_t mask = (k >= 64) ? ~0ULL : ((1ULL << k) - 1ULL);
    int h = (k + 1) / 2;
    uint64_t xk[4], mul[4];
    for (int r = 0; r < 4; ++r) {
        uint64_t key = oracle_splitmix64(seed, 4ULL * step + (uint64_t)r);
        xk[r] = key & mask;
        mul[r] = (key >> 32) | 1ULL;
    }
    for (int64_t t = 0; t < n_s; ++t) {
        uint64_t x = (uint64_t)t;
        do {
            for (int r = 0; r < 4; ++r) {
                x = (x ^ xk[r]) & mask;
                x = (x * mul[r]) & mask;
                x ^= x >> h;
            }
        } while (x >= (uint64_t)n);
        out[t] = (int64_t)x;
    }
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------ large cases: local FD
 * Central differences of the loss L = sum_p w (I_hat_p - I_p)^2 over a listed
 * pixel set, for selected parameters, at sizes where the all-pairs sums above
 * are too slow.  The closed form of Eq. 4 / Eq. 5 is unchanged; only which
 * pairs are visited differs: a pair whose exponent has exp(-1/2 v^T P v) < cut
 * is dropped (cut = 1e-12 keeps every pair that matters in float64), and the
 * pairs a pixel can have are found through a uniform grid of the Gaussian
 * means whose cell is at least the largest Euclidean radius of that cut.
 *  - predictions I_hat_p (float64) of every listed pixel -> pred_out, and per
 *    pixel the sum of |terms| with trunc_cut > exp(.) >= cut -> trunc_out
 *    (what a cut at trunc_cut drops);
 *  - a Gaussian parameter changes only that Gaussian's terms: the loss change
 *    is summed over the listed pixels within its cut under either perturbed
 *    value, from I_hat_p minus the old term plus the new one;
 *  - a slice-pose parameter moves that slice's pixels and PSF: its listed
 *    pixels are re-evaluated with the perturbed frame. */
typedef struct {
    double lo[3], cell;
    int64_t n[3];
    int64_t *start, *items;
} or_grid;

static int64_t grid_cell_of(const or_grid *G, const double *x, int64_t c[3]) {
    for (int a = 0; a < 3; ++a) {
        int64_t k = (int64_t)floor((x[a] - G->lo[a]) / G->cell);
        c[a] = k < 0 ? 0 : (k >= G->n[a] ? G->n[a] - 1 : k);
    }
    return (c[2] * G->n[1] + c[1]) * G->n[0] + c[0];
}

static int grid_build(or_grid *G, int64_t n, const double *pts, double cell, const double *lo, const double *hi) {
    G->cell = cell;
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        G->lo[a] = lo[a];
        G->n[a] = (int64_t)floor((hi[a] - lo[a]) / cell) + 1;
        if (G->n[a] < 1) G->n[a] = 1;
        total *= G->n[a];
    }
    G->start = (int64_t *)calloc((size_t)total + 1, sizeof(int64_t));
    G->items = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t *cellof = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (!G->start || !G->items || !cellof) return -1;
    for (int64_t k = 0; k < n; ++k) {
        int64_t c[3];
        cellof[k] = grid_cell_of(G, pts + 3 * k, c);
        G->start[cellof[k] + 1]++;
    }
    for (int64_t c = 0; c < total; ++c) G->start[c + 1] += G->start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)total);
    memcpy(fill, G->start, sizeof(int64_t) * (size_t)total);
    for (int64_t k = 0; k < n; ++k) G->items[fill[cellof[k]]++] = k;
    free(fill);
    free(cellof);
    return 0;
}

static void grid_free(or_grid *G) {
    free(G->start);
    free(G->items);
}

/* Sum over the Gaussians near x of c_l f exp(-1/2 v^T P v), pairs below the cut dropped. */
static double pred_near(const or_model *m, const or_grid *G, const double *mu, const or_frame *fr, const double *x,
                        int norm_mode, double r2cut, double rad2, double r2t, double *trunc, double *absum) {
    int64_t c[3];
    grid_cell_of(G, x, c);
    double s = 0.0;
    for (int64_t dz = -1; dz <= 1; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= G->n[0] || cy >= G->n[1] || cz >= G->n[2]) continue;
                int64_t cell = (cz * G->n[1] + cy) * G->n[0] + cx;
                for (int64_t q = G->start[cell]; q < G->start[cell + 1]; ++q) {
                    int64_t l = G->items[q];
                    double v0 = x[0] - mu[3 * l], v1 = x[1] - mu[3 * l + 1], v2 = x[2] - mu[3 * l + 2];
                    if (v0 * v0 + v1 * v1 + v2 * v2 > rad2) continue;  /* outside every pair's cut radius */
                    or_pair pr;
                    eval_pair(&m->g[l], fr, x, norm_mode, &pr);
                    double d2 = -2.0 * log(pr.e > 0.0 ? pr.e : 1e-300);
                    if (d2 <= r2cut) {
                        s += m->g[l].c * pr.g;
                        if (trunc && d2 > r2t) *trunc += fabs(m->g[l].c * pr.g);
                        if (absum) *absum += fabs(m->g[l].c * pr.g);
                    }
                }
            }
    return s;
}

int oracle_local_fd(int n_stacks, const or_stack *st, int64_t N, const double *theta, int64_t P, const int64_t *pix,
                    const double *I_obs, double w_pix, int norm_mode, double cut, int64_t K, const int64_t *params,
                    const double *h, double *fd_out, double *pred_out, double trunc_cut, double *trunc_out) {
    or_model m;
    if (model_setup(n_stacks, st, N, theta, &m)) return -1;
    const double r2cut = -2.0 * log(cut);
    /* the largest Euclidean cut radius over all pairs: r2cut (max Gaussian
     * variance + max PSF variance), with 1 % margin for the perturbations */
    double vmax = 0.0, pmax = 0.0;
    for (int64_t j = 0; j < N; ++j)
        for (int a = 0; a < 3; ++a) vmax = m.g[j].s2[a] > vmax ? m.g[j].s2[a] : vmax;
    for (int64_t i = 0; i < m.M; ++i)
        for (int a = 0; a < 3; ++a) pmax = m.sl[i].var[a] > pmax ? m.sl[i].var[a] : pmax;
    const double rad2 = r2cut * (vmax + pmax) * 1.02, rad = sqrt(rad2);
    double *mu = (double *)malloc(sizeof(double) * 3 * (size_t)(N ? N : 1));
    double *xp = (double *)malloc(sizeof(double) * 3 * (size_t)(P ? P : 1));
    int64_t *sp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P ? P : 1));
    double *pred = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    if (!mu || !xp || !sp || !pred) return -1;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t j = 0; j < N; ++j)
        for (int a = 0; a < 3; ++a) {
            mu[3 * j + a] = m.g[j].mu[a];
            lo[a] = mu[3 * j + a] < lo[a] ? mu[3 * j + a] : lo[a];
            hi[a] = mu[3 * j + a] > hi[a] ? mu[3 * j + a] : hi[a];
        }
    for (int64_t p = 0; p < P; ++p) {
        double u[3];
        pixel_world(&m, pix[p], &sp[p], u, xp + 3 * p);
        for (int a = 0; a < 3; ++a) {
            lo[a] = xp[3 * p + a] < lo[a] ? xp[3 * p + a] : lo[a];
            hi[a] = xp[3 * p + a] > hi[a] ? xp[3 * p + a] : hi[a];
        }
    }
    double cell = rad;
    for (;;) {  /* at most 2^24 cells */
        double cells = 1.0;
        for (int a = 0; a < 3; ++a) cells *= floor((hi[a] - lo[a]) / cell) + 1.0;
        if (cells <= 16777216.0) break;
        cell *= 1.25;
    }
    or_grid GG, GP;
    if (grid_build(&GG, N, mu, cell, lo, hi) || grid_build(&GP, P, xp, cell, lo, hi)) return -1;
    const double r2t = trunc_cut > 0.0 ? -2.0 * log(trunc_cut) : 1e300;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < P; ++p) {
        double t = 0.0;
        pred[p] = pred_near(&m, &GG, mu, &m.fr[sp[p]], xp + 3 * p, norm_mode, r2cut, rad2, r2t, &t, NULL);
        if (trunc_out) trunc_out[p] = t;
    }
    if (pred_out) memcpy(pred_out, pred, sizeof(double) * (size_t)P);
    /* listed pixels of each slice */
    int64_t *sl_start = (int64_t *)calloc((size_t)m.M + 1, sizeof(int64_t));
    int64_t *sl_items = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P ? P : 1));
    for (int64_t p = 0; p < P; ++p) sl_start[sp[p] + 1]++;
    for (int64_t i = 0; i < m.M; ++i) sl_start[i + 1] += sl_start[i];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m.M ? m.M : 1));
        memcpy(fill, sl_start, sizeof(int64_t) * (size_t)m.M);
        for (int64_t p = 0; p < P; ++p) sl_items[fill[sp[p]]++] = p;
        free(fill);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < K; ++k) {
        const int64_t q = params[k];
        double dL = 0.0;
        if (q < 11 * N) {
            const int64_t comp = q / N, j = q % N;
            double th[2][11];
            or_gauss gv[2];
            for (int s = 0; s < 2; ++s) {
                for (int e = 0; e < 11; ++e) th[s][e] = theta[e * N + j];
                th[s][comp] += (s == 0 ? 1.0 : -1.0) * h[k];
                gauss_setup(1, th[s], 0, &gv[s]);
            }
            int64_t c[3];
            grid_cell_of(&GP, m.g[j].mu, c);
            for (int64_t dz = -1; dz <= 1; ++dz)
                for (int64_t dy = -1; dy <= 1; ++dy)
                    for (int64_t dx = -1; dx <= 1; ++dx) {
                        int64_t cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
                        if (cx < 0 || cy < 0 || cz < 0 || cx >= GP.n[0] || cy >= GP.n[1] || cz >= GP.n[2]) continue;
                        int64_t cl = (cz * GP.n[1] + cy) * GP.n[0] + cx;
                        for (int64_t r = GP.start[cl]; r < GP.start[cl + 1]; ++r) {
                            int64_t p = GP.items[r];
                            const double *x = xp + 3 * p;
                            const or_frame *fr = &m.fr[sp[p]];
                            double old = 0.0, nw[2];
                            or_pair pr;
                            eval_pair(&m.g[j], fr, x, norm_mode, &pr);
                            if (-2.0 * log(pr.e > 0.0 ? pr.e : 1e-300) <= r2cut) old = m.g[j].c * pr.g;
                            for (int s = 0; s < 2; ++s) {
                                eval_pair(&gv[s], fr, x, norm_mode, &pr);
                                nw[s] = (-2.0 * log(pr.e > 0.0 ? pr.e : 1e-300) <= r2cut) ? gv[s].c * pr.g : 0.0;
                            }
                            if (old == 0.0 && nw[0] == 0.0 && nw[1] == 0.0) continue;
                            double rp = pred[p] - old + nw[0] - I_obs[p], rm = pred[p] - old + nw[1] - I_obs[p];
                            dL += w_pix * (rp * rp - rm * rm);
                        }
                    }
        } else {
            const int64_t i = (q - 11 * N) / 6, comp = (q - 11 * N) % 6;
            for (int s = 0; s < 2; ++s) {
                double pose[6];
                for (int e = 0; e < 6; ++e) pose[e] = theta[11 * N + 6 * i + e];
                pose[comp] += (s == 0 ? 1.0 : -1.0) * h[k];
                or_frame fr;
                slice_frame(&m.sl[i], pose, &fr);
                double part = 0.0;
                for (int64_t r = sl_start[i]; r < sl_start[i + 1]; ++r) {
                    int64_t p = sl_items[r];
                    double u[3], x[3];
                    pixel_local(&m.sl[i], pix[p], u);
                    mat_vec(fr.R, u, x);
                    for (int a = 0; a < 3; ++a) x[a] += fr.t[a];
                    double v = pred_near(&m, &GG, mu, &fr, x, norm_mode, r2cut, rad2, 1e300, NULL, NULL) - I_obs[p];
                    part += w_pix * v * v;
                }
                dL += (s == 0 ? 1.0 : -1.0) * part;
            }
        }
        fd_out[k] = dL / (2.0 * h[k]);
    }
    grid_free(&GG);
    grid_free(&GP);
    free(sl_start);
    free(sl_items);
    free(mu);
    free(xp);
    free(sp);
    free(pred);
    model_free(&m);
    return 0;
}

/* ------------------------------------------- large cases: analytic gradient
 * The analytic gradient of L = sum_p w (I_hat_p - I_p)^2 over a listed pixel
 * set, at sizes where the all-pairs loops of oracle_forward_backward are too
 * slow.  The per-pair expressions are those of oracle_forward_backward (the
 * derivative of Eq. 5's numerator with Sigma_obs of Eq. 4, chained through
 * Sigma = R S S^T R^T and the slice frame); only which pairs are visited
 * differs, exactly as in oracle_local_fd: a pair with exp(-1/2 v^T P v) < cut
 * is dropped, and the pairs are found through uniform grids of the Gaussian
 * means and of the pixel positions with cells no smaller than the largest
 * Euclidean radius of that cut.
 *   pred_out, trunc_pred: I_hat_p (float64) and the sum of |terms| of the
 *     pairs with trunc_cut > exp(.) >= cut (what a cut at trunc_cut drops);
 *   loss_out: the loss over the listed pixels;
 *   gsel, asel, tsel (11 x n_sel, entry k of selected Gaussian s at
 *     [k * n_sel + s], k in the parameter order mu, ls, q, c): the gradient of
 *     every component of the Gaussians sel[0..n_sel), the sum of |terms| of
 *     each (the same componentwise scales as oracle_forward_backward's
 *     absgrad) and that sum over the pairs below trunc_cut;
 *   gpose, apose, tpose (6 M): the same for every slice pose (r, tau);
 *   bsel (11 x n_sel), bpose (6 M): the sum of |terms| with each pixel's
 *     residual weight 2 w (I_hat_p - I_p) replaced by 2 w sum_j |c_j g_pj|, the
 *     scale at which a relative rounding error of the prediction I_hat_p
 *     (a sum of |terms| summing to that) moves the gradient;
 *   btsel (11 x n_sel), btpose (6 M): the same with the residual weight
 *     replaced by 2 w trunc_pred_p, how far dropping the pairs below trunc_cut
 *     from the predictions moves the gradient through the residuals. */
typedef struct {
    double a, dc, Go[9], gmu[3], dx[3], GR[9];
} or_pair_grad;

/* Contributions of one pair (residual weight rbar) to the gradient. */
static void pair_grad(const or_gauss *gj, const or_slice *s, const or_frame *fr, const or_pair *pr, const double *u,
                      double rbar, int norm_mode, or_pair_grad *o) {
    o->a = rbar * gj->c * pr->g;
    o->dc = rbar * pr->g;
    const double pk = norm_mode == 0 ? 1.0 : 0.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) o->Go[3 * r + c] = 0.5 * o->a * (pr->Pv[r] * pr->Pv[c] - pk * pr->P[3 * r + c]);
    for (int k = 0; k < 3; ++k) {
        o->gmu[k] = o->a * pr->Pv[k];
        o->dx[k] = -o->a * pr->Pv[k];
    }
    double D[9] = {s->var[0], 0, 0, 0, s->var[1], 0, 0, 0, s->var[2]}, RD[9], GoRD[9];
    mat_mul(fr->R, D, RD);
    mat_mul(o->Go, RD, GoRD);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) o->GR[3 * r + c] = o->dx[r] * u[c] + 2.0 * GoRD[3 * r + c];
}

/* Componentwise |.| scales of one pair's contributions: pose (6), log-scales
 * (3), quaternion (4). */
static void pair_grad_abs(const or_gauss *gj, const or_slice *s, const or_frame *fr, const double *pose,
                          const or_pair_grad *o, const double *u, int norm_mode, double *d6, double *als,
                          double *aq) {
    double Ga[9], RDa[9], GoRDa[9], GRa[9], dxa[3];
    double D[9] = {s->var[0], 0, 0, 0, s->var[1], 0, 0, 0, s->var[2]}, RD[9];
    mat_mul(fr->R, D, RD);
    for (int e = 0; e < 9; ++e) {
        Ga[e] = fabs(o->Go[e]);
        RDa[e] = fabs(RD[e]);
    }
    for (int k = 0; k < 3; ++k) dxa[k] = fabs(o->dx[k]);
    mat_mul(Ga, RDa, GoRDa);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) GRa[3 * r + c] = dxa[r] * fabs(u[c]) + 2.0 * GoRDa[3 * r + c];
    pose_chain_abs(s, pose, GRa, dxa, d6);
    double dls[3];
    cov_chain_abs(gj, Ga, dls, aq);
    for (int k = 0; k < 3; ++k) als[k] = dls[k] + (norm_mode == 0 ? fabs(o->a) : 0.0);
}

/* Indices of the grid items within Euclidean distance sqrt(rad2) of x
 * (the 27 cells around x's cell); returns the count, growing *buf. */
static int64_t grid_near(const or_grid *G, const double *pts, const double *x, double rad2, int64_t **buf,
                         int64_t *cap) {
    int64_t c[3], n = 0;
    grid_cell_of(G, x, c);
    for (int64_t dz = -1; dz <= 1; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= G->n[0] || cy >= G->n[1] || cz >= G->n[2]) continue;
                int64_t cell = (cz * G->n[1] + cy) * G->n[0] + cx;
                for (int64_t q = G->start[cell]; q < G->start[cell + 1]; ++q) {
                    int64_t l = G->items[q];
                    double v0 = x[0] - pts[3 * l], v1 = x[1] - pts[3 * l + 1], v2 = x[2] - pts[3 * l + 2];
                    if (v0 * v0 + v1 * v1 + v2 * v2 > rad2) continue;
                    if (n == *cap) {
                        *cap = *cap ? 2 * *cap : 4096;
                        *buf = (int64_t *)realloc(*buf, sizeof(int64_t) * (size_t)*cap);
                    }
                    (*buf)[n++] = l;
                }
            }
    return n;
}

int oracle_local_grad(int n_stacks, const or_stack *st, int64_t N, const double *theta, int64_t P,
                      const int64_t *pix, const double *I_obs, double w_pix, int norm_mode, double cut,
                      double trunc_cut, int64_t n_sel, const int64_t *sel, double *pred_out, double *trunc_pred,
                      double *loss_out, double *gsel, double *asel, double *tsel, double *gpose, double *apose,
                      double *tpose, double *bsel, double *bpose, double *btsel, double *btpose) {
    or_model m;
    if (model_setup(n_stacks, st, N, theta, &m)) return -1;
    const int64_t M = m.M;
    const double r2cut = -2.0 * log(cut);
    const double r2t = trunc_cut > 0.0 ? -2.0 * log(trunc_cut) : 1e300;
    double vmax = 0.0, pmax = 0.0;
    for (int64_t j = 0; j < N; ++j)
        for (int a = 0; a < 3; ++a) vmax = m.g[j].s2[a] > vmax ? m.g[j].s2[a] : vmax;
    for (int64_t i = 0; i < M; ++i)
        for (int a = 0; a < 3; ++a) pmax = m.sl[i].var[a] > pmax ? m.sl[i].var[a] : pmax;
    const double rad2 = r2cut * (vmax + pmax) * 1.02, rad = sqrt(rad2);
    double *mu = (double *)malloc(sizeof(double) * 3 * (size_t)(N ? N : 1));
    double *xp = (double *)malloc(sizeof(double) * 3 * (size_t)(P ? P : 1));
    double *up = (double *)malloc(sizeof(double) * 3 * (size_t)(P ? P : 1));
    int64_t *sp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P ? P : 1));
    double *pred = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *rbar = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *lt = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *rabs = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    double *rtr = (double *)malloc(sizeof(double) * (size_t)(P ? P : 1));
    if (!mu || !xp || !up || !sp || !pred || !rbar || !lt || !rabs || !rtr) return -1;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t j = 0; j < N; ++j)
        for (int a = 0; a < 3; ++a) {
            mu[3 * j + a] = m.g[j].mu[a];
            lo[a] = mu[3 * j + a] < lo[a] ? mu[3 * j + a] : lo[a];
            hi[a] = mu[3 * j + a] > hi[a] ? mu[3 * j + a] : hi[a];
        }
    for (int64_t p = 0; p < P; ++p) {
        pixel_world(&m, pix[p], &sp[p], up + 3 * p, xp + 3 * p);
        for (int a = 0; a < 3; ++a) {
            lo[a] = xp[3 * p + a] < lo[a] ? xp[3 * p + a] : lo[a];
            hi[a] = xp[3 * p + a] > hi[a] ? xp[3 * p + a] : hi[a];
        }
    }
    double cell = rad;
    for (;;) {
        double cells = 1.0;
        for (int a = 0; a < 3; ++a) cells *= floor((hi[a] - lo[a]) / cell) + 1.0;
        if (cells <= 16777216.0) break;
        cell *= 1.25;
    }
    or_grid GG, GP;
    if (grid_build(&GG, N, mu, cell, lo, hi) || grid_build(&GP, P, xp, cell, lo, hi)) return -1;

    /* predictions, residual weights and loss terms */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < P; ++p) {
        double t = 0.0, ab = 0.0;
        pred[p] = pred_near(&m, &GG, mu, &m.fr[sp[p]], xp + 3 * p, norm_mode, r2cut, rad2, r2t, &t, &ab);
        if (trunc_pred) trunc_pred[p] = t;
        const double r = pred[p] - I_obs[p];
        rbar[p] = 2.0 * w_pix * r;
        rabs[p] = 2.0 * w_pix * ab;
        rtr[p] = 2.0 * w_pix * t;
        lt[p] = w_pix * r * r;
    }
    if (pred_out) memcpy(pred_out, pred, sizeof(double) * (size_t)P);
    if (loss_out) *loss_out = sum_in_order(lt, P);

    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    /* slice poses: pixel-major, per-thread slice accumulators dL/dR_i (9),
     * dL/dt_i (3), |.| of the pose entries (6), |.| below trunc_cut (6), |.| at
     * the prediction-scale residual weights (6), |.| at the truncation-scale
     * residual weights (6) */
    double *pacc = (double *)calloc((size_t)nthreads * (size_t)(M ? M : 1) * 36, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = pacc + (size_t)tid * (size_t)(M ? M : 1) * 36;
        int64_t *buf = NULL, cap = 0;
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < P; ++p) {
            const int64_t i = sp[p];
            const double *x = xp + 3 * p, *u = up + 3 * p;
            const int64_t n = grid_near(&GG, mu, x, rad2, &buf, &cap);
            double *acc = my + 36 * i;
            for (int64_t k = 0; k < n; ++k) {
                const or_gauss *gj = &m.g[buf[k]];
                or_pair pr;
                eval_pair(gj, &m.fr[i], x, norm_mode, &pr);
                const double d2 = -2.0 * log(pr.e > 0.0 ? pr.e : 1e-300);
                if (d2 > r2cut) continue;
                or_pair_grad o;
                pair_grad(gj, &m.sl[i], &m.fr[i], &pr, u, rbar[p], norm_mode, &o);
                for (int e = 0; e < 9; ++e) acc[e] += o.GR[e];
                for (int a = 0; a < 3; ++a) acc[9 + a] += o.dx[a];
                double d6[6], als[3], aq[4];
                pair_grad_abs(gj, &m.sl[i], &m.fr[i], theta + 11 * N + 6 * i, &o, u, norm_mode, d6, als, aq);
                for (int a = 0; a < 6; ++a) acc[12 + a] += fabs(d6[a]);
                if (d2 > r2t)
                    for (int a = 0; a < 6; ++a) acc[18 + a] += fabs(d6[a]);
                or_pair_grad ob;
                pair_grad(gj, &m.sl[i], &m.fr[i], &pr, u, rabs[p], norm_mode, &ob);
                pair_grad_abs(gj, &m.sl[i], &m.fr[i], theta + 11 * N + 6 * i, &ob, u, norm_mode, d6, als, aq);
                for (int a = 0; a < 6; ++a) acc[24 + a] += fabs(d6[a]);
                pair_grad(gj, &m.sl[i], &m.fr[i], &pr, u, rtr[p], norm_mode, &ob);
                pair_grad_abs(gj, &m.sl[i], &m.fr[i], theta + 11 * N + 6 * i, &ob, u, norm_mode, d6, als, aq);
                for (int a = 0; a < 6; ++a) acc[30 + a] += fabs(d6[a]);
            }
        }
        free(buf);
    }
    for (int64_t i = 0; i < M; ++i) {
        double GR[9] = {0}, Gt[3] = {0}, ab[6] = {0}, tb[6] = {0}, bb[6] = {0}, bt[6] = {0};
        for (int t = 0; t < nthreads; ++t) {
            const double *acc = pacc + ((size_t)t * (size_t)M + (size_t)i) * 36;
            for (int e = 0; e < 9; ++e) GR[e] += acc[e];
            for (int a = 0; a < 3; ++a) Gt[a] += acc[9 + a];
            for (int a = 0; a < 6; ++a) ab[a] += acc[12 + a];
            for (int a = 0; a < 6; ++a) tb[a] += acc[18 + a];
            for (int a = 0; a < 6; ++a) bb[a] += acc[24 + a];
            for (int a = 0; a < 6; ++a) bt[a] += acc[30 + a];
        }
        double d6[6];
        pose_chain(&m.sl[i], theta + 11 * N + 6 * i, GR, Gt, d6);
        for (int a = 0; a < 6; ++a) {
            if (gpose) gpose[6 * i + a] = d6[a];
            if (apose) apose[6 * i + a] = ab[a];
            if (tpose) tpose[6 * i + a] = tb[a];
            if (bpose) bpose[6 * i + a] = bb[a];
            if (btpose) btpose[6 * i + a] = bt[a];
        }
    }
    free(pacc);

    /* selected Gaussians: Gaussian-major over the listed pixels near the mean */
#pragma omp parallel
    {
        int64_t *buf = NULL, cap = 0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < n_sel; ++s) {
            const int64_t j = sel[s];
            const or_gauss *gj = &m.g[j];
            double gmu[3] = {0, 0, 0}, GS[9] = {0}, gc = 0.0, gld = 0.0;
            double amu[3] = {0, 0, 0}, als[3] = {0, 0, 0}, aq[4] = {0, 0, 0, 0}, ac = 0.0;
            double tmu[3] = {0, 0, 0}, tls[3] = {0, 0, 0}, tq[4] = {0, 0, 0, 0}, tc = 0.0;
            double bmu[3] = {0, 0, 0}, bls[3] = {0, 0, 0}, bq[4] = {0, 0, 0, 0}, bc = 0.0;
            double umu[3] = {0, 0, 0}, uls[3] = {0, 0, 0}, uq[4] = {0, 0, 0, 0}, uc = 0.0;
            const int64_t n = grid_near(&GP, xp, gj->mu, rad2, &buf, &cap);
            for (int64_t k = 0; k < n; ++k) {
                const int64_t p = buf[k], i = sp[p];
                or_pair pr;
                eval_pair(gj, &m.fr[i], xp + 3 * p, norm_mode, &pr);
                const double d2 = -2.0 * log(pr.e > 0.0 ? pr.e : 1e-300);
                if (d2 > r2cut) continue;
                or_pair_grad o;
                pair_grad(gj, &m.sl[i], &m.fr[i], &pr, up + 3 * p, rbar[p], norm_mode, &o);
                gc += o.dc;
                for (int e = 0; e < 9; ++e) GS[e] += o.Go[e];
                for (int a = 0; a < 3; ++a) gmu[a] += o.gmu[a];
                if (norm_mode == 0) gld += 0.5 * o.a;
                double d6[6], pls[3], pq[4];
                pair_grad_abs(gj, &m.sl[i], &m.fr[i], theta + 11 * N + 6 * i, &o, up + 3 * p, norm_mode, d6, pls,
                              pq);
                const int below = d2 > r2t;
                for (int a = 0; a < 3; ++a) {
                    amu[a] += fabs(o.gmu[a]);
                    als[a] += pls[a];
                    if (below) {
                        tmu[a] += fabs(o.gmu[a]);
                        tls[a] += pls[a];
                    }
                }
                for (int a = 0; a < 4; ++a) {
                    aq[a] += pq[a];
                    if (below) tq[a] += pq[a];
                }
                ac += fabs(o.dc);
                if (below) tc += fabs(o.dc);
                or_pair_grad ob;
                pair_grad(gj, &m.sl[i], &m.fr[i], &pr, up + 3 * p, rabs[p], norm_mode, &ob);
                pair_grad_abs(gj, &m.sl[i], &m.fr[i], theta + 11 * N + 6 * i, &ob, up + 3 * p, norm_mode, d6, pls,
                              pq);
                for (int a = 0; a < 3; ++a) {
                    bmu[a] += fabs(ob.gmu[a]);
                    bls[a] += pls[a];
                }
                for (int a = 0; a < 4; ++a) bq[a] += pq[a];
                bc += fabs(ob.dc);
                pair_grad(gj, &m.sl[i], &m.fr[i], &pr, up + 3 * p, rtr[p], norm_mode, &ob);
                pair_grad_abs(gj, &m.sl[i], &m.fr[i], theta + 11 * N + 6 * i, &ob, up + 3 * p, norm_mode, d6, pls,
                              pq);
                for (int a = 0; a < 3; ++a) {
                    umu[a] += fabs(ob.gmu[a]);
                    uls[a] += pls[a];
                }
                for (int a = 0; a < 4; ++a) uq[a] += pq[a];
                uc += fabs(ob.dc);
            }
            double dls[3], dq[4];
            cov_chain(gj, GS, dls, dq);
            double g11[11], a11[11], t11[11], b11[11], u11[11];
            for (int a = 0; a < 3; ++a) {
                g11[a] = gmu[a];
                g11[3 + a] = dls[a] + 2.0 * gld;
                a11[a] = amu[a];
                a11[3 + a] = als[a];
                t11[a] = tmu[a];
                t11[3 + a] = tls[a];
                b11[a] = bmu[a];
                b11[3 + a] = bls[a];
                u11[a] = umu[a];
                u11[3 + a] = uls[a];
            }
            for (int a = 0; a < 4; ++a) {
                g11[6 + a] = dq[a];
                a11[6 + a] = aq[a];
                t11[6 + a] = tq[a];
                b11[6 + a] = bq[a];
                u11[6 + a] = uq[a];
            }
            g11[10] = gc;
            a11[10] = ac;
            t11[10] = tc;
            b11[10] = bc;
            u11[10] = uc;
            for (int a = 0; a < 11; ++a) {
                if (gsel) gsel[a * n_sel + s] = g11[a];
                if (asel) asel[a * n_sel + s] = a11[a];
                if (tsel) tsel[a * n_sel + s] = t11[a];
                if (bsel) bsel[a * n_sel + s] = b11[a];
                if (btsel) btsel[a * n_sel + s] = u11[a];
            }
        }
        free(buf);
    }
    grid_free(&GG);
    grid_free(&GP);
    free(mu);
    free(xp);
    free(up);
    free(sp);
    free(pred);
    free(rbar);
    free(lt);
    free(rabs);
    free(rtr);
    model_free(&m);
    return 0;
}
